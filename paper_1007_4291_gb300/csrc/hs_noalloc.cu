// hs_apply_noalloc: the sweep application z = M_alpha r without touching the
// allocator.  Some callers cannot call cudaMalloc at the point where they
// apply the preconditioner: applications that reserve all device memory at
// start-up for their own pool, latency-critical loops where cudaMalloc's
// implicit device synchronisation is not acceptable, and plug-in hosts that
// forbid a library from allocating after initialisation.  This entry point
// keeps every temporary it needs (the working vector in the solver layout,
// the per-column store of the chunk pass and the separator buffers) in one
// file-scope device array of fixed size instead of the plan's workspace.
//
// The plan is only read: its factors and tables are shared with every other
// call, its own workspace is not touched, so hs_apply or hs_solve on the same
// plan may run beside this call.  The static array, though, is shared by
// every hs_apply_noalloc call in the process on a device and keeps the
// contents of the last call.  No part of it has to start at zero: every
// kernel of the sweep writes each temporary before reading it.  Calls of this
// entry point that overlap on the GPU (on different streams, or from several
// host threads) race on it and must be serialised by the caller.
#include <mutex>
#include "hs_internal.cuh"

namespace hs {
namespace {

// Size of the static scratch: 32 MiB per device that loads the library.
constexpr size_t kScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_sweep_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_sweep_scratch for device `dev`, which must be current
// (looked up once per device; in host code the symbol itself is only a
// host-side stand-in).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return HS_EUNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_sweep_scratch);
    if (e != cudaSuccess || !ptr) return e != cudaSuccess ? cuda_status(e) : HS_ECUDA;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return HS_OK;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" int hs_apply_noalloc(hs_plan* plan, const void* r, void* z, int nrhs, int dtype, void* stream) {
  if (!plan || !r || !z) return HS_EINVAL;
  const Plan& p = *reinterpret_cast<const Plan*>(plan);
  if (nrhs < 1 || nrhs > p.max_nrhs || (dtype != HS_C64 && dtype != HS_C128)) return HS_EINVAL;
  if (p.dim != 2) return HS_EUNSUPPORTED;
  // the scratch of the current device must be the plan's device: the sweep
  // reads the plan's factors there
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev != p.device) return HS_EINVAL;
  int Wmax = 0;
  for (const auto& d : p.blocks) Wmax = d.W > Wmax ? d.W : Wmax;
  const size_t es = (p.prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  const size_t n2 = (size_t)p.n * p.n, R = (size_t)nrhs;
  const size_t bu = al256(n2 * R * es), bz = al256(2 * (size_t)p.n * R * Wmax * es);
  const size_t bs = al256(2 * (size_t)p.P * R * Wmax * es);
  if (bu + bz + 4 * bs > kScratchBytes) return HS_EINVAL;  // problem larger than the static scratch
  void* base = nullptr;
  int st = scratch_address(dev, &base);
  if (st != HS_OK) return st;
  plan_wait(p, (cudaStream_t)stream);
  char* q = static_cast<char*>(base);
  SweepWork w{};
  w.u = q; q += bu;
  w.z = q; q += bz;
  w.rc = q; q += bs;
  w.lc = q; q += bs;
  w.xs = q; q += bs;
  w.ps = q;
  cudaStream_t s = (cudaStream_t)stream;
  st = layout_to_internal(r, dtype, w.u, p.prec, (int)n2, nrhs, s);
  if (st == HS_OK) st = sweep_launch_work(p, w, nrhs, s);
  if (st == HS_OK) st = layout_from_internal(w.u, p.prec, z, dtype, (int)n2, nrhs, s);
  return st;
}
