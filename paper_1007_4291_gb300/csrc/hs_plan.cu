// Host side of libhs: option defaults, argument checks, the two-front block
// partition (Sec. 2.3), the PML tables (Eq. sigma and the stretch factors of
// Sec. 2.1, the moving profile of Eq. helma), device memory of the plan, and
// the status/error entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <complex>
#include <atomic>
#include <mutex>
#include "hs_internal.cuh"
#include "hs_device.cuh"
#include "hs3d.cuh"

namespace hs {

int cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HS_ENOMEM; }
  return HS_ECUDA;
}

int padded_width(int w) {
  if (w <= 0) return -1;
  if (w <= 8) return 8;
  if (w <= 12) return 12;
  if (w <= 16) return 16;
  if (w <= 24) return 24;
  if (w <= 32) return 32;
  return -1;
}

namespace {

using zc = std::complex<double>;

// Eq. sigma, two-sided quadratic ramp of width eta on [0,1].
double sigma_boundary(double t, double eta, double C) {
  if (t <= eta) { double q = (t - eta) / eta; return (C / eta) * q * q; }
  if (t >= 1.0 - eta) { double q = (t - 1.0 + eta) / eta; return (C / eta) * q * q; }
  return 0.0;
}
// sigma_2 of Eq. sigma: the ramp at t = 0 only (Dirichlet-top formulation).
double sigma_one_sided(double t, double eta, double C) {
  if (t <= eta) { double q = (t - eta) / eta; return (C / eta) * q * q; }
  return 0.0;
}
// One-sided moving profile of Eq. helma: distance d from the window's
// Dirichlet row, width eta_b; zero from depth eta_b on.
double sigma_moving(double d, double eta_b, double C) {
  if (d < 0.0 || d > eta_b) return 0.0;
  double q = (d - eta_b) / eta_b;
  return (C / eta_b) * q * q;
}
// 1/s = 1 + i sigma/omega (Sec. 2.1)
zc inv_stretch(double sig, double omega) { return zc(1.0, sig / omega); }
zc stretch(double sig, double omega) { return 1.0 / inv_stretch(sig, omega); }

// 2D plans draw their device buffers from one stream-ordered pool per device
// that keeps freed memory (release threshold at its maximum): a plan set up
// after another one destroyed reuses its memory without mapping it again
// (n = 2047, 64 RHS: cudaMalloc + cudaFree of a plan's buffers 6.1 ms, from
// the warm pool 0.06 ms).  hs_release_workspace() returns it to the device.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_plan_pool[kMaxPoolDevices] = {};
}  // namespace

int plan_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= kMaxPoolDevices) return HS_EUNSUPPORTED;
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_plan_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { cudaGetLastError(); return HS_ECUDA; }
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_plan_pool[dev] = pool;
  }
  *out = g_plan_pool[dev];
  return HS_OK;
}

void trim_plan_pools() {
  std::lock_guard<std::mutex> g(g_pool_mu);
  for (int d = 0; d < kMaxPoolDevices; ++d)
    if (g_plan_pool[d]) cudaMemPoolTrimTo(g_plan_pool[d], 0);
}

namespace {

c128 to_c(zc z) { return c128{z.real(), z.imag()}; }
c64 to_f(zc z) { return c64{(float)z.real(), (float)z.imag()}; }

template <typename T> int dalloc(Plan& p, T** ptr, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaMemPool_t pool = nullptr;
  int st = plan_pool(p.device, &pool);
  if (st != HS_OK) { *ptr = nullptr; return st; }
  cudaError_t e = cudaMallocFromPoolAsync((void**)ptr, bytes, pool, 0);
  if (e != cudaSuccess) { *ptr = nullptr; cudaGetLastError(); return HS_ENOMEM; }
  p.bytes += (long long)bytes;
  return HS_OK;
}
#define HS_TRY(expr) do { int _s = (expr); if (_s != HS_OK) return _s; } while (0)

}  // namespace

// Two-front partition: F, d-row lower blocks (last one takes the remainder),
// the middle layer (n+1)/2, and the mirrored upper front ending at E.
// Single front (Dirichlet top, Sec. 2.1-2.2): F, then d-row blocks upward to
// row n; the top block is solved once like the middle layer (it has no block
// above it to correct it in the backward sweep).  With k buffer rows the
// moving PML of a block sits k rows away from it (Sec. 2.2): window
// [lo - k - b + 1, hi] (lower) or [lo, hi + k + b - 1] (upper); a window that
// would cross the grid boundary is cut there and keeps the operator's own
// profile (the exact Schur inverse, as for the first layers of the paper).
void build_blocks(Plan& p) {
  const int n = p.n, bp = p.bp, b = p.b, dL = p.dL;
  const int kb = p.opt.buffer_rows;
  p.blocks.clear();
  p.stages.clear();
  auto add = [&](BlockDesc d) { p.blocks.push_back(d); return (int)p.blocks.size() - 1; };
  auto lower_block = [&](int lo, int hi) {
    BlockDesc Lb{}; Lb.kind = BK_LOWER; Lb.lo = lo; Lb.hi = hi; Lb.whi = hi;
    Lb.wlo = lo - kb - b + 1;
    if (Lb.wlo < 1) { Lb.wlo = 1; Lb.exact = 1; }
    Lb.prev_lo_row = lo - 1; Lb.prev_hi_row = 0; Lb.next_row = hi < n ? hi + 1 : 0; Lb.coup_local = hi - Lb.wlo;
    return Lb;
  };
  BlockDesc F{}; F.kind = BK_F; F.lo = 1; F.hi = bp; F.wlo = 1; F.whi = bp;
  F.prev_lo_row = 0; F.prev_hi_row = 0; F.next_row = bp + 1; F.coup_local = bp - 1;
  if (!p.opt.two_front) {
    std::vector<int> sizes;
    for (int r = n - bp; r > 0; r -= std::min(dL, r)) sizes.push_back(std::min(dL, r));
    p.stages.push_back({add(F)});
    int lo = bp + 1;
    for (size_t q = 0; q < sizes.size(); ++q) {
      const int hi = lo + sizes[q] - 1;
      if (q + 1 < sizes.size()) p.stages.push_back({add(lower_block(lo, hi))});
      else p.middle = add(lower_block(lo, hi));
      lo = hi + 1;
    }
  } else {
    const int m = (n + 1) / 2;
    const int rows_front = (n - 1) / 2 - bp;
    std::vector<int> sizes;
    for (int r = rows_front; r > 0; r -= std::min(dL, r)) sizes.push_back(std::min(dL, r));
    BlockDesc E{}; E.kind = BK_E; E.lo = n - bp + 1; E.hi = n; E.wlo = n - bp + 1; E.whi = n;
    E.prev_lo_row = 0; E.prev_hi_row = 0; E.next_row = n - bp; E.coup_local = 0;
    p.stages.push_back({add(F), add(E)});
    int lo = bp + 1;
    for (int d : sizes) {
      int hi = lo + d - 1;
      BlockDesc Lb = lower_block(lo, hi);
      int ulo = n + 1 - hi, uhi = n + 1 - lo;
      BlockDesc Ub{}; Ub.kind = BK_UPPER; Ub.lo = ulo; Ub.hi = uhi; Ub.wlo = ulo; Ub.whi = uhi + kb + b - 1;
      if (Ub.whi > n) { Ub.whi = n; Ub.exact = 1; }
      Ub.prev_lo_row = 0; Ub.prev_hi_row = uhi + 1; Ub.next_row = ulo - 1; Ub.coup_local = 0;
      p.stages.push_back({add(Lb), add(Ub)});
      lo = hi + 1;
    }
    BlockDesc M{}; M.kind = BK_MIDDLE; M.lo = m; M.hi = m; M.wlo = m - kb - b + 1; M.whi = m + kb + b - 1;
    M.prev_lo_row = m - 1; M.prev_hi_row = m + 1; M.next_row = 0; M.coup_local = -1;
    p.middle = add(M);
  }
  for (auto& d : p.blocks) {
    d.w = d.whi - d.wlo + 1;
    d.W = padded_width(d.w);
    d.out_off = d.lo - d.wlo;
    d.d_out = d.hi - d.lo + 1;
  }
}

}  // namespace hs

using namespace hs;

extern "C" int hs_default_options(hs_options* opt) {
  if (!opt) return HS_EINVAL;
  opt->alpha = 2.0;
  opt->pml_C = 20.0;
  opt->moving_pml_C = 0.0;
  opt->layers_per_step = 12;
  opt->factor_prec = HS_C64;
  opt->chunk = 0;
  opt->max_nrhs = 64;
  opt->restart = 20;
  opt->reorth = 0;
  opt->spin_budget = 1LL << 30;
  opt->graphs = 1;
  opt->frontal_gemm = 3;
  opt->krylov_basis = 1;
  opt->inner_tol = 1e-4;
  opt->tune_cache = nullptr;
  opt->sep_rhs_per_cta = 0;
  opt->two_front = 1;
  opt->buffer_rows = 0;
  opt->async_setup = 0;
  return HS_OK;
}

extern "C" const char* hs_strerror(int s) {
  switch (s) {
    case HS_OK: return "success";
    case HS_EINVAL: return "invalid argument";
    case HS_ENOMEM: return "device allocation failed";
    case HS_EBREAKDOWN: return "zero pivot in a subproblem factorisation";
    case HS_ETIMEOUT: return "bounded device wait expired";
    case HS_ENOCONV: return "FGMRES did not converge";
    case HS_ECUDA: return "CUDA runtime error";
    case HS_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

static void free_plan_memory(Plan* p) {
  void* ptrs[] = {p->d_inv_s1, p->d_a1, p->d_inv_s2, p->d_a2, p->f_inv_s1, p->f_a1, p->f_inv_s2, p->f_a2,
                  p->d_pml1, p->d_pml2, p->d_m0, p->f_m0, p->d_cinv2, p->d_s2win, p->d_blocks,
                  p->k_inv_s1, p->k_a1, p->k_inv_s2, p->k_a2, p->k_m0,
                  p->d_fac, p->d_red, p->d_cor, p->d_u, p->d_z, p->d_rc, p->d_lc, p->d_xs, p->d_ps,
                  p->d_status};
  // back to the plan pool, stream-ordered after everything already queued on
  // the legacy stream (the caller has synchronised the device)
  for (void* q : ptrs) if (q) cudaFreeAsync(q, 0);
}

extern "C" int hs_destroy(hs_plan* plan) {
  if (!plan) return HS_OK;
  Plan* p = reinterpret_cast<Plan*>(plan);
  // the plan's work and memory live on its own device, which need not be the
  // caller's current one
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->ready) cudaEventDestroy(p->ready);
  forget_batch_graphs(p->uid);
  release_sweep_graphs(*p);
  release_plan3(*p);
  free_plan_memory(p);
  const int dev = p->device;
  delete p;
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
  return HS_OK;
}

extern "C" int hs_setup_flops(const hs_plan* plan, double* gemm_flops, double* inverse_flops) {
  if (!plan) return HS_EINVAL;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  const Plan3* q = p->dim == 3 ? static_cast<const Plan3*>(p->p3) : nullptr;
  if (gemm_flops) *gemm_flops = q ? q->gemm_flops : 0.0;
  if (inverse_flops) *inverse_flops = q ? q->inv_flops : 0.0;
  return HS_OK;
}

extern "C" long long hs_plan_bytes(const hs_plan* plan) {
  if (!plan) return 0;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  return p->bytes;
}

std::atomic<long long> hs::g_launches{0};

extern "C" long long hs_kernel_launches(void) { return hs::g_launches.load(); }

extern "C" int hs_last_device_status(hs_plan* plan) {
  if (!plan) return HS_EINVAL;
  Plan* p = reinterpret_cast<Plan*>(plan);
  plan_wait_host(*p);
  int st[3] = {0, 0, 0};
  if (cudaMemcpy(st, p->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return HS_ECUDA;
  return st[0];
}

extern "C" int hs_sync(hs_plan* plan, void* stream) {
  if (!plan) return HS_EINVAL;
  plan_wait_host(*reinterpret_cast<Plan*>(plan));
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  return hs_last_device_status(plan);
}

// 3D plan: validation, the 1D stretch tables (all axes share the boundary
// profile), omega^2/c^2 and 1/c^2 per point, the block partition in x3
// layers, and the slab-solver workspace (hs3d.cu).
static int prepare_plan3d(const double* c, double omega, int n, int pml_width, int moving_pml_width,
                          const hs_options* opt_in, Plan** out) {
  if (n < 3 || n % 2 != 1 || pml_width < 1 || 2 * pml_width + 1 > n) return HS_EINVAL;
  if (moving_pml_width < 1 || moving_pml_width > pml_width + 1) return HS_EINVAL;
  if (n > 255) return HS_EUNSUPPORTED;
  hs_options opt;
  hs_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (!(opt.alpha >= 0.0) || !(opt.pml_C >= 0.0) || !(opt.moving_pml_C >= 0.0) || opt.layers_per_step < 1 || opt.max_nrhs < 1 ||
      opt.max_nrhs > 4096 || opt.restart < 1)
    return HS_EINVAL;
  if (opt.factor_prec != HS_C64 && opt.factor_prec != HS_C128) return HS_EINVAL;
  if (opt.frontal_gemm < 0 || opt.frontal_gemm > 4) return HS_EINVAL;
  if (opt.two_front != 1 || opt.buffer_rows != 0) return HS_EUNSUPPORTED;   // 3D: two fronts, no buffers
  const size_t N3 = (size_t)n * n * n;
  for (size_t k = 0; k < N3; ++k)
    if (!(c[k] > 0.0) || !std::isfinite(c[k])) return HS_EINVAL;
  Plan* p = new Plan();
  p->n = n; p->dim = 3; p->bp = pml_width; p->b = moving_pml_width; p->dL = opt.layers_per_step;
  p->omega = omega; p->alpha = opt.alpha; p->C = opt.pml_C; p->Cm = opt.moving_pml_C > 0.0 ? opt.moving_pml_C : opt.pml_C; p->h = 1.0 / (n + 1);
  p->prec = opt.factor_prec; p->max_nrhs = opt.max_nrhs; p->opt = opt;
  cudaGetDevice(&p->device);
  p->opt.tune_cache = nullptr;
  build_blocks(*p);
  int st = HS_OK;
  auto fail = [&](int code) { release_plan3(*p); free_plan_memory(p); delete p; return code; };
  const double h = p->h, eta = p->bp * h, C = p->C;
  std::vector<c128> inv_s(n + 2), a_half(n + 1);
  std::vector<unsigned char> pml(n + 2, 0);
  for (int k = 0; k <= n + 1; ++k) inv_s[k] = to_c(inv_stretch(sigma_boundary(k * h, eta, C), omega));
  for (int k = 0; k <= n; ++k) a_half[k] = to_c(stretch(sigma_boundary((k + 0.5) * h, eta, C), omega) / (h * h));
  std::vector<double> m0(N3), ci2(N3);
  for (size_t k = 0; k < N3; ++k) {
    ci2[k] = 1.0 / (c[k] * c[k]);
    m0[k] = omega * omega * ci2[k];
  }
  const size_t es = (p->prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  if ((st = dalloc(*p, &p->d_inv_s1, n + 2)) || (st = dalloc(*p, &p->d_a1, n + 1)) ||
      (st = dalloc(*p, &p->d_m0, N3)) || (st = dalloc(*p, &p->d_cinv2, N3)) ||
      (st = dalloc(*p, &p->d_blocks, p->blocks.size())) || (st = dalloc(*p, &p->d_status, 4)) ||
      (st = dalloc(*p, (char**)&p->d_u, N3 * (size_t)p->max_nrhs * es)))
    return fail(st);
  cudaMemcpy(p->d_inv_s1, inv_s.data(), (n + 2) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_a1, a_half.data(), (n + 1) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_m0, m0.data(), N3 * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_cinv2, ci2.data(), N3 * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(p->d_status, 0, 4 * sizeof(int));
  if ((st = prepare_plan3(*p)) != HS_OK) return fail(st);
  cudaMemcpy(p->d_blocks, p->blocks.data(), p->blocks.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice);
  if (cudaGetLastError() != cudaSuccess) return fail(HS_ECUDA);
  static std::atomic<long long> next_uid3{1LL << 40};
  p->uid = next_uid3.fetch_add(1);
  *out = p;
  return HS_OK;
}

// Validate the arguments, build the host tables of one problem and allocate
// and fill its device memory (no kernel launches).  On failure nothing is
// left allocated.
namespace hs {
// Per-point tables from the velocities already copied into m0: 1/c^2,
// omega^2/c^2 in double, float and double-float (same operations and
// rounding as a host loop would do, so the tables are exact copies).
__global__ void point_tables_kernel(double* m0, double* cinv2, float* fm0, float* km0, long long N, double omega2) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    const double cv = m0[k];
    const double ci = 1.0 / (cv * cv);
    const double m = omega2 * ci;
    const float hi = (float)m;
    cinv2[k] = ci;
    m0[k] = m;
    fm0[k] = hi;
    km0[2 * k] = hi;
    km0[2 * k + 1] = (float)(m - (double)hi);
  }
}
}  // namespace hs

static int prepare_plan(const double* c, double omega, int n, int dim, int pml_width, int moving_pml_width,
                        const hs_options* opt_in, Plan** out) {
  *out = nullptr;
  if (!c || !(omega > 0.0) || !std::isfinite(omega)) return HS_EINVAL;
  if (dim != 2 && dim != 3) return HS_EINVAL;
  if (dim == 3) return prepare_plan3d(c, omega, n, pml_width, moving_pml_width, opt_in, out);
  hs_options opt;
  hs_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.two_front != 0 && opt.two_front != 1) return HS_EINVAL;
  if (opt.buffer_rows < 0) return HS_EINVAL;
  if (opt.async_setup != 0 && opt.async_setup != 1) return HS_EINVAL;
  if (opt.two_front) {
    if (n < 3 || n % 2 != 1 || pml_width < 1 || 2 * pml_width + 1 > n) return HS_EINVAL;
    // the middle layer's window must fit inside the grid
    if ((n + 1) / 2 - opt.buffer_rows - moving_pml_width < 0) return HS_EINVAL;
  } else {
    if (n < 3 || pml_width < 1 || pml_width + 1 > n) return HS_EINVAL;
  }
  if (moving_pml_width < 1 || moving_pml_width > pml_width + 1) return HS_EINVAL;
  if (n > 32767) return HS_EUNSUPPORTED;   // point indices are 32-bit (n^2 < 2^30)
  if (!(opt.alpha >= 0.0) || !(opt.pml_C >= 0.0) || !(opt.moving_pml_C >= 0.0) || opt.layers_per_step < 1 || opt.max_nrhs < 1 ||
      opt.max_nrhs > 4096 || opt.restart < 1 || opt.chunk < 0 || opt.chunk == 1 || opt.spin_budget < 1)
    return HS_EINVAL;
  if (opt.factor_prec != HS_C64 && opt.factor_prec != HS_C128) return HS_EINVAL;
  if ((opt.krylov_basis != 0 && opt.krylov_basis != 1) || !(opt.inner_tol > 0.0 && opt.inner_tol < 1.0))
    return HS_EINVAL;
  if (opt.sep_rhs_per_cta != 0 && opt.sep_rhs_per_cta != 1 && opt.sep_rhs_per_cta != 2 && opt.sep_rhs_per_cta != 4)
    return HS_EINVAL;
  for (long long k = 0; k < (long long)n * n; ++k)
    if (!(c[k] > 0.0) || !std::isfinite(c[k])) return HS_EINVAL;

  Plan* p = new Plan();
  p->n = n; p->dim = dim; p->bp = pml_width; p->b = moving_pml_width; p->dL = opt.layers_per_step;
  p->omega = omega; p->alpha = opt.alpha; p->C = opt.pml_C; p->Cm = opt.moving_pml_C > 0.0 ? opt.moving_pml_C : opt.pml_C; p->h = 1.0 / (n + 1);
  p->prec = opt.factor_prec; p->max_nrhs = opt.max_nrhs; p->opt = opt;
  cudaGetDevice(&p->device);
  build_blocks(*p);
  int Wmax = 0;
  for (auto& d : p->blocks) {
    if (d.W < 0) { delete p; return HS_EUNSUPPORTED; }
    Wmax = std::max(Wmax, d.W);
  }
  // x1 chunking of the subproblem solves (>= 2 columns per chunk).  Default:
  // one chunk CTA of each front per pair of SMs, so that a sweep stage's
  // 2 P chunk CTAs fill the GPU in one wave.  The separator solve keeps the
  // right-hand sides of all separators of a chain in shared memory, which
  // bounds the separator count.
  int chunk = opt.chunk;
  if (chunk == 0) {
    int sep = 0;
    chunk = tuned_chunk(opt.tune_cache, n, pml_width, moving_pml_width, opt.layers_per_step, opt.factor_prec,
                        opt.max_nrhs, &sep);
    if (chunk && opt.sep_rhs_per_cta == 0) p->opt.sep_rhs_per_cta = sep;
  }
  p->opt.tune_cache = nullptr;  // the string belongs to the caller
  if (!chunk) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 2) sms = 2;
    const int per_front = sms / 2;
    chunk = (n + per_front - 1) / per_front;
  }
  p->L = chunk;
  p->L = std::max(p->L, (n + max_separators(Wmax, opt.factor_prec)) / (max_separators(Wmax, opt.factor_prec) + 1));
  if (p->L > n) p->L = n;
  if (p->L < 2) p->L = 2;
  p->P = (n + p->L - 1) / p->L;

  int st = HS_OK;
  auto fail = [&](int s) { free_plan_memory(p); delete p; return s; };
  const double h = p->h, eta = p->bp * h, eta_b = p->b * h, C = p->C, Cm = p->Cm;

  // ---- 1D tables of the x1 and x2 axes (Eq. sigma: two-sided in x1; in x2
  //      two-sided, or the one-sided sigma_2 for the Dirichlet-top formulation)
  const bool top = !opt.two_front;
  auto sig_axis = [&](int axis, double t) {
    return (axis == 2 && top) ? sigma_one_sided(t, eta, C) : sigma_boundary(t, eta, C);
  };
  std::vector<c128> inv_s(n + 2), a_half(n + 1), inv_s2(n + 2), a_half2(n + 1);
  std::vector<c64> f_inv_s(n + 2), f_a_half(n + 1), f_inv_s2(n + 2), f_a_half2(n + 1);
  std::vector<unsigned char> pml(n + 2, 0), pml2(n + 2, 0);
  auto fill_axis = [&](int axis, std::vector<c128>& is, std::vector<c128>& ah, std::vector<c64>& fis,
                       std::vector<c64>& fah, std::vector<unsigned char>& pm) {
    for (int k = 0; k <= n + 1; ++k) {
      zc v = inv_stretch(sig_axis(axis, k * h), omega);
      is[k] = to_c(v); fis[k] = to_f(v);
    }
    for (int k = 0; k <= n; ++k) {
      zc v = stretch(sig_axis(axis, (k + 0.5) * h), omega) / (h * h);
      ah[k] = to_c(v); fah[k] = to_f(v);
    }
    for (int k = 1; k <= n; ++k) {
      bool t = sig_axis(axis, k * h) != 0.0 || sig_axis(axis, (k - 0.5) * h) != 0.0 ||
               sig_axis(axis, (k + 0.5) * h) != 0.0;
      pm[k] = t ? 1 : 0;
    }
  };
  fill_axis(1, inv_s, a_half, f_inv_s, f_a_half, pml);
  fill_axis(2, inv_s2, a_half2, f_inv_s2, f_a_half2, pml2);
  if ((st = dalloc(*p, &p->d_inv_s1, n + 2)) || (st = dalloc(*p, &p->d_a1, n + 1)) ||
      (st = dalloc(*p, &p->d_inv_s2, n + 2)) || (st = dalloc(*p, &p->d_a2, n + 1)) ||
      (st = dalloc(*p, &p->f_inv_s1, n + 2)) || (st = dalloc(*p, &p->f_a1, n + 1)) ||
      (st = dalloc(*p, &p->f_inv_s2, n + 2)) || (st = dalloc(*p, &p->f_a2, n + 1)) ||
      (st = dalloc(*p, &p->d_pml1, n + 2)) || (st = dalloc(*p, &p->d_pml2, n + 2)))
    return fail(st);
  cudaMemcpy(p->d_inv_s1, inv_s.data(), (n + 2) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_inv_s2, inv_s2.data(), (n + 2) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_a1, a_half.data(), (n + 1) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_a2, a_half2.data(), (n + 1) * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->f_inv_s1, f_inv_s.data(), (n + 2) * sizeof(c64), cudaMemcpyHostToDevice);
  cudaMemcpy(p->f_inv_s2, f_inv_s2.data(), (n + 2) * sizeof(c64), cudaMemcpyHostToDevice);
  cudaMemcpy(p->f_a1, f_a_half.data(), (n + 1) * sizeof(c64), cudaMemcpyHostToDevice);
  cudaMemcpy(p->f_a2, f_a_half2.data(), (n + 1) * sizeof(c64), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_pml1, pml.data(), n + 2, cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_pml2, pml2.data(), n + 2, cudaMemcpyHostToDevice);
  {   // the PML-free points form one index range [lo, hi) per axis (sigma vanishes away from the boundary)
    int lo = 0;
    while (lo < n && pml[lo + 1]) ++lo;
    int hi = lo;
    while (hi < n && !pml[hi + 1]) ++hi;
    bool contiguous = true;
    for (int i = hi; i < n; ++i) contiguous = contiguous && pml[i + 1];
    p->int_lo = contiguous ? lo : 0;
    p->int_hi = contiguous ? hi : 0;
  }

  // ---- per-point omega^2/c^2 and 1/c^2 (and double-float copies)
  const size_t N2 = (size_t)n * n;
  {
    auto split = [](double x, float* o) {
      o[0] = (float)x;
      o[1] = (float)(x - (double)o[0]);
    };
    std::vector<float> kis(4 * (n + 2)), ka(4 * (n + 1)), kis2(4 * (n + 2)), ka2(4 * (n + 1));
    for (int k = 0; k <= n + 1; ++k) { split(inv_s[k].re, &kis[4 * k]); split(inv_s[k].im, &kis[4 * k + 2]); }
    for (int k = 0; k <= n; ++k) { split(a_half[k].re, &ka[4 * k]); split(a_half[k].im, &ka[4 * k + 2]); }
    for (int k = 0; k <= n + 1; ++k) { split(inv_s2[k].re, &kis2[4 * k]); split(inv_s2[k].im, &kis2[4 * k + 2]); }
    for (int k = 0; k <= n; ++k) { split(a_half2[k].re, &ka2[4 * k]); split(a_half2[k].im, &ka2[4 * k + 2]); }
    if ((st = dalloc(*p, &p->d_m0, N2)) || (st = dalloc(*p, &p->f_m0, N2)) || (st = dalloc(*p, &p->d_cinv2, N2)) ||
        (st = dalloc(*p, (float**)&p->k_m0, 2 * N2)) || (st = dalloc(*p, (float**)&p->k_inv_s1, 4 * (n + 2))) ||
        (st = dalloc(*p, (float**)&p->k_inv_s2, 4 * (n + 2))) || (st = dalloc(*p, (float**)&p->k_a1, 4 * (n + 1))) ||
        (st = dalloc(*p, (float**)&p->k_a2, 4 * (n + 1))))
      return fail(st);
    // velocities to the device once; the per-point tables are formed there
    cudaMemcpy(p->d_m0, c, N2 * sizeof(double), cudaMemcpyHostToDevice);
    const long long gb = std::min<long long>(((long long)N2 + 255) / 256, 4096);
    hs::point_tables_kernel<<<(int)gb, 256>>>(p->d_m0, p->d_cinv2, p->f_m0, (float*)p->k_m0, (long long)N2, omega * omega);
    if (cudaStreamSynchronize(0) != cudaSuccess) return fail(HS_ECUDA);
    cudaMemcpy(p->k_inv_s1, kis.data(), kis.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(p->k_inv_s2, kis2.data(), kis2.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(p->k_a1, ka.data(), ka.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(p->k_a2, ka2.data(), ka2.size() * sizeof(float), cudaMemcpyHostToDevice);
  }

  // ---- per-block window x2 tables (moving profile of Eq. helma or the
  //      boundary profile for F and E), and storage offsets
  std::vector<c128> s2win;
  // offsets below are counted in complex elements of the factor precision
  long long fac = 0, red = 0, cor = 0;
  for (auto& d : p->blocks) {
    d.s2_off = (int)s2win.size();
    // x2 absorption of the block's subproblem at coordinate x
    // (the moving profiles start at the rows just outside the window: its
    // Dirichlet rows wlo - 1 and whi + 1, b + k rows from the block)
    auto sig = [&](double x) {
      if (d.kind == BK_F || d.kind == BK_E || d.exact) return sig_axis(2, x);
      double s = 0.0;
      if (d.kind == BK_LOWER || d.kind == BK_MIDDLE) s += sigma_moving(x - (d.wlo - 1) * h, eta_b, Cm);
      if (d.kind == BK_UPPER || d.kind == BK_MIDDLE) s += sigma_moving((d.whi + 1) * h - x, eta_b, Cm);
      return s;
    };
    for (int q = 0; q < d.w; ++q) s2win.push_back(to_c(inv_stretch(sig((d.wlo + q) * h), omega)));
    for (int q = 0; q < d.w; ++q) s2win.push_back(to_c(stretch(sig((d.wlo + q + 0.5) * h), omega) / (h * h)));
    for (int q = 0; q < d.w; ++q) s2win.push_back(to_c(stretch(sig((d.wlo + q - 0.5) * h), omega) / (h * h)));
    d.fac_off = fac; fac += (long long)n * payload_elems(d.W, d.d_out);
    d.red_off = red; red += (long long)std::max(p->P - 1, 1) * red_elems(d.W);
    d.cor_off = cor; cor += (long long)p->P * cor_elems(d.W);
  }
  p->fac_elems = fac; p->red_elems = red; p->cor_elems = cor;
  const size_t es = (p->prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  if ((st = dalloc(*p, &p->d_s2win, s2win.size())) || (st = dalloc(*p, &p->d_blocks, p->blocks.size())) ||
      (st = dalloc(*p, (char**)&p->d_fac, fac * es)) || (st = dalloc(*p, (char**)&p->d_red, red * es)) ||
      (st = dalloc(*p, (char**)&p->d_cor, cor * es)) || (st = dalloc(*p, &p->d_status, 4)))
    return fail(st);
  cudaMemcpy(p->d_s2win, s2win.data(), s2win.size() * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_blocks, p->blocks.data(), p->blocks.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice);
  cudaMemset(p->d_status, 0, 4 * sizeof(int));

  // ---- sweep workspace for max_nrhs right-hand sides
  {
    const size_t R = (size_t)p->max_nrhs;
    if ((st = dalloc(*p, (char**)&p->d_u, N2 * R * es)) ||
        (st = dalloc(*p, (char**)&p->d_z, 2 * (size_t)n * R * Wmax * es)) ||
        (st = dalloc(*p, (char**)&p->d_rc, 2 * (size_t)p->P * R * Wmax * es)) ||
        (st = dalloc(*p, (char**)&p->d_lc, 2 * (size_t)p->P * R * Wmax * es)) ||
        (st = dalloc(*p, (char**)&p->d_xs, 2 * (size_t)p->P * R * Wmax * es)) ||
        (st = dalloc(*p, (char**)&p->d_ps, 2 * (size_t)p->P * R * Wmax * es)))
      return fail(st);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(HS_ECUDA);
  static std::atomic<long long> next_uid{1};
  p->uid = next_uid.fetch_add(1);
  *out = p;
  return HS_OK;
}

static void drop_plan(Plan* p) {
  release_sweep_graphs(*p);
  release_plan3(*p);
  free_plan_memory(p);
  delete p;
}

// Factor the prepared plans together and check their status words.
static int factor_plans(std::vector<Plan*>& ps, cudaStream_t s, bool async = false) {
  // the plan buffers were allocated stream-ordered on the legacy stream: the
  // setup kernels on `s` (and every later call) come after them
  if (cudaStreamSynchronize(0) != cudaSuccess) return HS_ECUDA;
  std::vector<Plan*> p2;
  for (Plan* p : ps) {
    if (p->dim == 3) {
      int st3 = setup3(*p, s);
      if (st3 != HS_OK) return st3;
    } else {
      p2.push_back(p);
    }
  }
  int st = launch_setup(p2, s, async);
  if (st != HS_OK) return st;
  if (async) {
    // later calls order themselves after this event; the status word is read
    // by the next synchronising call
    for (Plan* p : ps) {
      if (cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming) != cudaSuccess) return HS_ECUDA;
      if (cudaEventRecord(p->ready, s) != cudaSuccess) return HS_ECUDA;
    }
    return HS_OK;
  }
  for (Plan* p : ps) {
    int dst[3];
    if (cudaMemcpy(dst, p->d_status, sizeof(dst), cudaMemcpyDeviceToHost) != cudaSuccess) return HS_ECUDA;
    if (dst[0] != HS_OK) return dst[0];
  }
  return HS_OK;
}

extern "C" int hs_setup(const double* c, double omega, int n, int dim, int pml_width, int moving_pml_width,
                        const hs_options* opt, void* stream, hs_plan** out) {
  if (!out) return HS_EINVAL;
  *out = nullptr;
  Plan* p = nullptr;
  int st = prepare_plan(c, omega, n, dim, pml_width, moving_pml_width, opt, &p);
  if (st != HS_OK) return st;
  std::vector<Plan*> ps{p};
  st = factor_plans(ps, (cudaStream_t)stream, dim == 2 && p->opt.async_setup == 1);
  if (st != HS_OK) { drop_plan(p); return st; }
  *out = reinterpret_cast<hs_plan*>(p);
  return HS_OK;
}

namespace {
// Batched setup with options opt_of(k) for problem k (one factor precision).
template <typename OptOf>
int setup_batched(int nprob, const double* const* c, const double* omega, const int* n, int dim, int pml_width,
                  int moving_pml_width, OptOf opt_of, void* stream, hs_plan** out) {
  if (nprob < 1 || !c || !omega || !n || !out) return HS_EINVAL;
  for (int k = 0; k < nprob; ++k) out[k] = nullptr;
  hs_options d0;
  hs_default_options(&d0);
  const int prec0 = opt_of(0) ? opt_of(0)->factor_prec : d0.factor_prec;
  for (int k = 0; k < nprob; ++k) {
    const int pk = opt_of(k) ? opt_of(k)->factor_prec : d0.factor_prec;
    if ((pk != HS_C64 && pk != HS_C128) || pk != prec0) return HS_EINVAL;
  }
  std::vector<Plan*> ps;
  int st = HS_OK;
  for (int k = 0; k < nprob && st == HS_OK; ++k) {
    Plan* p = nullptr;
    st = prepare_plan(c[k], omega[k], n[k], dim, pml_width, moving_pml_width, opt_of(k), &p);
    if (st == HS_OK) ps.push_back(p);
  }
  if (st == HS_OK) st = factor_plans(ps, (cudaStream_t)stream);
  if (st != HS_OK) {
    for (Plan* p : ps) drop_plan(p);
    return st;
  }
  for (int k = 0; k < nprob; ++k) out[k] = reinterpret_cast<hs_plan*>(ps[k]);
  return HS_OK;
}
}  // namespace

extern "C" int hs_setup_batched(int nprob, const double* const* c, const double* omega, const int* n, int dim,
                                int pml_width, int moving_pml_width, const hs_options* opt, void* stream,
                                hs_plan** out) {
  return setup_batched(nprob, c, omega, n, dim, pml_width, moving_pml_width, [opt](int) { return opt; }, stream,
                       out);
}

extern "C" int hs_setup_batched_opts(int nprob, const double* const* c, const double* omega, const int* n, int dim,
                                     int pml_width, int moving_pml_width, const hs_options* opts, void* stream,
                                     hs_plan** out) {
  if (!opts) return HS_EINVAL;
  return setup_batched(nprob, c, omega, n, dim, pml_width, moving_pml_width,
                       [opts](int k) { return opts + k; }, stream, out);
}
