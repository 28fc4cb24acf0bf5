// Internal declarations of libhs: complex arithmetic, the plan, and the
// launchers shared between translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include <string>
#include <atomic>
#include <mutex>
#include "hs.h"

namespace hs {

// ---------------------------------------------------------------- complex
template <typename R> struct __align__(2 * sizeof(R)) cplx { R re, im; };
using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> cadd(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> csub(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __host__ __device__ __forceinline__ cplx<R> cscale(cplx<R> a, R s) { return {a.re * s, a.im * s}; }
template <typename R> __host__ __device__ __forceinline__ R cabs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename R> __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc -= a * b
template <typename R> __device__ __forceinline__ void cfms(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(-a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> __device__ __forceinline__ void cfmaconj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
template <typename R> __host__ __device__ __forceinline__ cplx<R> cinv(cplx<R> a) {
  R d = a.re * a.re + a.im * a.im;
  return {a.re / d, -a.im / d};
}
template <typename To, typename Ti> __host__ __device__ __forceinline__ cplx<To> ccast(cplx<Ti> a) {
  return {(To)a.re, (To)a.im};
}

// ---------------------------------------------------------------- blocks
// A subproblem block of the two-front partition (Sec. 2.3).  Rows are 1-based
// grid rows; window-local rows are 0..w-1 (global row = wlo + p).
enum BlockKind { BK_F = 0, BK_E = 1, BK_LOWER = 2, BK_UPPER = 3, BK_MIDDLE = 4 };

struct BlockDesc {
  int kind;
  int lo, hi;        // block rows (inputs/outputs of T~)
  int wlo, whi;      // window rows of H_B
  int w, W;          // window height and its padded height (W in {8,12,16,24,32})
  int out_off;       // window-local index of row lo
  int d_out;         // hi - lo + 1
  int prev_lo_row;   // forward sweep: grid row below whose value couples into row lo (0 = none)
  int prev_hi_row;   // forward sweep: grid row above whose value couples into row hi (0 = none)
  int next_row;      // backward sweep: grid row of the following block coupled to this block (0 = none)
  int coup_local;    // window-local row that couples to next_row
  long long fac_off; // offset (complex elements) of the per-column payloads
  long long red_off; // offset of the reduced (separator) system factors
  long long cor_off; // offset of the corner blocks used to build the reduced system
  int s2_off;        // offset (complex elements) of the window x2 tables (3*w values)
  int exact;         // 1: the window reaches the grid boundary on the eliminated side and keeps the
                     // operator's own x2 profile (T~_B is then the exact Schur inverse)
};

// ---------------------------------------------------------------- plan
struct Plan {
  int n = 0, dim = 2, bp = 0, b = 0, dL = 1;
  double omega = 0, alpha = 0, C = 0, Cm = 0, h = 0;   // C boundary PML, Cm moving PMLs
  int prec = HS_C64;  // factor precision
  int device = 0;     // CUDA device current at setup (owns every device buffer of the plan)
  cudaEvent_t ready = nullptr;   // asynchronous setup: recorded after the setup's last kernel
  int L = 32, P = 1;  // x1 chunk length and chunk count
  int max_nrhs = 64;
  hs_options opt{};
  std::vector<BlockDesc> blocks;            // host copy
  std::vector<std::vector<int>> stages;     // forward-sweep stages: block indices (lower, upper)
  int middle = -1;                          // index of the middle block
  // device tables (FP64 and FP32 copies)
  c128* d_inv_s1 = nullptr; c128* d_a1 = nullptr;  // 1/s1(ih) (i=0..n+1), s1((i+1/2)h)/h^2 (i=0..n)
  c128* d_inv_s2 = nullptr; c128* d_a2 = nullptr;
  c64* f_inv_s1 = nullptr; c64* f_a1 = nullptr; c64* f_inv_s2 = nullptr; c64* f_a2 = nullptr;
  unsigned char* d_pml1 = nullptr; unsigned char* d_pml2 = nullptr;  // 1 = PML affects column i / row j
  int int_lo = 0, int_hi = 0;   // 0-based index range of points no PML affects (same on both axes; empty if none)
  double* d_m0 = nullptr;   // omega^2 / c^2 per point
  float* f_m0 = nullptr;
  double* d_cinv2 = nullptr; // 1/c^2 per point
  // double-float copies for the Krylov solver of the complex64 path:
  // 1D tables as complex double-float, omega^2/c^2 per point as double-float
  void* k_inv_s1 = nullptr; void* k_a1 = nullptr; void* k_inv_s2 = nullptr; void* k_a2 = nullptr;
  void* k_m0 = nullptr;
  c128* d_s2win = nullptr;  // per-block window tables: 1/s2B(p), s2B(p+1/2)/h^2, s2B(p-1/2)/h^2
  BlockDesc* d_blocks = nullptr;
  void* d_fac = nullptr;    long long fac_elems = 0;   // factor payloads (c64 or c128 elements)
  void* d_red = nullptr;    long long red_elems = 0;
  void* d_cor = nullptr;    long long cor_elems = 0;
  // sweep workspace
  void* d_u = nullptr;      // working vector, internal layout [row][col][rhs]
  void* d_z = nullptr;      // z_j store for the backward chunk pass: [front][col][rhs][W]
  void* d_rc = nullptr;     // per chunk right contributions [front][chunk][rhs][W]
  void* d_lc = nullptr;     // per chunk left contributions
  void* d_xs = nullptr;     // separator solutions [front][sep][rhs][W]
  void* d_ps = nullptr;     // separator forward values psi
  int* d_status = nullptr;  // device status word(s): [0] code, [1] block, [2] column
  long long bytes = 0;
  long long uid = 0;        // process-unique id (keys of cached CUDA graphs)
  void* graphs = nullptr;   // cached executable graphs of this plan's sweep (hs_sweep.cu)
  void* cnn = nullptr;      // attached post-correction network (hs_cnn.cuh), not owned
  void* p3 = nullptr;       // 3D plan data (hs3d.cuh) when dim == 3
  long long npts() const { return dim == 3 ? (long long)n * n * n : (long long)n * n; }
};

// ---------------------------------------------------------------- helpers
int cuda_status(cudaError_t e);
// Number of kernels libhs has launched in this process (all streams).
extern std::atomic<long long> g_launches;
inline void note_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
#define HS_CUDA_TRY(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) return hs::cuda_status(_e); } while (0)

int padded_width(int w);   // 8, 12, 16, 24, 32 or -1
// block partition (rows in 2D, x3 layers in 3D) into p.blocks/stages/middle:
// two fronts (Sec. 2.3), or in 2D the single upward front of Sec. 2.1-2.2
// whose top block takes the place of the middle layer; buffer rows (Sec. 2.2)
// between each block and its moving PML
void build_blocks(Plan& p);

// Capture the launches body(stream) makes on `cap` into an executable graph.
// Kernels counted by note_launch during the capture did not run: they are
// taken back and returned in *kernels, to be counted at each replay.
template <typename F>
int capture_graph(cudaStream_t cap, F&& body, cudaGraphExec_t* exec, long long* kernels) {
  const long long before = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  const int st = body(cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);
  const long long k = g_launches.load() - before;
  g_launches.fetch_sub(k);
  if (st != HS_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != HS_OK ? st : cuda_status(e);
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e);
  *kernels = k;
  return HS_OK;
}

// launchers (defined in the .cu files)
// factor every block of every plan of `ps` (same factor precision): one
// launch over all chunks, one over all reduced systems; synchronises `s`
int launch_setup(const std::vector<Plan*>& ps, cudaStream_t s, bool async = false);
// Stream-ordered memory pool of the 2D plan buffers of device dev (created on
// first use, keeps freed memory), and the trim that returns that memory.
int plan_pool(int dev, cudaMemPool_t* out);
void trim_plan_pools();
// Order work on stream s after an asynchronous setup of plan p (no-op once
// the plan was set up synchronously).
inline void plan_wait(const Plan& p, cudaStream_t s) {
  if (p.ready) cudaStreamWaitEvent(s, p.ready, 0);
}
inline void plan_wait_host(const Plan& p) {
  if (p.ready) cudaEventSynchronize(p.ready);
}
// u <- M_alpha u on p.d_u.  graph: replay (or capture on first use) the
// stage chain as one CUDA graph keyed by nrhs and the scratch pointers.
int sweep_internal(Plan& p, int nrhs, cudaStream_t s, bool graph = false);
// direct launches of the stage chain (used inside captures)
int sweep_launch(Plan& p, int nrhs, cudaStream_t s);
// Sweep temporaries: the working vector (solver layout) and the chunk and
// separator buffers the stage kernels address.
struct SweepWork {
  void* u; void* z; void* rc; void* lc; void* xs; void* ps;
};
// direct launches of a 2D plan's stage chain on caller-provided temporaries
// (the plan itself is only read)
int sweep_launch_work(const Plan& p, const SweepWork& w, int nrhs, cudaStream_t s);
void release_sweep_graphs(Plan& p);
// chunk length stored by hs_autotune in `path` for this key (0 if none)
// chunk length (and separator grouping in *sep, 0 if not recorded) stored by
// hs_autotune for this key, or 0
int tuned_chunk(const char* path, int n, int bp, int b, int dL, int prec, int nrhs, int* sep);
// drop cached multi-plan graphs that contain plan `uid` (hs_batch.cu)
void forget_batch_graphs(long long uid);
// largest separator count per x1 partition the separator solve supports for
// window height W (shared-memory bound)
int max_separators(int W, int prec);
// set the shared-memory attributes of every sweep kernel (before a capture)
void sweep_prepare_attributes(int prec);
int layout_to_internal(const void* src, int dtype, void* dst, int prec, int n2, int R, cudaStream_t s);
int layout_from_internal(const void* src, int prec, void* dst, int dtype, int n2, int R, cudaStream_t s);
int matvec_abi(Plan& p, const void* x, void* y, int nrhs, int dtype, cudaStream_t s);
// internal-layout FP64 products: y = A x (x c64 or c128), or y = f - A x
int matvec_internal_f64(Plan& p, const void* x, bool x_is_c64, c128* y, const c128* f, int R, cudaStream_t s);
// y = A x in FP32 on solver-layout complex64 vectors (2D plans)
int matvec_internal_f32(Plan& p, const c64* x, c64* y, int R, cudaStream_t s);

}  // namespace hs
