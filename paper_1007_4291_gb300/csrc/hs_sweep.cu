// Application of the sweeping preconditioner, u <- M_alpha u (Algorithm 4
// with the two-front pattern and d layers per step, Sec. 2.3), on the GPU.
//
// The sweep is a chain of stages.  A forward stage applies T~_B to the
// lower-front block and the upper-front block of the same step at once
// (v_B = T~_B u_B, written over u_B; the coupling -A_{m+1,m} v_m of
// Algorithm 4 is folded into the next stage's input), the middle stage
// applies T~ of the middle layer, and the backward stages compute
// u_B = v_B - T~_B (A_{B,next} u_next) in reverse order.
//
// T~_B g is the block-row restriction of H_B^{-1}(0,..,0,g) (Eq. helma).
// With the x1 partition of the setup (chunks, separators, spikes) it is:
//   phase 1, per chunk in parallel: y_j = g_j - C_{j-1} z_{j-1},
//            z_j = G_j y_j (stored), and the two separator contributions
//            C_r z_r and C_{l-1} sum_j W_j^t g_j;
//   phase 2, per RHS: block LU solve of the separator system;
//   phase 3, per chunk in parallel: x_j = z_j - G_j C_j x_{j+1} from the
//            right separator, plus the left-spike correction -W_j C_{l-1} x_sep
//            on the output rows.
// Threads: T lanes share one right-hand side and split the W window rows;
// full vectors are exchanged by warp shuffles.  Per-column factor payloads
// (G_j | W_j rows | c_j) are double-buffered into shared memory with 1D TMA
// bulk copies completed on mbarriers (bounded waits -> HS_ETIMEOUT).
#include <algorithm>
#include "hs_internal.cuh"
#include "hs_device.cuh"

namespace hs {
namespace {

constexpr int NT = 128;  // threads per CTA of the chunk kernels

struct SweepArgs {
  int n, L, P, R, mode, nfront;
  BlockDesc blk[2];
  const void* fac;
  const void* red;
  void* u;
  void* z;
  void* rc;
  void* lc;
  void* xs;
  void* ps;
  const void* a2;      // x2 half-point table s2((j+1/2)h)/h^2 in the sweep precision
  const void* inv_s1;  // 1/s1(ih)
  int* status;
  long long spin;
};

template <int W> struct TPR { static constexpr int value = (W >= 24) ? 8 : 4; };

template <typename R>
__device__ __forceinline__ cplx<R> ncoup(const SweepArgs& a, int row, int j) {
  // x2 coupling N_{i,row} of A between grid rows row and row+1 at column i = j+1
  const cplx<R>* a2 = reinterpret_cast<const cplx<R>*>(a.a2);
  const cplx<R>* is1 = reinterpret_cast<const cplx<R>*>(a.inv_s1);
  return cmul(a2[row], is1[j + 1]);
}

// Right-hand side of T~_B at window row p, column j, RHS r.
template <typename R>
__device__ __forceinline__ cplx<R> sweep_input(const SweepArgs& a, const BlockDesc& d, int p, int j, int r) {
  const cplx<R>* u = reinterpret_cast<const cplx<R>*>(a.u);
  const long long rs = (long long)a.n * a.R;
  if (a.mode == 0) {
    if (p < d.out_off || p >= d.out_off + d.d_out) return cplx<R>{0, 0};
    const int jg = d.wlo + p;
    cplx<R> v = u[(jg - 1) * rs + (long long)j * a.R + r];
    if (jg == d.lo && d.prev_lo_row)
      cfms(v, ncoup<R>(a, d.lo - 1, j), u[(d.prev_lo_row - 1) * rs + (long long)j * a.R + r]);
    if (jg == d.hi && d.prev_hi_row)
      cfms(v, ncoup<R>(a, d.hi, j), u[(d.prev_hi_row - 1) * rs + (long long)j * a.R + r]);
    return v;
  } else {
    if (p != d.coup_local) return cplx<R>{0, 0};
    const int jg = d.wlo + p;
    const int rowN = min(jg, d.next_row);
    return cmul(ncoup<R>(a, rowN, j), u[(d.next_row - 1) * rs + (long long)j * a.R + r]);
  }
}

// Gather the full W-vector from the T lanes of this RHS (each owns ROWS rows).
template <typename R, int W, int T>
__device__ __forceinline__ void allgather(const cplx<R> (&own)[W / T], cplx<R> (&full)[W]) {
  constexpr int ROWS = W / T;
#pragma unroll
  for (int s = 0; s < T; ++s) {
#pragma unroll
    for (int q = 0; q < ROWS; ++q) full[s * ROWS + q] = shfl_c(own[q], s, T);
  }
}

// After a wait has expired: give the copies still in flight (uses t and t+1
// of the two barriers) one more bounded wait before the CTA exits.
__device__ __forceinline__ void drain_inflight(uint64_t* bars, int t, int nuses, long long spin) {
  if (threadIdx.x == 0) {
    for (int u = t; u < t + 2 && u < nuses; ++u) (void)mbar_wait_bounded(&bars[u & 1], (u >> 1) & 1, spin);
  }
}

template <typename R, int W>
struct ChunkSmem {
  static constexpr size_t bytes(int d_out) {
    return 128 + 2 * (((size_t)payload_elems(W, d_out) * sizeof(cplx<R>) + 127) / 128 * 128);
  }
};

// ---------------------------------------------------------------- phase 1
template <typename R, int W, int T>
__global__ void __launch_bounds__(NT) phase1_kernel(SweepArgs a) {
  using C = cplx<R>;
  constexpr int ROWS = W / T, LD = W + 1;
  constexpr int RT = NT / T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  const int front = blockIdx.z, k = blockIdx.x;
  const BlockDesc& d = a.blk[front];
  const long long pe = payload_elems(W, d.d_out);
  const uint32_t pbytes = (uint32_t)(pe * sizeof(C));
  const size_t bstride = ((size_t)pbytes + 127) / 128 * 128;
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  C* buf1 = reinterpret_cast<C*>(smem_raw + 128 + bstride);
  const C* fac = reinterpret_cast<const C*>(a.fac) + d.fac_off;
  const int tid = threadIdx.x, sl = tid % T;
  const int r = blockIdx.y * RT + tid / T;
  const bool valid = r < a.R;
  const int rr = (r < a.R) ? r : (a.R - 1);
  const int l = k * a.L;
  const int rgt = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
  const int ncol = rgt - l + 1;
  const bool has_left = k > 0;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], pbytes);
    tma_bulk_g2s(buf0, fac + (long long)l * pe, pbytes, &bars[0]);
    if (ncol > 1) {
      mbar_arrive_expect_tx(&bars[1], pbytes);
      tma_bulk_g2s(buf1, fac + (long long)(l + 1) * pe, pbytes, &bars[1]);
    }
  }
  C y[W], acc[W], zown[ROWS], cprev[ROWS];
#pragma unroll
  for (int q = 0; q < W; ++q) acc[q] = C{0, 0};
#pragma unroll
  for (int q = 0; q < ROWS; ++q) { zown[q] = C{0, 0}; cprev[q] = C{0, 0}; }
  C* zst = reinterpret_cast<C*>(a.z) + ((long long)front * a.n * a.R) * W;

  for (int t = 0; t < ncol; ++t) {
    const int j = l + t;
    const int b = t & 1;
    const C* G = b ? buf1 : buf0;
    const C* V = G + W * LD;
    const C* cc = V + d.d_out * LD;
    const bool ok = mbar_wait_bounded(&bars[b], (t >> 1) & 1, a.spin);
    C g[ROWS], yown[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int p = sl * ROWS + q;
      g[q] = sweep_input<R>(a, d, p, j, rr);
      yown[q] = g[q];
      if (t > 0) cfms(yown[q], cprev[q], zown[q]);
    }
    allgather<R, W, T>(yown, y);
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int p = sl * ROWS + q;
      C s0{0, 0}, s1{0, 0};
#pragma unroll
      for (int qq = 0; qq < W; qq += 2) {
        cfma(s0, G[p * LD + qq], y[qq]);
        cfma(s1, G[p * LD + qq + 1], y[qq + 1]);
      }
      zown[q] = cadd(s0, s1);
      cprev[q] = cc[p];
    }
    if (valid) {
      C* zp = zst + ((long long)j * a.R + r) * W + sl * ROWS;
#pragma unroll
      for (int q = 0; q < ROWS; ++q) zp[q] = zown[q];
    }
    if (has_left) {
#pragma unroll
      for (int q = 0; q < ROWS; ++q) {
        const int p = sl * ROWS + q;
        if (p >= d.out_off && p < d.out_off + d.d_out) {
          const C* vr = V + (p - d.out_off) * LD;
#pragma unroll
          for (int qq = 0; qq < W; ++qq) cfma(acc[qq], vr[qq], g[q]);
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(a.status, HS_ETIMEOUT, front, j);
      drain_inflight(bars, t, ncol, a.spin);
      return;
    }
    if (tid == 0 && t + 2 < ncol) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[b], pbytes);
      tma_bulk_g2s(b ? buf1 : buf0, fac + (long long)(j + 2) * pe, pbytes, &bars[b]);
    }
  }
  // separator contributions
  const long long sep_base = ((long long)front * a.P + k) * a.R;
  if (k < a.P - 1 && valid) {
    C* rc = reinterpret_cast<C*>(a.rc) + (sep_base + r) * W + sl * ROWS;
#pragma unroll
    for (int q = 0; q < ROWS; ++q) rc[q] = cmul(cprev[q], zown[q]);
  }
  if (has_left) {
#pragma unroll
    for (int m = 1; m < T; m <<= 1) {
#pragma unroll
      for (int qq = 0; qq < W; ++qq) acc[qq] = cadd(acc[qq], shfl_xor_c(acc[qq], m, T));
    }
    if (valid) {
      const C* cl = fac + (long long)(l - 1) * pe + (long long)(W + d.d_out) * LD;  // c_{l-1}
      C* lc = reinterpret_cast<C*>(a.lc) + (sep_base + r) * W + sl * ROWS;
#pragma unroll
      for (int q = 0; q < ROWS; ++q) {
        C av{0, 0};
#pragma unroll
        for (int s = 0; s < T; ++s)
          if (s == sl) av = acc[s * ROWS + q];  // static register index
        lc[q] = cmul(cl[sl * ROWS + q], av);
      }
    }
  }
}

// ---------------------------------------------------------------- phase 2
// One warp per right-hand side, lane p = window row p (p < W).
template <typename R, int W>
__global__ void __launch_bounds__(NT) phase2_kernel(SweepArgs a) {
  using C = cplx<R>;
  constexpr int LD = W + 1;
  constexpr int WPC = NT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  const int front = blockIdx.z;
  const BlockDesc& d = a.blk[front];
  const long long re = red_elems(W);
  const uint32_t rbytes = (uint32_t)(re * sizeof(C));
  const size_t bstride = ((size_t)rbytes + 127) / 128 * 128;
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  C* buf1 = reinterpret_cast<C*>(smem_raw + 128 + bstride);
  const C* red = reinterpret_cast<const C*>(a.red) + d.red_off;
  const int tid = threadIdx.x, lane = tid & 31;
  const int r = blockIdx.y * WPC + tid / 32;
  const bool valid = r < a.R;
  const int rr = valid ? r : (a.R - 1);
  const int nsep = a.P - 1;
  const int pl = lane < W ? lane : 0;
  const C* rcb = reinterpret_cast<const C*>(a.rc);
  const C* lcb = reinterpret_cast<const C*>(a.lc);
  C* xsb = reinterpret_cast<C*>(a.xs);
  C* psb = reinterpret_cast<C*>(a.ps);
  const long long fb = (long long)front * a.P;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    // payload use t reads separator t (forward, t < nsep) or 2 nsep - 1 - t
    // (backward); 2 nsep >= 2 uses always exist.
    const int k1 = (1 < nsep) ? 1 : 2 * nsep - 2;
    mbar_arrive_expect_tx(&bars[0], rbytes);
    tma_bulk_g2s(buf0, red, rbytes, &bars[0]);
    mbar_arrive_expect_tx(&bars[1], rbytes);
    tma_bulk_g2s(buf1, red + (long long)k1 * re, rbytes, &bars[1]);
  }
  // Forward: psi_k = rho_k - F_k psi_{k-1};  zeta_k = Gamma_k psi_k (stored)
  C psi{0, 0};
  int t = 0;  // barrier use counter
  for (int k = 0; k < nsep; ++k, ++t) {
    const int b = t & 1;
    const C* Gm = b ? buf1 : buf0;
    const C* F = Gm + W * LD;
    const bool ok = mbar_wait_bounded(&bars[b], (t >> 1) & 1, a.spin);
    const int s = (k + 1) * a.L - 1;
    C rho = sweep_input<R>(a, d, pl, s, rr);
    rho = csub(rho, rcb[((fb + k) * a.R + rr) * W + pl]);
    rho = csub(rho, lcb[((fb + k + 1) * a.R + rr) * W + pl]);
    C np = rho;
    if (k > 0) {
#pragma unroll
      for (int q = 0; q < W; ++q) cfms(np, F[pl * LD + q], shfl_c(psi, q));
    }
    psi = np;
    C zeta{0, 0};
#pragma unroll
    for (int q = 0; q < W; ++q) cfma(zeta, Gm[pl * LD + q], shfl_c(psi, q));
    if (valid && lane < W) psb[((fb + k) * a.R + r) * W + lane] = zeta;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(a.status, HS_ETIMEOUT, front, -2);
      drain_inflight(bars, t, 2 * nsep, a.spin);
      return;
    }
    if (tid == 0) {
      // next payload: forward continues with k+2, then the backward pass
      // reads separators nsep-1 down to 0.
      const int nt = t + 2;
      int kk = -1;
      if (nt < nsep) kk = nt;
      else if (nt < 2 * nsep) kk = 2 * nsep - 1 - nt;
      if (kk >= 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[b], rbytes);
        tma_bulk_g2s(b ? buf1 : buf0, red + (long long)kk * re, rbytes, &bars[b]);
      }
    }
  }
  __syncwarp();
  // Backward: x_k = zeta_k - F_{k+1}^t x_{k+1}; the payload of separator k
  // holds F_k, so the product with F_{k+1} uses the previous payload, kept
  // in registers as this lane's column of F_{k+1}.
  C x{0, 0};
  C fcol[W];
  for (int k = nsep - 1; k >= 0; --k, ++t) {
    const int b = t & 1;
    const C* Gm = b ? buf1 : buf0;
    const C* F = Gm + W * LD;
    const bool ok = mbar_wait_bounded(&bars[b], (t >> 1) & 1, a.spin);
    C xn = psb[((fb + k) * a.R + rr) * W + pl];
    if (k < nsep - 1) {
#pragma unroll
      for (int q = 0; q < W; ++q) cfms(xn, fcol[q], shfl_c(x, q));
    }
    x = xn;
#pragma unroll
    for (int q = 0; q < W; ++q) fcol[q] = F[q * LD + pl];
    if (valid && lane < W) xsb[((fb + k) * a.R + r) * W + lane] = x;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(a.status, HS_ETIMEOUT, front, -3);
      drain_inflight(bars, t, 2 * nsep, a.spin);
      return;
    }
    if (tid == 0) {
      const int nt = t + 2;
      if (nt < 2 * nsep) {
        const int kk = 2 * nsep - 1 - nt;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[b], rbytes);
        tma_bulk_g2s(b ? buf1 : buf0, red + (long long)kk * re, rbytes, &bars[b]);
      }
    }
  }
}

// ---------------------------------------------------------------- phase 3
template <typename R, int W, int T>
__global__ void __launch_bounds__(NT) phase3_kernel(SweepArgs a) {
  using C = cplx<R>;
  constexpr int ROWS = W / T, LD = W + 1;
  constexpr int RT = NT / T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  const int front = blockIdx.z, k = blockIdx.x;
  const BlockDesc& d = a.blk[front];
  const long long pe = payload_elems(W, d.d_out);
  const uint32_t pbytes = (uint32_t)(pe * sizeof(C));
  const size_t bstride = ((size_t)pbytes + 127) / 128 * 128;
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  C* buf1 = reinterpret_cast<C*>(smem_raw + 128 + bstride);
  const C* fac = reinterpret_cast<const C*>(a.fac) + d.fac_off;
  const int tid = threadIdx.x, sl = tid % T;
  const int r = blockIdx.y * RT + tid / T;
  const bool valid = r < a.R;
  const int rr = valid ? r : (a.R - 1);
  const int l = k * a.L;
  const int rgt = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
  const int ncol = rgt - l + 1;
  const bool has_left = k > 0, has_right = k < a.P - 1;
  C* u = reinterpret_cast<C*>(a.u);
  const long long rs = (long long)a.n * a.R;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], pbytes);
    tma_bulk_g2s(buf0, fac + (long long)rgt * pe, pbytes, &bars[0]);
    if (ncol > 1) {
      mbar_arrive_expect_tx(&bars[1], pbytes);
      tma_bulk_g2s(buf1, fac + (long long)(rgt - 1) * pe, pbytes, &bars[1]);
    }
  }
  const long long fb = (long long)front * a.P;
  const C* xsb = reinterpret_cast<const C*>(a.xs);
  C xnext[W], beta[W];
#pragma unroll
  for (int q = 0; q < W; ++q) {
    xnext[q] = has_right ? xsb[((fb + k) * a.R + rr) * W + q] : C{0, 0};
    beta[q] = C{0, 0};
  }
  if (has_left) {
    const C* cl = fac + (long long)(l - 1) * pe + (long long)(W + d.d_out) * LD;
#pragma unroll
    for (int q = 0; q < W; ++q) beta[q] = cmul(cl[q], xsb[((fb + k - 1) * a.R + rr) * W + q]);
  }
  const C* zst = reinterpret_cast<const C*>(a.z) + ((long long)front * a.n * a.R) * W;
  for (int t = 0; t < ncol; ++t) {
    const int j = rgt - t;
    const int b = t & 1;
    const C* G = b ? buf1 : buf0;
    const C* V = G + W * LD;
    const C* cc = V + d.d_out * LD;
    const bool ok = mbar_wait_bounded(&bars[b], (t >> 1) & 1, a.spin);
    C tv[W];
#pragma unroll
    for (int q = 0; q < W; ++q) tv[q] = cmul(cc[q], xnext[q]);
    C xown[ROWS];
    const C* zp = zst + ((long long)j * a.R + rr) * W + sl * ROWS;
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int p = sl * ROWS + q;
      C s0 = zp[q], s1{0, 0};
#pragma unroll
      for (int qq = 0; qq < W; qq += 2) {
        cfms(s0, G[p * LD + qq], tv[qq]);
        cfms(s1, G[p * LD + qq + 1], tv[qq + 1]);
      }
      xown[q] = cadd(s0, s1);
      if (valid && p >= d.out_off && p < d.out_off + d.d_out) {
        C o = xown[q];
        if (has_left) {
          const C* vr = V + (p - d.out_off) * LD;
#pragma unroll
          for (int qq = 0; qq < W; ++qq) cfms(o, vr[qq], beta[qq]);
        }
        C* up = u + (long long)(d.wlo + p - 1) * rs + (long long)j * a.R + r;
        *up = (a.mode == 0) ? o : csub(*up, o);
      }
    }
    allgather<R, W, T>(xown, xnext);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(a.status, HS_ETIMEOUT, front, j);
      drain_inflight(bars, t, ncol, a.spin);
      return;
    }
    if (tid == 0 && t + 2 < ncol) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[b], pbytes);
      tma_bulk_g2s(b ? buf1 : buf0, fac + (long long)(j - 2) * pe, pbytes, &bars[b]);
    }
  }
  if (has_right && valid) {
    const int s = rgt + 1;
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int p = sl * ROWS + q;
      if (p >= d.out_off && p < d.out_off + d.d_out) {
        C o = xsb[((fb + k) * a.R + r) * W + p];
        C* up = u + (long long)(d.wlo + p - 1) * rs + (long long)s * a.R + r;
        *up = (a.mode == 0) ? o : csub(*up, o);
      }
    }
  }
}

template <typename R, int W>
int run_stage_w(const Plan& p, SweepArgs a, cudaStream_t s) {
  constexpr int T = TPR<W>::value;
  constexpr int RT = NT / T;
  int dmax = std::max(a.blk[0].d_out, a.nfront > 1 ? a.blk[1].d_out : 0);
  const size_t sm13 = ChunkSmem<R, W>::bytes(dmax);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(phase1_kernel<R, W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    cudaFuncSetAttribute(phase3_kernel<R, W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    cudaFuncSetAttribute(phase2_kernel<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr_set = true;
  }
  dim3 g13(a.P, (a.R + RT - 1) / RT, a.nfront);
  note_launch();
  phase1_kernel<R, W, T><<<g13, NT, sm13, s>>>(a);
  if (a.P > 1) {
    const size_t sm2 = 128 + 2 * (((size_t)red_elems(W) * sizeof(cplx<R>) + 127) / 128 * 128);
    dim3 g2(1, (a.R + NT / 32 - 1) / (NT / 32), a.nfront);
    note_launch();
    phase2_kernel<R, W><<<g2, NT, sm2, s>>>(a);
  }
  note_launch();
  phase3_kernel<R, W, T><<<g13, NT, sm13, s>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

template <typename R>
int run_stage(const Plan& p, SweepArgs a, cudaStream_t s) {
  switch (a.blk[0].W) {
    case 8: return run_stage_w<R, 8>(p, a, s);
    case 12: return run_stage_w<R, 12>(p, a, s);
    case 16: return run_stage_w<R, 16>(p, a, s);
    case 24: return run_stage_w<R, 24>(p, a, s);
    case 32: return run_stage_w<R, 32>(p, a, s);
    default: return HS_EUNSUPPORTED;
  }
}

template <typename R>
int sweep_t(Plan& p, int nrhs, cudaStream_t s) {
  SweepArgs a{};
  a.n = p.n; a.L = p.L; a.P = p.P; a.R = nrhs;
  a.fac = p.d_fac; a.red = p.d_red; a.u = p.d_u;
  a.z = p.d_z; a.rc = p.d_rc; a.lc = p.d_lc; a.xs = p.d_xs; a.ps = p.d_ps;
  if (sizeof(R) == 4) { a.a2 = p.f_a2; a.inv_s1 = p.f_inv_s1; }
  else { a.a2 = p.d_a2; a.inv_s1 = p.d_inv_s1; }
  a.status = p.d_status;
  a.spin = p.opt.spin_budget;
  int st = HS_OK;
  const int S = (int)p.stages.size();
  // forward sweep of both fronts (v_B = T~_B u_B)
  for (int k = 0; k < S && st == HS_OK; ++k) {
    a.mode = 0; a.nfront = 2;
    a.blk[0] = p.blocks[p.stages[k][0]];
    a.blk[1] = p.blocks[p.stages[k][1]];
    st = run_stage<R>(p, a, s);
  }
  // middle layer with moving PMLs on both sides
  if (st == HS_OK) {
    a.mode = 0; a.nfront = 1;
    a.blk[0] = p.blocks[p.middle];
    a.blk[1] = a.blk[0];
    st = run_stage<R>(p, a, s);
  }
  // backward sweep: u_B = v_B - T~_B (A_{B,next} u_next)
  for (int k = S - 1; k >= 0 && st == HS_OK; --k) {
    a.mode = 1; a.nfront = 2;
    a.blk[0] = p.blocks[p.stages[k][0]];
    a.blk[1] = p.blocks[p.stages[k][1]];
    st = run_stage<R>(p, a, s);
  }
  return st;
}

// Layout conversion: ABI [rhs][point] <-> internal [point][rhs], with a
// precision change.  32x32 tiles through shared memory.
template <typename Ti, typename To, bool TO_INTERNAL>
__global__ void relayout_kernel(const cplx<Ti>* __restrict__ src, cplx<To>* __restrict__ dst, long long npts, int R) {
  __shared__ cplx<To> tile[32][33];
  const long long p0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    if (TO_INTERNAL) {
      // read ABI: src[(r0+yy)*npts + p0+tx]
      long long pt = p0 + tx; int r = r0 + yy;
      if (pt < npts && r < R) tile[yy][tx] = ccast<To>(src[(long long)r * npts + pt]);
    } else {
      // read internal: src[(p0+yy)*R + r0+tx]
      long long pt = p0 + yy; int r = r0 + tx;
      if (pt < npts && r < R) tile[yy][tx] = ccast<To>(src[pt * R + r]);
    }
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    if (TO_INTERNAL) {
      long long pt = p0 + yy; int r = r0 + tx;
      if (pt < npts && r < R) dst[pt * R + r] = tile[tx][yy];
    } else {
      long long pt = p0 + tx; int r = r0 + yy;
      if (pt < npts && r < R) dst[(long long)r * npts + pt] = tile[tx][yy];
    }
  }
}

template <typename Ti, typename To, bool TI>
int relayout(const void* src, void* dst, long long npts, int R, cudaStream_t s) {
  dim3 grid((unsigned)((npts + 31) / 32), (R + 31) / 32);
  note_launch();
  relayout_kernel<Ti, To, TI><<<grid, dim3(32, 8), 0, s>>>(reinterpret_cast<const cplx<Ti>*>(src),
                                                           reinterpret_cast<cplx<To>*>(dst), npts, R);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

}  // namespace

int sweep_internal(Plan& p, int nrhs, cudaStream_t s) {
  return (p.prec == HS_C64) ? sweep_t<float>(p, nrhs, s) : sweep_t<double>(p, nrhs, s);
}

int layout_to_internal(const void* src, int dtype, void* dst, int prec, int n2, int R, cudaStream_t s) {
  if (dtype == HS_C64 && prec == HS_C64) return relayout<float, float, true>(src, dst, n2, R, s);
  if (dtype == HS_C64 && prec == HS_C128) return relayout<float, double, true>(src, dst, n2, R, s);
  if (dtype == HS_C128 && prec == HS_C64) return relayout<double, float, true>(src, dst, n2, R, s);
  return relayout<double, double, true>(src, dst, n2, R, s);
}

int layout_from_internal(const void* src, int prec, void* dst, int dtype, int n2, int R, cudaStream_t s) {
  if (dtype == HS_C64 && prec == HS_C64) return relayout<float, float, false>(src, dst, n2, R, s);
  if (dtype == HS_C64 && prec == HS_C128) return relayout<double, float, false>(src, dst, n2, R, s);
  if (dtype == HS_C128 && prec == HS_C64) return relayout<float, double, false>(src, dst, n2, R, s);
  return relayout<double, double, false>(src, dst, n2, R, s);
}

}  // namespace hs

using namespace hs;

extern "C" int hs_apply(hs_plan* plan, const void* r, void* z, int nrhs, int dtype, void* stream) {
  if (!plan || !r || !z) return HS_EINVAL;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (nrhs < 1 || nrhs > p.max_nrhs || (dtype != HS_C64 && dtype != HS_C128)) return HS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int n2 = p.n * p.n;
  int st = layout_to_internal(r, dtype, p.d_u, p.prec, n2, nrhs, s);
  if (st == HS_OK) st = sweep_internal(p, nrhs, s);
  if (st == HS_OK) st = layout_from_internal(p.d_u, p.prec, z, dtype, n2, nrhs, s);
  return st;
}
