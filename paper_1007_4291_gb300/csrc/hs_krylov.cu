// Outer Krylov solver of Sec. 2.3: GMRES preconditioned by the sweep M_alpha.
// Implemented as right-preconditioned flexible GMRES(m): z_j = M_alpha v_j in
// the factor precision, w = A z_j, classical Gram-Schmidt (optionally with a
// second pass when the norm drops below 1/sqrt(2) of its value, DGKS),
// Givens rotations on the host, and the true residual ||f - A u|| at every
// restart.  All right-hand sides advance in lock step; a right-hand side that
// has converged at the start of a cycle is carried with a zero basis vector
// and receives no update.
//
// Two arithmetics for the Arnoldi vectors, the iterate and the residual:
//  * complex128 factors: native FP64 (the plain double-precision solver);
//  * complex64 factors: double-float (two floats per real, 48-bit
//    significand, see hs_df64.cuh) on the FP32 pipes, because GB300 runs
//    FP64 at 1/64 of its FP32 rate and these kernels would otherwise be
//    FP64-ALU-bound instead of memory-bound.
// The preconditioned vectors z_j are stored in the factor precision.
//
// Vectors inside the solver use the RHS-inner layout [point][rhs].
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <mutex>
#include <type_traits>
#include <vector>
#include "hs_internal.cuh"
#include "hs_df64.cuh"
#include "hs_cnn.cuh"

namespace hs {
namespace {

constexpr int KT = 256;  // threads per CTA: 8 warps x 32 RHS lanes

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

// ---------------------------------------------------------------- arithmetic
// Element operations of the two solver arithmetics.
struct F64 {
  using V = c128;    // Krylov vector element
  using A = c128;    // dot-product accumulator
  using N = double;  // norm accumulator
  static __device__ __forceinline__ A zero() { return c128{0, 0}; }
  static __device__ __forceinline__ void acc_conj(A& acc, V v, V w) { cfmaconj(acc, v, w); }
  static __device__ __forceinline__ void norm_zero(N& n) { n = 0.0; }
  static __device__ __forceinline__ void norm_acc(N& nrm, V w) { nrm = fma(w.re, w.re, fma(w.im, w.im, nrm)); }
  static __device__ __forceinline__ double norm_out(N n) { return n; }
  static __device__ __forceinline__ c128 to_c128(A a) { return a; }
  static __device__ __forceinline__ V coef(c128 h) { return h; }
  static __device__ __forceinline__ void sub_prod(V& w, V h, V v) { cfms(w, h, v); }
  template <typename ZT>
  static __device__ __forceinline__ void add_prod_z(V& x, V y, cplx<ZT> z) {
    cfma(x, y, c128{(double)z.re, (double)z.im});
  }
  static __device__ __forceinline__ c64 to_c64(V v) { return c64{(float)v.re, (float)v.im}; }
  static __device__ __forceinline__ V from_c128(c128 v) { return v; }
  static __device__ __forceinline__ c128 out_c128(V v) { return v; }
};

struct DF64 {
  using V = cdf;
  using A = cdf;
  using N = df;
  static __device__ __forceinline__ A zero() { return cdf{df{0.f, 0.f}, df{0.f, 0.f}}; }
  static __device__ __forceinline__ void acc_conj(A& acc, V v, V w) { cdf_fma_conj(acc, v, w); }
  static __device__ __forceinline__ void norm_zero(N& n) { n = df{0.f, 0.f}; }
  static __device__ __forceinline__ void norm_acc(N& nrm, V w) {
    df_fma(nrm, w.re, w.re);
    df_fma(nrm, w.im, w.im);
  }
  static __device__ __forceinline__ double norm_out(N n) { return df_to_double(n); }
  static __device__ __forceinline__ c128 to_c128(A a) { return cdf_to_c128(a); }
  static __device__ __forceinline__ V coef(c128 h) { return cdf_from_c128(h); }
  static __device__ __forceinline__ void sub_prod(V& w, V h, V v) { cdf_fms(w, h, v); }
  template <typename ZT>
  static __device__ __forceinline__ void add_prod_z(V& x, V y, cplx<ZT> z) {
    cdf_fma_c64(x, y, c64{(float)z.re, (float)z.im});
  }
  static __device__ __forceinline__ c64 to_c64(V v) { return c64{v.re.h, v.im.h}; }
  static __device__ __forceinline__ V from_c128(c128 v) { return cdf_from_c128(v); }
  static __device__ __forceinline__ c128 out_c128(V v) { return cdf_to_c128(v); }
};

// Single precision, for the basis of the refinement mode: FP32 products with
// per-thread FP32 partial sums, combined in FP64 across threads and CTAs.
struct F32 {
  using V = c64;
  using A = c64;
  using N = float;
  static __device__ __forceinline__ A zero() { return c64{0.f, 0.f}; }
  static __device__ __forceinline__ void acc_conj(A& acc, V v, V w) { cfmaconj(acc, v, w); }
  static __device__ __forceinline__ void norm_zero(N& n) { n = 0.f; }
  static __device__ __forceinline__ void norm_acc(N& nrm, V w) { nrm = fmaf(w.re, w.re, fmaf(w.im, w.im, nrm)); }
  static __device__ __forceinline__ double norm_out(N n) { return (double)n; }
  static __device__ __forceinline__ c128 to_c128(A a) { return c128{(double)a.re, (double)a.im}; }
  static __device__ __forceinline__ V coef(c128 h) { return c64{(float)h.re, (float)h.im}; }
  static __device__ __forceinline__ void sub_prod(V& w, V h, V v) { cfms(w, h, v); }
  template <typename ZT>
  static __device__ __forceinline__ void add_prod_z(V& x, V y, cplx<ZT> z) {
    cfma(x, y, c64{(float)z.re, (float)z.im});
  }
  static __device__ __forceinline__ c64 to_c64(V v) { return v; }
  static __device__ __forceinline__ V from_c128(c128 v) { return c64{(float)v.re, (float)v.im}; }
  static __device__ __forceinline__ c128 out_c128(V v) { return c128{(double)v.re, (double)v.im}; }
};

// ---------------------------------------------------------------- kernels
// part[cta][i][r] = sum over this CTA's points of conj(V_i) w ; slot nv holds |w|^2.
template <typename AR, int MAXJ>
__global__ void __launch_bounds__(KT) dots_kernel(const typename AR::V* __restrict__ V, long long vstride, int nv,
                                                  const typename AR::V* __restrict__ w, long long npts, int R,
                                                  c128* __restrict__ part) {
  __shared__ double sre[MAXJ + 1][32], sim[MAXJ + 1][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  for (int t = threadIdx.x; t < (MAXJ + 1) * 32; t += KT) {
    sre[t / 32][t % 32] = 0.0;
    sim[t / 32][t % 32] = 0.0;
  }
  __syncthreads();
  typename AR::A acc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) acc[i] = AR::zero();
  typename AR::N nrm;
  AR::norm_zero(nrm);
  if (r < R) {
    // two points per iteration with every load of both issued before the
    // products (up to 16 vectors; n = 2047, 64 RHS, 9 vectors: 3.0 ms against
    // 13.8 ms one point at a time, where the loads queue behind the products)
    const long long stride = (long long)gridDim.x * 8;
    long long pt = (long long)blockIdx.x * 8 + warp;
    for (; MAXJ <= 16 && pt + stride < npts; pt += 2 * stride) {
      const long long e0 = pt * R + r, e1 = (pt + stride) * R + r;
      const typename AR::V w0 = w[e0], w1 = w[e1];
      typename AR::V v0[MAXJ], v1[MAXJ];
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) { v0[i] = V[i * vstride + e0]; v1[i] = V[i * vstride + e1]; }
      AR::norm_acc(nrm, w0);
      AR::norm_acc(nrm, w1);
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) { AR::acc_conj(acc[i], v0[i], w0); AR::acc_conj(acc[i], v1[i], w1); }
    }
    for (; pt < npts; pt += stride) {
      const long long e = pt * R + r;
      const typename AR::V wv = w[e];
      AR::norm_acc(nrm, wv);
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) AR::acc_conj(acc[i], V[i * vstride + e], wv);
    }
  }
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) {
    if (i < nv) {
      const c128 a = AR::to_c128(acc[i]);
      atomicAdd(&sre[i][lane], a.re);
      atomicAdd(&sim[i][lane], a.im);
    }
  }
  atomicAdd(&sre[MAXJ][lane], AR::norm_out(nrm));
  __syncthreads();
  const long long cta = blockIdx.x;
  for (int t = threadIdx.x; t < (nv + 1) * 32; t += KT) {
    const int i = t / 32, l = t % 32, rr = blockIdx.y * 32 + l;
    if (rr >= R) continue;
    const int src = (i == nv) ? MAXJ : i;
    part[(cta * (MAXJ + 1) + i) * R + rr] = c128{sre[src][l], sim[src][l]};
  }
}

// out[i][r] = sum over CTAs of part[cta][i][r] (fixed order)
__global__ void reduce_parts_kernel(const c128* __restrict__ part, int nctas, int stride_i, int nv1, int R,
                                    c128* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv1 * R) return;
  const int i = t / R, r = t % R;
  c128 s{0, 0};
  for (int c = 0; c < nctas; ++c) s = cadd(s, part[((long long)c * stride_i + i) * R + r]);
  out[i * R + r] = s;
}

// w -= sum_i h[i][r] s[i][r] V_i (s = 1 when `iscale` is NULL: scaled
// coefficients let the basis vectors stay unnormalised); also copied to
// `wcopy` when given; part[cta][r] = partial |w_new|^2
template <typename AR, int MAXJ>
__global__ void __launch_bounds__(KT) update_kernel(const typename AR::V* __restrict__ V, long long vstride, int nv,
                                                    const c128* __restrict__ h, typename AR::V* __restrict__ w,
                                                    long long npts, int R, c128* __restrict__ part,
                                                    const double* __restrict__ iscale = nullptr,
                                                    typename AR::V* __restrict__ wcopy = nullptr) {
  __shared__ double snrm[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (threadIdx.x < 32) snrm[threadIdx.x] = 0.0;
  __syncthreads();
  typename AR::V hc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) {
    c128 hv = (i < nv && r < R) ? h[i * R + r] : c128{0, 0};
    if (iscale && i < nv && r < R) hv = cscale(hv, iscale[i * R + r]);
    hc[i] = AR::coef(hv);
  }
  typename AR::N nrm;
  AR::norm_zero(nrm);
  if (r < R) {
    // two points per iteration with every load of both issued before the
    // products (up to 16 vectors; n = 2047, 64 RHS, 5-8 vectors: 2.6-3.4 ms
    // against 3.2-4.4 ms one point at a time)
    const long long stride = (long long)gridDim.x * 8;
    long long pt = (long long)blockIdx.x * 8 + warp;
    for (; MAXJ <= 16 && pt + stride < npts; pt += 2 * stride) {
      const long long e0 = pt * R + r, e1 = (pt + stride) * R + r;
      typename AR::V w0 = w[e0], w1 = w[e1];
      typename AR::V v0[MAXJ], v1[MAXJ];
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) { v0[i] = V[i * vstride + e0]; v1[i] = V[i * vstride + e1]; }
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) { AR::sub_prod(w0, hc[i], v0[i]); AR::sub_prod(w1, hc[i], v1[i]); }
      w[e0] = w0;
      w[e1] = w1;
      if (wcopy) { wcopy[e0] = w0; wcopy[e1] = w1; }
      AR::norm_acc(nrm, w0);
      AR::norm_acc(nrm, w1);
    }
    for (; pt < npts; pt += stride) {
      const long long e = pt * R + r;
      typename AR::V wv = w[e];
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) AR::sub_prod(wv, hc[i], V[i * vstride + e]);
      w[e] = wv;
      if (wcopy) wcopy[e] = wv;
      AR::norm_acc(nrm, wv);
    }
  }
  atomicAdd(&snrm[lane], AR::norm_out(nrm));
  __syncthreads();
  const int rr = blockIdx.y * 32 + threadIdx.x;
  if (threadIdx.x < 32 && rr < R) part[(long long)blockIdx.x * R + rr] = c128{snrm[threadIdx.x], 0.0};
}

// v = w * s[r]
__global__ void scale_f64_kernel(const c128* __restrict__ w, const double* __restrict__ s, c128* __restrict__ v,
                                 long long total, int R) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double f = s[e % R];
    v[e] = c128{w[e].re * f, w[e].im * f};
  }
}
__global__ void scale_df_kernel(const cdf* __restrict__ w, const df* __restrict__ s, cdf* __restrict__ v,
                                long long total, int R) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    v[e] = cdf_scale(w[e], s[e % R]);
}
// The RHS index of a grid-stride element loop, advanced by the stride's
// residue instead of a 64-bit remainder per element.
struct RhsCursor {
  int r, step, R;
  __device__ RhsCursor(long long e0, long long stride, int R_) : r((int)(e0 % R_)), step((int)(stride % R_)), R(R_) {}
  __device__ void advance() {
    r += step;
    if (r >= R) r -= R;
  }
};
// v = w * s[r], also written to v2 when given (the next sweep's input)
__global__ void scale_f32_kernel(const c64* w, const float* __restrict__ s, c64* v, long long total, int R,
                                 c64* __restrict__ v2 = nullptr) {
  const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  RhsCursor rc(e0, stride, R);
  for (long long e = e0; e < total; e += stride, rc.advance()) {
    const float f = s[rc.r];
    const c64 a{w[e].re * f, w[e].im * f};
    v[e] = a;
    if (v2) v2[e] = a;
  }
}
// v = complex64 (r * s[r]) from a double-float vector (the scaled residual
// that starts a refinement cycle; FP32 rounding is all the cycle keeps)
__global__ void df_to_c64_scaled_kernel(const cdf* __restrict__ r, const float* __restrict__ s, c64* __restrict__ v,
                                        long long total, int R, c64* __restrict__ v2) {
  const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  RhsCursor rc(e0, stride, R);
  for (long long e = e0; e < total; e += stride, rc.advance()) {
    const float f = s[rc.r];
    const cdf a = r[e];
    const c64 b{(a.re.h + a.re.l) * f, (a.im.h + a.im.l) * f};
    v[e] = b;
    v2[e] = b;
  }
}
template <typename AR>
__global__ void to_c64_kernel(const typename AR::V* __restrict__ v, c64* __restrict__ z, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    z[e] = AR::to_c64(v[e]);
}

// x += sum_i y[i][r] Z_i
template <typename AR, int MAXJ, typename ZT>
__global__ void __launch_bounds__(KT) xupdate_kernel(const cplx<ZT>* __restrict__ Z, long long zstride, int k,
                                                     const c128* __restrict__ y, typename AR::V* __restrict__ x,
                                                     long long npts, int R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  typename AR::V yc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) yc[i] = AR::coef((i < k) ? y[i * R + r] : c128{0, 0});
  for (long long pt = (long long)blockIdx.x * 8 + warp; pt < npts; pt += (long long)gridDim.x * 8) {
    const long long e = pt * R + r;
    typename AR::V xv = x[e];
#pragma unroll
    for (int i = 0; i < MAXJ; ++i)
      if (i < k) AR::add_prod_z(xv, yc[i], Z[i * zstride + e]);
    x[e] = xv;
  }
}

// Refinement update x += d with the cycle's correction d = sum_i y_i Z_i
// formed in FP32 (it only has to be as accurate as the cycle that made it)
// and added to the double-float iterate exactly.
template <int MAXJ>
__global__ void __launch_bounds__(KT) xcorrect_kernel(const c64* __restrict__ Z, long long zstride, int k,
                                                      const c128* __restrict__ y, cdf* __restrict__ x,
                                                      long long npts, int R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  c64 yc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) {
    const c128 v = (i < k) ? y[i * R + r] : c128{0, 0};
    yc[i] = c64{(float)v.re, (float)v.im};
  }
  // two points per iteration with every load of both issued before the
  // products (up to 16 vectors), then single points
  const long long stride = (long long)gridDim.x * 8;
  long long pt = (long long)blockIdx.x * 8 + warp;
  for (; MAXJ <= 16 && pt + stride < npts; pt += 2 * stride) {
    const long long e0 = pt * R + r, e1 = (pt + stride) * R + r;
    c64 z0[MAXJ], z1[MAXJ];
#pragma unroll
    for (int i = 0; i < MAXJ; ++i)
      if (i < k) { z0[i] = Z[i * zstride + e0]; z1[i] = Z[i * zstride + e1]; }
    cdf x0 = x[e0], x1 = x[e1];
    c64 d0{0.f, 0.f}, d1{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < MAXJ; ++i)
      if (i < k) { cfma(d0, yc[i], z0[i]); cfma(d1, yc[i], z1[i]); }
    x0.re = df_add(x0.re, df{d0.re, 0.f});
    x0.im = df_add(x0.im, df{d0.im, 0.f});
    x1.re = df_add(x1.re, df{d1.re, 0.f});
    x1.im = df_add(x1.im, df{d1.im, 0.f});
    x[e0] = x0;
    x[e1] = x1;
  }
  for (; pt < npts; pt += stride) {
    const long long e = pt * R + r;
    c64 d{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < MAXJ; ++i)
      if (i < k) cfma(d, yc[i], Z[i * zstride + e]);
    cdf xv = x[e];
    xv.re = df_add(xv.re, df{d.re, 0.f});
    xv.im = df_add(xv.im, df{d.im, 0.f});
    x[e] = xv;
  }
}

// Layout conversion ABI [rhs][point] (complex128) <-> solver [point][rhs] (V).
// Each CTA moves 32 x 32 tiles (points x RHS) through shared memory, looping
// over point tiles; each thread fetches its four entries of the next tile
// before it writes out the current one, so loads stay in flight across the
// tile's barriers.
template <typename AR, bool TO_INTERNAL>
__global__ void relayout_v_kernel(const void* __restrict__ srcv, void* __restrict__ dstv, long long npts, int R) {
  using V = typename AR::V;
  __shared__ V tile[32][33];
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long step = (long long)gridDim.x * 32;
  V pre[4];
  auto fetch = [&](long long p0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int yy = ty + 8 * q;
      if (TO_INTERNAL) {
        const c128* src = reinterpret_cast<const c128*>(srcv);
        const long long pt = p0 + tx;
        const int r = r0 + yy;
        if (pt < npts && r < R) pre[q] = AR::from_c128(src[(long long)r * npts + pt]);
      } else {
        const V* src = reinterpret_cast<const V*>(srcv);
        const long long pt = p0 + yy;
        const int r = r0 + tx;
        if (pt < npts && r < R) pre[q] = src[pt * R + r];
      }
    }
  };
  long long p0 = (long long)blockIdx.x * 32;
  if (p0 < npts) fetch(p0);
  for (; p0 < npts; p0 += step) {
#pragma unroll
    for (int q = 0; q < 4; ++q) tile[ty + 8 * q][tx] = pre[q];
    __syncthreads();
    if (p0 + step < npts) fetch(p0 + step);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int yy = ty + 8 * q;
      if (TO_INTERNAL) {
        V* dst = reinterpret_cast<V*>(dstv);
        const long long pt = p0 + yy;
        const int r = r0 + tx;
        if (pt < npts && r < R) dst[pt * R + r] = tile[tx][yy];
      } else {
        c128* dst = reinterpret_cast<c128*>(dstv);
        const long long pt = p0 + tx;
        const int r = r0 + yy;
        if (pt < npts && r < R) dst[(long long)r * npts + pt] = AR::out_c128(tile[tx][yy]);
      }
    }
    __syncthreads();
  }
}

// Eq. helmd in double-float: y = A x (x complex float or double-float), or
// y = f - A x.  Interior points use the real form (sum of the four
// neighbours)(n+1)^2 + (omega^2/c^2 - 4(n+1)^2) x; PML points the complex
// coefficients built from the double-float stretch tables.
struct DfTabs {
  const cdf* inv_s1; const cdf* a1; const cdf* inv_s2; const cdf* a2;
  const df* m0; const unsigned char* pml1; const unsigned char* pml2;
  float ih2;   // (n+1)^2, exact in FP32 for n < 4095
};

template <bool XDF>
__device__ __forceinline__ cdf ld_x(const void* x, long long k) {
  if (XDF) return reinterpret_cast<const cdf*>(x)[k];
  const c64 v = reinterpret_cast<const c64*>(x)[k];
  return cdf{df{v.re, 0.f}, df{v.im, 0.f}};
}

// One warp per grid point and 32 consecutive RHS (coordinates and
// coefficients warp-uniform, neighbour rows contiguous).  Each warp takes two
// points per iteration and issues all loads of both before it computes, so
// that twice as many loads are in flight.
template <bool XDF, bool RESID>
__global__ void __launch_bounds__(256) matvec_df_kernel(const void* __restrict__ x, cdf* __restrict__ y,
                                                        const cdf* __restrict__ f, DfTabs t, int n, int R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  const int n2 = n * n;
  const cdf zero{df{0.f, 0.f}, df{0.f, 0.f}};
  const long long sx = R, sy = (long long)n * R;
  struct Pt {
    cdf xc, xe, xw, xn, xs, fv;
    df m0;
    int i, j;
    bool pml;
  };
  auto load = [&](int pt, Pt& q) {
    q.j = pt / n;
    q.i = pt - q.j * n;
    const long long e = (long long)pt * R + r;
    q.xc = ld_x<XDF>(x, e);
    q.xe = (q.i + 1 < n) ? ld_x<XDF>(x, e + sx) : zero;
    q.xw = (q.i > 0) ? ld_x<XDF>(x, e - sx) : zero;
    q.xn = (q.j + 1 < n) ? ld_x<XDF>(x, e + sy) : zero;
    q.xs = (q.j > 0) ? ld_x<XDF>(x, e - sy) : zero;
    q.fv = RESID ? f[e] : zero;
    q.m0 = t.m0[pt];
    q.pml = t.pml1[q.i + 1] || t.pml2[q.j + 1];
  };
  auto apply = [&](int pt, const Pt& q) {
    cdf acc;
    if (!q.pml) {
      const df dg = df_add(q.m0, df{-4.f * t.ih2, 0.f});
      const cdf s4 = cdf_add(cdf_add(q.xe, q.xw), cdf_add(q.xn, q.xs));
      acc.re = df_add(df_mul_f(s4.re, t.ih2), df_mul(dg, q.xc.re));
      acc.im = df_add(df_mul_f(s4.im, t.ih2), df_mul(dg, q.xc.im));
    } else {
      const int i = q.i, j = q.j;
      const cdf is1 = t.inv_s1[i + 1], is2 = t.inv_s2[j + 1];
      const cdf E = cdf_mul(t.a1[i + 1], is2), Wc = cdf_mul(t.a1[i], is2);
      const cdf N = cdf_mul(t.a2[j + 1], is1), S = cdf_mul(t.a2[j], is1);
      const cdf ss = cdf_mul(is1, is2);
      const cdf D = cdf_sub(cdf{df_mul(ss.re, q.m0), df_mul(ss.im, q.m0)}, cdf_add(cdf_add(E, Wc), cdf_add(N, S)));
      acc = cdf_mul(D, q.xc);
      acc = cdf_add(acc, cdf_mul(E, q.xe));
      acc = cdf_add(acc, cdf_mul(Wc, q.xw));
      acc = cdf_add(acc, cdf_mul(N, q.xn));
      acc = cdf_add(acc, cdf_mul(S, q.xs));
    }
    y[(long long)pt * R + r] = RESID ? cdf_sub(q.fv, acc) : acc;
  };
  const int stride = gridDim.x * 8;
  int pt = blockIdx.x * 8 + warp;
  for (; pt + stride < n2; pt += 2 * stride) {
    Pt a, b;
    load(pt, a);
    load(pt + stride, b);
    apply(pt, a);
    apply(pt + stride, b);
  }
  if (pt < n2) {
    Pt a;
    load(pt, a);
    apply(pt, a);
  }
}


// ---------------------------------------------------------------- workspace
// Process-wide Krylov workspace: one device allocation reused by every
// hs_solve (held under a mutex for the duration of a solve, so concurrent
// solves from several host threads serialise instead of racing).  It grows
// when a solve needs more and is returned by hs_release_workspace().
struct KrylovPool {
  std::mutex mu;
  char* base = nullptr;
  size_t bytes = 0;
};
KrylovPool& pool() {
  static KrylovPool kp;
  return kp;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct Work {
  void* C;      // network correction of the current direction (factor precision), or null
  void* Wc;     // A applied to it (solver precision), or null
  void* V;      // (m+1) Arnoldi vectors (c128 or cdf, 16 bytes per element)
  void* Z;      // m preconditioned vectors (factor precision)
  void* x;      // iterate
  void* f;      // right-hand side
  c128* part;   // CTA partial sums
  c128* h;      // small coefficient vectors (34 rows of R)
  void* s;      // per-RHS scale factors (double or double-float)
};

int carve_workspace(const Plan& p, int m, int R, Work& w, bool judge) {
  KrylovPool& kp = pool();
  const size_t ves = 16;
  const size_t zes = (p.prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  const size_t npts = (size_t)p.npts(), vs = npts * R;
  const size_t nct = (size_t)sm_count() * 2;
  const size_t b1 = al256((m + 1) * vs * ves), b2 = al256(m * vs * zes), b3 = al256(vs * ves);
  const size_t b4 = al256(nct * 33 * R * sizeof(c128)), b5 = al256(34 * R * sizeof(c128)), b6 = al256(R * 8);
  const size_t b7 = judge ? al256(vs * zes) + al256(vs * ves) + al256(R * (2 * sizeof(double) + sizeof(int))) : 0;
  const size_t need = b1 + b2 + 2 * b3 + b4 + b5 + b6 + b7;
  if (kp.bytes < need) {
    if (kp.base) cudaFree(kp.base);
    kp.base = nullptr;
    kp.bytes = 0;
    if (cudaMalloc(&kp.base, need) != cudaSuccess) {
      cudaGetLastError();
      kp.base = nullptr;
      return HS_ENOMEM;
    }
    kp.bytes = need;
  }
  char* q = kp.base;
  w.V = q; q += b1;
  w.Z = q; q += b2;
  w.x = q; q += b3;
  w.f = q; q += b3;
  w.part = (c128*)q; q += b4;
  w.h = (c128*)q; q += b5;
  w.s = q; q += b6;
  w.C = w.Wc = nullptr;
  if (judge) {
    w.C = q; q += al256(vs * zes);
    w.Wc = q;
  }
  return HS_OK;
}

using zc = std::complex<double>;

void givens(zc a, zc b, double& c, zc& s) {
  if (b == 0.0) { c = 1.0; s = 0.0; return; }
  if (a == 0.0) { c = 0.0; s = std::conj(b) / std::abs(b); return; }
  const double na = std::hypot(std::abs(a), std::abs(b));
  c = std::abs(a) / na;
  s = (a / std::abs(a)) * std::conj(b) / na;
}

// ---------------------------------------------------------------- post-correction judge
// acc[r] += |v - w|^2, acc[R + r] += |v - w - wc|^2 over the points of RHS r:
// the FP64 residual of the preconditioned direction without (w = A z) and
// with (w + wc = A (z + c)) the network's correction c.
template <typename AR>
__global__ void judge_kernel(const typename AR::V* __restrict__ v, const typename AR::V* __restrict__ w,
                             const typename AR::V* __restrict__ wc, long long total, int R, double* acc) {
  extern __shared__ double sacc[];
  for (int i = threadIdx.x; i < 2 * R; i += blockDim.x) sacc[i] = 0.0;
  __syncthreads();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % R);
    const c128 a = AR::out_c128(v[e]), b = AR::out_c128(w[e]), c = AR::out_c128(wc[e]);
    const double pr = a.re - b.re, pi = a.im - b.im;
    const double qr = pr - c.re, qi = pi - c.im;
    atomicAdd(&sacc[r], pr * pr + pi * pi);
    atomicAdd(&sacc[R + r], qr * qr + qi * qi);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * R; i += blockDim.x) atomicAdd(&acc[i], sacc[i]);
}

// For the RHS the judge kept (use[r] != 0): z += c and w += wc.
template <typename AR, typename ZT>
__global__ void keep_correction_kernel(cplx<ZT>* __restrict__ z, const cplx<ZT>* __restrict__ c,
                                       typename AR::V* __restrict__ w, const typename AR::V* __restrict__ wc,
                                       long long total, int R, const int* __restrict__ use) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    if (!use[e % R]) continue;
    z[e] = cadd(z[e], c[e]);
    const c128 a = AR::out_c128(w[e]), b = AR::out_c128(wc[e]);
    w[e] = AR::from_c128(c128{a.re + b.re, a.im + b.im});
  }
}

// ---------------------------------------------------------------- solver
template <typename AR>
struct Solver {
  using V = typename AR::V;
  Plan& p;
  int R;
  long long npts, vs;
  cudaStream_t s;
  Work w;
  int nctas;
  std::vector<float> scratch;   // host staging for double-float scale factors
  dim3 grid() const { return dim3(nctas, (R + 31) / 32); }

  // h[i][r] (i < nv) and |v|^2 (slot nv) into w.h
  void dots(const V* Vb, int nv, const V* v) {
    const dim3 g = grid();
    note_launch();
    // the smallest instantiation that holds nv vectors: the per-thread
    // accumulators and loads of the larger ones cost registers, and with
    // them resident warps (DF64 with room for 8 vectors: 165 registers, one
    // CTA per SM, 1.3 TB/s for a norm)
    if (nv <= 1) dots_kernel<AR, 1><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    else if (nv <= 4) dots_kernel<AR, 4><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    else if (nv <= 8) dots_kernel<AR, 8><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    else if (nv <= 12) dots_kernel<AR, 12><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    else if (nv <= 16) dots_kernel<AR, 16><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    else dots_kernel<AR, 32><<<g, KT, 0, s>>>(Vb, vs, nv, v, npts, R, w.part);
    const int mj = (nv <= 1) ? 1 : (nv <= 4) ? 4 : (nv <= 8) ? 8 : (nv <= 12) ? 12 : (nv <= 16) ? 16 : 32;
    note_launch();
    reduce_parts_kernel<<<((nv + 1) * R + 255) / 256, 256, 0, s>>>(w.part, nctas, mj + 1, nv + 1, R, w.h);
  }
  // v -= V h ; |v|^2 -> w.h row `slot`
  void update(const V* Vb, int nv, V* v, int slot, const double* iscale = nullptr, V* vcopy = nullptr) {
    const dim3 g = grid();
    note_launch();
    if (nv <= 4) update_kernel<AR, 4><<<g, KT, 0, s>>>(Vb, vs, nv, w.h, v, npts, R, w.part, iscale, vcopy);
    else if (nv <= 8) update_kernel<AR, 8><<<g, KT, 0, s>>>(Vb, vs, nv, w.h, v, npts, R, w.part, iscale, vcopy);
    else if (nv <= 12) update_kernel<AR, 12><<<g, KT, 0, s>>>(Vb, vs, nv, w.h, v, npts, R, w.part, iscale, vcopy);
    else if (nv <= 16) update_kernel<AR, 16><<<g, KT, 0, s>>>(Vb, vs, nv, w.h, v, npts, R, w.part, iscale, vcopy);
    else update_kernel<AR, 32><<<g, KT, 0, s>>>(Vb, vs, nv, w.h, v, npts, R, w.part, iscale, vcopy);
    note_launch();
    reduce_parts_kernel<<<(R + 255) / 256, 256, 0, s>>>(w.part, nctas, 1, 1, R, w.h + (long long)slot * R);
  }
  void norm2(const V* v, int slot) {
    note_launch();
    dots_kernel<AR, 1><<<grid(), KT, 0, s>>>(nullptr, vs, 0, v, npts, R, w.part);
    note_launch();
    reduce_parts_kernel<<<(R + 255) / 256, 256, 0, s>>>(w.part, nctas, 2, 1, R, w.h + (long long)slot * R);
  }
  // dst = src * f[r]; the host factors are copied synchronously (tiny)
  void scale(const V* src, const std::vector<double>& f, V* dst) {
    note_launch();
    if constexpr (std::is_same<AR, F32>::value) {
      scratch.resize(R);
      for (int r = 0; r < R; ++r) scratch[r] = (float)f[r];
      cudaMemcpyAsync(w.s, scratch.data(), R * sizeof(float), cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
      scale_f32_kernel<<<sm_count() * 8, 256, 0, s>>>(src, (const float*)w.s, dst, vs, R);
    } else if constexpr (std::is_same<AR, F64>::value) {
      cudaMemcpyAsync(w.s, f.data(), R * sizeof(double), cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
      scale_f64_kernel<<<sm_count() * 8, 256, 0, s>>>(src, (const double*)w.s, dst, vs, R);
    } else {
      scratch.resize(2 * R);
      for (int r = 0; r < R; ++r) {
        scratch[2 * r] = (float)f[r];
        scratch[2 * r + 1] = (float)(f[r] - (double)scratch[2 * r]);
      }
      cudaMemcpyAsync(w.s, scratch.data(), 2 * R * sizeof(float), cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
      scale_df_kernel<<<sm_count() * 8, 256, 0, s>>>(src, (const df*)w.s, dst, vs, R);
    }
  }
  template <typename ZT>
  void xupdate(const cplx<ZT>* Z, int k, V* x) {
    const dim3 g = grid();
    note_launch();
    if (k <= 8) xupdate_kernel<AR, 8, ZT><<<g, KT, 0, s>>>(Z, vs, k, w.h, x, npts, R);
    else if (k <= 16) xupdate_kernel<AR, 16, ZT><<<g, KT, 0, s>>>(Z, vs, k, w.h, x, npts, R);
    else xupdate_kernel<AR, 32, ZT><<<g, KT, 0, s>>>(Z, vs, k, w.h, x, npts, R);
  }
  // y = A x, or y = f - A x when f is given.  x is a solver vector
  // (solver_vec) or a preconditioned vector in the factor precision.
  void matvec(const void* x, bool solver_vec, V* y, const V* f) {
    if constexpr (std::is_same<AR, F64>::value) {
      matvec_internal_f64(p, x, !solver_vec && p.prec == HS_C64, y, f, R, s);
    } else {
      DfTabs t{(const cdf*)p.k_inv_s1, (const cdf*)p.k_a1, (const cdf*)p.k_inv_s2, (const cdf*)p.k_a2,
               (const df*)p.k_m0, p.d_pml1, p.d_pml2, (float)((double)(p.n + 1) * (p.n + 1))};
      const int gy = (R + 31) / 32;
      const dim3 g((unsigned)std::min<long long>(((long long)p.n * p.n + 7) / 8, std::max(1, sm_count() * 8 / gy)), gy);
      note_launch();
      if (solver_vec) {
        if (f) matvec_df_kernel<true, true><<<g, 256, 0, s>>>(x, y, f, t, p.n, R);
        else matvec_df_kernel<true, false><<<g, 256, 0, s>>>(x, y, f, t, p.n, R);
      } else {
        if (f) matvec_df_kernel<false, true><<<g, 256, 0, s>>>(x, y, f, t, p.n, R);
        else matvec_df_kernel<false, false><<<g, 256, 0, s>>>(x, y, f, t, p.n, R);
      }
    }
  }
  void to_c64(const V* v, c64* z) {
    note_launch();
    to_c64_kernel<AR><<<sm_count() * 8, 256, 0, s>>>(v, z, vs);
  }
  void relayout(const void* src, void* dst, bool to_internal) {
    const long long tiles = (npts + 31) / 32;
    dim3 gr((unsigned)std::min<long long>(tiles, (long long)sm_count() * 8), (R + 31) / 32);
    note_launch();
    if (to_internal) relayout_v_kernel<AR, true><<<gr, dim3(32, 8), 0, s>>>(src, dst, npts, R);
    else relayout_v_kernel<AR, false><<<gr, dim3(32, 8), 0, s>>>(src, dst, npts, R);
  }
};

template <typename AR>
int solve_t(Plan& p, const void* f, void* u, int nrhs, double tol, int maxit, hs_solve_info* info, cudaStream_t s) {
  using V = typename AR::V;
  const auto t0 = std::chrono::steady_clock::now();
  const int R = nrhs;
  const int m = std::min(std::max(p.opt.restart, 1), 32);
  std::lock_guard<std::mutex> guard(pool().mu);
  Solver<AR> K{p, R, p.npts(), p.npts() * R, s, Work{}, sm_count() * 2, {}};
  Cnn* net = p.dim == 2 ? static_cast<Cnn*>(p.cnn) : nullptr;
  int st = carve_workspace(p, m, R, K.w, net != nullptr);
  if (st != HS_OK) return st;
  const long long vs = K.vs;
  V* Vb = (V*)K.w.V;
  V* x = (V*)K.w.x;
  V* fi = (V*)K.w.f;
  c64* Z = (c64*)K.w.Z;                      // complex64 factors: preconditioned vectors in c64
  c128* Z2 = (c128*)K.w.Z;                   // complex128 factors
  K.relayout(f, fi, true);
  K.relayout(u, x, true);

  cudaEvent_t ev[4];
  for (auto& e : ev) cudaEventCreate(&e);
  double t_apply = 0, t_mv = 0, t_orth = 0;
  auto elapsed = [](cudaEvent_t a, cudaEvent_t b) { float ms = 0; cudaEventElapsedTime(&ms, a, b); return (double)ms; };

  std::vector<c128> hbuf(34 * R);
  auto fetch_h = [&](int rows) {
    cudaMemcpyAsync(hbuf.data(), K.w.h, (size_t)rows * R * sizeof(c128), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
  };
  K.norm2(fi, 0);
  fetch_h(1);
  std::vector<double> fn(R);
  for (int r = 0; r < R; ++r) fn[r] = std::sqrt(hbuf[r].re);

  std::vector<zc> H((size_t)R * (m + 1) * m), g((size_t)R * (m + 1)), sn((size_t)R * m);
  std::vector<double> cs((size_t)R * m), relres(R, 1.0), scl(R);
  std::vector<char> active(R);
  int it = 0, cycles = 0, applies = 0, cnn_applies = 0;
  void* const u_saved = p.d_u;
  const bool cnn_on = net != nullptr;
  const size_t zes = (p.prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  double* judge_acc = nullptr;
  int* judge_use = nullptr;
  if (cnn_on) {
    judge_acc = reinterpret_cast<double*>(static_cast<char*>(K.w.Wc) + al256(vs * 16));
    judge_use = reinterpret_cast<int*>(judge_acc + 2 * R);
  }
  std::vector<double> jacc(2 * R);
  std::vector<int> juse(R);
  while (true) {
    // true residual r = f - A x -> V_0
    K.matvec(x, true, Vb, fi);
    K.norm2(Vb, 0);
    fetch_h(1);
    bool all = true;
    for (int r = 0; r < R; ++r) {
      const double beta = std::sqrt(hbuf[r].re);
      relres[r] = (fn[r] > 0) ? beta / fn[r] : 0.0;
      active[r] = relres[r] > tol;
      all = all && !active[r];
      scl[r] = active[r] ? 1.0 / beta : 0.0;
      g[(size_t)r * (m + 1)] = active[r] ? beta : 0.0;
      for (int q = 1; q <= m; ++q) g[(size_t)r * (m + 1) + q] = 0.0;
    }
    if (all || it >= maxit) break;
    ++cycles;
    K.scale(Vb, scl, Vb);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      V* Vj = Vb + (long long)j * vs;
      V* W1 = Vb + (long long)(j + 1) * vs;
      // z_j = M_alpha v_j in the factor precision, computed in place in Z_j
      // (2D: z_j moves with j, direct launches).  3D vectors are small and
      // the slab sweep is many short launches: the sweep runs on the plan's
      // own vector as a replayed CUDA graph and z_j is copied out.
      cudaEventRecord(ev[0], s);
      const bool g3 = p.dim == 3 && p.opt.graphs != 0;
      void* zj = (p.prec == HS_C64) ? (void*)(Z + (long long)j * vs) : (void*)(Z2 + (long long)j * vs);
      void* work = g3 ? u_saved : zj;
      if (p.prec == HS_C64) K.to_c64(Vj, (c64*)work);
      else cudaMemcpyAsync(work, Vj, vs * sizeof(c128), cudaMemcpyDeviceToDevice, s);
      p.d_u = work;
      st = sweep_internal(p, R, s, g3);
      p.d_u = u_saved;
      if (st == HS_OK && g3) cudaMemcpyAsync(zj, work, vs * zes, cudaMemcpyDeviceToDevice, s);
      if (st == HS_OK && cnn_on) {      // correction c = s N(z_j / s) of the sweep output
        cudaMemsetAsync(K.w.C, 0, vs * zes, s);
        st = cnn_correct(*net, zj, K.w.C, p.prec, R, p.n, s);
      }
      if (st != HS_OK) break;
      ++applies;
      cudaEventRecord(ev[1], s);
      K.matvec(zj, false, W1, nullptr);     // w = A z_j
      if (cnn_on) {
        // the FP64 residual judges the correction, per RHS and direction:
        // keep z_j + c where |v_j - A (z_j + c)| < |v_j - A z_j|
        V* Wc = static_cast<V*>(K.w.Wc);
        K.matvec(K.w.C, false, Wc, nullptr);
        cudaMemsetAsync(judge_acc, 0, 2 * R * sizeof(double), s);
        static std::once_flag once;
        std::call_once(once, [] {
          cudaFuncSetAttribute(judge_kernel<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8);
        });
        note_launch();
        judge_kernel<AR><<<sm_count() * 4, 256, 2 * R * sizeof(double), s>>>(Vj, W1, Wc, vs, R, judge_acc);
        cudaMemcpyAsync(jacc.data(), judge_acc, 2 * R * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        int kept = 0;
        for (int r = 0; r < R; ++r) {
          juse[r] = (active[r] && jacc[R + r] < jacc[r]) ? 1 : 0;
          kept += juse[r];
        }
        if (kept) {
          cudaMemcpyAsync(judge_use, juse.data(), R * sizeof(int), cudaMemcpyHostToDevice, s);
          note_launch();
          if (p.prec == HS_C64)
            keep_correction_kernel<AR, float><<<sm_count() * 4, 256, 0, s>>>(
                static_cast<c64*>(zj), static_cast<const c64*>(K.w.C), W1, Wc, vs, R, judge_use);
          else
            keep_correction_kernel<AR, double><<<sm_count() * 4, 256, 0, s>>>(
                static_cast<c128*>(zj), static_cast<const c128*>(K.w.C), W1, Wc, vs, R, judge_use);
        }
        cnn_applies += kept;
      }
      cudaEventRecord(ev[2], s);
      // classical Gram-Schmidt with an optional DGKS second pass
      K.dots(Vb, j + 1, W1);          // h[0..j] = V^H w, h[j+1] = |w|^2
      cudaMemcpyAsync(K.w.h + 33 * R, K.w.h + (long long)(j + 1) * R, R * sizeof(c128), cudaMemcpyDeviceToDevice, s);
      K.update(Vb, j + 1, W1, 32);    // |w'|^2 -> h[32]
      fetch_h(34);
      std::vector<c128> h1(hbuf.begin(), hbuf.begin() + (size_t)(j + 1) * R);
      bool need2 = false;
      for (int r = 0; r < R; ++r)
        if (active[r] && hbuf[32 * R + r].re < 0.5 * hbuf[33 * R + r].re) need2 = true;
      std::vector<double> nw(R);
      for (int r = 0; r < R; ++r) nw[r] = std::sqrt(hbuf[32 * R + r].re);
      if (need2 && p.opt.reorth) {
        K.dots(Vb, j + 1, W1);
        K.update(Vb, j + 1, W1, 32);
        fetch_h(33);
        for (size_t q = 0; q < h1.size(); ++q) { h1[q].re += hbuf[q].re; h1[q].im += hbuf[q].im; }
        for (int r = 0; r < R; ++r) nw[r] = std::sqrt(hbuf[32 * R + r].re);
      }
      std::vector<double> inv(R);
      for (int r = 0; r < R; ++r) inv[r] = (active[r] && nw[r] > 0) ? 1.0 / nw[r] : 0.0;
      K.scale(W1, inv, W1);
      cudaEventRecord(ev[3], s);
      cudaEventSynchronize(ev[3]);
      t_apply += elapsed(ev[0], ev[1]);
      t_mv += elapsed(ev[1], ev[2]);
      t_orth += elapsed(ev[2], ev[3]);
      // Givens rotations per RHS
      bool conv_all = true;
      for (int r = 0; r < R; ++r) {
        zc* Hr = &H[(size_t)r * (m + 1) * m];
        zc* gr = &g[(size_t)r * (m + 1)];
        double* cr = &cs[(size_t)r * m];
        zc* sr = &sn[(size_t)r * m];
        for (int i = 0; i <= j; ++i) Hr[i * m + j] = active[r] ? zc(h1[i * R + r].re, h1[i * R + r].im) : 0.0;
        Hr[(j + 1) * m + j] = active[r] ? nw[r] : 0.0;
        for (int i = 0; i < j; ++i) {
          zc t = cr[i] * Hr[i * m + j] + sr[i] * Hr[(i + 1) * m + j];
          Hr[(i + 1) * m + j] = -std::conj(sr[i]) * Hr[i * m + j] + cr[i] * Hr[(i + 1) * m + j];
          Hr[i * m + j] = t;
        }
        givens(Hr[j * m + j], Hr[(j + 1) * m + j], cr[j], sr[j]);
        Hr[j * m + j] = cr[j] * Hr[j * m + j] + sr[j] * Hr[(j + 1) * m + j];
        Hr[(j + 1) * m + j] = 0.0;
        gr[j + 1] = -std::conj(sr[j]) * gr[j];
        gr[j] = cr[j] * gr[j];
        if (active[r] && std::abs(gr[j + 1]) > tol * fn[r]) conv_all = false;
      }
      ++it;
      k = j + 1;
      if (conv_all || it >= maxit) break;
    }
    if (st != HS_OK) break;
    // y = H^{-1} g per RHS (upper triangular k x k), x += Z y
    std::vector<c128> y((size_t)k * R);
    for (int r = 0; r < R; ++r) {
      zc* Hr = &H[(size_t)r * (m + 1) * m];
      zc* gr = &g[(size_t)r * (m + 1)];
      std::vector<zc> yr(k);
      for (int i = k - 1; i >= 0; --i) {
        zc acc = active[r] ? gr[i] : 0.0;
        for (int q = i + 1; q < k; ++q) acc -= Hr[i * m + q] * yr[q];
        yr[i] = (active[r] && Hr[i * m + i] != 0.0) ? acc / Hr[i * m + i] : 0.0;
      }
      for (int i = 0; i < k; ++i) y[(size_t)i * R + r] = c128{yr[i].real(), yr[i].imag()};
    }
    cudaMemcpyAsync(K.w.h, y.data(), y.size() * sizeof(c128), cudaMemcpyHostToDevice, s);
    if (p.prec == HS_C64) K.xupdate(Z, k, x);
    else K.xupdate(Z2, k, x);
    cudaStreamSynchronize(s);
  }
  p.d_u = u_saved;
  if (st == HS_OK) K.relayout(x, u, false);
  cudaError_t e = cudaStreamSynchronize(s);
  for (auto& q : ev) cudaEventDestroy(q);
  if (st == HS_OK && e != cudaSuccess) st = cuda_status(e);
  if (st == HS_OK) {
    int w3[3];
    cudaMemcpy(w3, p.d_status, sizeof(w3), cudaMemcpyDeviceToHost);
    if (w3[0] != HS_OK) st = w3[0];
  }
  double mx = 0;
  bool nan = false;
  for (int r = 0; r < R; ++r) { mx = std::max(mx, relres[r]); if (!std::isfinite(relres[r])) nan = true; }
  if (info) {
    info->iterations = it;
    info->restarts = cycles;
    info->applies = applies;
    info->max_relres = mx;
    info->t_apply_ms = t_apply;
    info->t_matvec_ms = t_mv;
    info->t_orth_ms = t_orth;
    info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->cnn_applies = cnn_applies;
  }
  if (st == HS_OK && (mx > tol || nan)) st = HS_ENOCONV;
  return st;
}

// Mixed-precision refinement (2D, complex64 factors): each cycle restarts
// from the true residual r = f - A x computed in double-float and runs
// FGMRES with an FP32 Arnoldi basis (complex64 vectors, FP32 products A z_j,
// FP32 Gram-Schmidt) until its Givens estimate has fallen by inner_tol (or
// reaches tol ||f||); the cycle's correction is formed in FP32 and added to
// the double-float iterate.
// FP64-class arithmetic is kept exactly where the iterate and the residual
// that decides convergence are formed.
int solve_refine(Plan& p, const void* f, void* u, int nrhs, double tol, int maxit, hs_solve_info* info,
                 cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int R = nrhs;
  const int m = std::min(std::max(p.opt.restart, 1), 32);
  const double inner = p.opt.inner_tol;
  std::lock_guard<std::mutex> guard(pool().mu);
  KrylovPool& kp = pool();
  const size_t npts = (size_t)p.npts(), vs = npts * R;
  const size_t nct = (size_t)sm_count() * 2;
  const size_t b1 = al256((m + 1) * vs * sizeof(c64)), b2 = al256(m * vs * sizeof(c64)), b3 = al256(vs * sizeof(cdf));
  const size_t b4 = al256(nct * 33 * R * sizeof(c128)), b5 = al256(34 * R * sizeof(c128)), b6 = al256(R * 16);
  const size_t b7 = al256((size_t)(m + 1) * R * sizeof(double));
  const size_t need = b1 + b2 + 3 * b3 + b4 + b5 + b6 + b7;
  if (kp.bytes < need) {
    if (kp.base) cudaFree(kp.base);
    kp.base = nullptr;
    kp.bytes = 0;
    if (cudaMalloc(&kp.base, need) != cudaSuccess) { cudaGetLastError(); return HS_ENOMEM; }
    kp.bytes = need;
  }
  Work w{};
  char* q = kp.base;
  w.V = q; q += b1;
  w.Z = q; q += b2;
  w.x = q; q += b3;
  w.f = q; q += b3;
  cdf* rb = (cdf*)q; q += b3;
  w.part = (c128*)q; q += b4;
  w.h = (c128*)q; q += b5;
  w.s = q; q += b6;
  double* d_inu2 = (double*)q;     // 1 / |V_i|^2 per basis vector and RHS
  Solver<DF64> K{p, R, (long long)npts, (long long)vs, s, w, sm_count() * 2, {}};
  Solver<F32> B{p, R, (long long)npts, (long long)vs, s, w, sm_count() * 2, {}};
  c64* Vb = (c64*)w.V;
  c64* Z = (c64*)w.Z;
  cdf* x = (cdf*)w.x;
  cdf* fi = (cdf*)w.f;
  K.relayout(f, fi, true);
  K.relayout(u, x, true);
  cudaEvent_t ev[4];
  for (auto& e : ev) cudaEventCreate(&e);
  double t_apply = 0, t_mv = 0, t_orth = 0;
  auto elapsed = [](cudaEvent_t a, cudaEvent_t b) { float ms = 0; cudaEventElapsedTime(&ms, a, b); return (double)ms; };
  std::vector<c128> hbuf(34 * R);
  auto fetch_h = [&](int rows) {
    cudaMemcpyAsync(hbuf.data(), w.h, (size_t)rows * R * sizeof(c128), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
  };
  K.norm2(fi, 0);
  fetch_h(1);
  std::vector<double> fn(R), beta0(R);
  for (int r = 0; r < R; ++r) fn[r] = std::sqrt(hbuf[r].re);
  std::vector<zc> H((size_t)R * (m + 1) * m), g((size_t)R * (m + 1)), sn((size_t)R * m);
  std::vector<double> cs((size_t)R * m), relres(R, 1.0), scl(R);
  std::vector<float> sclf(R);
  std::vector<char> active(R);
  // The basis vectors V_i are kept unnormalised: v_i = V_i / nu_i.  The
  // update divides its coefficients by nu_i^2 and writes the next sweep input
  // in the same pass, and the Hessenberg entries and the final combination
  // take the norms on the host, so no pass rescales the vectors.
  std::vector<double> nu((size_t)(m + 1) * R, 0.0), inu2((size_t)(m + 1) * R, 0.0);
  int it = 0, cycles = 0, applies = 0, st = HS_OK;
  void* const u_saved = p.d_u;
  while (true) {
    K.matvec(x, true, rb, fi);                 // r = f - A x (double-float)
    K.norm2(rb, 0);
    fetch_h(1);
    bool all = true;
    for (int r = 0; r < R; ++r) {
      const double beta = std::sqrt(hbuf[r].re);
      relres[r] = (fn[r] > 0) ? beta / fn[r] : 0.0;
      active[r] = relres[r] > tol;
      all = all && !active[r];
      scl[r] = active[r] ? 1.0 / beta : 0.0;
      beta0[r] = beta;
      g[(size_t)r * (m + 1)] = active[r] ? beta : 0.0;
      for (int k = 1; k <= m; ++k) g[(size_t)r * (m + 1) + k] = 0.0;
    }
    if (all || it >= maxit) break;
    ++cycles;
    for (int r = 0; r < R; ++r) sclf[r] = (float)scl[r];
    cudaMemcpyAsync(w.s, sclf.data(), R * sizeof(float), cudaMemcpyHostToDevice, s);
    note_launch();
    df_to_c64_scaled_kernel<<<sm_count() * 8, 256, 0, s>>>(rb, (const float*)w.s, Vb, vs, R, Z);   // v_0, z_0 input
    for (int r = 0; r < R; ++r) {          // V_0 = r / |r| (zero for converged RHS)
      nu[r] = active[r] ? 1.0 : 0.0;
      inu2[r] = nu[r];
    }
    cudaMemcpyAsync(d_inu2, inu2.data(), R * sizeof(double), cudaMemcpyHostToDevice, s);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      c64* W1 = Vb + (long long)(j + 1) * vs;
      c64* Zj = Z + (long long)j * vs;
      cudaEventRecord(ev[0], s);
      p.d_u = Zj;                                 // holds v_j: the sweep overwrites it with z_j
      st = sweep_internal(p, R, s);
      p.d_u = u_saved;
      if (st != HS_OK) break;
      ++applies;
      cudaEventRecord(ev[1], s);
      st = matvec_internal_f32(p, Zj, W1, R, s);   // A z_j in FP32 (the cycle's precision)
      if (st != HS_OK) break;
      cudaEventRecord(ev[2], s);
      // FP32 classical Gram-Schmidt on the unnormalised basis: d_i = V_i^H W,
      // W -= sum_i (d_i / nu_i^2) V_i, written also as the next sweep's input
      B.dots(Vb, j + 1, W1);
      B.update(Vb, j + 1, W1, 32, d_inu2, j + 1 < m ? Zj + vs : nullptr);
      fetch_h(33);
      // W = A M V_j = nu_j A z_j: the normalised entries are d_i / (nu_i nu_j),
      // and |W'| = nu_j |w'|, so nu_{j+1} = |W'| and h_{j+1,j} = nu_{j+1} / nu_j
      std::vector<c128> h1((size_t)(j + 1) * R);
      std::vector<double> nw(R);
      double* nu_j = &nu[(size_t)j * R];
      double* nu_n = &nu[(size_t)(j + 1) * R];
      for (int r = 0; r < R; ++r) {
        nu_n[r] = std::sqrt(hbuf[32 * R + r].re);
        inu2[(size_t)(j + 1) * R + r] = nu_n[r] > 0 ? 1.0 / (nu_n[r] * nu_n[r]) : 0.0;
        nw[r] = nu_j[r] > 0 ? nu_n[r] / nu_j[r] : 0.0;
        for (int i = 0; i <= j; ++i) {
          const double den = nu[(size_t)i * R + r] * nu_j[r];
          const c128 d = hbuf[(size_t)i * R + r];
          h1[(size_t)i * R + r] = den > 0 ? c128{d.re / den, d.im / den} : c128{0, 0};
        }
      }
      cudaMemcpyAsync(d_inu2 + (size_t)(j + 1) * R, &inu2[(size_t)(j + 1) * R], R * sizeof(double),
                      cudaMemcpyHostToDevice, s);
      cudaEventRecord(ev[3], s);
      cudaEventSynchronize(ev[3]);
      t_apply += elapsed(ev[0], ev[1]);
      t_mv += elapsed(ev[1], ev[2]);
      t_orth += elapsed(ev[2], ev[3]);
      bool conv_all = true;
      for (int r = 0; r < R; ++r) {
        zc* Hr = &H[(size_t)r * (m + 1) * m];
        zc* gr = &g[(size_t)r * (m + 1)];
        double* cr = &cs[(size_t)r * m];
        zc* sr = &sn[(size_t)r * m];
        for (int i = 0; i <= j; ++i) Hr[i * m + j] = active[r] ? zc(h1[i * R + r].re, h1[i * R + r].im) : 0.0;
        Hr[(j + 1) * m + j] = active[r] ? nw[r] : 0.0;
        for (int i = 0; i < j; ++i) {
          zc t = cr[i] * Hr[i * m + j] + sr[i] * Hr[(i + 1) * m + j];
          Hr[(i + 1) * m + j] = -std::conj(sr[i]) * Hr[i * m + j] + cr[i] * Hr[(i + 1) * m + j];
          Hr[i * m + j] = t;
        }
        givens(Hr[j * m + j], Hr[(j + 1) * m + j], cr[j], sr[j]);
        Hr[j * m + j] = cr[j] * Hr[j * m + j] + sr[j] * Hr[(j + 1) * m + j];
        Hr[(j + 1) * m + j] = 0.0;
        gr[j + 1] = -std::conj(sr[j]) * gr[j];
        gr[j] = cr[j] * gr[j];
        if (active[r] && std::abs(gr[j + 1]) > std::max(tol * fn[r], inner * beta0[r])) conv_all = false;
      }
      ++it;
      k = j + 1;
      if (conv_all || it >= maxit) break;
    }
    if (st != HS_OK) break;
    std::vector<c128> y((size_t)k * R);
    for (int r = 0; r < R; ++r) {
      zc* Hr = &H[(size_t)r * (m + 1) * m];
      zc* gr = &g[(size_t)r * (m + 1)];
      std::vector<zc> yr(k);
      for (int i = k - 1; i >= 0; --i) {
        zc acc = active[r] ? gr[i] : 0.0;
        for (int q2 = i + 1; q2 < k; ++q2) acc -= Hr[i * m + q2] * yr[q2];
        yr[i] = (active[r] && Hr[i * m + i] != 0.0) ? acc / Hr[i * m + i] : 0.0;
      }
      // x += sum_i y_i z_i, z_i = Z_i / nu_i
      for (int i = 0; i < k; ++i) {
        const double ni = nu[(size_t)i * R + r];
        const zc yi = ni > 0 ? yr[i] / ni : zc(0.0);
        y[(size_t)i * R + r] = c128{yi.real(), yi.imag()};
      }
    }
    cudaMemcpyAsync(w.h, y.data(), y.size() * sizeof(c128), cudaMemcpyHostToDevice, s);
    {
      const dim3 g = K.grid();
      note_launch();
      if (k <= 8) xcorrect_kernel<8><<<g, KT, 0, s>>>(Z, (long long)vs, k, w.h, x, (long long)npts, R);
      else if (k <= 12) xcorrect_kernel<12><<<g, KT, 0, s>>>(Z, (long long)vs, k, w.h, x, (long long)npts, R);
      else if (k <= 16) xcorrect_kernel<16><<<g, KT, 0, s>>>(Z, (long long)vs, k, w.h, x, (long long)npts, R);
      else xcorrect_kernel<32><<<g, KT, 0, s>>>(Z, (long long)vs, k, w.h, x, (long long)npts, R);
    }
    cudaStreamSynchronize(s);
  }
  p.d_u = u_saved;
  if (st == HS_OK) K.relayout(x, u, false);
  cudaError_t e = cudaStreamSynchronize(s);
  for (auto& q3 : ev) cudaEventDestroy(q3);
  if (st == HS_OK && e != cudaSuccess) st = cuda_status(e);
  if (st == HS_OK) {
    int w3[3];
    cudaMemcpy(w3, p.d_status, sizeof(w3), cudaMemcpyDeviceToHost);
    if (w3[0] != HS_OK) st = w3[0];
  }
  double mx = 0;
  bool nan = false;
  for (int r = 0; r < R; ++r) { mx = std::max(mx, relres[r]); if (!std::isfinite(relres[r])) nan = true; }
  if (info) {
    info->iterations = it;
    info->restarts = cycles;
    info->applies = applies;
    info->max_relres = mx;
    info->t_apply_ms = t_apply;
    info->t_matvec_ms = t_mv;
    info->t_orth_ms = t_orth;
    info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->cnn_applies = 0;
  }
  if (st == HS_OK && (mx > tol || nan)) st = HS_ENOCONV;
  return st;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" int hs_solve(hs_plan* plan, const void* f, void* u, int nrhs, double tol, int maxit,
                        hs_solve_info* info, void* stream) {
  if (!plan || !f || !u || !(tol > 0.0) || maxit < 1) return HS_EINVAL;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (nrhs < 1 || nrhs > p.max_nrhs) return HS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  plan_wait(p, s);
  // 3D plans keep the Krylov vectors in FP64 (the double-float kernels are 2D)
  if (p.prec == HS_C64 && p.dim == 2 && p.opt.krylov_basis == 1 && !p.cnn)
    return solve_refine(p, f, u, nrhs, tol, maxit, info, s);
  return (p.prec == HS_C64 && p.dim == 2) ? solve_t<DF64>(p, f, u, nrhs, tol, maxit, info, s)
                                          : solve_t<F64>(p, f, u, nrhs, tol, maxit, info, s);
}

extern "C" int hs_attach_cnn(hs_plan* plan, hs_cnn* net) {
  if (!plan) return HS_EINVAL;
  if (reinterpret_cast<Plan*>(plan)->dim != 2) return HS_EUNSUPPORTED;
  reinterpret_cast<Plan*>(plan)->cnn = net;
  return HS_OK;
}

extern "C" int hs_release_workspace(void) {
  KrylovPool& kp = pool();
  std::lock_guard<std::mutex> guard(kp.mu);
  if (kp.base) cudaFree(kp.base);
  kp.base = nullptr;
  kp.bytes = 0;
  trim_plan_pools();
  return HS_OK;
}
