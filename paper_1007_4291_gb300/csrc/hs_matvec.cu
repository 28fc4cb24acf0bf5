// 5-point PML-stretched Helmholtz operator y = A x (Sec. 2.1, Eq. helmd):
//   (1/h^2)(s1/s2)_{i+-1/2,j} u_{i+-1,j} + (1/h^2)(s2/s1)_{i,j+-1/2} u_{i,j+-1}
//   + (omega^2 / ((s1 s2)_ij c_ij^2) - sum of the four) u_ij,
// zero Dirichlet values outside 1..n.  Coefficients come from 1D stretch
// tables and the per-point omega^2/c^2; points away from every PML take the
// real-coefficient form (x_e + x_w + x_n + x_s) / h^2 + (omega^2/c^2 - 4/h^2) x.
//
// Both vector layouts are supported: RHS-outer (the ABI layout, x1 fastest;
// a CTA walks consecutive points of one RHS) and RHS-inner (the solver's
// layout; a warp holds 32 RHS of one point).
#include <algorithm>
#include "hs_internal.cuh"
#include "hs3d.cuh"

namespace hs {
namespace {

template <typename Rc> struct Tabs {
  const cplx<Rc>* inv_s1; const cplx<Rc>* a1; const cplx<Rc>* inv_s2; const cplx<Rc>* a2;
  const Rc* m0; const unsigned char* pml1; const unsigned char* pml2;
  Rc ih2;
};

// The operator at one point (i, j) (0-based) given its value and four
// neighbours (zero outside the grid).
template <typename Rc>
__device__ __forceinline__ cplx<Rc> apply_point(const Tabs<Rc>& t, int n, int i, int j, int pt, cplx<Rc> xc,
                                                cplx<Rc> xe, cplx<Rc> xw, cplx<Rc> xn, cplx<Rc> xs) {
  using C = cplx<Rc>;
  const Rc m0 = t.m0[pt];
  if (!t.pml1[i + 1] && !t.pml2[j + 1]) {
    const C sum = cadd(cadd(xe, xw), cadd(xn, xs));
    const Rc dg = m0 - Rc(4) * t.ih2;
    return C{fma(t.ih2, sum.re, dg * xc.re), fma(t.ih2, sum.im, dg * xc.im)};
  }
  const C is1 = t.inv_s1[i + 1], is2 = t.inv_s2[j + 1];
  const C E = cmul(t.a1[i + 1], is2), Wc = cmul(t.a1[i], is2);
  const C N = cmul(t.a2[j + 1], is1), S = cmul(t.a2[j], is1);
  const C D = csub(cscale(cmul(is1, is2), m0), cadd(cadd(E, Wc), cadd(N, S)));
  C acc = cmul(D, xc);
  cfma(acc, E, xe);
  cfma(acc, Wc, xw);
  cfma(acc, N, xn);
  cfma(acc, S, xs);
  return acc;
}

template <typename Tx, typename Rc>
__device__ __forceinline__ cplx<Rc> ldc(const cplx<Tx>* x, long long k) {
  const cplx<Tx> v = x[k];
  return cplx<Rc>{(Rc)v.re, (Rc)v.im};
}

template <typename Ty, typename Rc, bool RESID>
__device__ __forceinline__ void store_y(cplx<Ty>* y, const cplx<Ty>* f, long long e, cplx<Rc> acc) {
  if (RESID) {
    const cplx<Ty> fv = f[e];
    y[e] = cplx<Ty>{(Ty)(fv.re - acc.re), (Ty)(fv.im - acc.im)};
  } else {
    y[e] = cplx<Ty>{(Ty)acc.re, (Ty)acc.im};
  }
}

// The points are split into the PML-free square [lo, hi)^2, where the
// operator has the real form and needs only omega^2/c^2, and the PML band
// around it (a few percent of the points), which takes the complex
// coefficients.  The square's kernel keeps few registers, so every SM holds
// its full thread count and each thread keeps UNR points' loads in flight;
// the band's kernel runs after it on the same stream.
constexpr int UNR = 2;

struct Square {
  int lo, ni;   // first index and width of the PML-free range
};
// point q of the PML band (i, j outside the square on some axis), row by row
__device__ __forceinline__ void band_point(long long q, int n, Square sq, int& i, int& j) {
  const long long below = (long long)sq.lo * n;
  const int hi = sq.lo + sq.ni, side = n - sq.ni;
  if (q < below) { j = (int)(q / n); i = (int)(q - (long long)j * n); return; }
  q -= below;
  const long long mid = (long long)sq.ni * side;
  if (q < mid) {
    const int row = (int)(q / side), k = (int)(q - (long long)row * side);
    j = sq.lo + row;
    i = k < sq.lo ? k : hi + (k - sq.lo);
    return;
  }
  q -= mid;
  j = hi + (int)(q / n);
  i = (int)(q - (long long)(j - hi) * n);
}

// ABI layout (RHS outermost, x1 fastest): blockIdx.y walks the RHS, the
// threads of a CTA consecutive points of one RHS.
template <typename Tx, typename Ty, typename Rc, bool RESID>
__global__ void __launch_bounds__(256) square_outer_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                           const cplx<Ty>* __restrict__ f, const Rc* __restrict__ m0t,
                                                           Rc ih2, int n, int R, Square sq) {
  using C = cplx<Rc>;
  const int nq = sq.ni * sq.ni;
  const int step = gridDim.x * blockDim.x;
  const Rc four = Rc(4) * ih2;
  for (int r = blockIdx.y; r < R; r += gridDim.y) {
    const long long base = (long long)r * n * n;
    for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < nq; q0 += step * UNR) {
      C xc[UNR], s4[UNR];
      int pt[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int q = q0 + u * step;
        if (q < nq) {
          const int jj = q / sq.ni, j = sq.lo + jj, i = sq.lo + (q - jj * sq.ni);
          pt[u] = j * n + i;
          const long long e = base + pt[u];
          xc[u] = ldc<Tx, Rc>(x, e);
          const C xe = (i + 1 < n) ? ldc<Tx, Rc>(x, e + 1) : C{0, 0};
          const C xw = (i > 0) ? ldc<Tx, Rc>(x, e - 1) : C{0, 0};
          const C xn = (j + 1 < n) ? ldc<Tx, Rc>(x, e + n) : C{0, 0};
          const C xs = (j > 0) ? ldc<Tx, Rc>(x, e - n) : C{0, 0};
          s4[u] = cadd(cadd(xe, xw), cadd(xn, xs));
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        if (q0 + u * step < nq) {
          const Rc dg = m0t[pt[u]] - four;
          store_y<Ty, Rc, RESID>(y, f, base + pt[u],
                                 C{fma(ih2, s4[u].re, dg * xc[u].re), fma(ih2, s4[u].im, dg * xc[u].im)});
        }
      }
    }
  }
}

template <typename Tx, typename Ty, typename Rc, bool RESID>
__global__ void __launch_bounds__(256) band_outer_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                         const cplx<Ty>* __restrict__ f, Tabs<Rc> t, int n, int R,
                                                         Square sq) {
  using C = cplx<Rc>;
  const long long nb = (long long)n * n - (long long)sq.ni * sq.ni;
  for (int r = blockIdx.y; r < R; r += gridDim.y) {
    const long long base = (long long)r * n * n;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
      int i, j;
      band_point(q, n, sq, i, j);
      const int pt = j * n + i;
      const long long e = base + pt;
      const C xc = ldc<Tx, Rc>(x, e);
      const C xe = (i + 1 < n) ? ldc<Tx, Rc>(x, e + 1) : C{0, 0};
      const C xw = (i > 0) ? ldc<Tx, Rc>(x, e - 1) : C{0, 0};
      const C xn = (j + 1 < n) ? ldc<Tx, Rc>(x, e + n) : C{0, 0};
      const C xs = (j > 0) ? ldc<Tx, Rc>(x, e - n) : C{0, 0};
      store_y<Ty, Rc, RESID>(y, f, e, apply_point(t, n, i, j, pt, xc, xe, xw, xn, xs));
    }
  }
}

// Solver layout (RHS fastest): one warp per grid point and 32 consecutive
// RHS, so the point's coordinates and coefficients are warp-uniform and
// every neighbour load is a contiguous 32-element row segment.
template <typename Tx, typename Ty, typename Rc, bool RESID>
__global__ void __launch_bounds__(256) square_inner_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                           const cplx<Ty>* __restrict__ f, const Rc* __restrict__ m0t,
                                                           Rc ih2, int n, int R, Square sq) {
  using C = cplx<Rc>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  const int nq = sq.ni * sq.ni;
  const int step = gridDim.x * 8;
  const long long sx = R, sy = (long long)n * R;
  const Rc four = Rc(4) * ih2;
  for (int q0 = blockIdx.x * 8 + warp; q0 < nq; q0 += step * UNR) {
    C xc[UNR], s4[UNR];
    int pt[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int q = q0 + u * step;
      if (q < nq) {
        const int jj = q / sq.ni, j = sq.lo + jj, i = sq.lo + (q - jj * sq.ni);
        pt[u] = j * n + i;
        const long long e = (long long)pt[u] * R + r;
        xc[u] = ldc<Tx, Rc>(x, e);
        const C xe = (i + 1 < n) ? ldc<Tx, Rc>(x, e + sx) : C{0, 0};
        const C xw = (i > 0) ? ldc<Tx, Rc>(x, e - sx) : C{0, 0};
        const C xn = (j + 1 < n) ? ldc<Tx, Rc>(x, e + sy) : C{0, 0};
        const C xs = (j > 0) ? ldc<Tx, Rc>(x, e - sy) : C{0, 0};
        s4[u] = cadd(cadd(xe, xw), cadd(xn, xs));
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (q0 + u * step < nq) {
        const Rc dg = m0t[pt[u]] - four;
        store_y<Ty, Rc, RESID>(y, f, (long long)pt[u] * R + r,
                               C{fma(ih2, s4[u].re, dg * xc[u].re), fma(ih2, s4[u].im, dg * xc[u].im)});
      }
    }
  }
}

template <typename Tx, typename Ty, typename Rc, bool RESID>
__global__ void __launch_bounds__(256) band_inner_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                         const cplx<Ty>* __restrict__ f, Tabs<Rc> t, int n, int R,
                                                         Square sq) {
  using C = cplx<Rc>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  const long long nb = (long long)n * n - (long long)sq.ni * sq.ni;
  const long long sx = R, sy = (long long)n * R;
  for (long long q = (long long)blockIdx.x * 8 + warp; q < nb; q += (long long)gridDim.x * 8) {
    int i, j;
    band_point(q, n, sq, i, j);
    const int pt = j * n + i;
    const long long e = (long long)pt * R + r;
    const C xc = ldc<Tx, Rc>(x, e);
    const C xe = (i + 1 < n) ? ldc<Tx, Rc>(x, e + sx) : C{0, 0};
    const C xw = (i > 0) ? ldc<Tx, Rc>(x, e - sx) : C{0, 0};
    const C xn = (j + 1 < n) ? ldc<Tx, Rc>(x, e + sy) : C{0, 0};
    const C xs = (j > 0) ? ldc<Tx, Rc>(x, e - sy) : C{0, 0};
    store_y<Ty, Rc, RESID>(y, f, e, apply_point(t, n, i, j, pt, xc, xe, xw, xn, xs));
  }
}

template <typename Rc> Tabs<Rc> tabs(const Plan& p);
template <> Tabs<double> tabs<double>(const Plan& p) {
  return Tabs<double>{p.d_inv_s1, p.d_a1, p.d_inv_s2, p.d_a2, p.d_m0, p.d_pml1, p.d_pml2,
                      (double)(p.n + 1) * (p.n + 1)};
}
template <> Tabs<float> tabs<float>(const Plan& p) {
  return Tabs<float>{p.f_inv_s1, p.f_a1, p.f_inv_s2, p.f_a2, p.f_m0, p.d_pml1, p.d_pml2,
                     (float)((double)(p.n + 1) * (p.n + 1))};
}

int sm_total() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

// CTAs of 256 threads: 8 per SM over the whole grid (x: points, y: RHS)
dim3 outer_grid(long long points, int R) {
  const long long per_rhs = std::max(1LL, (points + 255) / 256);
  const int gy = std::min(R, 65535);
  const long long gx = std::max(1LL, std::min(per_rhs, ((long long)sm_total() * 8 + gy - 1) / gy));
  return dim3((unsigned)gx, (unsigned)gy);
}
dim3 inner_grid(long long points, int R) {
  const int gy = (R + 31) / 32;
  const long long want = std::max(1LL, (points + 7) / 8);
  const long long cap = std::max(1LL, (long long)sm_total() * 8 / gy);
  return dim3((unsigned)std::min(want, cap), (unsigned)gy);
}

// y = A x (or f - A x): the PML-free square, then the PML band
template <typename Tx, typename Ty, typename Rc, bool RESID, bool INNER>
void launch_matvec(const Plan& p, const cplx<Tx>* x, cplx<Ty>* y, const cplx<Ty>* f, int R, cudaStream_t s) {
  const Tabs<Rc> t = tabs<Rc>(p);
  const Square sq{p.int_lo, p.int_hi - p.int_lo};
  const long long nsq = (long long)sq.ni * sq.ni, nband = (long long)p.n * p.n - nsq;
  if (nsq > 0) {
    note_launch();
    if (INNER)
      square_inner_kernel<Tx, Ty, Rc, RESID><<<inner_grid(nsq, R), 256, 0, s>>>(x, y, f, t.m0, t.ih2, p.n, R, sq);
    else
      square_outer_kernel<Tx, Ty, Rc, RESID><<<outer_grid(nsq, R), 256, 0, s>>>(x, y, f, t.m0, t.ih2, p.n, R, sq);
  }
  if (nband > 0) {
    note_launch();
    if (INNER)
      band_inner_kernel<Tx, Ty, Rc, RESID><<<inner_grid(nband, R), 256, 0, s>>>(x, y, f, t, p.n, R, sq);
    else
      band_outer_kernel<Tx, Ty, Rc, RESID><<<outer_grid(nband, R), 256, 0, s>>>(x, y, f, t, p.n, R, sq);
  }
}

}  // namespace

int matvec_abi(Plan& p, const void* x, void* y, int nrhs, int dtype, cudaStream_t s) {
  if (dtype == HS_C128)
    launch_matvec<double, double, double, false, false>(p, (const c128*)x, (c128*)y, nullptr, nrhs, s);
  else
    launch_matvec<float, float, float, false, false>(p, (const c64*)x, (c64*)y, nullptr, nrhs, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

int matvec_internal_f32(Plan& p, const c64* x, c64* y, int R, cudaStream_t s) {
  if (p.dim != 2) return HS_EUNSUPPORTED;
  launch_matvec<float, float, float, false, true>(p, x, y, nullptr, R, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

int matvec_internal_f64(Plan& p, const void* x, bool x_is_c64, c128* y, const c128* f, int R, cudaStream_t s) {
  if (p.dim == 3) return matvec3_internal_f64(p, x, x_is_c64, y, f, R, s);
  if (x_is_c64) {
    if (f) launch_matvec<float, double, double, true, true>(p, (const c64*)x, y, f, R, s);
    else launch_matvec<float, double, double, false, true>(p, (const c64*)x, y, f, R, s);
  } else {
    if (f) launch_matvec<double, double, double, true, true>(p, (const c128*)x, y, f, R, s);
    else launch_matvec<double, double, double, false, true>(p, (const c128*)x, y, f, R, s);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

}  // namespace hs

using namespace hs;

extern "C" int hs_matvec(hs_plan* plan, const void* x, void* y, int nrhs, int dtype, void* stream) {
  if (!plan || !x || !y || x == y) return HS_EINVAL;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (nrhs < 1 || (dtype != HS_C64 && dtype != HS_C128)) return HS_EINVAL;
  plan_wait(p, (cudaStream_t)stream);
  if (p.dim == 3) return matvec3_abi(p, x, y, nrhs, dtype, (cudaStream_t)stream);
  return matvec_abi(p, x, y, nrhs, dtype, (cudaStream_t)stream);
}
