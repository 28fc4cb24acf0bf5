// 5-point PML-stretched Helmholtz operator y = A x (Sec. 2.1, Eq. helmd):
//   (1/h^2)(s1/s2)_{i+-1/2,j} u_{i+-1,j} + (1/h^2)(s2/s1)_{i,j+-1/2} u_{i,j+-1}
//   + (omega^2 / ((s1 s2)_ij c_ij^2) - sum of the four) u_ij,
// zero Dirichlet values outside 1..n.  Coefficients come from 1D stretch
// tables and the per-point omega^2/c^2; points away from every PML take the
// real-coefficient form (x_e + x_w + x_n + x_s) / h^2 + (omega^2/c^2 - 4/h^2) x.
//
// One thread per (point, RHS) element; both vector layouts are supported:
// RHS-outer (the ABI layout, x1 fastest) and RHS-inner (the solver's layout).
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

template <typename Tx, typename Ty, typename Rc, bool INNER, bool RESID>
__global__ void __launch_bounds__(256) matvec_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                     const cplx<Ty>* __restrict__ f, Tabs<Rc> t, int n, int R) {
  using C = cplx<Rc>;
  const long long n2 = (long long)n * n;
  const long long total = n2 * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long pt; int r;
    if (INNER) { pt = e / R; r = (int)(e - pt * R); }
    else { r = (int)(e / n2); pt = e - (long long)r * n2; }
    const int j = (int)(pt / n), i = (int)(pt - (long long)j * n);  // 0-based
    const long long sx = INNER ? R : 1;             // stride of x1 neighbours
    const long long sy = INNER ? (long long)n * R : n;  // stride of x2 neighbours
    auto ld = [&](long long k) { const cplx<Tx> v = x[k]; return C{(Rc)v.re, (Rc)v.im}; };
    const C xc = ld(e);
    const C xe = (i + 1 < n) ? ld(e + sx) : C{0, 0};
    const C xw = (i > 0) ? ld(e - sx) : C{0, 0};
    const C xn = (j + 1 < n) ? ld(e + sy) : C{0, 0};
    const C xs = (j > 0) ? ld(e - sy) : C{0, 0};
    const Rc m0 = t.m0[pt];
    C acc;
    if (!t.pml1[i + 1] && !t.pml2[j + 1]) {
      const C sum = cadd(cadd(xe, xw), cadd(xn, xs));
      const Rc dg = m0 - Rc(4) * t.ih2;
      acc = C{fma(t.ih2, sum.re, dg * xc.re), fma(t.ih2, sum.im, dg * xc.im)};
    } else {
      const C is1 = t.inv_s1[i + 1], is2 = t.inv_s2[j + 1];
      const C E = cmul(t.a1[i + 1], is2), Wc = cmul(t.a1[i], is2);
      const C N = cmul(t.a2[j + 1], is1), S = cmul(t.a2[j], is1);
      const C D = csub(cscale(cmul(is1, is2), m0), cadd(cadd(E, Wc), cadd(N, S)));
      acc = cmul(D, xc);
      cfma(acc, E, xe);
      cfma(acc, Wc, xw);
      cfma(acc, N, xn);
      cfma(acc, S, xs);
    }
    if (RESID) {
      const cplx<Ty> fv = f[e];
      y[e] = cplx<Ty>{(Ty)(fv.re - acc.re), (Ty)(fv.im - acc.im)};
    } else {
      y[e] = cplx<Ty>{(Ty)acc.re, (Ty)acc.im};
    }
  }
}

// Solver layout, same arithmetic: one warp per grid point and 32 consecutive
// RHS, so the point's coordinates and coefficients are warp-uniform and
// every neighbour load is a contiguous 32-element row segment.
template <typename Rc>
__global__ void __launch_bounds__(256) matvec_inner_kernel(const cplx<Rc>* __restrict__ x, cplx<Rc>* __restrict__ y,
                                                           Tabs<Rc> t, int n, int R) {
  using C = cplx<Rc>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  const int n2 = n * n;
  const long long sx = R, sy = (long long)n * R;
  for (int pt = blockIdx.x * 8 + warp; pt < n2; pt += gridDim.x * 8) {
    const int j = pt / n, i = pt - j * n;
    const long long e = (long long)pt * R + r;
    const C xc = x[e];
    const C xe = (i + 1 < n) ? x[e + sx] : C{0, 0};
    const C xw = (i > 0) ? x[e - sx] : C{0, 0};
    const C xn = (j + 1 < n) ? x[e + sy] : C{0, 0};
    const C xs = (j > 0) ? x[e - sy] : C{0, 0};
    const Rc m0 = t.m0[pt];
    C acc;
    if (!t.pml1[i + 1] && !t.pml2[j + 1]) {
      const C sum = cadd(cadd(xe, xw), cadd(xn, xs));
      const Rc dg = m0 - Rc(4) * t.ih2;
      acc = C{fma(t.ih2, sum.re, dg * xc.re), fma(t.ih2, sum.im, dg * xc.im)};
    } else {
      const C is1 = t.inv_s1[i + 1], is2 = t.inv_s2[j + 1];
      const C E = cmul(t.a1[i + 1], is2), Wc = cmul(t.a1[i], is2);
      const C N = cmul(t.a2[j + 1], is1), S = cmul(t.a2[j], is1);
      const C D = csub(cscale(cmul(is1, is2), m0), cadd(cadd(E, Wc), cadd(N, S)));
      acc = cmul(D, xc);
      cfma(acc, E, xe);
      cfma(acc, Wc, xw);
      cfma(acc, N, xn);
      cfma(acc, S, xs);
    }
    y[e] = acc;
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

int grid_for(long long total) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  long long g = (total + 255) / 256;
  long long cap = (long long)sms * 8 * 4;  // 8 CTAs of 256 per SM, 4 waves in flight
  return (int)(g < cap ? g : cap);
}

}  // namespace

int matvec_abi(Plan& p, const void* x, void* y, int nrhs, int dtype, cudaStream_t s) {
  const long long total = (long long)p.n * p.n * nrhs;
  if (dtype == HS_C128) {
    note_launch();
    matvec_kernel<double, double, double, false, false><<<grid_for(total), 256, 0, s>>>(
        (const c128*)x, (c128*)y, nullptr, tabs<double>(p), p.n, nrhs);
  } else {
    note_launch();
    matvec_kernel<float, float, float, false, false><<<grid_for(total), 256, 0, s>>>(
        (const c64*)x, (c64*)y, nullptr, tabs<float>(p), p.n, nrhs);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

int matvec_internal_f32(Plan& p, const c64* x, c64* y, int R, cudaStream_t s) {
  if (p.dim != 2) return HS_EUNSUPPORTED;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int gy = (R + 31) / 32;
  const long long want = ((long long)p.n * p.n + 7) / 8;
  const long long cap = std::max(1LL, (long long)sms * 8 / gy);   // 8 CTAs of 256 per SM
  note_launch();
  matvec_inner_kernel<float><<<dim3((unsigned)std::min(want, cap), gy), 256, 0, s>>>(x, y, tabs<float>(p), p.n, R);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

int matvec_internal_f64(Plan& p, const void* x, bool x_is_c64, c128* y, const c128* f, int R, cudaStream_t s) {
  if (p.dim == 3) return matvec3_internal_f64(p, x, x_is_c64, y, f, R, s);
  const long long total = (long long)p.n * p.n * R;
  const int g = grid_for(total);
  note_launch();
  if (x_is_c64) {
    if (f) matvec_kernel<float, double, double, true, true><<<g, 256, 0, s>>>((const c64*)x, y, f, tabs<double>(p), p.n, R);
    else matvec_kernel<float, double, double, true, false><<<g, 256, 0, s>>>((const c64*)x, y, f, tabs<double>(p), p.n, R);
  } else {
    if (f) matvec_kernel<double, double, double, true, true><<<g, 256, 0, s>>>((const c128*)x, y, f, tabs<double>(p), p.n, R);
    else matvec_kernel<double, double, double, true, false><<<g, 256, 0, s>>>((const c128*)x, y, f, tabs<double>(p), p.n, R);
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
  if (p.dim == 3) return matvec3_abi(p, x, y, nrhs, dtype, (cudaStream_t)stream);
  return matvec_abi(p, x, y, nrhs, dtype, (cudaStream_t)stream);
}
