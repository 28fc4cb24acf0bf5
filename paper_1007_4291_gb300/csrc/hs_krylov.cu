// Outer Krylov solver of Sec. 2.3: GMRES preconditioned by the sweep M_alpha.
// Implemented as right-preconditioned flexible GMRES(m): z_j = M_alpha v_j in
// the factor precision, w = A z_j in FP64, classical Gram-Schmidt in FP64 with
// a second pass when the norm drops below 1/sqrt(2) of its value (DGKS),
// Givens rotations on the host, and the FP64 true residual ||f - A u|| at
// every restart.  All right-hand sides advance in lock step; a right-hand
// side that has converged at the start of a cycle is carried with a zero
// basis vector and receives no update.
//
// Vectors inside the solver use the RHS-inner layout [point][rhs].
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>
#include "hs_internal.cuh"

namespace hs {
namespace {

constexpr int KT = 256;  // threads per CTA: 8 warps x 32 RHS lanes

// part[cta][i][r] = sum over this CTA's points of conj(V_i) w ; slot i = nv holds |w|^2.
template <int MAXJ>
__global__ void __launch_bounds__(KT) dots_kernel(const c128* __restrict__ V, long long vstride, int nv,
                                                  const c128* __restrict__ w, long long npts, int R,
                                                  c128* __restrict__ part) {
  __shared__ double sre[MAXJ + 1][32], sim[MAXJ + 1][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  for (int t = threadIdx.x; t < (MAXJ + 1) * 32; t += KT) {
    sre[t / 32][t % 32] = 0.0;
    sim[t / 32][t % 32] = 0.0;
  }
  __syncthreads();
  c128 acc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) acc[i] = c128{0, 0};
  double nrm = 0.0;
  if (r < R) {
    for (long long pt = (long long)blockIdx.x * 8 + warp; pt < npts; pt += (long long)gridDim.x * 8) {
      const long long e = pt * R + r;
      const c128 wv = w[e];
      nrm = fma(wv.re, wv.re, fma(wv.im, wv.im, nrm));
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) cfmaconj(acc[i], V[i * vstride + e], wv);
    }
  }
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) {
    if (i < nv) {
      atomicAdd(&sre[i][lane], acc[i].re);
      atomicAdd(&sim[i][lane], acc[i].im);
    }
  }
  atomicAdd(&sre[MAXJ][lane], nrm);
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

// w -= sum_i h[i][r] V_i ; part[cta][0][r] = partial |w_new|^2
template <int MAXJ>
__global__ void __launch_bounds__(KT) update_kernel(const c128* __restrict__ V, long long vstride, int nv,
                                                    const c128* __restrict__ h, c128* __restrict__ w,
                                                    long long npts, int R, c128* __restrict__ part) {
  __shared__ double snrm[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (threadIdx.x < 32) snrm[threadIdx.x] = 0.0;
  __syncthreads();
  c128 hc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) hc[i] = (i < nv && r < R) ? h[i * R + r] : c128{0, 0};
  double nrm = 0.0;
  if (r < R) {
    for (long long pt = (long long)blockIdx.x * 8 + warp; pt < npts; pt += (long long)gridDim.x * 8) {
      const long long e = pt * R + r;
      c128 wv = w[e];
#pragma unroll
      for (int i = 0; i < MAXJ; ++i)
        if (i < nv) cfms(wv, hc[i], V[i * vstride + e]);
      w[e] = wv;
      nrm = fma(wv.re, wv.re, fma(wv.im, wv.im, nrm));
    }
  }
  atomicAdd(&snrm[lane], nrm);
  __syncthreads();
  const int rr = blockIdx.y * 32 + threadIdx.x;
  if (threadIdx.x < 32 && rr < R) part[(long long)blockIdx.x * R + rr] = c128{snrm[threadIdx.x], 0.0};
}

// v = w * s[r]  (c128), or z = (c64) v
__global__ void scale_kernel(const c128* __restrict__ w, const double* __restrict__ s, c128* __restrict__ v,
                             long long total, int R) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const double f = s[e % R];
    v[e] = c128{w[e].re * f, w[e].im * f};
  }
}
__global__ void to_c64_kernel(const c128* __restrict__ v, c64* __restrict__ z, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    z[e] = c64{(float)v[e].re, (float)v[e].im};
}

// x += sum_i y[i][r] Z_i
template <int MAXJ, typename ZT>
__global__ void __launch_bounds__(KT) xupdate_kernel(const cplx<ZT>* __restrict__ Z, long long zstride, int k,
                                                     const c128* __restrict__ y, c128* __restrict__ x,
                                                     long long npts, int R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 32 + lane;
  if (r >= R) return;
  c128 yc[MAXJ];
#pragma unroll
  for (int i = 0; i < MAXJ; ++i) yc[i] = (i < k) ? y[i * R + r] : c128{0, 0};
  for (long long pt = (long long)blockIdx.x * 8 + warp; pt < npts; pt += (long long)gridDim.x * 8) {
    const long long e = pt * R + r;
    c128 xv = x[e];
#pragma unroll
    for (int i = 0; i < MAXJ; ++i)
      if (i < k) {
        const cplx<ZT> zv = Z[i * zstride + e];
        cfma(xv, yc[i], c128{(double)zv.re, (double)zv.im});
      }
    x[e] = xv;
  }
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

struct Kry {
  Plan& p;
  int R;
  long long npts, vstride;
  cudaStream_t s;
  int nctas;
  dim3 grid() const { return dim3(nctas, (R + 31) / 32); }

  // h[i][r] (i < nv) and |w|^2 (slot nv) into p.d_h
  void dots(const c128* V, int nv, const c128* w) {
    const dim3 g = grid();
    note_launch();
    if (nv <= 8) dots_kernel<8><<<g, KT, 0, s>>>(V, vstride, nv, w, npts, R, p.d_part);
    else if (nv <= 16) dots_kernel<16><<<g, KT, 0, s>>>(V, vstride, nv, w, npts, R, p.d_part);
    else dots_kernel<32><<<g, KT, 0, s>>>(V, vstride, nv, w, npts, R, p.d_part);
    const int mj = (nv <= 8) ? 8 : (nv <= 16) ? 16 : 32;
    const int tot = (nv + 1) * R;
    note_launch();
    reduce_parts_kernel<<<(tot + 255) / 256, 256, 0, s>>>(p.d_part, nctas, mj + 1, nv + 1, R, p.d_h);
  }
  // w -= V h ; |w|^2 -> p.d_h row `slot`
  void update(const c128* V, int nv, const c128* h, c128* w, int slot) {
    const dim3 g = grid();
    note_launch();
    if (nv <= 8) update_kernel<8><<<g, KT, 0, s>>>(V, vstride, nv, h, w, npts, R, p.d_part);
    else if (nv <= 16) update_kernel<16><<<g, KT, 0, s>>>(V, vstride, nv, h, w, npts, R, p.d_part);
    else update_kernel<32><<<g, KT, 0, s>>>(V, vstride, nv, h, w, npts, R, p.d_part);
    note_launch();
    reduce_parts_kernel<<<(R + 255) / 256, 256, 0, s>>>(p.d_part, nctas, 1, 1, R, p.d_h + (long long)slot * R);
  }
  void norm2(const c128* w, int slot) {
    note_launch();
    dots_kernel<8><<<grid(), KT, 0, s>>>(nullptr, vstride, 0, w, npts, R, p.d_part);
    note_launch();
    reduce_parts_kernel<<<(R + 255) / 256, 256, 0, s>>>(p.d_part, nctas, 9, 1, R, p.d_h + (long long)slot * R);
  }
  void scale(const c128* w, const std::vector<double>& f, c128* v) {
    cudaMemcpyAsync(p.d_nrm, f.data(), R * sizeof(double), cudaMemcpyHostToDevice, s);
    note_launch();
    scale_kernel<<<sm_count() * 8, 256, 0, s>>>(w, p.d_nrm, v, npts * R, R);
  }
  template <typename ZT>
  void xupdate(const cplx<ZT>* Z, int k, const c128* y, c128* x) {
    const dim3 g = grid();
    note_launch();
    if (k <= 8) xupdate_kernel<8, ZT><<<g, KT, 0, s>>>(Z, vstride, k, y, x, npts, R);
    else if (k <= 16) xupdate_kernel<16, ZT><<<g, KT, 0, s>>>(Z, vstride, k, y, x, npts, R);
    else xupdate_kernel<32, ZT><<<g, KT, 0, s>>>(Z, vstride, k, y, x, npts, R);
  }
};

using zc = std::complex<double>;

void givens(zc a, zc b, double& c, zc& s) {
  if (b == 0.0) { c = 1.0; s = 0.0; return; }
  if (a == 0.0) { c = 0.0; s = std::conj(b) / std::abs(b); return; }
  const double na = std::hypot(std::abs(a), std::abs(b));
  c = std::abs(a) / na;
  s = (a / std::abs(a)) * std::conj(b) / na;
}

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

int carve_workspace(Plan& p, int m, int R) {
  KrylovPool& kp = pool();
  const size_t zes = (p.prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  const size_t npts = (size_t)p.n * p.n, vs = npts * R;
  const size_t nct = (size_t)sm_count() * 2;
  const size_t b1 = al256((m + 1) * vs * sizeof(c128)), b2 = al256(m * vs * zes), b3 = al256(vs * sizeof(c128));
  const size_t b4 = al256(nct * 33 * R * sizeof(c128)), b5 = al256(34 * R * sizeof(c128)), b6 = al256(R * sizeof(double));
  const size_t need = b1 + b2 + 2 * b3 + b4 + b5 + b6;
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
  p.d_V = (c128*)q; q += b1;
  p.d_Zk = (c64*)q; q += b2;
  p.d_x = (c128*)q; q += b3;
  p.d_f = (c128*)q; q += b3;
  p.d_part = (c128*)q; q += b4;
  p.d_h = (c128*)q; q += b5;
  p.d_nrm = (double*)q;
  p.kry_m = m; p.kry_R = R;
  p.kry_bytes = (long long)need;
  return HS_OK;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" int hs_solve(hs_plan* plan, const void* f, void* u, int nrhs, double tol, int maxit,
                        hs_solve_info* info, void* stream) {
  if (!plan || !f || !u || !(tol > 0.0) || maxit < 1) return HS_EINVAL;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (nrhs < 1 || nrhs > p.max_nrhs) return HS_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const int R = nrhs;
  const int m = std::min(std::max(p.opt.restart, 1), 32);
  std::lock_guard<std::mutex> guard(pool().mu);
  int st = carve_workspace(p, m, R);
  if (st != HS_OK) return st;
  const long long npts = (long long)p.n * p.n, vs = npts * R;
  Kry K{p, R, npts, vs, s, sm_count() * 2};
  c128* V = p.d_V;
  c64* Z = p.d_Zk;                       // c64 basis (factor precision c64)
  c128* Z2 = reinterpret_cast<c128*>(p.d_Zk);  // c128 basis (factor precision c128)
  c128* x = p.d_x;
  c128* fi = p.d_f;
  if ((st = layout_to_internal(f, HS_C128, fi, HS_C128, (int)npts, R, s)) != HS_OK) return st;
  if ((st = layout_to_internal(u, HS_C128, x, HS_C128, (int)npts, R, s)) != HS_OK) return st;

  cudaEvent_t ev[6];
  for (auto& e : ev) cudaEventCreate(&e);
  double t_apply = 0, t_mv = 0, t_orth = 0;
  auto elapsed = [](cudaEvent_t a, cudaEvent_t b) { float ms = 0; cudaEventElapsedTime(&ms, a, b); return (double)ms; };

  std::vector<c128> hbuf(34 * R);
  auto fetch_h = [&](int rows) {
    cudaMemcpyAsync(hbuf.data(), p.d_h, (size_t)rows * R * sizeof(c128), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
  };
  // ||f|| per RHS
  K.norm2(fi, 0);
  fetch_h(1);
  std::vector<double> fn(R);
  for (int r = 0; r < R; ++r) fn[r] = std::sqrt(hbuf[r].re);

  std::vector<zc> H((size_t)R * (m + 1) * m), g((size_t)R * (m + 1)), sn((size_t)R * m);
  std::vector<double> cs((size_t)R * m), relres(R, 1.0), scl(R);
  std::vector<char> active(R);
  int it = 0, cycles = 0, applies = 0;
  bool done = false;
  void* const u_saved = p.d_u;
  while (!done) {
    // true residual r = f - A x -> V_0
    matvec_internal_f64(p, x, false, V, fi, R, s);
    K.norm2(V, 0);
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
    K.scale(V, scl, V);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      c128* Vj = V + (long long)j * vs;
      c128* W1 = V + (long long)(j + 1) * vs;
      c64* Zj = Z + (long long)j * vs;
      c128* Zj2 = Z2 + (long long)j * vs;
      // z_j = M_alpha v_j in the factor precision, computed in place in Z_j
      cudaEventRecord(ev[0], s);
      if (p.prec == HS_C64) {
        note_launch();
        to_c64_kernel<<<sm_count() * 8, 256, 0, s>>>(Vj, Zj, vs);
        p.d_u = Zj;
      } else {
        cudaMemcpyAsync(Zj2, Vj, vs * sizeof(c128), cudaMemcpyDeviceToDevice, s);
        p.d_u = Zj2;
      }
      st = sweep_internal(p, R, s);
      p.d_u = u_saved;
      if (st != HS_OK) break;
      ++applies;
      cudaEventRecord(ev[1], s);
      // w = A z_j (FP64)
      if (p.prec == HS_C64) matvec_internal_f64(p, Zj, true, W1, nullptr, R, s);
      else matvec_internal_f64(p, Zj2, false, W1, nullptr, R, s);
      cudaEventRecord(ev[2], s);
      // classical Gram-Schmidt, FP64, with a DGKS second pass
      K.dots(V, j + 1, W1);          // d_h[0..j] = V^H w, d_h[j+1] = |w|^2
      cudaMemcpyAsync(p.d_h + 33 * R, p.d_h + (long long)(j + 1) * R, R * sizeof(c128), cudaMemcpyDeviceToDevice, s);
      K.update(V, j + 1, p.d_h, W1, 32);   // |w'|^2 -> d_h[32]
      fetch_h(34);
      std::vector<c128> h1(hbuf.begin(), hbuf.begin() + (size_t)(j + 1) * R);
      bool need2 = false;
      for (int r = 0; r < R; ++r)
        if (active[r] && hbuf[32 * R + r].re < 0.5 * hbuf[33 * R + r].re) need2 = true;
      std::vector<double> nw(R);
      for (int r = 0; r < R; ++r) nw[r] = std::sqrt(hbuf[32 * R + r].re);
      if (need2 && p.opt.reorth) {
        K.dots(V, j + 1, W1);
        K.update(V, j + 1, p.d_h, W1, 32);
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
    cudaMemcpyAsync(p.d_h, y.data(), y.size() * sizeof(c128), cudaMemcpyHostToDevice, s);
    if (p.prec == HS_C64) K.xupdate(Z, k, p.d_h, x);
    else K.xupdate(Z2, k, p.d_h, x);
    cudaStreamSynchronize(s);
  }
  p.d_u = u_saved;
  if (st == HS_OK) st = layout_from_internal(x, HS_C128, u, HS_C128, (int)npts, R, s);
  cudaError_t e = cudaStreamSynchronize(s);
  for (auto& q : ev) cudaEventDestroy(q);
  if (st == HS_OK && e != cudaSuccess) st = cuda_status(e);
  int dst = HS_OK;
  if (st == HS_OK) {
    int w3[3];
    cudaMemcpy(w3, p.d_status, sizeof(w3), cudaMemcpyDeviceToHost);
    dst = w3[0];
    if (dst != HS_OK) st = dst;
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
  }
  if (st == HS_OK && (mx > tol || nan)) st = HS_ENOCONV;
  return st;
}

extern "C" int hs_release_workspace(void) {
  KrylovPool& kp = pool();
  std::lock_guard<std::mutex> guard(kp.mu);
  if (kp.base) cudaFree(kp.base);
  kp.base = nullptr;
  kp.bytes = 0;
  return HS_OK;
}
