// Setup of the sweeping factorisation (Algorithm 3, Sec. 2.3) on the GPU.
//
// Every subproblem H_B (Eq. helma on the block's window of w rows and all n
// columns) is, in the x2-first ordering of Sec. 2.2, block tridiagonal along
// x1 with w x w tridiagonal diagonal blocks D_j and diagonal couplings
// C_j = diag(c_j) between columns j and j+1.  Its banded LU is therefore the
// block LDL^t recursion S_j = D_j - C_{j-1} S_{j-1}^{-1} C_{j-1} over the
// columns.  To run the later solves in parallel along x1, the columns are
// split into chunks of L: the last column of every chunk but the last is a
// separator, the others form an interior.  Each interior is factored on its
// own (G_j = S_j^{-1}, left to right), together with its left spike
// W_j = (A_II^{-1})_{j,l} (a right-to-left factorisation gives
// W_l = (S^R_l)^{-1}, W_{j+1} = -(S^R_{j+1})^{-1} C_j W_j), and the
// separators form a block-tridiagonal reduced system whose block LU is
// computed by a second kernel.  This re-association along x1 is exact: the
// same T~_B in exact arithmetic, different rounding.
//
// Each diagonal block inverse uses Gauss-Jordan elimination with partial
// pivoting inside the block (the block recursion itself is pivot-free);
// a zero pivot sets HS_EBREAKDOWN in the plan's status word.
//
// One warp owns one (block, chunk) work item; lanes own matrix rows and all
// work matrices live in shared memory (row stride W+1 complex, conflict-free).
#include <algorithm>
#include "hs_internal.cuh"
#include "hs_device.cuh"

namespace hs {
namespace {

struct FactorArgs {
  int n, L, P, nitems, nblocks;
  const int* block_ids;
  const BlockDesc* blocks;
  const c128* inv_s1;
  const c128* a1;
  const double* cinv2;
  const c128* s2win;
  c128 wst2;  // (omega + i alpha)^2
  void* fac;
  void* red;
  void* cor;
  int* status;
};

// Entries of row p of D_j (column j, 0-based) of H_B: diagonal, coupling to
// row p+1 and to row p-1 (Eq. helmd with the window's x2 stretch).
__device__ __forceinline__ void d_entries(const FactorArgs& a, const BlockDesc& d, const c128* s2, int j, int p,
                                          c128& diag, c128& up, c128& dn) {
  const int i = j + 1;  // grid column
  const c128 inv2 = s2[p], upc = s2[d.w + p], dnc = s2[2 * d.w + p];
  const c128 is1 = a.inv_s1[i];
  const c128 E = cmul(a.a1[i], inv2), Wc = cmul(a.a1[i - 1], inv2);
  up = cmul(upc, is1);
  dn = cmul(dnc, is1);
  const int jg = d.wlo + p;
  const double ci2 = a.cinv2[(size_t)(jg - 1) * a.n + (i - 1)];
  c128 m = cmul(cmul(cscale(a.wst2, ci2), is1), inv2);
  diag = csub(m, cadd(cadd(E, Wc), cadd(up, dn)));
}

// coupling between columns j and j+1 on window row p (zero on padded rows)
template <typename R>
__device__ __forceinline__ cplx<R> coupling(const FactorArgs& a, const BlockDesc& d, const c128* s2, int j, int p) {
  if (p >= d.w || j + 1 > a.n) return cplx<R>{0, 0};
  return ccast<R>(cmul(a.a1[j + 1], s2[p]));
}

// A (W x LD) <- D_j, lane p writes row p.
template <typename R, int W>
__device__ __forceinline__ void build_d(const FactorArgs& a, const BlockDesc& d, const c128* s2, int j,
                                        cplx<R>* A, int lane) {
  constexpr int LD = W + 1;
  if (lane < W) {
    cplx<R>* row = A + lane * LD;
#pragma unroll
    for (int q = 0; q < W; ++q) row[q] = cplx<R>{0, 0};
    if (lane < d.w) {
      c128 dg, up, dn;
      d_entries(a, d, s2, j, lane, dg, up, dn);
      row[lane] = ccast<R>(dg);
      if (lane + 1 < d.w) row[lane + 1] = ccast<R>(up);
      if (lane >= 1) row[lane - 1] = ccast<R>(dn);
    } else {
      row[lane] = cplx<R>{1, 0};
    }
  }
  __syncwarp();
}

// A -= diag(cv) G diag(cv)
template <typename R, int W>
__device__ __forceinline__ void sub_cgc(cplx<R>* A, const cplx<R>* G, const cplx<R>* cv, int lane) {
  constexpr int LD = W + 1;
  if (lane < W) {
    const cplx<R> cp = cv[lane];
#pragma unroll 4
    for (int q = 0; q < W; ++q) {
      cplx<R> t = cmul(cmul(cp, G[lane * LD + q]), cv[q]);
      A[lane * LD + q] = csub(A[lane * LD + q], t);
    }
  }
  __syncwarp();
}

// In-place Gauss-Jordan inversion with partial (row) pivoting of the W x W
// matrix A; column interchanges undo the row swaps at the end.  Returns
// false (uniformly) on a zero or non-finite pivot.
template <typename R, int W>
__device__ bool invert_inplace(cplx<R>* A, int* piv, int lane) {
  constexpr int LD = W + 1;
  bool ok = true;
  for (int k = 0; k < W; ++k) {
    R v = (lane < W && lane >= k) ? cabs2(A[lane * LD + k]) : R(-1);
    int idx = lane;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      R ov = Shfl<R>::xr(v, m);
      int oi = __shfl_xor_sync(0xffffffffu, idx, m);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (!(v > R(0)) || !isfinite(v)) ok = false;
    const int pr = idx;
    if (lane == 0) piv[k] = pr;
    if (pr != k && lane < W) {
      cplx<R> t = A[k * LD + lane];
      A[k * LD + lane] = A[pr * LD + lane];
      A[pr * LD + lane] = t;
    }
    __syncwarp();
    const cplx<R> pinv = cinv(A[k * LD + k]);
    cplx<R> f = (lane < W) ? A[lane * LD + k] : cplx<R>{0, 0};
    __syncwarp();
    if (lane < W) {
      // scale the pivot row (lane = column)
      cplx<R> e = A[k * LD + lane];
      A[k * LD + lane] = (lane == k) ? pinv : cmul(e, pinv);
    }
    __syncwarp();
    if (lane < W && lane != k) {
      cplx<R>* row = A + lane * LD;
      const cplx<R>* prow = A + k * LD;
#pragma unroll 4
      for (int q = 0; q < W; ++q) {
        if (q == k) continue;
        cfms(row[q], f, prow[q]);
      }
      row[k] = cmul(cplx<R>{-f.re, -f.im}, pinv);
    }
    __syncwarp();
  }
  for (int k = W - 1; k >= 0; --k) {
    const int pr = piv[k];
    if (pr != k && lane < W) {
      cplx<R> t = A[lane * LD + k];
      A[lane * LD + k] = A[lane * LD + pr];
      A[lane * LD + pr] = t;
    }
    __syncwarp();
  }
  return __all_sync(0xffffffffu, ok);
}

// Copy rows row0 .. row0+nrows-1 of a shared W x (W+1) matrix to global
// memory with row stride `ld` (payload_ld(W) for payloads, W+1 for corners).
template <typename R, int W>
__device__ __forceinline__ void store_rows(cplx<R>* dst, const cplx<R>* src, int lane, int row0, int nrows, int ld) {
  constexpr int LD = W + 1;
  if (lane >= row0 && lane < row0 + nrows) {
#pragma unroll 4
    for (int q = 0; q < W; ++q) dst[(lane - row0) * ld + q] = src[lane * LD + q];
  }
}

template <typename R, int W>
__global__ void __launch_bounds__(32) factor_chunks_kernel(FactorArgs a) {
  using C = cplx<R>;
  constexpr int LD = W + 1;          // shared work matrices
  constexpr int LDP = W + 2;         // global payload rows (payload_ld)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufG = bufA + W * LD;
  C* bufW = bufG + W * LD;
  C* bufT = bufW + W * LD;
  C* cv = bufT + W * LD;
  c128* s2 = reinterpret_cast<c128*>(cv + 2 * W);
  int* piv = reinterpret_cast<int*>(s2 + 3 * 32);
  const int lane = threadIdx.x;
  C* facb = reinterpret_cast<C*>(a.fac);
  C* corb = reinterpret_cast<C*>(a.cor);

  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int bi = a.block_ids[item / a.P];
    const int k = (int)(item % a.P);
    const BlockDesc d = a.blocks[bi];
    const long long pe = payload_elems(W, d.d_out);
    C* fac = facb + d.fac_off;
    C* cor = corb + d.cor_off + (long long)k * cor_elems(W);
    const int l = k * a.L;
    const int r = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
    const bool has_left = k > 0, has_right = k < a.P - 1;
    for (int t = lane; t < 3 * d.w; t += 32) s2[t] = a.s2win[d.s2_off + t];
    __syncwarp();
    C *A = bufA, *G = bufG, *Wsp = bufW, *Tm = bufT;
    bool ok = true;

    // Pass 1: right-to-left factorisation of the interior, for the spike.
    if (has_left) {
      for (int j = r; j >= l; --j) {
        build_d<R, W>(a, d, s2, j, A, lane);
        if (j < r) {
          if (lane < W) cv[lane] = coupling<R>(a, d, s2, j, lane);
          __syncwarp();
          sub_cgc<R, W>(A, G, cv, lane);
        }
        ok &= invert_inplace<R, W>(A, piv, lane);
        store_rows<R, W>(fac + (long long)j * pe, A, lane, 0, W, LDP);
        C* t = A; A = G; G = t;
        __syncwarp();
      }
    }
    // Pass 2: left-to-right factorisation G_j and the spike W_j.
    for (int j = l; j <= r; ++j) {
      C* slot = fac + (long long)j * pe;
      if (lane < W) cv[W + lane] = (j > l) ? coupling<R>(a, d, s2, j - 1, lane) : C{0, 0};
      __syncwarp();
      if (has_left) {
        if (lane < W) {
#pragma unroll 4
          for (int q = 0; q < W; ++q) Tm[lane * LD + q] = slot[lane * LDP + q];
        }
        __syncwarp();
        if (j > l) {
          // new spike row p: -sum_q Tm[p][q] c_{j-1}[q] Wsp[q][:]
          C acc[W];
#pragma unroll
          for (int q = 0; q < W; ++q) acc[q] = C{0, 0};
          if (lane < W) {
            for (int q = 0; q < W; ++q) {
              C t = cmul(Tm[lane * LD + q], cv[W + q]);
#pragma unroll
              for (int qq = 0; qq < W; ++qq) cfms(acc[qq], t, Wsp[q * LD + qq]);
            }
          }
          __syncwarp();
          if (lane < W) {
#pragma unroll
            for (int q = 0; q < W; ++q) Tm[lane * LD + q] = acc[q];
          }
          __syncwarp();
        }
        C* t = Wsp; Wsp = Tm; Tm = t;    // Wsp = W_j
        store_rows<R, W>(slot + (long long)W * LDP, Wsp, lane, d.out_off, d.d_out, LDP);
        if (j == l) store_rows<R, W>(cor + (long long)W * LD, Wsp, lane, 0, W, LD);
        if (j == r) store_rows<R, W>(cor + 2LL * W * LD, Wsp, lane, 0, W, LD);
        __syncwarp();
      }
      build_d<R, W>(a, d, s2, j, A, lane);
      if (j > l) sub_cgc<R, W>(A, G, cv + W, lane);
      ok &= invert_inplace<R, W>(A, piv, lane);
      store_rows<R, W>(slot, A, lane, 0, W, LDP);
      if (j == r) store_rows<R, W>(cor, A, lane, 0, W, LD);
      C* t = A; A = G; G = t;
      // coupling c_j of this column (and of the separator that follows)
      C* cslot = slot + (long long)(W + d.d_out) * LDP;
      if (lane < W) cslot[lane] = coupling<R>(a, d, s2, j, lane);
      __syncwarp();
    }
    if (has_right) {
      const int s = r + 1;
      C* cslot = fac + (long long)s * pe + (long long)(W + d.d_out) * LDP;
      if (lane < W) cslot[lane] = coupling<R>(a, d, s2, s, lane);
    }
    if (!ok && lane == 0) set_status(a.status, HS_EBREAKDOWN, bi, l);
    __syncwarp();
  }
}

// Block LU of the reduced (separator) system of each block:
//   Sigma_kk   = D_s - C_{s-1} G^{(k)}_r C_{s-1} - C_s W^{(k+1)}_l C_s
//   Sigma_k,k-1 = -C_{s-1} W^{(k)}_r C_{s'}        (s' = previous separator)
//   F_k = Sigma_k,k-1 Gamma_{k-1},  Gamma_k = (Sigma_kk - F_k Sigma_k,k-1^t)^{-1}
template <typename R, int W>
__global__ void __launch_bounds__(32) factor_reduced_kernel(FactorArgs a) {
  using C = cplx<R>;
  constexpr int LD = W + 1;          // shared work matrices and corner blocks
  constexpr int LDP = W + 2;         // global payload rows (payload_ld)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufG = bufA + W * LD;
  C* bufS = bufG + W * LD;
  C* bufF = bufS + W * LD;
  C* cv = bufF + W * LD;
  c128* s2 = reinterpret_cast<c128*>(cv + 2 * W);
  int* piv = reinterpret_cast<int*>(s2 + 3 * 32);
  const int lane = threadIdx.x;
  C* facb = reinterpret_cast<C*>(a.fac);
  C* corb = reinterpret_cast<C*>(a.cor);
  C* redb = reinterpret_cast<C*>(a.red);
  for (int item = blockIdx.x; item < a.nblocks; item += gridDim.x) {
    const int bi = a.block_ids[item];
    const BlockDesc d = a.blocks[bi];
    (void)facb;
    for (int t = lane; t < 3 * d.w; t += 32) s2[t] = a.s2win[d.s2_off + t];
    __syncwarp();
    C *A = bufA, *Gam = bufG, *Sig = bufS, *F = bufF;
    bool ok = true;
    for (int k = 0; k + 1 < a.P; ++k) {
      const int s = (k + 1) * a.L - 1;
      const C* corL = corb + d.cor_off + (long long)k * cor_elems(W);        // interior k (left)
      const C* corR = corb + d.cor_off + (long long)(k + 1) * cor_elems(W);  // interior k+1 (right)
      C* red = redb + d.red_off + (long long)k * red_elems(W);
      build_d<R, W>(a, d, s2, s, A, lane);
      // - C_{s-1} Gr_k C_{s-1}
      if (lane < W) cv[lane] = coupling<R>(a, d, s2, s - 1, lane);
      if (lane < W) cv[W + lane] = coupling<R>(a, d, s2, s, lane);
      __syncwarp();
      if (lane < W) {
        const C cp = cv[lane], cq = cv[W + lane];
        for (int q = 0; q < W; ++q) {
          C t1 = cmul(cmul(cp, corL[lane * LD + q]), cv[q]);
          C t2 = cmul(cmul(cq, corR[(long long)W * LD + lane * LD + q]), cv[W + q]);
          A[lane * LD + q] = csub(csub(A[lane * LD + q], t1), t2);
        }
      }
      __syncwarp();
      if (k >= 1) {
        const int sp = k * a.L - 1;
        // Sig[p][q] = -c_{s-1}[p] Wr_k[p][q] c_{sp}[q]
        if (lane < W) cv[W + lane] = coupling<R>(a, d, s2, sp, lane);
        __syncwarp();
        if (lane < W) {
          const C cp = cv[lane];
          for (int q = 0; q < W; ++q) {
            C t = cmul(cmul(cp, corL[2LL * W * LD + lane * LD + q]), cv[W + q]);
            Sig[lane * LD + q] = C{-t.re, -t.im};
          }
        }
        __syncwarp();
        // F = Sig * Gam_prev
        C acc[W];
#pragma unroll
        for (int q = 0; q < W; ++q) acc[q] = C{0, 0};
        if (lane < W) {
          for (int q = 0; q < W; ++q) {
            C t = Sig[lane * LD + q];
#pragma unroll
            for (int qq = 0; qq < W; ++qq) cfma(acc[qq], t, Gam[q * LD + qq]);
          }
#pragma unroll
          for (int q = 0; q < W; ++q) F[lane * LD + q] = acc[q];
        }
        __syncwarp();
        // A -= F Sig^t
        if (lane < W) {
          for (int q = 0; q < W; ++q) {
            C t{0, 0};
            for (int u = 0; u < W; ++u) cfma(t, F[lane * LD + u], Sig[q * LD + u]);
            A[lane * LD + q] = csub(A[lane * LD + q], t);
          }
        }
        __syncwarp();
        store_rows<R, W>(red + (long long)W * LDP, F, lane, 0, W, LDP);
      }
      ok &= invert_inplace<R, W>(A, piv, lane);
      store_rows<R, W>(red, A, lane, 0, W, LDP);
      C* t = A; A = Gam; Gam = t;
      __syncwarp();
    }
    if (!ok && lane == 0) set_status(a.status, HS_EBREAKDOWN, bi, -1);
    __syncwarp();
  }
}

template <typename R, int W>
int launch_w(Plan& p, FactorArgs a, const std::vector<int>& ids, cudaStream_t s) {
  if (ids.empty()) return HS_OK;
  int* d_ids = nullptr;
  HS_CUDA_TRY(cudaMalloc(&d_ids, ids.size() * sizeof(int)));
  cudaMemcpyAsync(d_ids, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  a.block_ids = d_ids;
  a.nblocks = (int)ids.size();
  a.nitems = (int)ids.size() * p.P;
  const size_t smem = 4 * sizeof(cplx<R>) * W * (W + 1) + 2 * sizeof(cplx<R>) * W + 3 * 32 * sizeof(c128) +
                      32 * sizeof(int);
  cudaFuncSetAttribute(factor_chunks_kernel<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(factor_reduced_kernel<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // One persistent launch over all (block, chunk) work items of this width.
  int grid = std::min<long long>(a.nitems, (long long)sms * 16);
  note_launch();
  factor_chunks_kernel<R, W><<<grid, 32, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && p.P > 1) {
    int g2 = std::min(a.nblocks, sms * 16);
    note_launch();
    factor_reduced_kernel<R, W><<<g2, 32, smem, s>>>(a);
    e = cudaGetLastError();
  }
  cudaStreamSynchronize(s);
  cudaFree(d_ids);
  if (e != cudaSuccess) return cuda_status(e);
  return HS_OK;
}

template <typename R>
int launch_setup_t(Plan& p, cudaStream_t s) {
  FactorArgs a{};
  a.n = p.n; a.L = p.L; a.P = p.P;
  a.blocks = p.d_blocks;
  a.inv_s1 = p.d_inv_s1; a.a1 = p.d_a1; a.cinv2 = p.d_cinv2; a.s2win = p.d_s2win;
  const double wr = p.omega, wi = p.alpha;
  a.wst2 = c128{wr * wr - wi * wi, 2 * wr * wi};
  a.fac = p.d_fac; a.red = p.d_red; a.cor = p.d_cor; a.status = p.d_status;
  std::vector<int> by_w[33];
  for (int i = 0; i < (int)p.blocks.size(); ++i) by_w[p.blocks[i].W].push_back(i);
  int st = HS_OK;
  if (st == HS_OK) st = launch_w<R, 8>(p, a, by_w[8], s);
  if (st == HS_OK) st = launch_w<R, 12>(p, a, by_w[12], s);
  if (st == HS_OK) st = launch_w<R, 16>(p, a, by_w[16], s);
  if (st == HS_OK) st = launch_w<R, 24>(p, a, by_w[24], s);
  if (st == HS_OK) st = launch_w<R, 32>(p, a, by_w[32], s);
  return st;
}

}  // namespace

int launch_setup(Plan& p, cudaStream_t s) {
  return (p.prec == HS_C64) ? launch_setup_t<float>(p, s) : launch_setup_t<double>(p, s);
}

}  // namespace hs
