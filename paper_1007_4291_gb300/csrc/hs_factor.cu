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
// One warp owns one (problem, block, chunk) work item and a single persistent
// launch covers the items of every problem of a batch (any n, any window
// height); lanes own matrix rows and all
// work matrices live in shared memory (row stride W+1 complex, conflict-free).
#include <algorithm>
#include "hs_internal.cuh"
#include "hs_device.cuh"

namespace hs {
namespace {

struct FactorArgs {
  int n, L, P;
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
    int pr;
    if constexpr (sizeof(R) == 4) {
      // |a|^2 >= 0 orders like its bit pattern: one warp max-reduction, then
      // the lowest lane holding the maximum (ties as in a scan from row k)
      const unsigned key = (lane < W && lane >= k) ? __float_as_uint(cabs2(A[lane * LD + k])) + 1u : 0u;
      const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
      pr = __ffs(__ballot_sync(0xffffffffu, key == kmax)) - 1;
      const float v = __uint_as_float(kmax - 1u);
      if (!(v > 0.f) || !isfinite(v)) ok = false;
    } else {
      R v = (lane < W && lane >= k) ? cabs2(A[lane * LD + k]) : R(-1);
      int idx = lane;
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        R ov = Shfl<R>::xr(v, m);
        int oi = __shfl_xor_sync(0xffffffffu, idx, m);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
      }
      if (!(v > R(0)) || !isfinite(v)) ok = false;
      pr = idx;
    }
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
      // every column, k included (row[k] is then replaced by -f pinv)
      cplx<R>* row = A + lane * LD;
      const cplx<R>* prow = A + k * LD;
#pragma unroll
      for (int q = 0; q < W; ++q) cfms(row[q], f, prow[q]);
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

// Factor chunk k of block bi: interior G_j, spikes, corner blocks.
template <typename R, int W>
__device__ __forceinline__ void chunk_item(const FactorArgs& a, const int bi, const int k) {
  using C = cplx<R>;
  constexpr int LD = W + 1;          // shared work matrices
  constexpr int LDP = W + 2;         // global payload rows (payload_ld)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufG = bufA + W * LD;
  C* bufW = bufG + W * LD;
  C* cv = bufW + W * LD;
  c128* s2 = reinterpret_cast<c128*>(cv + 2 * W);
  int* piv = reinterpret_cast<int*>(s2 + 3 * 32);
  const int lane = threadIdx.x;
  C* facb = reinterpret_cast<C*>(a.fac);
  C* corb = reinterpret_cast<C*>(a.cor);

  {
    const BlockDesc d = a.blocks[bi];
    const long long pe = payload_elems(W, d.d_out);
    C* fac = facb + d.fac_off;
    C* cor = corb + d.cor_off + (long long)k * cor_elems(W);
    const int l = k * a.L;
    const int r = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
    const bool has_left = k > 0, has_right = k < a.P - 1;
    for (int t = lane; t < 3 * d.w; t += 32) s2[t] = a.s2win[d.s2_off + t];
    __syncwarp();
    // three work matrices: A (the column being factored), G (the previous
    // column's inverse) and the spike; the spike update of pass 2 stages
    // (S^R_j)^{-1} in A's buffer, which is free until the column is built
    C *A = bufA, *G = bufG, *Wsp = bufW;
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
        C* Tm = A;
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
        A = Wsp;                         // the previous spike's buffer is free now
        Wsp = Tm;                        // Wsp = W_j
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

// Twisted block LU of the reduced (separator) system of each block: the
// separators s_0..s_{K-1} form a block-tridiagonal system with
//   Sigma_kk     = D_s - C_{s-1} G^{(k)}_r C_{s-1} - C_s W^{(k+1)}_l C_s
//   Sigma_k,k-1  = -C_{s-1} W^{(k)}_r C_{s'}        (s' = previous separator)
// eliminated from both ends toward the twist m = K/2:
//   top    (k < m):  F_k = Sigma_k,k-1 Gamma_{k-1},   Gamma_k  = (Sigma_kk - F_k Sigma_k,k-1^t)^{-1}
//   bottom (k > m):  F'_k = Sigma_k+1,k^t Gamma'_{k+1}, Gamma'_k = (Sigma_kk - F'_k Sigma_k+1,k)^{-1}
//   twist:           Gamma_m = (Sigma_mm - F_m Sigma_m,m-1^t - F'_m Sigma_m+1,m)^{-1}
// Slot k stores [Gamma_k or Gamma'_k | F_k or F'_k | F'_m at the twist].  The
// two chains of the separator solve are then half as long.
template <typename R, int W>
__device__ __forceinline__ void reduced_item(const FactorArgs& a, const int bi) {
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
  C* corb = reinterpret_cast<C*>(a.cor);
  C* redb = reinterpret_cast<C*>(a.red);
  const BlockDesc d = a.blocks[bi];
  for (int t = lane; t < 3 * d.w; t += 32) s2[t] = a.s2win[d.s2_off + t];
  __syncwarp();
  const int K = a.P - 1, m = twist_index(K);
  auto sep_col = [&](int k) { return (k + 1) * a.L - 1; };
  auto slot = [&](int k) { return redb + d.red_off + (long long)k * red_elems(W); };
  // A = Sigma_kk
  auto build_diag = [&](C* A, int k) {
    const int s = sep_col(k);
    const C* corL = corb + d.cor_off + (long long)k * cor_elems(W);        // interior k (left)
    const C* corR = corb + d.cor_off + (long long)(k + 1) * cor_elems(W);  // interior k+1 (right)
    build_d<R, W>(a, d, s2, s, A, lane);
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
  };
  // Sig = Sigma_{k,k-1} (k >= 1): -c_{s-1}[p] Wr_k[p][q] c_{s'}[q]
  auto build_sub = [&](C* Sig, int k) {
    const int s = sep_col(k), sp = sep_col(k - 1);
    const C* corL = corb + d.cor_off + (long long)k * cor_elems(W);
    if (lane < W) cv[lane] = coupling<R>(a, d, s2, s - 1, lane);
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
  };
  // F = op(Sig) Gam, op = identity (top) or transpose (bottom)
  auto mul_sg = [&](C* F, const C* Sig, const C* Gam, bool trans) {
    C acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = C{0, 0};
    if (lane < W) {
      for (int u = 0; u < W; ++u) {
        const C t = trans ? Sig[u * LD + lane] : Sig[lane * LD + u];
#pragma unroll
        for (int qq = 0; qq < W; ++qq) cfma(acc[qq], t, Gam[u * LD + qq]);
      }
#pragma unroll
      for (int q = 0; q < W; ++q) F[lane * LD + q] = acc[q];
    }
    __syncwarp();
  };
  // A -= F op(Sig): op = transpose (top: Sigma_k,k-1^t) or identity (bottom: Sigma_k+1,k)
  auto sub_fs = [&](C* A, const C* F, const C* Sig, bool trans) {
    if (lane < W) {
      for (int q = 0; q < W; ++q) {
        C t{0, 0};
        for (int u = 0; u < W; ++u) cfma(t, F[lane * LD + u], trans ? Sig[q * LD + u] : Sig[u * LD + q]);
        A[lane * LD + q] = csub(A[lane * LD + q], t);
      }
    }
    __syncwarp();
  };
  C *A = bufA, *Gam = bufG, *Sig = bufS, *F = bufF;
  bool ok = true;
  // top chain k = 0 .. m (the twist gets its top coupling but is not inverted yet)
  for (int k = 0; k <= m; ++k) {
    build_diag(A, k);
    if (k >= 1) {
      build_sub(Sig, k);
      mul_sg(F, Sig, Gam, false);
      sub_fs(A, F, Sig, true);
      store_rows<R, W>(slot(k) + (long long)W * LDP, F, lane, 0, W, LDP);
    }
    if (k < m) {
      ok &= invert_inplace<R, W>(A, piv, lane);
      store_rows<R, W>(slot(k), A, lane, 0, W, LDP);
      C* t = A; A = Gam; Gam = t;
      __syncwarp();
    }
  }
  // park Sigma_mm - F_m Sigma_m,m-1^t in the twist's Gamma slot
  store_rows<R, W>(slot(m), A, lane, 0, W, LDP);
  __syncwarp();
  // bottom chain k = K-1 .. m+1
  for (int k = K - 1; k > m; --k) {
    build_diag(A, k);
    if (k < K - 1) {
      build_sub(Sig, k + 1);
      mul_sg(F, Sig, Gam, true);
      sub_fs(A, F, Sig, false);
      store_rows<R, W>(slot(k) + (long long)W * LDP, F, lane, 0, W, LDP);
    }
    ok &= invert_inplace<R, W>(A, piv, lane);
    store_rows<R, W>(slot(k), A, lane, 0, W, LDP);
    C* t = A; A = Gam; Gam = t;
    __syncwarp();
  }
  // twist: Gamma_m = (parked - F'_m Sigma_m+1,m)^{-1}
  {
    const C* parked = slot(m);
    if (lane < W)
      for (int q = 0; q < W; ++q) A[lane * LD + q] = parked[lane * LDP + q];
    __syncwarp();
    if (m < K - 1) {
      build_sub(Sig, m + 1);
      mul_sg(F, Sig, Gam, true);
      sub_fs(A, F, Sig, false);
      store_rows<R, W>(slot(m) + 2LL * W * LDP, F, lane, 0, W, LDP);
    }
    ok &= invert_inplace<R, W>(A, piv, lane);
    store_rows<R, W>(slot(m), A, lane, 0, W, LDP);
    __syncwarp();
  }
  if (!ok && lane == 0) set_status(a.status, HS_EBREAKDOWN, bi, -1);
  __syncwarp();
}

// One work item of the batched setup: a chunk of a block of a problem.
struct FactorItem {
  int prob, block, chunk, W;
};

// Persistent launches over the work items of all problems of a batch; the
// window height W (uniform per item) selects the instantiation.
template <typename R>
__global__ void __launch_bounds__(32) factor_chunks_kernel(const FactorArgs* probs, const FactorItem* items, int nitems) {
  for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
    const FactorItem it = items[i];
    const FactorArgs a = probs[it.prob];
    switch (it.W) {
      case 8: chunk_item<R, 8>(a, it.block, it.chunk); break;
      case 12: chunk_item<R, 12>(a, it.block, it.chunk); break;
      case 16: chunk_item<R, 16>(a, it.block, it.chunk); break;
      case 24: chunk_item<R, 24>(a, it.block, it.chunk); break;
      case 32: chunk_item<R, 32>(a, it.block, it.chunk); break;
      default: if (threadIdx.x == 0) set_status(a.status, HS_EUNSUPPORTED, it.block, it.chunk);
    }
    __syncwarp();
  }
}

template <typename R>
__global__ void __launch_bounds__(32) factor_reduced_kernel(const FactorArgs* probs, const FactorItem* items, int nitems) {
  for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
    const FactorItem it = items[i];
    const FactorArgs a = probs[it.prob];
    switch (it.W) {
      case 8: reduced_item<R, 8>(a, it.block); break;
      case 12: reduced_item<R, 12>(a, it.block); break;
      case 16: reduced_item<R, 16>(a, it.block); break;
      case 24: reduced_item<R, 24>(a, it.block); break;
      case 32: reduced_item<R, 32>(a, it.block); break;
      default: if (threadIdx.x == 0) set_status(a.status, HS_EUNSUPPORTED, it.block, -1);
    }
    __syncwarp();
  }
}

template <typename R>
size_t factor_smem(int W, int nmat) {
  return nmat * sizeof(cplx<R>) * W * (W + 1) + 2 * sizeof(cplx<R>) * W + 3 * 32 * sizeof(c128) + 32 * sizeof(int);
}
// work matrices: three for a chunk, four for a reduced system (fewer shared
// bytes per one-warp CTA leave room for more resident CTAs)
constexpr int kChunkMats = 3, kReducedMats = 4;

template <typename R>
int launch_setup_t(const std::vector<Plan*>& ps, cudaStream_t s, bool async) {
  std::vector<FactorArgs> args;
  std::vector<FactorItem> items, reduced;
  int Wmax = 8;
  for (int q = 0; q < (int)ps.size(); ++q) {
    const Plan& p = *ps[q];
    FactorArgs a{};
    a.n = p.n; a.L = p.L; a.P = p.P;
    a.blocks = p.d_blocks;
    a.inv_s1 = p.d_inv_s1; a.a1 = p.d_a1; a.cinv2 = p.d_cinv2; a.s2win = p.d_s2win;
    const double wr = p.omega, wi = p.alpha;
    a.wst2 = c128{wr * wr - wi * wi, 2 * wr * wi};
    a.fac = p.d_fac; a.red = p.d_red; a.cor = p.d_cor; a.status = p.d_status;
    args.push_back(a);
    for (int b = 0; b < (int)p.blocks.size(); ++b) {
      const int W = p.blocks[b].W;
      Wmax = std::max(Wmax, W);
      for (int k = 0; k < p.P; ++k) items.push_back({q, b, k, W});
      if (p.P > 1) reduced.push_back({q, b, 0, W});
    }
  }
  // longest items first: windows of height W cost ~W^3 per column
  auto wider = [](const FactorItem& x, const FactorItem& y) { return x.W > y.W; };
  std::stable_sort(items.begin(), items.end(), wider);
  std::stable_sort(reduced.begin(), reduced.end(), wider);
  const size_t abytes = ((args.size() * sizeof(FactorArgs) + 255) / 256) * 256;
  const size_t ibytes = items.size() * sizeof(FactorItem), rbytes = reduced.size() * sizeof(FactorItem);
  // the launch arguments live in stream-ordered memory, released on the
  // stream after the kernels (no device-wide synchronisation)
  char* buf = nullptr;
  HS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&buf), abytes + ibytes + rbytes + 16, s));
  FactorArgs* d_args = reinterpret_cast<FactorArgs*>(buf);
  FactorItem* d_items = reinterpret_cast<FactorItem*>(buf + abytes);
  FactorItem* d_red = reinterpret_cast<FactorItem*>(buf + abytes + ibytes);
  cudaMemcpyAsync(d_args, args.data(), args.size() * sizeof(FactorArgs), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_items, items.data(), ibytes, cudaMemcpyHostToDevice, s);
  if (rbytes) cudaMemcpyAsync(d_red, reduced.data(), rbytes, cudaMemcpyHostToDevice, s);
  const size_t smem = factor_smem<R>(Wmax, kChunkMats), smem_r = factor_smem<R>(Wmax, kReducedMats);
  cudaFuncSetAttribute(factor_chunks_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(factor_reduced_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  if (!items.empty()) {
    const int grid = (int)std::min<long long>((long long)items.size(), (long long)sms * 16);
    note_launch();
    factor_chunks_kernel<R><<<grid, 32, smem, s>>>(d_args, d_items, (int)items.size());
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !reduced.empty()) {
    const int g2 = (int)std::min<long long>((long long)reduced.size(), (long long)sms * 16);
    note_launch();
    factor_reduced_kernel<R><<<g2, 32, smem_r, s>>>(d_args, d_red, (int)reduced.size());
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return cuda_status(e);
  if (async) return HS_OK;
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e2 != cudaSuccess) return cuda_status(e2);
  return HS_OK;
}

}  // namespace

int launch_setup(const std::vector<Plan*>& ps, cudaStream_t s, bool async) {
  if (ps.empty()) return HS_OK;
  return (ps[0]->prec == HS_C64) ? launch_setup_t<float>(ps, s, async) : launch_setup_t<double>(ps, s, async);
}

}  // namespace hs
