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
// Phases 1 and 3: each consumer thread owns a few window rows of two RHS;
// the vector carried from column to column goes through shared memory, one
// named barrier per column.  Per-column factor payloads (G_j | W_j rows |
// c_j) stream into a shared-memory ring with 1D TMA bulk copies completed on
// mbarriers (bounded waits -> HS_ETIMEOUT), issued by two producer warps that
// take the columns in turn.  Phase 2: one or a few RHS per CTA, two chain
// warps per half chain of each RHS (complex64; one for complex128), two
// producer warps per half (see below).
#include <algorithm>
#include "hs_internal.cuh"
#include "hs_device.cuh"
#include "hs3d.cuh"

namespace hs {
namespace {

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

constexpr int S13 = 4;        // TMA ring depth of the chunk kernels (phases 1 and 3)
// Producer warps of the chunk kernels: two, taking the columns in turn (one
// thread keeps about one bulk copy in flight; n = 2047, 64 RHS: 29.9 -> 29.5 ms
// per application, one RHS 15.7 -> 15.0 ms; four producers 30.2 ms).
constexpr int P13 = 2;
static_assert(S13 % P13 == 0, "each producer owns every P13-th stage");

__host__ __device__ __forceinline__ size_t round128(size_t b) { return (b + 127) / 128 * 128; }

// Per-thread description of the right-hand side of T~_B on the thread's own
// window rows: a direct term (forward sweep: the block rows of u) and up to
// two coupling terms k * inv_s1(j) * u[row'] (forward sweep: minus the
// coupling to the previous blocks' rows; backward sweep: the coupling to the
// next block's row).  Offsets count rows of u (n*R elements); -1 = none.
template <typename R, int ROWS>
struct RhsTerms {
  int drow[ROWS], crow1[ROWS], crow2[ROWS];
  cplx<R> k1[ROWS], k2[ROWS];

  // own rows p0, p0 + pstride, ..., p0 + (ROWS-1) pstride
  __device__ __forceinline__ void init(const SweepArgs& a, const BlockDesc& d, int p0, int pstride = 1) {
    const cplx<R>* a2 = reinterpret_cast<const cplx<R>*>(a.a2);
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int p = p0 + q * pstride, jg = d.wlo + p;
      drow[q] = crow1[q] = crow2[q] = -1;
      k1[q] = k2[q] = cplx<R>{0, 0};
      if (a.mode == 0) {
        if (p >= d.out_off && p < d.out_off + d.d_out) {
          drow[q] = jg - 1;
          if (jg == d.lo && d.prev_lo_row) { crow1[q] = d.prev_lo_row - 1; k1[q] = cplx<R>{-a2[d.lo - 1].re, -a2[d.lo - 1].im}; }
          if (jg == d.hi && d.prev_hi_row) { crow2[q] = d.prev_hi_row - 1; k2[q] = cplx<R>{-a2[d.hi].re, -a2[d.hi].im}; }
        }
      } else if (p == d.coup_local) {
        crow1[q] = d.next_row - 1;
        k1[q] = a2[min(jg, d.next_row)];
      }
    }
  }
  // Raw operands of the right-hand side at column j (loads only; combine()
  // forms the value later, so the loads can be in flight meanwhile).
  struct Raw {
    cplx<R> d[ROWS], c1[ROWS], c2[ROWS], s;
  };
  __device__ __forceinline__ void load_raw(Raw& w, const cplx<R>* ur, const cplx<R>* is1, int n, int R_,
                                           int j) const {
    w.s = is1[j + 1];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      w.d[q] = (drow[q] >= 0) ? ur[((long long)drow[q] * n + j) * R_] : cplx<R>{0, 0};
      w.c1[q] = (crow1[q] >= 0) ? ur[((long long)crow1[q] * n + j) * R_] : cplx<R>{0, 0};
      w.c2[q] = (crow2[q] >= 0) ? ur[((long long)crow2[q] * n + j) * R_] : cplx<R>{0, 0};
    }
  }
  __device__ __forceinline__ void combine(cplx<R> (&g)[ROWS], const Raw& w) const {
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      cplx<R> v = w.d[q];
      if (crow1[q] >= 0) cfma(v, cmul(k1[q], w.s), w.c1[q]);
      if (crow2[q] >= 0) cfma(v, cmul(k2[q], w.s), w.c2[q]);
      g[q] = v;
    }
  }
  // right-hand side at column j for the RHS whose first element is ur = u + r
  __device__ __forceinline__ void load(cplx<R> (&g)[ROWS], const cplx<R>* ur, const cplx<R>* is1, int n, int R_,
                                       int j) const {
    const cplx<R> s = is1[j + 1];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      cplx<R> v{0, 0};
      if (drow[q] >= 0) v = ur[((long long)drow[q] * n + j) * R_];
      if (crow1[q] >= 0) cfma(v, cmul(k1[q], s), ur[((long long)crow1[q] * n + j) * R_]);
      if (crow2[q] >= 0) cfma(v, cmul(k2[q], s), ur[((long long)crow2[q] * n + j) * R_]);
      g[q] = v;
    }
  }
};

// Producer of a ring: issues uses first, first + step, ... (< nuses) into
// stage t % S once the consumers have released use t - S.  Returns after every
// copy it issued has landed (bounded waits; an expired wait records
// HS_ETIMEOUT).  Several producers may share a ring when step divides S: each
// then owns the stages t % S with t = first (mod step), so the uses of a stage
// stay in one producer's order.  One thread keeps about one bulk copy in
// flight at a time, so two producers per ring halve the step time of a ring
// whose consumer is fast.
template <typename F>
__device__ __forceinline__ void ring_producer(uint64_t* full, uint64_t* empty, int S, int nuses, long long spin,
                                              int* status, int front, F&& issue, int first = 0, int step = 1) {
  int t = first;
  for (; t < nuses; t += step) {
    if (t >= S && !mbar_wait_bounded(&empty[t % S], ((t / S) - 1) & 1, spin)) {
      set_status(status, HS_ETIMEOUT, front, -4);
      break;
    }
    issue(t);
  }
  // drain: copies already issued must land before the CTA may exit, so this
  // wait does not shrink with a small `spin` (a copy lands in microseconds)
  const long long drain = spin > (1LL << 27) ? spin : (1LL << 27);
  for (int u = first; u < t; u += step)
    if (u >= t - S) (void)mbar_wait_bounded(&full[u % S], (u / S) & 1, drain);
}

// ---------------------------------------------------------------- phases 1 and 3
// One CTA owns one chunk of one block for a group of RG right-hand sides.
// Each consumer thread owns a tile of ROWS window rows x RPT RHS; the
// per-column product (W x W) * (W x RG) reads G_j from the TMA ring and the
// vector being carried from shared memory (written by its owners before a
// named barrier), so every column costs one barrier.  Two producer warps
// stream the column payloads.
// SM: the small tile for at most 16 right-hand sides: CTAs of 16 RHS, one
// window row per thread, so that the per-column chain of a thread (which sets
// the pace when few warps share an SM) is a third as long.
template <typename R, int W, bool SM = false> struct Tile13 {
  static constexpr int ROWS = SM ? 1 : (W == 12) ? 3 : W / 8;  // window rows per thread
  static constexpr int NRG = W / ROWS;                // row groups
  static constexpr int RPT = 2;                       // RHS per thread
  static constexpr int RG = SM ? 16 : (sizeof(R) == 4 ? 64 : 32); // RHS per CTA
  static constexpr int NHG = RG / RPT;                // RHS groups
  static constexpr int NCONS = NRG * NHG;             // consumer threads
  static constexpr int LDR = RG + 2;                  // row stride of the [W][RG] exchange arrays
  static_assert(NCONS % 32 == 0, "producer warps follow whole consumer warps");
};

// Two adjacent complex values of shared memory (one 128-bit access for c64).
template <typename R>
__device__ __forceinline__ void ld2(const cplx<R>* p, cplx<R>& a, cplx<R>& b) {
  a = p[0];
  b = p[1];
}
template <>
__device__ __forceinline__ void ld2<float>(const cplx<float>* p, cplx<float>& a, cplx<float>& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = cplx<float>{v.x, v.y};
  b = cplx<float>{v.z, v.w};
}
template <typename R>
__device__ __forceinline__ void st2(cplx<R>* p, cplx<R> a, cplx<R> b) {
  p[0] = a;
  p[1] = b;
}
template <>
__device__ __forceinline__ void st2<float>(cplx<float>* p, cplx<float> a, cplx<float> b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}

__device__ __forceinline__ void consumer_barrier(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Consumer barrier that also returns the AND of `v` over the consumer
// threads: after a bounded wait every consumer learns whether all of them
// got their data, so they continue or stop together (a thread that stopped
// alone would leave the others blocked on the next barrier).
__device__ __forceinline__ bool consumer_barrier_and(int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Depth of phase 3's staging of the previous u values (backward stages, full
// tile): each thread copies its own output entries OD - 1 columns ahead with
// cp.async (n = 2047, 64 RHS: 29.5 -> 29.1 ms per application; depths 4 and 5
// the same).  The 16-RHS tile keeps register prefetches (staged: 0.6-0.75 ms
// slower at 1-16 RHS).
constexpr int OD = 3;

// Shared-memory bytes of phases 1 and 3.
template <typename R, int W, bool SM>
size_t tile_smem(int d_out, bool p3) {
  using TL = Tile13<R, W, SM>;
  const size_t pb = round128((size_t)payload_elems(W, d_out) * sizeof(cplx<R>));
  const size_t vb = round128((size_t)W * TL::LDR * sizeof(cplx<R>));  // one W x RG array (padded)
  const size_t ob = SM ? 0 : round128((size_t)OD * d_out * TL::LDR * sizeof(cplx<R>));   // [OD][d_out][LDR]
  // phase 1: ring of payloads, Y and g double buffers
  // phase 3: ring of (payload + z tile), tv double buffer, beta, old-u staging
  return p3 ? 256 + S13 * (pb + vb) + 3 * vb + ob : 256 + S13 * pb + 4 * vb;
}

// Forward elimination over the chunk's interior columns:
//   y_j = g_j - C_{j-1} z_{j-1},  z_j = G_j y_j  (z_j stored for phase 3),
// the left-spike sum sum_j W_j^t g_j, and the separator term C_r z_r - g(s).
// Thread (rg, hg) owns rows rg + NRG*i (i < ROWS) and RHS 2hg, 2hg+1 of the group.
template <typename R, int W, bool SM>
__global__ void __launch_bounds__(Tile13<R, W, SM>::NCONS + 32 * P13) phase1_kernel(SweepArgs a) {
  using C = cplx<R>;
  using TL = Tile13<R, W, SM>;
  constexpr int ROWS = TL::ROWS, NRG = TL::NRG, RPT = TL::RPT, RG = TL::RG, NCONS = TL::NCONS, LDR = TL::LDR;
  constexpr int LDP = W + 2;
  static_assert(RPT == 2, "tiles carry two right-hand sides");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + S13;
  const int front = blockIdx.z, k = blockIdx.x;
  const BlockDesc& d = a.blk[front];
  const long long pe = payload_elems(W, d.d_out);
  const uint32_t pbytes = (uint32_t)(pe * sizeof(C));
  const size_t pstride = round128(pbytes);
  const size_t vb = round128((size_t)W * LDR * sizeof(C));
  C* ybuf = reinterpret_cast<C*>(smem_raw + 256 + S13 * pstride);            // [2][W][LDR]
  C* gbuf = reinterpret_cast<C*>(smem_raw + 256 + S13 * pstride + 2 * vb);   // [2][W][LDR]
  const C* fac = reinterpret_cast<const C*>(a.fac) + d.fac_off;
  const int tid = threadIdx.x;
  const int l = k * a.L;
  const int rgt = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
  const int ncol = rgt - l + 1;
  auto stage = [&](int u) { return reinterpret_cast<const C*>(smem_raw + 256 + (size_t)(u % S13) * pstride); };

  if (tid == 0) {
    for (int u = 0; u < S13; ++u) {
      mbar_init(&full[u], 1);
      mbar_init(&empty[u], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= NCONS) {
    const int sub = (tid - NCONS) >> 5;
    if ((tid & 31) == 0 && sub < ncol) {
      ring_producer(
          full, empty, S13, ncol, a.spin, a.status, front,
          [&](int t) {
            mbar_arrive_expect_tx(&full[t % S13], pbytes);
            tma_bulk_g2s(const_cast<C*>(stage(t)), fac + (long long)(l + t) * pe, pbytes, &full[t % S13]);
          },
          sub, P13);
    }
    return;
  }
  const int rg = tid % NRG, hg = tid / NRG;
  const int c0 = hg * RPT;                 // first own RHS of the group
  const int rbase = blockIdx.y * RG;
  bool valid[RPT];
  const C* ur[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    valid[q] = rbase + c0 + q < a.R;
    ur[q] = reinterpret_cast<const C*>(a.u) + min(rbase + c0 + q, a.R - 1);
  }
  const C* is1 = reinterpret_cast<const C*>(a.inv_s1);
  RhsTerms<R, ROWS> rhs;
  rhs.init(a, d, rg, NRG);
  const bool has_left = k > 0;
  const int in_lo = (a.mode == 0) ? d.out_off : d.coup_local;
  const int in_hi = (a.mode == 0) ? d.out_off + d.d_out : d.coup_local + 1;
  C* zbase = reinterpret_cast<C*>(a.z) + ((long long)front * a.n * a.R) * W;

  using Raw = typename RhsTerms<R, ROWS>::Raw;
  auto load_g = [&](C (&g)[RPT][ROWS], int j) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) rhs.load(g[q], ur[q], is1, a.n, a.R, j);
  };
  auto load_raw = [&](Raw (&w)[RPT], int j) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) rhs.load_raw(w[q], ur[q], is1, a.n, a.R, j);
  };
  auto put_tile = [&](C* buf, const C (&v)[RPT][ROWS]) {
#pragma unroll
    for (int i = 0; i < ROWS; ++i) st2(buf + (rg + NRG * i) * LDR + c0, v[0][i], v[1][i]);
  };
  C z[RPT][ROWS], sp[RPT][ROWS];
  Raw ra[RPT], rb[RPT];   // raw right-hand sides, fetched two columns ahead
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int i = 0; i < ROWS; ++i) sp[q][i] = C{0, 0};
  {
    C g0[RPT][ROWS];
    load_g(g0, l);
    put_tile(ybuf, g0);     // y_l = g_l
    put_tile(gbuf, g0);
  }
  if (ncol > 1) load_raw(ra, l + 1);
  if (ncol > 2) load_raw(rb, l + 2);
  consumer_barrier(NCONS);
  bool ok = true;
  // one column step; wn = raw right-hand side of the next column
  auto step = [&](int t, const Raw (&wn)[RPT]) {
    const int j = l + t;
    const C* G = stage(t);
    const C* V = G + W * LDP;
    const C* cc = V + d.d_out * LDP;
    const C* Y = ybuf + (t & 1) * (W * LDR);
    const C* Gi = gbuf + (t & 1) * (W * LDR);
    const bool landed = mbar_wait_bounded(&full[t % S13], (t / S13) & 1, a.spin);
    if (landed) {
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int i = 0; i < ROWS; ++i) z[q][i] = C{0, 0};
#pragma unroll
    for (int kk = 0; kk < W; kk += 2) {
      C g0[ROWS], g1[ROWS], y00, y01, y10, y11;
#pragma unroll
      for (int i = 0; i < ROWS; ++i) ld2(G + (rg + NRG * i) * LDP + kk, g0[i], g1[i]);
      ld2(Y + kk * LDR + c0, y00, y01);
      ld2(Y + (kk + 1) * LDR + c0, y10, y11);
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        cfma(z[0][i], g0[i], y00);
        cfma(z[1][i], g0[i], y01);
        cfma(z[0][i], g1[i], y10);
        cfma(z[1][i], g1[i], y11);
      }
    }
    // store z_j (layout [front][col][rhs][W])
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (valid[q]) {
        C* zp = zbase + ((long long)j * a.R + rbase + c0 + q) * W + rg;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) zp[NRG * i] = z[q][i];
      }
    if (has_left) {
      // sp[own rows] += sum over input rows o of W_j[o][own rows] g_j[o]
      for (int o = in_lo; o < in_hi; ++o) {
        const C* vr = V + (o - d.out_off) * LDP + rg;
        C go0, go1;
        ld2(Gi + o * LDR + c0, go0, go1);
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          const C v = vr[NRG * i];
          cfma(sp[0][i], v, go0);
          cfma(sp[1][i], v, go1);
        }
      }
    }
    if (t + 1 < ncol) {
      // y_{j+1} = g_{j+1} - C_j z_j
      C gn[RPT][ROWS], yn[RPT][ROWS];
#pragma unroll
      for (int q = 0; q < RPT; ++q) rhs.combine(gn[q], wn[q]);
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        const C ci = cc[rg + NRG * i];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          yn[q][i] = gn[q][i];
          cfms(yn[q][i], ci, z[q][i]);
        }
      }
      put_tile(ybuf + ((t + 1) & 1) * (W * LDR), yn);
      put_tile(gbuf + ((t + 1) & 1) * (W * LDR), gn);
    }
    }  // landed
    ok = consumer_barrier_and(NCONS, landed);
    if (ok && tid == 0) mbar_arrive(&empty[t % S13]);
  };
  for (int t = 0; t < ncol; t += 2) {
    step(t, ra);
    if (!ok) break;
    if (t + 3 < ncol) load_raw(ra, l + t + 3);
    if (t + 1 < ncol) {
      step(t + 1, rb);
      if (!ok) break;
      if (t + 4 < ncol) load_raw(rb, l + t + 4);
    }
  }
  if (!ok) {
    if ((tid & 31) == 0) set_status(a.status, HS_ETIMEOUT, front, l);
    return;
  }
  // separator contributions (z holds z_r of the last column)
  const long long sep_base = ((long long)front * a.P + k) * a.R + rbase + c0;
  const C* cr = fac + (long long)rgt * pe + (long long)(W + d.d_out) * LDP;   // c_r
  if (k < a.P - 1) {
    C gs[RPT][ROWS];
    load_g(gs, rgt + 1);
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (valid[q]) {
        C* rc = reinterpret_cast<C*>(a.rc) + (sep_base + q) * W + rg;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) rc[NRG * i] = csub(cmul(cr[rg + NRG * i], z[q][i]), gs[q][i]);
      }
  }
  if (has_left) {
    const C* cl = fac + (long long)(l - 1) * pe + (long long)(W + d.d_out) * LDP;   // c_{l-1}
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (valid[q]) {
        C* lc = reinterpret_cast<C*>(a.lc) + (sep_base + q) * W + rg;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) lc[NRG * i] = cmul(cl[rg + NRG * i], sp[q][i]);
      }
  }
}

// ---------------------------------------------------------------- phase 2
// Twisted block LU solve of the separator system (see the setup): for each
// RHS the top half and the bottom half run the two half chains at once,
//   top     psi_k  = rho_k - F_k psi_{k-1}            k = 0 .. m-1
//   bottom  psi'_k = rho_k - F'_k psi'_{k+1}          k = K-1 .. m+1
//   twist   x_m = Gamma_m (rho_m - F_m psi_{m-1} - F'_m psi'_{m+1})
//   top     x_k = Gamma_k psi_k - F_{k+1}^t x_{k+1}    k = m-1 .. 0
//   bottom  x_k = Gamma'_k psi'_k - F'_{k-1}^t x_{k-1} k = m+1 .. K-1
// (lane p = row p).  Each half is two warps that split the W columns of
// every block product: each forms the partial sums of its columns, they
// exchange them through shared memory on a named barrier (which also
// carries their agreement on the bounded waits), and both finish the step,
// so each keeps the chain variable it needs in its own registers and
// shared-memory copy.  rho_k = -(rc_k + lc_{k+1}) is gathered into shared
// memory first.  The four warps of a RHS meet twice on a named barrier
// (psi'_{m+1}, then x_m); each half has its own producer warps streaming the
// separator factors through an S2-deep TMA ring in the order its chain uses
// them.
// RHS per CTA (wpc, from the block size): one while the RHS of both fronts
// fit on the SMs one CTA each (the chain warps then run on SMs the chunk
// phases leave idle), else two or four so that the separator solve stays
// within one wave.
constexpr int WPC_MAX = 4;
// Column parts per half: two for complex64; complex128 keeps one warp per
// half (its products are bound by the FP64 pipe, and the exchange only adds
// latency there), with at most two RHS per CTA so that the threads keep the
// registers of the double-precision products.
template <typename R> constexpr int npart() { return sizeof(R) == 4 ? 2 : 1; }
template <typename R> constexpr int wpc_max() { return sizeof(R) == 4 ? WPC_MAX : 2; }
// Producer warps per half chain; they take the ring's uses in turn (each owns
// every other stage), which halves the ring's step time against one producer
// (n = 2047, 64 RHS: 30.4 -> 29.8 ms per application).
constexpr int PPH = 2;
constexpr int P2_PROD_THREADS = 2 * PPH * 32;
// TMA ring depth: 4 stages per half, 2 when the separator factors are large
template <typename R, int W> struct Ring2 {
  static constexpr int S = (8LL * 3 * W * (W + 2) * 2 * (long long)sizeof(R) <= 128 * 1024) ? 4 : 2;
};

// per RHS: rho/psi [K] + x_m + two exchange vectors (one per half) and the
// partial sums [step parity][half][part]
template <typename R, int W>
size_t phase2_smem(int nsep, int wpc) {
  return 256 + (size_t)2 * Ring2<R, W>::S * round128((size_t)red_elems(W) * sizeof(cplx<R>)) +
         (size_t)wpc * ((nsep + 3) * W + 8 * W) * sizeof(cplx<R>);
}
int phase2_wpc(int R, int nfront, int maxw) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int wpc = 1;
  while (wpc < maxw && (long long)((R + wpc - 1) / wpc) * nfront > sms) wpc *= 2;
  return wpc;
}

// Named barrier of `nthreads` threads, returning the AND of `v` over them.
__device__ __forceinline__ bool named_barrier_and(int id, int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <typename R, int W>
__global__ void __launch_bounds__(2 * npart<R>() * wpc_max<R>() * 32 + P2_PROD_THREADS) phase2_kernel(SweepArgs a) {
  using C = cplx<R>;
  constexpr int LDP = W + 2;
  constexpr int S2 = Ring2<R, W>::S;
  static_assert(S2 % PPH == 0, "each producer owns every PPH-th stage");
  constexpr int NP = npart<R>();     // column parts per half
  constexpr int P2W = 2 * NP;        // consumer warps per RHS
  constexpr int WH = W / NP;         // columns per part (even for every supported W)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);     // [2][S2]
  uint64_t* empty = full + 2 * S2;                            // [2][S2]
  const int front = blockIdx.z;
  const BlockDesc& d = a.blk[front];
  const long long re = red_elems(W);
  const uint32_t rbytes = (uint32_t)(re * sizeof(C));
  const size_t sstride = round128(rbytes);
  const int K = a.P - 1, m = twist_index(K), nb = K - 1 - m;
  const int nuse[2] = {2 * m + 1, nb > 0 ? 2 * nb + 1 : 0};
  C* rz = reinterpret_cast<C*>(smem_raw + 256 + (size_t)2 * S2 * sstride);
  const C* red = reinterpret_cast<const C*>(a.red) + d.red_off;
  const int tid = threadIdx.x;
  const int wpc = ((int)blockDim.x - P2_PROD_THREADS) / (P2W * 32);   // RHS per CTA
  auto stage = [&](int h, int u) { return reinterpret_cast<C*>(smem_raw + 256 + (size_t)(h * S2 + u % S2) * sstride); };
  // separator of use u of half h
  auto slot_of = [&](int h, int u) {
    if (h == 0) return u <= m ? u : 2 * m - u;              // 0..m-1, m, m-1..0
    return u < nb ? K - 1 - u : m + (u - nb);               // K-1..m+1, m..K-1
  };

  if (tid == 0) {
    for (int u = 0; u < 2 * S2; ++u) {
      mbar_init(&full[u], 1);
      mbar_init(&empty[u], NP * wpc);    // every column part of every RHS releases each use
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= P2W * wpc * 32) {
    const int pw = (tid - P2W * wpc * 32) >> 5;
    const int h = pw / PPH, sub = pw % PPH;
    if ((tid & 31) == 0 && nuse[h] > sub)
      ring_producer(
          full + h * S2, empty + h * S2, S2, nuse[h], a.spin, a.status, front,
          [&](int t) {
            mbar_arrive_expect_tx(&full[h * S2 + t % S2], rbytes);
            tma_bulk_g2s(stage(h, t), red + (long long)slot_of(h, t) * re, rbytes, &full[h * S2 + t % S2]);
          },
          sub, PPH);
    return;
  }
  const int lane = tid & 31, wq = tid >> 5;
  const int rhs = wq % wpc, role = wq / wpc, half = role / NP, part = role % NP;
  const int q0 = part * WH;          // first column of this warp's part
  const int r = blockIdx.y * wpc + rhs;
  const bool valid = r < a.R;
  const int rr = valid ? r : (a.R - 1);
  const int pl = lane < W ? lane : 0;
  const int pair_id = 1 + rhs, half_id = 1 + WPC_MAX + 2 * rhs + half;
  const C* rcb = reinterpret_cast<const C*>(a.rc);
  const C* lcb = reinterpret_cast<const C*>(a.lc);
  C* xsb = reinterpret_cast<C*>(a.xs);
  const long long fb = (long long)front * a.P;
  // [0..K-1] rho/psi, [K] x_m, [K+1+half] exchange of the half, then the
  // partial sums [parity][half][part][W]
  C* myrz = rz + (size_t)rhs * ((K + 3) * W + 8 * W);
  C* xm = myrz + (size_t)K * W;
  C* xch = myrz + (size_t)(K + 1 + half) * W;
  C* pbuf = myrz + (size_t)(K + 3) * W;
  auto my_part = [&](int par) { return pbuf + ((par * 2 + half) * 2 + part) * W; };
  auto other_part = [&](int par) { return pbuf + ((par * 2 + half) * 2 + (1 - part)) * W; };
  uint64_t* fl = full + half * S2;
  uint64_t* em = empty + half * S2;
  // rho_k of this half's separators (top: 0..m, bottom: m+1..K-1); both
  // parts write the same values
  const int k_lo = half == 0 ? 0 : m + 1, k_hi = half == 0 ? m + 1 : K;
  for (int k0 = k_lo; k0 < k_hi; k0 += 16) {
    C v1[16], v2[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int k = min(k0 + q, k_hi - 1);
      v1[q] = rcb[((fb + k) * a.R + rr) * W + pl];
      v2[q] = lcb[((fb + k + 1) * a.R + rr) * W + pl];
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (k0 + q < k_hi && lane < W) myrz[(k0 + q) * W + lane] = C{-(v1[q].re + v2[q].re), -(v1[q].im + v2[q].im)};
  }
  __syncwarp();
  // partial sum over this part's columns of row pl of a W x W block (row
  // stride LDP) times a W-vector in shared memory.  Rows and vectors start on
  // 16-byte boundaries (W and WH even), so both move two complex values per
  // access; the row reads of one quarter warp fall in distinct bank groups.
  auto part_dot = [&](const C* Mrow, const C* vec) {
    C s[4] = {C{0, 0}, C{0, 0}, C{0, 0}, C{0, 0}};
#pragma unroll
    for (int q = 0; q < WH; q += 2) {
      C m0, m1, p0, p1;
      ld2(Mrow + q0 + q, m0, m1);
      ld2(vec + q0 + q, p0, p1);
      cfma(s[q & 3], m0, p0);
      cfma(s[(q & 3) + 1], m1, p1);
    }
    return cadd(cadd(s[0], s[1]), cadd(s[2], s[3]));
  };
  // partial of F^t x over this part's rows of F (F's column pl held in fc)
  auto fcol_dot = [&](const C (&fc)[WH], const C* xv) {
    C s[4] = {C{0, 0}, C{0, 0}, C{0, 0}, C{0, 0}};
#pragma unroll
    for (int q = 0; q < WH; q += 2) {
      C x0, x1;
      ld2(xv + q0 + q, x0, x1);
      cfma(s[q & 3], fc[q], x0);
      cfma(s[(q & 3) + 1], fc[q + 1], x1);
    }
    return cadd(cadd(s[0], s[1]), cadd(s[2], s[3]));
  };
  auto load_fcol = [&](C (&fc)[WH], const C* Fblk) {   // column pl of F, this part's rows
#pragma unroll
    for (int q = 0; q < WH; ++q) fc[q] = Fblk[(q0 + q) * LDP + pl];
  };
  // both parts publish their partial sums and meet; the result is the AND of
  // `landed` over the two warps, and on success `total` is part 0's partial
  // plus part 1's in that order (the same bits in both warps)
  int sc = 0;
  auto exchange = [&](C own, bool landed, C& total) {
    if constexpr (NP == 1) {        // one warp per half: its own agreement
      total = own;
      return landed;
    }
    const int par = sc++ & 1;
    if (lane < W) my_part(par)[lane] = own;
    const bool both = named_barrier_and(half_id, 64, landed);
    if (both) {
      const C oth = other_part(par)[pl];
      total = part == 0 ? cadd(own, oth) : cadd(oth, own);
    }
    return both;
  };
  auto waitp = [&](int u) { return __all_sync(0xffffffffu, mbar_wait_bounded(&fl[u % S2], (u / S2) & 1, a.spin)); };
  auto release = [&](int u) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&em[u % S2]);
  };
  bool ok = true;
  int t = 0;
  // ---- forward half chains: every step ends with the parts' exchange, so a
  // step with no product (the first) still carries the wait agreement
  if (half == 0) {
    for (int k = 0; k < m; ++k, ++t) {
      const bool landed = waitp(t);
      const C v = myrz[k * W + pl];            // rho_k, read before the exchange
      C own{0, 0}, tot{0, 0};
      if (landed && k > 0) own = part_dot(stage(0, t) + W * LDP + pl * LDP, myrz + (k - 1) * W);
      ok = exchange(own, landed, tot);
      if (!ok) break;
      if (k > 0 && lane < W) myrz[k * W + lane] = csub(v, tot);
      release(t);
    }
  } else {
    for (int u = 0; u < nb; ++u, ++t) {
      const int k = K - 1 - u;
      const bool landed = waitp(t);
      const C v = myrz[k * W + pl];
      C own{0, 0}, tot{0, 0};
      if (landed && k < K - 1) own = part_dot(stage(1, t) + W * LDP + pl * LDP, myrz + (k + 1) * W);
      ok = exchange(own, landed, tot);
      if (!ok) break;
      if (k < K - 1 && lane < W) myrz[k * W + lane] = csub(v, tot);
      release(t);
    }
  }
  ok = named_barrier_and(pair_id, P2W * 32, ok);
  // ---- twist (top half)
  C fcol[WH];
  if (half == 0 && ok) {
    const bool landed = waitp(t);
    const C* Gm = stage(0, t);
    const C v = myrz[m * W + pl];
    C own{0, 0}, tot{0, 0}, x{0, 0};
    if (landed) {
      if (m >= 1) own = part_dot(Gm + W * LDP + pl * LDP, myrz + (m - 1) * W);
      if (m < K - 1) own = cadd(own, part_dot(Gm + 2 * W * LDP + pl * LDP, myrz + (m + 1) * W));
    }
    ok = exchange(own, landed, tot);
    own = C{0, 0};
    if (ok) {
      if (lane < W) xch[lane] = csub(v, tot);  // both parts write the same vector
      __syncwarp();
      own = part_dot(Gm + pl * LDP, xch);     // Gamma_m is symmetric: row pl for column pl
    }
    ok = exchange(own, ok, x);
    if (ok) {
      load_fcol(fcol, Gm + W * LDP);           // F_m
      __syncwarp();
      if (lane < W) { xm[lane] = x; xch[lane] = x; }
      if (valid && part == 0 && lane < W) xsb[((fb + m) * a.R + r) * W + lane] = x;
      release(t);
      ++t;
    }
  }
  ok = named_barrier_and(pair_id, P2W * 32, ok);
  // ---- backward half chains
  if (half == 0 && ok) {
    for (int k = m - 1; k >= 0; --k, ++t) {
      const bool landed = waitp(t);
      const C* Gm = stage(0, t);
      C own{0, 0}, x{0, 0};
      if (landed) own = csub(part_dot(Gm + pl * LDP, myrz + k * W), fcol_dot(fcol, xch));   // Gamma_k psi_k - F_{k+1}^t x_{k+1}
      ok = exchange(own, landed, x);
      if (!ok) break;
      load_fcol(fcol, Gm + W * LDP);           // F_k for the next step
      __syncwarp();
      if (lane < W) xch[lane] = x;
      if (valid && part == 0 && lane < W) xsb[((fb + k) * a.R + r) * W + lane] = x;
      release(t);
    }
  } else if (half == 1 && ok && nb > 0) {
    // F'_m column from the twist slot, then k = m+1 .. K-1
    const bool landed = waitp(t);
    if (landed) load_fcol(fcol, stage(1, t) + 2 * W * LDP);
    C dummy{0, 0};
    ok = exchange(C{0, 0}, landed, dummy);
    if (ok) {
      __syncwarp();
      if (lane < W) xch[lane] = xm[lane];
      release(t);
      ++t;
      for (int k = m + 1; k < K; ++k, ++t) {
        const bool landed2 = waitp(t);
        const C* Gk = stage(1, t);
        C own{0, 0}, x{0, 0};
        if (landed2) own = csub(part_dot(Gk + pl * LDP, myrz + k * W), fcol_dot(fcol, xch));   // - F'_{k-1}^t x_{k-1}
        ok = exchange(own, landed2, x);
        if (!ok) break;
        load_fcol(fcol, Gk + W * LDP);
        __syncwarp();
        if (lane < W) xch[lane] = x;
        if (valid && part == 0 && lane < W) xsb[((fb + k) * a.R + r) * W + lane] = x;
        release(t);
      }
    }
  }
  if (!ok && lane == 0) set_status(a.status, HS_ETIMEOUT, front, -2);
}

// ---------------------------------------------------------------- phase 3
// Back substitution over the chunk's interior columns from the right
// separator: x_j = z_j - G_j (C_j x_{j+1}); output rows get the left-spike
// correction -W_j beta, beta = C_{l-1} x_{left separator}.  Each ring stage
// brings the column payload and the CTA's tile of the stored z_j.  Thread
// (rg, hg) owns rows rg + NRG*i and RHS 2hg, 2hg+1 of the group.
template <typename R, int W, bool SM>
__global__ void __launch_bounds__(Tile13<R, W, SM>::NCONS + 32 * P13) phase3_kernel(SweepArgs a) {
  using C = cplx<R>;
  using TL = Tile13<R, W, SM>;
  constexpr int ROWS = TL::ROWS, NRG = TL::NRG, RPT = TL::RPT, RG = TL::RG, NCONS = TL::NCONS, LDR = TL::LDR;
  constexpr int LDP = W + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + S13;
  const int front = blockIdx.z, k = blockIdx.x;
  const BlockDesc& d = a.blk[front];
  const long long pe = payload_elems(W, d.d_out);
  const uint32_t pbytes = (uint32_t)(pe * sizeof(C));
  const size_t pstride = round128(pbytes);
  const size_t vb = round128((size_t)W * LDR * sizeof(C));
  const size_t sstride = pstride + vb;
  C* tvbuf = reinterpret_cast<C*>(smem_raw + 256 + S13 * sstride);            // [2][W][LDR]
  C* beta = reinterpret_cast<C*>(smem_raw + 256 + S13 * sstride + 2 * vb);     // [W][LDR]
  C* olds = reinterpret_cast<C*>(smem_raw + 256 + S13 * sstride + 3 * vb);     // [OD][d_out][LDR]
  const C* fac = reinterpret_cast<const C*>(a.fac) + d.fac_off;
  const int tid = threadIdx.x;
  const int rbase = blockIdx.y * RG;
  const int nvalid = min(RG, a.R - rbase);
  const uint32_t zbytes = (uint32_t)((size_t)nvalid * W * sizeof(C));
  const int l = k * a.L;
  const int rgt = (k < a.P - 1) ? (k + 1) * a.L - 2 : a.n - 1;
  const int ncol = rgt - l + 1;
  const bool has_left = k > 0, has_right = k < a.P - 1;
  const C* zst = reinterpret_cast<const C*>(a.z) + ((long long)front * a.n * a.R) * W;
  auto pay = [&](int t) { return reinterpret_cast<C*>(smem_raw + 256 + (size_t)(t % S13) * sstride); };
  auto ztile = [&](int t) { return reinterpret_cast<C*>(smem_raw + 256 + (size_t)(t % S13) * sstride + pstride); };

  if (tid == 0) {
    for (int u = 0; u < S13; ++u) {
      mbar_init(&full[u], 1);
      mbar_init(&empty[u], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= NCONS) {
    const int sub = (tid - NCONS) >> 5;
    if ((tid & 31) == 0 && sub < ncol)
      ring_producer(
          full, empty, S13, ncol, a.spin, a.status, front,
          [&](int t) {
            const int j = rgt - t;
            mbar_arrive_expect_tx(&full[t % S13], pbytes + zbytes);
            tma_bulk_g2s(pay(t), fac + (long long)j * pe, pbytes, &full[t % S13]);
            tma_bulk_g2s(ztile(t), zst + ((long long)j * a.R + rbase) * W, zbytes, &full[t % S13]);
          },
          sub, P13);
    return;
  }
  const int rg = tid % NRG, hg = tid / NRG;
  const int c0 = hg * RPT;
  bool valid[RPT];
  int rr[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    valid[q] = rbase + c0 + q < a.R;
    rr[q] = min(rbase + c0 + q, a.R - 1);
  }
  const long long fb = (long long)front * a.P;
  const C* xsb = reinterpret_cast<const C*>(a.xs);
  C* u = reinterpret_cast<C*>(a.u);
  const long long rs = (long long)a.n * a.R;
  const bool bwd = a.mode == 1;
  // beta = C_{l-1} x_{left separator}; x = x_{right separator} (own tile)
  C x[RPT][ROWS];
  {
    const C* cl = fac + (long long)(l > 0 ? l - 1 : 0) * pe + (long long)(W + d.d_out) * LDP;
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      const int p = rg + NRG * i;
      C bv[RPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        bv[q] = has_left ? cmul(cl[p], xsb[((fb + k - 1) * a.R + rr[q]) * W + p]) : C{0, 0};
        x[q][i] = has_right ? xsb[((fb + k) * a.R + rr[q]) * W + p] : C{0, 0};
      }
      st2(beta + p * LDR + c0, bv[0], bv[1]);
    }
  }
  // beta does not change along the chunk: for complex64 windows up to 24 rows
  // every thread keeps the beta column of its two RHS in registers, so that
  // the spike correction reads only W_j from shared memory
  constexpr bool BREG = sizeof(R) == 4 && W <= 24;
  C bb[BREG ? W : 1][RPT];
  if constexpr (BREG) {
    consumer_barrier(NCONS);
#pragma unroll
    for (int kk = 0; kk < W; ++kk) {
      if (has_left) ld2(beta + kk * LDR + c0, bb[kk][0], bb[kk][1]);
      else bb[kk][0] = bb[kk][1] = C{0, 0};
    }
  }
  bool isout[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) isout[i] = (rg + NRG * i >= d.out_off) && (rg + NRG * i < d.out_off + d.d_out);
  // backward stages subtract from the previous u: each thread copies its own
  // output entries of column rgt - t into staging slot t % OD (one commit
  // group per column, empty when there is nothing to copy)
  auto old_slot = [&](int t, int i) {
    return olds + ((size_t)(t % OD) * d.d_out + (rg + NRG * i - d.out_off)) * LDR + c0;
  };
  auto issue_old = [&](int t) {
    if (t < ncol) {
      const int j = rgt - t;
#pragma unroll
      for (int i = 0; i < ROWS; ++i)
        if (isout[i]) {
          C* dst = old_slot(t, i);
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const C* src = u + (long long)(d.wlo + rg + NRG * i - 1) * rs + (long long)j * a.R + rr[q];
            if constexpr (sizeof(R) == 4) cp_async8(dst + q, src);
            else cp_async16(dst + q, src);
          }
        }
    }
    cp_async_commit();
  };
  auto read_old = [&](int t, C (&uo)[RPT][ROWS]) {
    cp_async_wait<OD - 1>();      // column t's group has landed
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
      if (isout[i]) {
        const C* src = old_slot(t, i);
#pragma unroll
        for (int q = 0; q < RPT; ++q) uo[q][i] = src[q];
      }
  };
  // register prefetch of the same entries (16-RHS tile)
  auto load_old = [&](C (&o)[RPT][ROWS], int j) {
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int i = 0; i < ROWS; ++i)
        o[q][i] = (bwd && isout[i]) ? u[(long long)(d.wlo + rg + NRG * i - 1) * rs + (long long)j * a.R + rr[q]]
                                    : C{0, 0};
  };
  bool ok = true;
  auto step = [&](int t, const C (&uo)[RPT][ROWS]) {
    const int j = rgt - t;
    const C* G = pay(t);
    const C* V = G + W * LDP;
    const C* cc = V + d.d_out * LDP;
    const C* zt = ztile(t);
    C* TV = tvbuf + (t & 1) * (W * LDR);
    const bool landed = mbar_wait_bounded(&full[t % S13], (t / S13) & 1, a.spin);
    // tv = C_j x_{j+1} (own tile), shared through shared memory
    if (landed) {
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        const C ci = cc[rg + NRG * i];
        st2(TV + (rg + NRG * i) * LDR + c0, cmul(ci, x[0][i]), cmul(ci, x[1][i]));
      }
    }
    ok = consumer_barrier_and(NCONS, landed);
    if (!ok) return;
    if (tid == 0 && t > 0) mbar_arrive(&empty[(t - 1) % S13]);   // every read of stage t-1 is done
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int i = 0; i < ROWS; ++i) x[q][i] = zt[(c0 + q) * W + rg + NRG * i];
#pragma unroll
    for (int kk = 0; kk < W; kk += 2) {
      C g0[ROWS], g1[ROWS], t00, t01, t10, t11;
#pragma unroll
      for (int i = 0; i < ROWS; ++i) ld2(G + (rg + NRG * i) * LDP + kk, g0[i], g1[i]);
      ld2(TV + kk * LDR + c0, t00, t01);
      ld2(TV + (kk + 1) * LDR + c0, t10, t11);
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        cfms(x[0][i], g0[i], t00);
        cfms(x[1][i], g0[i], t01);
        cfms(x[0][i], g1[i], t10);
        cfms(x[1][i], g1[i], t11);
      }
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      if (isout[i]) {
        const int p = rg + NRG * i;
        C o0 = x[0][i], o1 = x[1][i];
        if (BREG && has_left) {
          const C* vr = V + (p - d.out_off) * LDP;
#pragma unroll
          for (int kk = 0; kk < W; kk += 2) {
            C v0, v1;
            ld2(vr + kk, v0, v1);
            cfms(o0, v0, bb[kk][0]);
            cfms(o1, v0, bb[kk][1]);
            cfms(o0, v1, bb[BREG ? kk + 1 : 0][0]);
            cfms(o1, v1, bb[BREG ? kk + 1 : 0][1]);
          }
        } else if (has_left) {
          const C* vr = V + (p - d.out_off) * LDP;
#pragma unroll 4
          for (int kk = 0; kk < W; kk += 2) {
            C v0, v1, b00, b01, b10, b11;
            ld2(vr + kk, v0, v1);
            ld2(beta + kk * LDR + c0, b00, b01);
            ld2(beta + (kk + 1) * LDR + c0, b10, b11);
            cfms(o0, v0, b00);
            cfms(o1, v0, b01);
            cfms(o0, v1, b10);
            cfms(o1, v1, b11);
          }
        }
        C* up = u + (long long)(d.wlo + p - 1) * rs + (long long)j * a.R + rbase + c0;
        if (valid[0]) up[0] = bwd ? csub(uo[0][i], o0) : o0;
        if (valid[1]) up[1] = bwd ? csub(uo[1][i], o1) : o1;
      }
    }
  };
  if constexpr (!SM) {
    if (bwd)
      for (int t = 0; t < OD - 1; ++t) issue_old(t);
    for (int t = 0; t < ncol; ++t) {
      C uo[RPT][ROWS] = {};
      if (bwd) {
        issue_old(t + OD - 1);
        read_old(t, uo);
      }
      step(t, uo);
      if (!ok) break;
    }
    if (bwd) cp_async_wait_all();
  } else {
    C o0[RPT][ROWS], o1[RPT][ROWS];
    load_old(o0, rgt);
    if (ncol > 1) load_old(o1, rgt - 1);
    for (int t = 0; t < ncol; t += 2) {
      step(t, o0);
      if (!ok) break;
      if (t + 2 < ncol) load_old(o0, rgt - t - 2);
      if (t + 1 < ncol) {
        step(t + 1, o1);
        if (!ok) break;
        if (t + 3 < ncol) load_old(o1, rgt - t - 3);
      }
    }
  }
  if (!ok) {
    if ((tid & 31) == 0) set_status(a.status, HS_ETIMEOUT, front, rgt);
    return;
  }
  consumer_barrier(NCONS);
  if (tid == 0) mbar_arrive(&empty[(ncol - 1) % S13]);
  if (has_right) {
    const int sc = rgt + 1;
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
      if (isout[i]) {
        const int p = rg + NRG * i;
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (valid[q]) {
            const C o = xsb[((fb + k) * a.R + rr[q]) * W + p];
            C* up = u + (long long)(d.wlo + p - 1) * rs + (long long)sc * a.R + rbase + c0 + q;
            *up = bwd ? csub(*up, o) : o;
          }
      }
  }
}

template <typename R, int W>
void set_attrs_w() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(phase1_kernel<R, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(phase3_kernel<R, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(phase1_kernel<R, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(phase3_kernel<R, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(phase2_kernel<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
}

template <typename R>
void set_attrs() {
  set_attrs_w<R, 8>(); set_attrs_w<R, 12>(); set_attrs_w<R, 16>(); set_attrs_w<R, 24>(); set_attrs_w<R, 32>();
}

// One stage: chunk tiles of 16 RHS when the stage has at most 16, else the
// full tile.
template <typename R, int W, bool SM>
int run_stage_t(const Plan& p, SweepArgs a, cudaStream_t s) {
  using TL = Tile13<R, W, SM>;
  const int dmax = std::max(a.blk[0].d_out, a.nfront > 1 ? a.blk[1].d_out : 0);
  const size_t sm1 = tile_smem<R, W, SM>(dmax, false);
  const size_t sm3 = tile_smem<R, W, SM>(dmax, true);
  set_attrs_w<R, W>();
  const int wpc = p.opt.sep_rhs_per_cta > 0 ? std::min(p.opt.sep_rhs_per_cta, wpc_max<R>())
                                            : phase2_wpc(a.R, a.nfront, wpc_max<R>());
  if (sm1 > 220 * 1024 || sm3 > 220 * 1024 || phase2_smem<R, W>(a.P - 1, wpc) > 220 * 1024) return HS_EUNSUPPORTED;
  dim3 g13(a.P, (a.R + TL::RG - 1) / TL::RG, a.nfront);
  note_launch();
  phase1_kernel<R, W, SM><<<g13, TL::NCONS + 32 * P13, sm1, s>>>(a);
  if (a.P > 1) {
    dim3 g2(1, (a.R + wpc - 1) / wpc, a.nfront);
    note_launch();
    phase2_kernel<R, W><<<g2, 2 * npart<R>() * wpc * 32 + P2_PROD_THREADS, phase2_smem<R, W>(a.P - 1, wpc), s>>>(a);
  }
  note_launch();
  phase3_kernel<R, W, SM><<<g13, TL::NCONS + 32 * P13, sm3, s>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

template <typename R, int W>
int run_stage_w(const Plan& p, SweepArgs a, cudaStream_t s) {
  return a.R <= Tile13<R, W, true>::RG ? run_stage_t<R, W, true>(p, a, s) : run_stage_t<R, W, false>(p, a, s);
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
int sweep_t(const Plan& p, const SweepWork& w, int nrhs, cudaStream_t s) {
  SweepArgs a{};
  a.n = p.n; a.L = p.L; a.P = p.P; a.R = nrhs;
  a.fac = p.d_fac; a.red = p.d_red; a.u = w.u;
  a.z = w.z; a.rc = w.rc; a.lc = w.lc; a.xs = w.xs; a.ps = w.ps;
  if (sizeof(R) == 4) { a.a2 = p.f_a2; a.inv_s1 = p.f_inv_s1; }
  else { a.a2 = p.d_a2; a.inv_s1 = p.d_inv_s1; }
  a.status = p.d_status;
  a.spin = p.opt.spin_budget;
  int st = HS_OK;
  const int S = (int)p.stages.size();
  // forward sweep of both fronts, or of the single front (v_B = T~_B u_B)
  for (int k = 0; k < S && st == HS_OK; ++k) {
    a.mode = 0; a.nfront = (int)p.stages[k].size();
    a.blk[0] = p.blocks[p.stages[k][0]];
    a.blk[1] = p.blocks[p.stages[k][a.nfront - 1]];
    st = run_stage<R>(p, a, s);
  }
  // middle layer with moving PMLs on both sides (single front: the top
  // block, which has no block above it to correct it afterwards)
  if (st == HS_OK) {
    a.mode = 0; a.nfront = 1;
    a.blk[0] = p.blocks[p.middle];
    a.blk[1] = a.blk[0];
    st = run_stage<R>(p, a, s);
  }
  // backward sweep: u_B = v_B - T~_B (A_{B,next} u_next)
  for (int k = S - 1; k >= 0 && st == HS_OK; --k) {
    a.mode = 1; a.nfront = (int)p.stages[k].size();
    a.blk[0] = p.blocks[p.stages[k][0]];
    a.blk[1] = p.blocks[p.stages[k][a.nfront - 1]];
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

namespace {
template <typename R, int W>
int max_sep_w() {
  int k = 1;
  while (k < 4096 && phase2_smem<R, W>(k + 1, wpc_max<R>()) <= 220 * 1024) ++k;   // the largest CTA
  return k;
}
template <typename R>
int max_sep_r(int W) {
  switch (W) {
    case 8: return max_sep_w<R, 8>();
    case 12: return max_sep_w<R, 12>();
    case 16: return max_sep_w<R, 16>();
    case 24: return max_sep_w<R, 24>();
    default: return max_sep_w<R, 32>();
  }
}
}  // namespace

int max_separators(int W, int prec) {
  return prec == HS_C64 ? max_sep_r<float>(W) : max_sep_r<double>(W);
}

void sweep_prepare_attributes(int prec) {
  if (prec == HS_C64) set_attrs<float>(); else set_attrs<double>();
}

int sweep_launch_work(const Plan& p, const SweepWork& w, int nrhs, cudaStream_t s) {
  return (p.prec == HS_C64) ? sweep_t<float>(p, w, nrhs, s) : sweep_t<double>(p, w, nrhs, s);
}

int sweep_launch(Plan& p, int nrhs, cudaStream_t s) {
  const SweepWork w{p.d_u, p.d_z, p.d_rc, p.d_lc, p.d_xs, p.d_ps};
  return sweep_launch_work(p, w, nrhs, s);
}

namespace {
// Executable graphs of one plan's stage chain, keyed by the number of RHS and
// the scratch buffers the kernels address.
struct SweepGraphs {
  struct Entry {
    int nrhs;
    void* ptrs[6];
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::mutex m;
  std::vector<Entry> list;
  cudaStream_t cap = nullptr;
};
}  // namespace

int sweep_internal(Plan& p, int nrhs, cudaStream_t s, bool graph) {
  auto launch = [&p, nrhs](cudaStream_t c) -> int { return p.dim == 3 ? sweep3(p, nrhs, c) : sweep_launch(p, nrhs, c); };
  if (!graph) return launch(s);
  if (!p.graphs) p.graphs = new SweepGraphs();
  SweepGraphs& gs = *static_cast<SweepGraphs*>(p.graphs);
  std::lock_guard<std::mutex> lock(gs.m);
  void* const ptrs[6] = {p.d_u, p.d_z, p.d_rc, p.d_lc, p.d_xs, p.d_ps};
  for (auto& e : gs.list) {
    if (e.nrhs == nrhs && std::equal(ptrs, ptrs + 6, e.ptrs)) {
      note_launch(e.kernels);
      cudaError_t ce = cudaGraphLaunch(e.exec, s);
      return ce == cudaSuccess ? HS_OK : cuda_status(ce);
    }
  }
  if (p.dim == 2) sweep_prepare_attributes(p.prec);
  if (!gs.cap) HS_CUDA_TRY(cudaStreamCreateWithFlags(&gs.cap, cudaStreamNonBlocking));
  SweepGraphs::Entry e{};
  e.nrhs = nrhs;
  std::copy(ptrs, ptrs + 6, e.ptrs);
  int st = capture_graph(gs.cap, launch, &e.exec, &e.kernels);
  if (st != HS_OK) return st;
  gs.list.push_back(e);
  note_launch(e.kernels);
  cudaError_t ce = cudaGraphLaunch(e.exec, s);
  return ce == cudaSuccess ? HS_OK : cuda_status(ce);
}

void release_sweep_graphs(Plan& p) {
  if (!p.graphs) return;
  SweepGraphs* gs = static_cast<SweepGraphs*>(p.graphs);
  for (auto& e : gs->list) cudaGraphExecDestroy(e.exec);
  if (gs->cap) cudaStreamDestroy(gs->cap);
  delete gs;
  p.graphs = nullptr;
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
  plan_wait(p, s);
  const int n2 = (int)p.npts();
  int st = layout_to_internal(r, dtype, p.d_u, p.prec, n2, nrhs, s);
  if (st == HS_OK) st = sweep_internal(p, nrhs, s, p.opt.graphs != 0);
  if (st == HS_OK) st = layout_from_internal(p.d_u, p.prec, z, dtype, n2, nrhs, s);
  return st;
}
