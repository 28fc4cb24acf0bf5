// 3D: the 7-point operator (Eq. helmd3) and the slab sweep of Sec. 4
// (Algorithms 5 and 6 with the two-front pattern and d layers per step).
//
// Each slab problem H_B lives on the window of w x3 layers of the block and
// all n x n points of the (x1, x2) plane.  Its exact solve is a multifrontal
// LDL^t-style elimination in the order of a nested dissection of the plane
// (Sec. 4.2): the plane is bisected recursively across its longer side; the
// separator line of a node (or all points of a leaf region) is eliminated
// at that node, every plane point keeping its w unknowns of the x3 column
// together.  A node's front holds its own unknowns (S) and the unknowns on
// the ring of plane points just outside its region (Bd, all on ancestor
// separators).  Setup, per level from the leaves up and for all slabs of
// all stages at once:
//   assemble   F = original entries of the node's rows + children's updates
//   invert     G = F11^{-1}                   (Gauss-Jordan, partial pivoting)
//   GEMM       L = F21 G                      (Bd x S)
//   GEMM       U = F22 - L F12                (the update passed to the parent)
// The solve with a right-hand side X over the slab (Algorithm 6 applies T~
// as H_B^{-1} of a vector that lives on a few layers), per level:
//   leaves up:  t = G X_own (kept),  X_bnd -= L X_own
//   root down:  X_own = t - L^t X_bnd          (F is complex symmetric)
// T~_B is unique, so this equals the oracle's sparse LU solve up to rounding.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>
#include "hs_internal.cuh"
#include "hs_device.cuh"
#include "hs3d.cuh"
#include "hs3d_tc.cuh"

namespace hs {
namespace {

// ---------------------------------------------------------------- nested dissection
// Front point position P of plane point (i, j) in node nd, or -1 if the point
// is eliminated by a descendant or lies outside the front.  Own points come
// first, then the four boundary segments (left, right, bottom, top).
__host__ __device__ inline int front_pos(const Node3& nd, int i, int j, int n) {
  if (i >= nd.x0 && i < nd.x1 && j >= nd.y0 && j < nd.y1) {
    if (nd.kind == 0) return (j - nd.y0) * (nd.x1 - nd.x0) + (i - nd.x0);
    if (nd.kind == 1) return (i == nd.mid) ? (j - nd.y0) : -1;
    return (j == nd.mid) ? (i - nd.x0) : -1;
  }
  int P = nd.nown;
  const int h = nd.y1 - nd.y0, wd = nd.x1 - nd.x0;
  if (nd.x0 > 0) { if (i == nd.x0 - 1 && j >= nd.y0 && j < nd.y1) return P + (j - nd.y0); P += h; }
  if (nd.x1 < n) { if (i == nd.x1 && j >= nd.y0 && j < nd.y1) return P + (j - nd.y0); P += h; }
  if (nd.y0 > 0) { if (j == nd.y0 - 1 && i >= nd.x0 && i < nd.x1) return P + (i - nd.x0); P += wd; }
  if (nd.y1 < n) { if (j == nd.y1 && i >= nd.x0 && i < nd.x1) return P + (i - nd.x0); }
  return -1;
}

// Plane index j * n + i of front point position P of node nd.
__host__ __device__ inline int front_point(const Node3& nd, int P, int n) {
  if (P < nd.nown) {
    if (nd.kind == 0) { const int wd = nd.x1 - nd.x0; return (nd.y0 + P / wd) * n + nd.x0 + P % wd; }
    if (nd.kind == 1) return (nd.y0 + P) * n + nd.mid;
    return nd.mid * n + nd.x0 + P;
  }
  int q = P - nd.nown;
  const int h = nd.y1 - nd.y0, wd = nd.x1 - nd.x0;
  if (nd.x0 > 0) { if (q < h) return (nd.y0 + q) * n + nd.x0 - 1; q -= h; }
  if (nd.x1 < n) { if (q < h) return (nd.y0 + q) * n + nd.x1; q -= h; }
  if (nd.y0 > 0) { if (q < wd) return (nd.y0 - 1) * n + nd.x0 + q; q -= wd; }
  return nd.y1 * n + nd.x0 + q;
}

int build_nd(std::vector<Node3>& nodes, int x0, int x1, int y0, int y1, int level, int parent, int n) {
  Node3 nd{};
  nd.x0 = x0; nd.x1 = x1; nd.y0 = y0; nd.y1 = y1;
  nd.level = level; nd.parent = parent;
  nd.child[0] = nd.child[1] = -1;
  const int wd = x1 - x0, h = y1 - y0;
  if (wd * h <= 16 || (wd <= 3 && h <= 3)) {
    nd.kind = 0;
    nd.nown = wd * h;
  } else if (wd >= h) {
    nd.kind = 1;
    nd.mid = (x0 + x1) / 2;
    nd.nown = h;
  } else {
    nd.kind = 2;
    nd.mid = (y0 + y1) / 2;
    nd.nown = wd;
  }
  nd.nbnd = (x0 > 0 ? h : 0) + (x1 < n ? h : 0) + (y0 > 0 ? wd : 0) + (y1 < n ? wd : 0);
  const int id = (int)nodes.size();
  nodes.push_back(nd);
  if (nd.kind == 1) {
    if (nd.mid > x0) nodes[id].child[0] = build_nd(nodes, x0, nd.mid, y0, y1, level + 1, id, n);
    if (nd.mid + 1 < x1) nodes[id].child[1] = build_nd(nodes, nd.mid + 1, x1, y0, y1, level + 1, id, n);
  } else if (nd.kind == 2) {
    if (nd.mid > y0) nodes[id].child[0] = build_nd(nodes, x0, x1, y0, nd.mid, level + 1, id, n);
    if (nd.mid + 1 < y1) nodes[id].child[1] = build_nd(nodes, x0, x1, nd.mid + 1, y1, level + 1, id, n);
  }
  return id;
}

// ---------------------------------------------------------------- coefficients
struct Coef3 {
  int n;
  const c128* inv_s;    // 1/s(k h), k = 0..n+1 (every axis)
  const c128* a;        // s((k+1/2) h)/h^2, k = 0..n
  const double* cinv2;  // 1/c^2 per point [k][j][i]
  const c128* s3;       // per block window: 1/s3(q), s3(q+1/2)/h^2, s3(q-1/2)/h^2
  c128 wst2;            // (omega + i alpha)^2
};

// Eq. helmd3 entries of H_B at plane point (i, j) (0-based), window layer q:
// couplings E, W, N, S (plane), Up, Dn (x3) and the diagonal.
struct Row3 { c128 E, W, N, S, Up, Dn, D; };
__device__ inline Row3 row3(const Coef3& c, const BlockDesc& d, int i, int j, int q) {
  const c128* s3 = c.s3 + d.s2_off;
  const c128 is1 = c.inv_s[i + 1], is2 = c.inv_s[j + 1], is3 = s3[q];
  const c128 i12 = cmul(is1, is2);
  Row3 r;
  r.E = cmul(c.a[i + 1], cmul(is2, is3));
  r.W = cmul(c.a[i], cmul(is2, is3));
  r.N = cmul(c.a[j + 1], cmul(is1, is3));
  r.S = cmul(c.a[j], cmul(is1, is3));
  r.Up = cmul(s3[d.w + q], i12);
  r.Dn = cmul(s3[2 * d.w + q], i12);
  const int k0 = d.wlo - 1 + q;
  const double ci2 = c.cinv2[((long long)k0 * c.n + j) * c.n + i];
  const c128 m = cmul(cscale(c.wst2, ci2), cmul(i12, is3));
  r.D = csub(m, cadd(cadd(cadd(r.E, r.W), cadd(r.N, r.S)), cadd(r.Up, r.Dn)));
  return r;
}

// ---------------------------------------------------------------- setup kernels
struct SetupItem {
  int block, node, S, Bd;   // S = nown * w, Bd = nbnd * w
  long long f_off;          // front (S+Bd)^2 in its level buffer
  long long g_off, l_off;   // G (S x S) and L (Bd x S) in the factor storage
  int child_item[2];        // items of the children (previous level), -1 if none
};

template <typename R>
__global__ void __launch_bounds__(256) assemble_kernel(Coef3 c, const BlockDesc* blocks, const Node3* nodes,
                                                       const SetupItem* items, cplx<R>* F, const SetupItem* citems,
                                                       const cplx<R>* Fchild) {
  using C = cplx<R>;
  const SetupItem it = items[blockIdx.x];
  const BlockDesc d = blocks[it.block];
  const Node3 nd = nodes[it.node];
  const int n = c.n, w = d.w;
  const int LD = it.S + it.Bd;
  C* f = F + it.f_off;
  for (long long e = threadIdx.x; e < (long long)LD * LD; e += blockDim.x) f[e] = C{0, 0};
  __syncthreads();
  // original entries of the node's own rows (and their symmetric boundary columns)
  for (int row = threadIdx.x; row < it.S; row += blockDim.x) {
    const int a = row / w, q = row % w;
    const int p = front_point(nd, a, n), i = p % n, j = p / n;
    const Row3 r = row3(c, d, i, j, q);
    f[(long long)row * LD + row] = ccast<R>(r.D);
    if (q + 1 < w) f[(long long)row * LD + row + 1] = ccast<R>(r.Up);
    if (q > 0) f[(long long)row * LD + row - 1] = ccast<R>(r.Dn);
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    const c128 cf[4] = {r.E, r.W, r.N, r.S};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int ii = i + di[t], jj = j + dj[t];
      if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
      const int P = front_pos(nd, ii, jj, n);
      if (P < 0) continue;                      // eliminated below: in a child's update
      const int col = P * w + q;
      f[(long long)row * LD + col] = ccast<R>(cf[t]);
      if (P >= nd.nown) f[(long long)col * LD + row] = ccast<R>(cf[t]);
    }
  }
  // extend-add of the children's updates U = F22 (one child at a time)
  for (int ch = 0; ch < 2; ++ch) {
    __syncthreads();
    const int ci = it.child_item[ch];
    if (ci < 0) continue;
    const SetupItem cit = citems[ci];
    const Node3 cn = nodes[cit.node];
    const int LDc = cit.S + cit.Bd;
    const C* U = Fchild + cit.f_off + (long long)cit.S * LDc + cit.S;
    for (long long e = threadIdx.x; e < (long long)cit.Bd * cit.Bd; e += blockDim.x) {
      const int r1 = (int)(e / cit.Bd), r2 = (int)(e % cit.Bd);
      const int b1 = r1 / w, q1 = r1 % w, b2 = r2 / w, q2 = r2 % w;
      const int p1 = front_point(cn, cn.nown + b1, n), p2 = front_point(cn, cn.nown + b2, n);
      const int P1 = front_pos(nd, p1 % n, p1 / n, n), P2 = front_pos(nd, p2 % n, p2 / n, n);
      if (P1 < 0 || P2 < 0) continue;   // cannot happen for a dissection tree; keeps writes in bounds
      C& dst = f[(long long)(P1 * w + q1) * LD + P2 * w + q2];
      dst = cadd(dst, U[(long long)r1 * LDc + r2]);
    }
  }
}

// In-place Gauss-Jordan inverse (partial pivoting by rows, undone by column
// swaps) of the leading S x S block of each front; a zero pivot records
// HS_EBREAKDOWN.  One CTA per front; the matrix stays in global memory (L2).
template <typename R>
__global__ void __launch_bounds__(512) invert_kernel(const SetupItem* items, cplx<R>* F, int* status) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const SetupItem it = items[blockIdx.x];
  const int S = it.S, LD = it.S + it.Bd;
  C* A = F + it.f_off;
  C* colk = reinterpret_cast<C*>(smraw);
  C* rowk = colk + S;
  int* piv = reinterpret_cast<int*>(rowk + S);
  __shared__ R bestv[32];
  __shared__ int besti[32];
  __shared__ int pr_s;
  bool ok = true;
  for (int k = 0; k < S; ++k) {
    R v = R(-1);
    int idx = k;
    for (int i = k + threadIdx.x; i < S; i += blockDim.x) {
      const R a = cabs2(A[(long long)i * LD + k]);
      if (a > v) { v = a; idx = i; }
    }
    for (int m = 16; m > 0; m >>= 1) {
      const R ov = Shfl<R>::xr(v, m);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, m);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bestv[threadIdx.x >> 5] = v; besti[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      R bv = bestv[0];
      int bi = besti[0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
        if (bestv[q] > bv || (bestv[q] == bv && besti[q] < bi)) { bv = bestv[q]; bi = besti[q]; }
      if (!(bv > R(0)) || !isfinite(bv)) { ok = false; bi = k; }
      pr_s = bi;
      piv[k] = bi;
    }
    __syncthreads();
    const int pr = pr_s;
    if (pr != k)
      for (int j = threadIdx.x; j < S; j += blockDim.x) {
        const C t = A[(long long)k * LD + j];
        A[(long long)k * LD + j] = A[(long long)pr * LD + j];
        A[(long long)pr * LD + j] = t;
      }
    __syncthreads();
    const C pinv = cinv(A[(long long)k * LD + k]);
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
      colk[i] = A[(long long)i * LD + k];
      rowk[i] = (i == k) ? pinv : cmul(A[(long long)k * LD + i], pinv);
    }
    __syncthreads();
    // rank-1 update: rows over warps, columns over lanes (coalesced rows)
    const int nw = (int)(blockDim.x >> 5), lane = threadIdx.x & 31;
    for (int i = (int)(threadIdx.x >> 5); i < S; i += nw) {
      C* Ai = A + (long long)i * LD;
      const C ci = colk[i];
      if (i == k) {
        for (int j = lane; j < S; j += 32) Ai[j] = rowk[j];
      } else {
        for (int j = lane; j < S; j += 32) Ai[j] = (j == k) ? cmul(C{-ci.re, -ci.im}, pinv) : csub(Ai[j], cmul(ci, rowk[j]));
      }
    }
    __syncthreads();
  }
  for (int k = S - 1; k >= 0; --k) {
    const int pr = piv[k];
    if (pr != k)
      for (int i = threadIdx.x; i < S; i += blockDim.x) {
        const C t = A[(long long)i * LD + k];
        A[(long long)i * LD + k] = A[(long long)i * LD + pr];
        A[(long long)i * LD + pr] = t;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0 && !ok) set_status(status, HS_EBREAKDOWN, it.block, it.node);
}

// Batched complex GEMM  C = beta C + alpha A B  (64 x 64 tiles, FP32/FP64 FMA).
struct GemmJob {
  const void* A; const void* B; void* C;
  int lda, ldb, ldc, M, N, K;
  int alpha, beta;      // alpha in {1, -1}, beta in {0, 1}
};
struct GemmTile { int job, tm, tn; };

template <typename R>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmJob* jobs, const GemmTile* tiles) {
  using C = cplx<R>;
  __shared__ C As[16][65];
  __shared__ C Bs[16][65];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const C* A = static_cast<const C*>(jb.A);
  const C* B = static_cast<const C*>(jb.B);
  C* Cm = static_cast<C*>(jb.C);
  const int m0 = tl.tm * 64, n0 = tl.tn * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = C{0, 0};
  for (int k0 = 0; k0 < jb.K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < jb.M && gk < jb.K) ? A[(long long)gm * jb.lda + gk] : C{0, 0};
      const int gn = n0 + mm;
      Bs[kk][mm] = (gk < jb.K && gn < jb.N) ? B[(long long)gk * jb.ldb + gn] : C{0, 0};
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      C av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gm = m0 + ty + 16 * a, gn = n0 + tx + 16 * b;
      if (gm < jb.M && gn < jb.N) {
        C& dst = Cm[(long long)gm * jb.ldc + gn];
        const C v = jb.alpha > 0 ? acc[a][b] : C{-acc[a][b].re, -acc[a][b].im};
        dst = jb.beta ? cadd(dst, v) : v;
      }
    }
}

template <typename R>
__global__ void copy_g_kernel(const SetupItem* items, const cplx<R>* F, cplx<R>* G) {
  const SetupItem it = items[blockIdx.x];
  const int LD = it.S + it.Bd;
  for (long long e = threadIdx.x; e < (long long)it.S * it.S; e += blockDim.x) {
    const int i = (int)(e / it.S), j = (int)(e % it.S);
    G[it.g_off + e] = F[it.f_off + (long long)i * LD + j];
  }
}

// ---------------------------------------------------------------- solve kernels
// Work item of one level of a stage: rows [tile * 64, +64) of G (part 0) or
// of L (part 1) of node `node` of front f (forward), or rows of x_own (back).
struct SolveItem { int f, node, part, tile; };

struct SolveArgs {
  int n, R, w[2];
  long long g_base[2];   // per front: index of the block's (node 0) storage offsets in the tables
  const long long* g_off; const long long* l_off; const long long* t_off;   // per (block, node) / per node
  const Node3* nodes;
  const void* G; const void* L;
  void* T; long long t_front;   // T scratch per front: t_off[node] * R + ...
  void* X; long long x_front;   // slab vectors per front (elements)
};

// C_tile[64][16] = A[rows][0..K) Y[0..K)[16 RHS], A and Y given by functors.
template <typename R, typename FA, typename FY, typename FO>
__device__ inline void tile_product(int K, FA&& a_at, FY&& y_at, FO&& out) {
  using C = cplx<R>;
  __shared__ C As[32][65];
  __shared__ C Ys[32][17];
  const int row = threadIdx.x % 64, cg = threadIdx.x / 64;   // 4 groups of 4 RHS
  C acc[4] = {C{0, 0}, C{0, 0}, C{0, 0}, C{0, 0}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      As[kk][mm] = (k0 + kk < K) ? a_at(mm, k0 + kk) : C{0, 0};
    }
    for (int e = threadIdx.x; e < 32 * 16; e += 256) {
      const int kk = e / 16, rr = e % 16;
      Ys[kk][rr] = (k0 + kk < K) ? y_at(k0 + kk, rr) : C{0, 0};
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const C av = As[kk][row];
#pragma unroll
      for (int q = 0; q < 4; ++q) cfma(acc[q], av, Ys[kk][cg * 4 + q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) out(row, cg * 4 + q, acc[q]);
}

template <typename R>
__global__ void __launch_bounds__(256) fwd_level_kernel(SolveArgs a, const SolveItem* items, int r0) {
  using C = cplx<R>;
  const SolveItem it = items[blockIdx.x];
  const Node3 nd = a.nodes[it.node];
  const int w = a.w[it.f], n = a.n, R_ = a.R;
  const int S = nd.nown * w, Bd = nd.nbnd * w;
  const long long gi = a.g_base[it.f] + it.node;
  C* X = static_cast<C*>(a.X) + it.f * a.x_front;
  const int rbase = it.tile * 64;
  const int nrows = it.part == 0 ? S : Bd;
  const C* M = static_cast<const C*>(it.part == 0 ? a.G : a.L) + (it.part == 0 ? a.g_off[gi] : a.l_off[gi]);
  auto xidx = [&](int P, int q, int r) { return ((long long)front_point(nd, P, n) * w + q) * R_ + r; };
  auto a_at = [&](int mm, int k) { const int rr = rbase + mm; return rr < nrows ? M[(long long)rr * S + k] : C{0, 0}; };
  auto y_at = [&](int k, int r) { const int rr = r0 + r; return rr < R_ ? X[xidx(k / w, k % w, rr)] : C{0, 0}; };
  C* T = static_cast<C*>(a.T) + it.f * a.t_front + a.t_off[it.node] * w * R_;
  tile_product<R>(S, a_at, y_at, [&](int mm, int r, C v) {
    const int rr = rbase + mm, rhs = r0 + r;
    if (rr >= nrows || rhs >= R_) return;
    if (it.part == 0) {
      T[(long long)rr * R_ + rhs] = v;
    } else {
      const int P = nd.nown + rr / w, q = rr % w;
      R* dst = reinterpret_cast<R*>(X + xidx(P, q, rhs));
      atomicAdd(dst, -v.re);
      atomicAdd(dst + 1, -v.im);
    }
  });
}

template <typename R>
__global__ void __launch_bounds__(256) bwd_level_kernel(SolveArgs a, const SolveItem* items, int r0) {
  using C = cplx<R>;
  const SolveItem it = items[blockIdx.x];
  const Node3 nd = a.nodes[it.node];
  const int w = a.w[it.f], n = a.n, R_ = a.R;
  const int S = nd.nown * w, Bd = nd.nbnd * w;
  const long long gi = a.g_base[it.f] + it.node;
  C* X = static_cast<C*>(a.X) + it.f * a.x_front;
  const int rbase = it.tile * 64;
  const C* Lm = static_cast<const C*>(a.L) + a.l_off[gi];
  const C* T = static_cast<const C*>(a.T) + it.f * a.t_front + a.t_off[it.node] * w * R_;
  auto xidx = [&](int P, int q, int r) { return ((long long)front_point(nd, P, n) * w + q) * R_ + r; };
  auto a_at = [&](int mm, int k) { const int rr = rbase + mm; return rr < S ? Lm[(long long)k * S + rr] : C{0, 0}; };
  auto y_at = [&](int k, int r) { const int rr = r0 + r; return rr < R_ ? X[xidx(nd.nown + k / w, k % w, rr)] : C{0, 0}; };
  tile_product<R>(Bd, a_at, y_at, [&](int mm, int r, C v) {
    const int rr = rbase + mm, rhs = r0 + r;
    if (rr >= S || rhs >= R_) return;
    X[xidx(rr / w, rr % w, rhs)] = csub(T[(long long)rr * R_ + rhs], v);
  });
}

// Stage input: X = 0 except the input layers (mode 0: the block layers of u;
// mode 1: the coupling layer, A_{B,next} u_next).
template <typename R>
__global__ void stage_init_kernel(const BlockDesc* blocks, int b0, int b1, int nfront, int mode, int wmax, int n, int R_,
                                  const c128* inv_s, const c128* a_half, const cplx<R>* u, cplx<R>* X, long long x_front) {
  using C = cplx<R>;
  const int f = blockIdx.y;
  if (f >= nfront) return;
  const BlockDesc d = blocks[f == 0 ? b0 : b1];
  const long long n2 = (long long)n * n;
  const long long tot = n2 * d.w * R_;
  C* Xf = X + f * x_front;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % R_);
    const long long pq = e / R_;
    const int q = (int)(pq % d.w);
    const long long p = pq / d.w;
    C v{0, 0};
    if (mode == 0) {
      if (q >= d.out_off && q < d.out_off + d.d_out) v = u[((long long)(d.wlo - 1 + q) * n2 + p) * R_ + r];
    } else if (q == d.coup_local) {
      const int i = (int)(p % n), j = (int)(p / n);
      const int kc = d.next_row > d.hi ? d.hi : d.next_row;   // coupling across layers kc, kc+1 (1-based)
      const c128 cf = cmul(a_half[kc], cmul(inv_s[i + 1], inv_s[j + 1]));
      v = cmul(ccast<R>(cf), u[((long long)(d.next_row - 1) * n2 + p) * R_ + r]);
    }
    Xf[e] = v;
  }
}

// Stage output: mode 0: u_B = X on the block layers and, for the fronts, the
// forward coupling u_next -= A_{next,B} v_B; mode 1: u_B -= X.
template <typename R>
__global__ void stage_finish_kernel(const BlockDesc* blocks, int b0, int b1, int nfront, int mode, int n, int R_,
                                    const c128* inv_s, const c128* a_half, cplx<R>* u, const cplx<R>* X,
                                    long long x_front) {
  using C = cplx<R>;
  const int f = blockIdx.y;
  if (f >= nfront) return;
  const BlockDesc d = blocks[f == 0 ? b0 : b1];
  const long long n2 = (long long)n * n;
  const long long tot = n2 * d.d_out * R_;
  const C* Xf = X + f * x_front;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % R_);
    const long long pl = e / R_;
    const long long p = pl % n2;
    const int l = (int)(pl / n2);                 // block layer index 0..d_out-1
    const int q = d.out_off + l;
    const C xv = Xf[(p * d.w + q) * R_ + r];
    C& dst = u[((long long)(d.lo - 1 + l) * n2 + p) * R_ + r];
    if (mode == 0) {
      dst = xv;
      const bool last = (d.next_row == d.hi + 1) ? (l == d.d_out - 1) : (l == 0);
      if (d.kind != BK_MIDDLE && last) {
        const int i = (int)(p % n), j = (int)(p / n);
        const int kc = d.next_row > d.hi ? d.hi : d.next_row;
        const c128 cf = cmul(a_half[kc], cmul(inv_s[i + 1], inv_s[j + 1]));
        // both fronts may couple into the middle layer in the same launch
        const C dv = cmul(ccast<R>(cf), xv);
        R* nx = reinterpret_cast<R*>(u + ((long long)(d.next_row - 1) * n2 + p) * R_ + r);
        atomicAdd(nx, -dv.re);
        atomicAdd(nx + 1, -dv.im);
      }
    } else {
      dst = csub(dst, xv);
    }
  }
}

// ---------------------------------------------------------------- 7-point matvec
template <typename Tx, typename Ty, bool INNER, bool RESID>
__global__ void __launch_bounds__(256) matvec3_kernel(const cplx<Tx>* __restrict__ x, cplx<Ty>* __restrict__ y,
                                                      const cplx<Ty>* __restrict__ f, const c128* inv_s,
                                                      const c128* a_half, const double* m0, int n, int R) {
  using C = c128;
  const long long n2 = (long long)n * n, n3 = n2 * n;
  const long long total = n3 * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    long long pt;
    int r;
    if (INNER) { pt = e / R; r = (int)(e - pt * R); }
    else { r = (int)(e / n3); pt = e - (long long)r * n3; }
    const int k = (int)(pt / n2), j = (int)((pt / n) % n), i = (int)(pt % n);
    const long long s1 = INNER ? R : 1, s2 = INNER ? (long long)n * R : n, s3 = INNER ? n2 * R : n2;
    auto ld = [&](long long q) { const cplx<Tx> v = x[q]; return C{(double)v.re, (double)v.im}; };
    const C is1 = inv_s[i + 1], is2 = inv_s[j + 1], is3 = inv_s[k + 1];
    const C E = cmul(a_half[i + 1], cmul(is2, is3)), W = cmul(a_half[i], cmul(is2, is3));
    const C N = cmul(a_half[j + 1], cmul(is1, is3)), S = cmul(a_half[j], cmul(is1, is3));
    const C U = cmul(a_half[k + 1], cmul(is1, is2)), Dn = cmul(a_half[k], cmul(is1, is2));
    const C D = csub(cscale(cmul(cmul(is1, is2), is3), m0[pt]), cadd(cadd(cadd(E, W), cadd(N, S)), cadd(U, Dn)));
    C acc = cmul(D, ld(e));
    if (i + 1 < n) cfma(acc, E, ld(e + s1));
    if (i > 0) cfma(acc, W, ld(e - s1));
    if (j + 1 < n) cfma(acc, N, ld(e + s2));
    if (j > 0) cfma(acc, S, ld(e - s2));
    if (k + 1 < n) cfma(acc, U, ld(e + s3));
    if (k > 0) cfma(acc, Dn, ld(e - s3));
    if (RESID) {
      const cplx<Ty> fv = f[e];
      y[e] = cplx<Ty>{(Ty)(fv.re - acc.re), (Ty)(fv.im - acc.im)};
    } else {
      y[e] = cplx<Ty>{(Ty)acc.re, (Ty)acc.im};
    }
  }
}

int grid3(long long total) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const long long g = (total + 255) / 256, cap = (long long)sms * 32;
  return (int)(g < cap ? g : cap);
}

using zc = std::complex<double>;
c128 to_c(zc z) { return c128{z.real(), z.imag()}; }
double sigma_b(double t, double eta, double C) {
  if (t <= eta) { const double q = (t - eta) / eta; return (C / eta) * q * q; }
  if (t >= 1.0 - eta) { const double q = (t - 1.0 + eta) / eta; return (C / eta) * q * q; }
  return 0.0;
}
double sigma_m(double dd, double eta_b, double C) {
  if (dd < 0.0 || dd > eta_b) return 0.0;
  const double q = (dd - eta_b) / eta_b;
  return (C / eta_b) * q * q;
}

}  // namespace

// ---------------------------------------------------------------- host
void release_plan3(Plan& p) {
  Plan3* q = static_cast<Plan3*>(p.p3);
  if (!q) return;
  void* ptrs[] = {q->d_nodes, q->d_g_off, q->d_l_off, q->d_t_off, q->d_G, q->d_L, q->d_T, q->d_X, q->d_s3,
                  q->d_items, q->d_jobs};
  for (void* x : ptrs) if (x) cudaFree(x);
  delete q;
  p.p3 = nullptr;
}

// Blocked Gauss-Jordan inverse of the large front pivot blocks (S > 64): the
// same partial pivoting by rows and the same in-place result as
// invert_kernel, with the work of every NB-column panel split in two.
//  * panel_kernel: the panel's NB pivot steps on its own columns only (one
//    CTA per front, rows over warps, one lane per panel column): pivot search
//    over rows >= k, row swap inside the panel, Gauss-Jordan update.  The
//    panel columns then hold E[:, P], the columns of the panel's accumulated
//    transformation E = I + (E[:, P] - I[:, P]) e_P^t.
//  * swap_rest_kernel applies the panel's row swaps to every other column,
//    copy_rows_kernel saves the pivot rows T = A[P, :], and the deferred
//    update of the other columns is two batched GEMMs:
//      A[i, c] += E[i, P] T[:, c]   (i not in P),   A[P, c] = E[P, P] T[:, c]
//    run by the frontal-update GEMM path (tensor cores, in the split form of
//    the chosen operand type, or FMA).
//  * unpivot_kernel undoes the row pivoting by column swaps at the end.
constexpr int INV_NB = 32;        // panel width
constexpr int INV_DIRECT = 64;    // fronts up to this size keep the one-kernel inverse

template <typename R>
__global__ void __launch_bounds__(512) panel_kernel(const SetupItem* items, cplx<R>* F, int k0, int* piv_all,
                                                    const long long* piv_off, int* status) {
  using C = cplx<R>;
  __shared__ C rowk[INV_NB];
  __shared__ R bestv[16];
  __shared__ int besti[16];
  __shared__ int pr_s;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* colk = reinterpret_cast<C*>(smraw);
  const SetupItem it = items[blockIdx.x];
  const int S = it.S, LD = it.S + it.Bd;
  if (k0 >= S) return;
  const int kb = min(INV_NB, S - k0);
  C* A = F + it.f_off;
  int* piv = piv_all + piv_off[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  bool ok = true;
  for (int kk = 0; kk < kb; ++kk) {
    const int k = k0 + kk;
    R v = R(-1);
    int idx = k;
    for (int i = k + threadIdx.x; i < S; i += blockDim.x) {
      const R a = cabs2(A[(long long)i * LD + k]);
      if (a > v) { v = a; idx = i; }
    }
    for (int m = 16; m > 0; m >>= 1) {
      const R ov = Shfl<R>::xr(v, m);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, m);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { bestv[warp] = v; besti[warp] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      R bv = bestv[0];
      int bi = besti[0];
      for (int q = 1; q < nw; ++q)
        if (bestv[q] > bv || (bestv[q] == bv && besti[q] < bi)) { bv = bestv[q]; bi = besti[q]; }
      if (!(bv > R(0)) || !isfinite(bv)) { ok = false; bi = k; }
      pr_s = bi;
      piv[k] = bi;
    }
    __syncthreads();
    const int pr = pr_s;
    if (pr != k && threadIdx.x < kb) {
      C* a = A + (long long)k * LD + k0 + threadIdx.x;
      C* b = A + (long long)pr * LD + k0 + threadIdx.x;
      const C t = *a;
      *a = *b;
      *b = t;
    }
    __syncthreads();
    const C pinv = cinv(A[(long long)k * LD + k]);
    for (int i = threadIdx.x; i < S; i += blockDim.x) colk[i] = A[(long long)i * LD + k];
    if (threadIdx.x < kb) rowk[threadIdx.x] = (threadIdx.x == kk) ? pinv : cmul(A[(long long)k * LD + k0 + threadIdx.x], pinv);
    __syncthreads();
    if (lane < kb)
      for (int i = warp; i < S; i += nw) {
        C& x = A[(long long)i * LD + k0 + lane];
        if (i == k) x = rowk[lane];
        else if (lane == kk) x = cmul(C{-colk[i].re, -colk[i].im}, pinv);
        else x = csub(x, cmul(colk[i], rowk[lane]));
      }
    __syncthreads();
  }
  if (threadIdx.x == 0 && !ok) set_status(status, HS_EBREAKDOWN, it.block, it.node);
}

// the panel's row swaps (in order) on every column outside the panel
template <typename R>
__global__ void __launch_bounds__(256) swap_rest_kernel(const SetupItem* items, cplx<R>* F, int k0, const int* piv_all,
                                                        const long long* piv_off) {
  using C = cplx<R>;
  const SetupItem it = items[blockIdx.x];
  const int S = it.S, LD = it.S + it.Bd;
  if (k0 >= S) return;
  const int kb = min(INV_NB, S - k0);
  C* A = F + it.f_off;
  const int* piv = piv_all + piv_off[blockIdx.x];
  for (int kk = 0; kk < kb; ++kk) {
    const int k = k0 + kk, pr = piv[k];
    if (pr != k)
      for (int j = threadIdx.x; j < S; j += blockDim.x) {
        if (j >= k0 && j < k0 + kb) continue;
        const C t = A[(long long)k * LD + j];
        A[(long long)k * LD + j] = A[(long long)pr * LD + j];
        A[(long long)pr * LD + j] = t;
      }
    __syncthreads();
  }
}

// T[q][j] = A[k0 + q][j], the panel's pivot rows before the deferred update
template <typename R>
__global__ void __launch_bounds__(256) copy_rows_kernel(const SetupItem* items, const cplx<R>* F, int k0,
                                                        cplx<R>* T, const long long* t_off) {
  const SetupItem it = items[blockIdx.x];
  const int S = it.S, LD = it.S + it.Bd;
  if (k0 >= S) return;
  const int kb = min(INV_NB, S - k0);
  const cplx<R>* A = F + it.f_off;
  cplx<R>* Tb = T + t_off[blockIdx.x];
  for (int e = threadIdx.x; e < kb * S; e += blockDim.x) {
    const int q = e / S, j = e - q * S;
    Tb[e] = A[(long long)(k0 + q) * LD + j];
  }
}

// undo the row pivoting: column swaps in reverse order
template <typename R>
__global__ void __launch_bounds__(256) unpivot_kernel(const SetupItem* items, cplx<R>* F, const int* piv_all,
                                                      const long long* piv_off) {
  using C = cplx<R>;
  const SetupItem it = items[blockIdx.x];
  const int S = it.S, LD = it.S + it.Bd;
  C* A = F + it.f_off;
  const int* piv = piv_all + piv_off[blockIdx.x];
  for (int k = S - 1; k >= 0; --k) {
    const int pr = piv[k];
    if (pr != k)
      for (int i = threadIdx.x; i < S; i += blockDim.x) {
        const C t = A[(long long)i * LD + k];
        A[(long long)i * LD + k] = A[(long long)i * LD + pr];
        A[(long long)i * LD + pr] = t;
      }
    __syncthreads();
  }
}

// Host side of the blocked inverse for the large fronts of one tree level.
// All panels' GEMM jobs are formed up front (their operands sit at fixed
// places) and uploaded once; the level is synchronised by the caller.
template <typename R>
int blocked_inverse(Plan& p, const std::vector<SetupItem>& large, cplx<R>* F, cudaStream_t s) {
  using C = cplx<R>;
  const int nl = (int)large.size();
  if (nl == 0) return HS_OK;
  int Smax = 0;
  std::vector<long long> piv_off(nl), t_off(nl);
  long long ptot = 0, ttot = 0;
  for (int i = 0; i < nl; ++i) {
    Smax = std::max(Smax, large[i].S);
    piv_off[i] = ptot; ptot += large[i].S;
    t_off[i] = ttot; ttot += (long long)INV_NB * large[i].S;
  }
  const bool tc = sizeof(R) == 4 && p.opt.frontal_gemm != 0;
  const int npan = (Smax + INV_NB - 1) / INV_NB;
  // GEMM jobs of every panel: rows outside the panel (A += E[R, P] T[:, c])
  // and the panel rows (A[P, c] = E[P, P] T[:, c]), columns outside the panel
  std::vector<GemmJob> gj;
  std::vector<GemmTile> gt;
  std::vector<TcGemmJob> tj;
  std::vector<TcGemmTile> tt;
  std::vector<int> pan_tile(npan + 1, 0);
  for (int pn = 0; pn < npan; ++pn) {
    const int k0 = pn * INV_NB;
    std::vector<GemmJob> jobs;
    for (int i = 0; i < nl; ++i) {
      const SetupItem& it = large[i];
      const int S = it.S, LD = it.S + it.Bd;
      if (k0 >= S) continue;
      const int kb = std::min(INV_NB, S - k0);
      C* A = F + it.f_off;
      C* Tb = nullptr;   // device address formed after allocation: offset kept in ldb-free form below
      (void)Tb;
      const int rr[2][2] = {{0, k0}, {k0 + kb, S}};
      for (auto& cr : rr) {
        const int c0 = cr[0], nc = cr[1] - cr[0];
        if (nc <= 0) continue;
        for (auto& rw : rr) {
          const int r0 = rw[0], nr = rw[1] - rw[0];
          if (nr <= 0) continue;
          // B operand recorded as an offset into T; fixed up below
          jobs.push_back(GemmJob{A + (long long)r0 * LD + k0, reinterpret_cast<void*>(t_off[i] + c0), A + (long long)r0 * LD + c0,
                                 LD, S, LD, nr, nc, kb, 1, 1});
        }
        jobs.push_back(GemmJob{A + (long long)k0 * LD + k0, reinterpret_cast<void*>(t_off[i] + c0), A + (long long)k0 * LD + c0,
                               LD, S, LD, kb, nc, kb, 1, 0});
      }
    }
    for (auto& j : jobs) {
      if (tc) {
        TcGemmJob t{j.A, j.B, j.C, j.lda, j.ldb, j.ldc, j.M, j.N, j.K, (float)j.alpha, j.beta};
        tj.push_back(t);
      } else {
        gj.push_back(j);
      }
    }
    pan_tile[pn + 1] = pan_tile[pn];
    if (tc) {
      const size_t before = tt.size();
      std::vector<TcGemmJob> last(tj.end() - jobs.size(), tj.end());
      zgemm_tc_tiles(last, (int)(tj.size() - jobs.size()), tt);
      pan_tile[pn + 1] += (int)(tt.size() - before);
    } else {
      for (int t = (int)(gj.size() - jobs.size()); t < (int)gj.size(); ++t)
        for (int tm = 0; tm < (gj[t].M + 63) / 64; ++tm)
          for (int tn = 0; tn < (gj[t].N + 63) / 64; ++tn) {
            gt.push_back({t, tm, tn});
            ++pan_tile[pn + 1];
          }
    }
  }
  SetupItem* d_items = nullptr;
  int* d_piv = nullptr;
  long long *d_poff = nullptr, *d_toff = nullptr;
  C* d_T = nullptr;
  void* d_jobs = nullptr;
  void* d_tiles = nullptr;
  const size_t njob = tc ? tj.size() : gj.size(), ntile = tc ? tt.size() : gt.size();
  const size_t jsz = tc ? sizeof(TcGemmJob) : sizeof(GemmJob), tsz = tc ? sizeof(TcGemmTile) : sizeof(GemmTile);
  int st = HS_OK;
  if (cudaMalloc(&d_items, nl * sizeof(SetupItem)) != cudaSuccess || cudaMalloc(&d_piv, ptot * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&d_poff, nl * sizeof(long long)) != cudaSuccess || cudaMalloc(&d_toff, nl * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&d_T, std::max<long long>(ttot, 1) * sizeof(C)) != cudaSuccess ||
      cudaMalloc(&d_jobs, std::max<size_t>(njob, 1) * jsz) != cudaSuccess ||
      cudaMalloc(&d_tiles, std::max<size_t>(ntile, 1) * tsz) != cudaSuccess) {
    cudaGetLastError();
    st = HS_ENOMEM;
  }
  if (st == HS_OK) {
    // B operands: offsets into T -> device addresses
    for (auto& j : gj) j.B = d_T + reinterpret_cast<long long>(j.B);
    for (auto& j : tj) j.B = d_T + reinterpret_cast<long long>(j.B);
    cudaMemcpyAsync(d_items, large.data(), nl * sizeof(SetupItem), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_poff, piv_off.data(), nl * sizeof(long long), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_toff, t_off.data(), nl * sizeof(long long), cudaMemcpyHostToDevice, s);
    if (njob) cudaMemcpyAsync(d_jobs, tc ? (const void*)tj.data() : (const void*)gj.data(), njob * jsz, cudaMemcpyHostToDevice, s);
    if (ntile) cudaMemcpyAsync(d_tiles, tc ? (const void*)tt.data() : (const void*)gt.data(), ntile * tsz, cudaMemcpyHostToDevice, s);
    const size_t psm = (size_t)Smax * sizeof(C);
    if (psm > 48 * 1024) cudaFuncSetAttribute(panel_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    for (int pn = 0; pn < npan && st == HS_OK; ++pn) {
      const int k0 = pn * INV_NB;
      note_launch(3);
      panel_kernel<R><<<nl, 512, psm, s>>>(d_items, F, k0, d_piv, d_poff, p.d_status);
      swap_rest_kernel<R><<<nl, 256, 0, s>>>(d_items, F, k0, d_piv, d_poff);
      copy_rows_kernel<R><<<nl, 256, 0, s>>>(d_items, F, k0, d_T, d_toff);
      const int t0 = pan_tile[pn], tn = pan_tile[pn + 1] - pan_tile[pn];
      if (tn > 0) {
        if (tc) {
          // the inverse keeps FP32-level accuracy: the split form of the mode's operand type
          const int mode = p.opt.frontal_gemm == 1 ? 3 : p.opt.frontal_gemm == 2 ? 4 : p.opt.frontal_gemm;
          st = zgemm_tc_launch(static_cast<const TcGemmJob*>(d_jobs), static_cast<const TcGemmTile*>(d_tiles) + t0, tn,
                               mode, p.d_status, p.opt.spin_budget, s);
        } else {
          note_launch();
          gemm_kernel<R><<<tn, 256, 0, s>>>(static_cast<const GemmJob*>(d_jobs), static_cast<const GemmTile*>(d_tiles) + t0);
        }
      }
    }
    note_launch();
    unpivot_kernel<R><<<nl, 256, 0, s>>>(d_items, F, d_piv, d_poff);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == HS_OK && e != cudaSuccess) st = cuda_status(e);
  }
  for (void* x : {(void*)d_items, (void*)d_piv, (void*)d_poff, (void*)d_toff, (void*)d_T, d_jobs, d_tiles})
    if (x) cudaFree(x);
  return st;
}

template <typename R>
int setup3_t(Plan& p, Plan3& q, cudaStream_t s) {
  using C = cplx<R>;
  const int nb = (int)p.blocks.size(), nn = (int)q.nodes.size();
  const int maxl = q.nlevels - 1;
  // items per level (all blocks), factor offsets
  std::vector<std::vector<SetupItem>> lv(q.nlevels);
  std::vector<int> item_of((size_t)nb * nn, -1);
  q.g_off.assign((size_t)nb * nn, 0);
  q.l_off.assign((size_t)nb * nn, 0);
  long long gtot = 0, ltot = 0;
  for (int L = maxl; L >= 0; --L)
    for (int b = 0; b < nb; ++b)
      for (int id : q.by_level[L]) {
        const Node3& nd = q.nodes[id];
        const int w = p.blocks[b].w;
        SetupItem it{};
        it.block = b; it.node = id; it.S = nd.nown * w; it.Bd = nd.nbnd * w;
        it.g_off = gtot; gtot += (long long)it.S * it.S;
        it.l_off = ltot; ltot += (long long)it.Bd * it.S;
        q.g_off[(size_t)b * nn + id] = it.g_off;
        q.l_off[(size_t)b * nn + id] = it.l_off;
        it.child_item[0] = it.child_item[1] = -1;
        for (int c = 0; c < 2; ++c)
          if (nd.child[c] >= 0) it.child_item[c] = item_of[(size_t)b * nn + nd.child[c]];
        item_of[(size_t)b * nn + id] = (int)lv[L].size();
        lv[L].push_back(it);
      }
  const size_t es = sizeof(C);
  HS_CUDA_TRY(cudaMalloc(&q.d_G, std::max<long long>(gtot, 1) * es));
  HS_CUDA_TRY(cudaMalloc(&q.d_L, std::max<long long>(ltot, 1) * es));
  p.bytes += (gtot + ltot) * (long long)es;
  Coef3 cf{p.n, p.d_inv_s1, p.d_a1, p.d_cinv2, q.d_s3, c128{p.omega * p.omega - p.alpha * p.alpha, 2 * p.omega * p.alpha}};
  void* prevF = nullptr;
  SetupItem* prevItems = nullptr;
  int st = HS_OK;
  for (int L = maxl; L >= 0 && st == HS_OK; --L) {
    std::vector<SetupItem>& its = lv[L];
    long long ftot = 0;
    int Smax = 0;
    for (auto& it : its) {
      it.f_off = ftot;
      ftot += (long long)(it.S + it.Bd) * (it.S + it.Bd);
      Smax = std::max(Smax, it.S);
    }
    void* F = nullptr;
    SetupItem* d_its = nullptr;
    if (cudaMalloc(&F, std::max<long long>(ftot, 1) * es) != cudaSuccess ||
        cudaMalloc(&d_its, its.size() * sizeof(SetupItem)) != cudaSuccess) {
      cudaGetLastError();
      if (F) cudaFree(F);
      st = HS_ENOMEM;
      break;
    }
    cudaMemcpyAsync(d_its, its.data(), its.size() * sizeof(SetupItem), cudaMemcpyHostToDevice, s);
    note_launch();
    assemble_kernel<R><<<(int)its.size(), 256, 0, s>>>(cf, p.d_blocks, q.d_nodes, d_its, (C*)F, prevItems,
                                                        (const C*)prevF);
    // pivot-block inverses: one kernel for the small fronts, the blocked
    // Gauss-Jordan (panels + GEMM updates) for the large ones
    {
      std::vector<SetupItem> small, large;
      int Ssmall = 0;
      for (auto& it : its) {
        if (it.S > INV_DIRECT) large.push_back(it);
        else { small.push_back(it); Ssmall = std::max(Ssmall, it.S); }
      }
      SetupItem* d_small = nullptr;
      if (!small.empty()) {
        if (cudaMalloc(&d_small, small.size() * sizeof(SetupItem)) != cudaSuccess) { cudaGetLastError(); st = HS_ENOMEM; }
        else {
          cudaMemcpyAsync(d_small, small.data(), small.size() * sizeof(SetupItem), cudaMemcpyHostToDevice, s);
          const size_t ism = (size_t)Ssmall * 2 * es + (size_t)Ssmall * sizeof(int);
          if (ism > 48 * 1024) cudaFuncSetAttribute(invert_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
          note_launch();
          invert_kernel<R><<<(int)small.size(), 512, ism, s>>>(d_small, (C*)F, p.d_status);
        }
      }
      if (st == HS_OK) st = blocked_inverse<R>(p, large, (C*)F, s);
      if (d_small) { cudaStreamSynchronize(s); cudaFree(d_small); }
      if (st != HS_OK) { cudaFree(F); cudaFree(d_its); break; }
    }
    // L = F21 G ; F22 -= L F12
    std::vector<GemmJob> j1, j2;
    for (auto& it : its) {
      if (it.Bd == 0) continue;
      const int LD = it.S + it.Bd;
      C* f = (C*)F + it.f_off;
      C* Lm = (C*)q.d_L + it.l_off;
      j1.push_back(GemmJob{f + (long long)it.S * LD, f, Lm, LD, LD, it.S, it.Bd, it.S, it.S, 1, 0});
      j2.push_back(GemmJob{Lm, f + it.S, f + (long long)it.S * LD + it.S, it.S, LD, LD, it.Bd, it.Bd, it.S, -1, 1});
    }
    for (auto& it : its) q.inv_flops += 8.0 * it.S * (double)it.S * it.S;
    for (auto* jobs : {&j1, &j2})
      for (auto& g : *jobs) q.gemm_flops += 8.0 * g.M * (double)g.N * g.K;
    const bool tc = sizeof(R) == 4 && p.opt.frontal_gemm != 0;
    for (auto* jobs : {&j1, &j2}) {
      if (jobs->empty()) continue;
      if (tc) {
        std::vector<TcGemmJob> tj;
        for (auto& g : *jobs) tj.push_back(TcGemmJob{g.A, g.B, g.C, g.lda, g.ldb, g.ldc, g.M, g.N, g.K, (float)g.alpha, g.beta});
        const int s2 = zgemm_tc_batched(tj, p.opt.frontal_gemm, p.d_status, p.opt.spin_budget, s);
        if (s2 != HS_OK) { st = s2; break; }
        continue;
      }
      std::vector<GemmTile> tiles;
      for (int t = 0; t < (int)jobs->size(); ++t)
        for (int tm = 0; tm < ((*jobs)[t].M + 63) / 64; ++tm)
          for (int tn = 0; tn < ((*jobs)[t].N + 63) / 64; ++tn) tiles.push_back({t, tm, tn});
      GemmJob* dj = nullptr;
      GemmTile* dt = nullptr;
      cudaMalloc(&dj, jobs->size() * sizeof(GemmJob));
      cudaMalloc(&dt, tiles.size() * sizeof(GemmTile));
      cudaMemcpyAsync(dj, jobs->data(), jobs->size() * sizeof(GemmJob), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(GemmTile), cudaMemcpyHostToDevice, s);
      note_launch();
      gemm_kernel<R><<<(int)tiles.size(), 256, 0, s>>>(dj, dt);
      cudaStreamSynchronize(s);
      cudaFree(dj);
      cudaFree(dt);
    }
    note_launch();
    copy_g_kernel<R><<<(int)its.size(), 256, 0, s>>>(d_its, (const C*)F, (C*)q.d_G);
    cudaError_t e = cudaStreamSynchronize(s);
    if (prevF) cudaFree(prevF);
    if (prevItems) cudaFree(prevItems);
    prevF = F;
    prevItems = d_its;
    if (e != cudaSuccess) st = cuda_status(e);
  }
  if (prevF) cudaFree(prevF);
  if (prevItems) cudaFree(prevItems);
  return st;
}

int prepare_plan3(Plan& p) {
  Plan3* q = new Plan3();
  p.p3 = q;
  const int n = p.n;
  build_nd(q->nodes, 0, n, 0, n, 0, -1, n);
  q->nlevels = 0;
  for (auto& nd : q->nodes) q->nlevels = std::max(q->nlevels, nd.level + 1);
  q->by_level.assign(q->nlevels, {});
  for (int i = 0; i < (int)q->nodes.size(); ++i) q->by_level[q->nodes[i].level].push_back(i);
  // T offsets per node (points)
  q->t_off.assign(q->nodes.size(), 0);
  long long tp = 0;
  for (size_t i = 0; i < q->nodes.size(); ++i) { q->t_off[i] = tp; tp += q->nodes[i].nown; }
  int wmax = 0;
  for (auto& d : p.blocks) wmax = std::max(wmax, d.w);
  q->wmax = wmax;
  const size_t es = (p.prec == HS_C64) ? sizeof(c64) : sizeof(c128);
  const long long n2 = (long long)n * n;
  q->x_front = n2 * wmax * p.max_nrhs;
  q->t_front = tp * wmax * p.max_nrhs;
  // moving-PML window tables of x3 (same rules as the 2D x2 windows)
  const double h = p.h, eta = p.bp * h, eta_b = p.b * h, C = p.C;
  std::vector<c128> s3;
  for (auto& d : p.blocks) {
    d.s2_off = (int)s3.size();
    auto sig = [&](double x) {
      if (d.kind == BK_F || d.kind == BK_E) return sigma_b(x, eta, C);
      double sg = 0.0;
      if (d.kind == BK_LOWER || d.kind == BK_MIDDLE) sg += sigma_m(x - (d.lo - p.b) * h, eta_b, p.Cm);
      if (d.kind == BK_UPPER || d.kind == BK_MIDDLE) sg += sigma_m((d.hi + p.b) * h - x, eta_b, p.Cm);
      return sg;
    };
    auto inv = [&](double sg) { return zc(1.0, sg / p.omega); };
    for (int t = 0; t < d.w; ++t) s3.push_back(to_c(inv(sig((d.wlo + t) * h))));
    for (int t = 0; t < d.w; ++t) s3.push_back(to_c(1.0 / inv(sig((d.wlo + t + 0.5) * h)) / (h * h)));
    for (int t = 0; t < d.w; ++t) s3.push_back(to_c(1.0 / inv(sig((d.wlo + t - 0.5) * h)) / (h * h)));
  }
  HS_CUDA_TRY(cudaMalloc(&q->d_s3, s3.size() * sizeof(c128)));
  HS_CUDA_TRY(cudaMalloc(&q->d_nodes, q->nodes.size() * sizeof(Node3)));
  HS_CUDA_TRY(cudaMalloc(&q->d_t_off, q->t_off.size() * sizeof(long long)));
  HS_CUDA_TRY(cudaMalloc(&q->d_T, 2 * q->t_front * es));
  HS_CUDA_TRY(cudaMalloc(&q->d_X, 2 * q->x_front * es));
  p.bytes += (long long)(2 * q->t_front + 2 * q->x_front) * (long long)es;
  cudaMemcpy(q->d_s3, s3.data(), s3.size() * sizeof(c128), cudaMemcpyHostToDevice);
  cudaMemcpy(q->d_nodes, q->nodes.data(), q->nodes.size() * sizeof(Node3), cudaMemcpyHostToDevice);
  cudaMemcpy(q->d_t_off, q->t_off.data(), q->t_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
  return HS_OK;
}

int setup3(Plan& p, cudaStream_t s) {
  Plan3& q = *static_cast<Plan3*>(p.p3);
  int st = (p.prec == HS_C64) ? setup3_t<float>(p, q, s) : setup3_t<double>(p, q, s);
  if (st != HS_OK) return st;
  const size_t nb = p.blocks.size(), nn = q.nodes.size();
  HS_CUDA_TRY(cudaMalloc(&q.d_g_off, nb * nn * sizeof(long long)));
  HS_CUDA_TRY(cudaMalloc(&q.d_l_off, nb * nn * sizeof(long long)));
  cudaMemcpy(q.d_g_off, q.g_off.data(), nb * nn * sizeof(long long), cudaMemcpyHostToDevice);
  cudaMemcpy(q.d_l_off, q.l_off.data(), nb * nn * sizeof(long long), cudaMemcpyHostToDevice);
  // solve work lists: per distinct window height pair of a stage and level
  // (items depend only on the nodes and w), built for every stage
  std::vector<SolveItem> all;
  auto stage_lists = [&](int wa, int wb, int nfront, StageLists& sl) {
    sl.fwd_off.assign(q.nlevels, 0); sl.fwd_cnt.assign(q.nlevels, 0);
    sl.bwd_off.assign(q.nlevels, 0); sl.bwd_cnt.assign(q.nlevels, 0);
    for (int L = 0; L < q.nlevels; ++L) {
      sl.fwd_off[L] = (int)all.size();
      for (int f = 0; f < nfront; ++f) {
        const int w = f == 0 ? wa : wb;
        for (int id : q.by_level[L]) {
          const Node3& nd = q.nodes[id];
          for (int t = 0; t < (nd.nown * w + 63) / 64; ++t) all.push_back({f, id, 0, t});
          for (int t = 0; t < (nd.nbnd * w + 63) / 64; ++t) all.push_back({f, id, 1, t});
        }
      }
      sl.fwd_cnt[L] = (int)all.size() - sl.fwd_off[L];
      sl.bwd_off[L] = (int)all.size();
      for (int f = 0; f < nfront; ++f) {
        const int w = f == 0 ? wa : wb;
        for (int id : q.by_level[L]) {
          const Node3& nd = q.nodes[id];
          for (int t = 0; t < (nd.nown * w + 63) / 64; ++t) all.push_back({f, id, 0, t});
        }
      }
      sl.bwd_cnt[L] = (int)all.size() - sl.bwd_off[L];
    }
  };
  q.stage_lists.clear();
  for (auto& stg : p.stages) {
    StageLists sl;
    stage_lists(p.blocks[stg[0]].w, p.blocks[stg[1]].w, 2, sl);
    q.stage_lists.push_back(sl);
  }
  stage_lists(p.blocks[p.middle].w, p.blocks[p.middle].w, 1, q.middle_lists);
  HS_CUDA_TRY(cudaMalloc(&q.d_items, std::max<size_t>(all.size(), 1) * sizeof(SolveItem)));
  cudaMemcpy(q.d_items, all.data(), all.size() * sizeof(SolveItem), cudaMemcpyHostToDevice);
  return HS_OK;
}

template <typename R>
int run_stage3(Plan& p, Plan3& q, int b0, int b1, int nfront, int mode, const StageLists& sl, int R_, cudaStream_t s) {
  using C = cplx<R>;
  SolveArgs a{};
  a.n = p.n; a.R = R_;
  a.w[0] = p.blocks[b0].w; a.w[1] = p.blocks[b1].w;
  const long long nn = (long long)q.nodes.size();
  a.g_base[0] = b0 * nn; a.g_base[1] = b1 * nn;
  a.g_off = q.d_g_off; a.l_off = q.d_l_off; a.t_off = q.d_t_off;
  a.nodes = q.d_nodes; a.G = q.d_G; a.L = q.d_L;
  a.T = q.d_T; a.t_front = q.t_front;
  a.X = q.d_X; a.x_front = q.x_front;
  const SolveItem* items = static_cast<const SolveItem*>(q.d_items);
  const long long n2 = (long long)p.n * p.n;
  C* u = static_cast<C*>(p.d_u);
  note_launch();
  stage_init_kernel<R><<<dim3(grid3(n2 * q.wmax * R_), nfront), 256, 0, s>>>(
      p.d_blocks, b0, b1, nfront, mode, q.wmax, p.n, R_, p.d_inv_s1, p.d_a1, u, (C*)q.d_X, q.x_front);
  for (int r0 = 0; r0 < R_; r0 += 16) {
    for (int L = q.nlevels - 1; L >= 0; --L) {
      if (!sl.fwd_cnt[L]) continue;
      note_launch();
      fwd_level_kernel<R><<<sl.fwd_cnt[L], 256, 0, s>>>(a, items + sl.fwd_off[L], r0);
    }
    for (int L = 0; L < q.nlevels; ++L) {
      if (!sl.bwd_cnt[L]) continue;
      note_launch();
      bwd_level_kernel<R><<<sl.bwd_cnt[L], 256, 0, s>>>(a, items + sl.bwd_off[L], r0);
    }
  }
  note_launch();
  stage_finish_kernel<R><<<dim3(grid3(n2 * std::max(p.blocks[b0].d_out, p.blocks[b1].d_out) * R_), nfront), 256, 0, s>>>(
      p.d_blocks, b0, b1, nfront, mode, p.n, R_, p.d_inv_s1, p.d_a1, u, (const C*)q.d_X, q.x_front);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

template <typename R>
int sweep3_t(Plan& p, int R_, cudaStream_t s) {
  Plan3& q = *static_cast<Plan3*>(p.p3);
  const int S = (int)p.stages.size();
  int st = HS_OK;
  for (int k = 0; k < S && st == HS_OK; ++k)
    st = run_stage3<R>(p, q, p.stages[k][0], p.stages[k][1], 2, 0, q.stage_lists[k], R_, s);
  if (st == HS_OK) st = run_stage3<R>(p, q, p.middle, p.middle, 1, 0, q.middle_lists, R_, s);
  for (int k = S - 1; k >= 0 && st == HS_OK; --k)
    st = run_stage3<R>(p, q, p.stages[k][0], p.stages[k][1], 2, 1, q.stage_lists[k], R_, s);
  return st;
}

int sweep3(Plan& p, int nrhs, cudaStream_t s) {
  return (p.prec == HS_C64) ? sweep3_t<float>(p, nrhs, s) : sweep3_t<double>(p, nrhs, s);
}

int matvec3_abi(Plan& p, const void* x, void* y, int nrhs, int dtype, cudaStream_t s) {
  const long long total = (long long)p.n * p.n * p.n * nrhs;
  note_launch();
  if (dtype == HS_C128)
    matvec3_kernel<double, double, false, false><<<grid3(total), 256, 0, s>>>(
        (const c128*)x, (c128*)y, nullptr, p.d_inv_s1, p.d_a1, p.d_m0, p.n, nrhs);
  else
    matvec3_kernel<float, float, false, false><<<grid3(total), 256, 0, s>>>(
        (const c64*)x, (c64*)y, nullptr, p.d_inv_s1, p.d_a1, p.d_m0, p.n, nrhs);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

int matvec3_internal_f64(Plan& p, const void* x, bool x_is_c64, c128* y, const c128* f, int R, cudaStream_t s) {
  const long long total = (long long)p.n * p.n * p.n * R;
  const int g = grid3(total);
  note_launch();
  if (x_is_c64) {
    if (f) matvec3_kernel<float, double, true, true><<<g, 256, 0, s>>>((const c64*)x, y, f, p.d_inv_s1, p.d_a1, p.d_m0, p.n, R);
    else matvec3_kernel<float, double, true, false><<<g, 256, 0, s>>>((const c64*)x, y, f, p.d_inv_s1, p.d_a1, p.d_m0, p.n, R);
  } else {
    if (f) matvec3_kernel<double, double, true, true><<<g, 256, 0, s>>>((const c128*)x, y, f, p.d_inv_s1, p.d_a1, p.d_m0, p.n, R);
    else matvec3_kernel<double, double, true, false><<<g, 256, 0, s>>>((const c128*)x, y, f, p.d_inv_s1, p.d_a1, p.d_m0, p.n, R);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

}  // namespace hs
