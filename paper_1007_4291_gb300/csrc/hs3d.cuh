// 3D plans: nested-dissection tree of the (x1, x2) plane, per-slab
// multifrontal factors and the work lists of the slab solves (hs3d.cu).
#pragma once
#include <vector>
#include "hs_internal.cuh"

namespace hs {

// A node of the nested dissection of the n x n plane: region [x0,x1) x [y0,y1)
// (0-based), eliminated set = the whole region (leaf, kind 0), the column
// x = mid (kind 1) or the row y = mid (kind 2).
struct Node3 {
  int x0, x1, y0, y1;
  int kind, mid;
  int nown, nbnd;        // plane points eliminated here / on the ring outside the region
  int level, parent;
  int child[2];
};

struct StageLists {
  std::vector<int> fwd_off, fwd_cnt, bwd_off, bwd_cnt;   // per level, into the solve item array
};

struct Plan3 {
  std::vector<Node3> nodes;
  std::vector<std::vector<int>> by_level;
  int nlevels = 0, wmax = 0;
  std::vector<long long> g_off, l_off, t_off;
  Node3* d_nodes = nullptr;
  long long* d_g_off = nullptr;
  long long* d_l_off = nullptr;
  long long* d_t_off = nullptr;
  void* d_G = nullptr;     // G = F11^{-1} of every (block, node), S x S
  void* d_L = nullptr;     // L = F21 G, Bd x S
  void* d_T = nullptr;     // solve scratch t = G X_own, per front
  void* d_X = nullptr;     // slab vectors of the two fronts [point][layer][rhs]
  long long t_front = 0, x_front = 0;
  c128* d_s3 = nullptr;    // per block: 1/s3, s3(+1/2)/h^2, s3(-1/2)/h^2 on the window layers
  void* d_items = nullptr; // solve work items of every stage
  void* d_jobs = nullptr;
  std::vector<StageLists> stage_lists;
  StageLists middle_lists;
  double gemm_flops = 0;     // real flops of the frontal Schur-update GEMMs of the setup (8 per complex MAC)
  double inv_flops = 0;      // real flops of the front pivot-block inversions (8 S^3 each)
};

int prepare_plan3(Plan& p);                 // tree, window tables, solve workspace
int setup3(Plan& p, cudaStream_t s);        // factor every slab (Algorithm 5)
int sweep3(Plan& p, int nrhs, cudaStream_t s);   // u <- M_alpha u on p.d_u (Algorithm 6)
void release_plan3(Plan& p);
int matvec3_abi(Plan& p, const void* x, void* y, int nrhs, int dtype, cudaStream_t s);
int matvec3_internal_f64(Plan& p, const void* x, bool x_is_c64, c128* y, const c128* f, int R, cudaStream_t s);

}  // namespace hs
