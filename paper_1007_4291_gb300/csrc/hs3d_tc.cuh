// Batched complex64 GEMMs on the tensor cores (TF32 or BF16, FP32 accumulation) for
// the frontal updates of the 3D setup (hs3d_tc.cu).
#pragma once
#include <vector>
#include "hs_internal.cuh"

namespace hs {

struct TcGemmJob {
  const void* A;   // complex64, M x K, row stride lda (elements)
  const void* B;   // complex64, K x N, row stride ldb
  void* C;         // complex64, M x N, row stride ldc
  int lda, ldb, ldc, M, N, K;
  float alpha;     // C = beta C + alpha A B
  int beta;        // 0 or 1
};
struct TcGemmTile { int job, tm, tn; };

// mode 1: one TF32 pass; 3: 3xTF32 (a_hi b_hi + a_hi b_lo + a_lo b_hi,
// FP32-level accuracy); 2: one BF16 pass; 4: 3xBF16.  Synchronises `s`.
int zgemm_tc_batched(const std::vector<TcGemmJob>& jobs, int mode, int* status, long long spin, cudaStream_t s);
// The same on job and tile lists already on the device (no allocation, no
// synchronisation); zgemm_tc_tiles appends the tiles of `jobs`, numbered
// from job0, to `tiles`.
int zgemm_tc_launch(const TcGemmJob* d_jobs, const TcGemmTile* d_tiles, int ntiles, int mode, int* status,
                    long long spin, cudaStream_t s);
void zgemm_tc_tiles(const std::vector<TcGemmJob>& jobs, int job0, std::vector<TcGemmTile>& tiles);

}  // namespace hs
