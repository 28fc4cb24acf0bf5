// Batched complex64 GEMMs on the tensor cores (TF32, FP32 accumulation) for
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

// split = 1: 3xTF32 (a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32-level accuracy);
// 0: one TF32 pass.  Synchronises `s`.
int zgemm_tf32_batched(const std::vector<TcGemmJob>& jobs, int split, int* status, long long spin, cudaStream_t s);

}  // namespace hs
