// Frontal updates of the 3D multifrontal setup on the tensor cores: batched
// complex GEMMs C = beta C + alpha A B (complex64) as real TF32 GEMMs with
// FP32 accumulation in tensor memory.
//
// Complex product as one real product (the "4M" form): with A read as the
// real M x 2K matrix of its interleaved (re, im) storage and
//   Bt[2n + c][2k + d] = { Br, -Bi ; Bi, Br }[c][d]   (rows = output columns),
// the interleaved complex result is A Bt^t.  Precision modes: one TF32 pass
// (operands truncated to 10-bit mantissas), the 3xTF32 split a = a_hi + a_lo
// with a_hi b_hi + a_hi b_lo + a_lo b_hi, which restores FP32 accuracy, and
// the same two with BF16 operands (8-bit mantissas, rounded to nearest; the
// split keeps about 16 bits).
//
// A CTA computes a 128 x 32 complex tile (MMA M = 128, N = 64 real columns)
// and loops over K in chunks of 16 complex (32 real) values: its threads
// write the A and Bt chunks to shared memory in the K-major non-swizzled
// core-matrix layout ([k/4][row][4] floats), one thread issues the MMAs
// (K = 8 each) and commits them, and every thread waits on the mbarrier
// (bounded) before the chunk's buffers are reused.  The epilogue reads the
// accumulator rows of each warp's TMEM lane quarter.
#include <algorithm>
#include <cuda_bf16.h>
#include "hs_internal.cuh"
#include "hs_device.cuh"
#include "hs_tc.cuh"
#include "hs3d_tc.cuh"

namespace hs {
namespace {

constexpr int TM = 128;        // tile rows (MMA M)
constexpr int TNC = 32;        // tile columns, complex
constexpr int TN = 2 * TNC;    // MMA N (real)
constexpr int KC = 16;         // complex K per chunk
constexpr int KR = 2 * KC;     // real K per chunk
// K-adjacent core matrices are LBO bytes apart: one 16-byte pad after each
// k-group of rows keeps the 16-byte stores of 8 consecutive k-groups in
// distinct banks.
constexpr uint32_t A_LBO = TM * 16 + 16, B_LBO = TN * 16 + 16;

// Operand formats: TF32 (4-byte elements, core-matrix rows of 4 k-values,
// MMA K = 8, kind::tf32) or BF16 (2-byte elements, rows of 8 k-values,
// MMA K = 16, kind::f16 with BF16 inputs).  Both accumulate in FP32.
template <bool BF> struct Fmt {
  using E = float;
  static constexpr int G = 4;                 // k-values per 16-byte core-matrix row
  static constexpr int MK = 8;                // K of one MMA
  static constexpr uint32_t IDESC = tc_idesc(2u, TM, TN);
  static __device__ __forceinline__ E hi(float x, bool split) {
    return split ? __uint_as_float(__float_as_uint(x) & 0xFFFFE000u) : x;
  }
  static __device__ __forceinline__ float val(E x) { return x; }
  static __device__ __forceinline__ E lo(float x, E h) { return x - h; }
  static __device__ __forceinline__ void mma(uint32_t t, uint64_t a, uint64_t b, uint32_t acc) {
    tc_mma_tf32(t, a, b, IDESC, acc);
  }
};
template <> struct Fmt<true> {
  using E = __nv_bfloat16;
  static constexpr int G = 8;
  static constexpr int MK = 16;
  static constexpr uint32_t IDESC = tc_idesc(1u, TM, TN);
  static __device__ __forceinline__ E hi(float x, bool) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float val(E x) { return __bfloat162float(x); }
  static __device__ __forceinline__ E lo(float x, E h) { return __float2bfloat16_rn(x - __bfloat162float(h)); }
  static __device__ __forceinline__ void mma(uint32_t t, uint64_t a, uint64_t b, uint32_t acc) {
    tc_mma_f16(t, a, b, IDESC, acc);
  }
};

template <bool BF> constexpr uint32_t a_bytes() { return (KR / Fmt<BF>::G) * A_LBO; }
template <bool BF> constexpr uint32_t b_bytes() { return (KR / Fmt<BF>::G) * B_LBO; }
// Shared memory: the two precision halves of A and B plus the barrier.
template <bool BF> constexpr uint32_t smem_bytes() { return 2 * a_bytes<BF>() + 2 * b_bytes<BF>() + 16; }

// element (row r, real k) of a [k/G][rows][G] operand with row groups lbo bytes apart
template <typename E, int G>
__device__ __forceinline__ void put(E* buf, uint32_t lbo, int r, int k, E v) {
  buf[(k / G) * (lbo / sizeof(E)) + r * G + (k % G)] = v;
}

template <bool BF>
__global__ void __launch_bounds__(128, 4) zgemm_tc_kernel(const TcGemmJob* jobs, const TcGemmTile* tiles, int split,
                                                         int* status, long long spin) {
  using F = Fmt<BF>;
  using E = typename F::E;
  constexpr int G = F::G;
  constexpr uint32_t AB = a_bytes<BF>(), BB = b_bytes<BF>();
  extern __shared__ __align__(1024) unsigned char sm[];
  E* Ah = reinterpret_cast<E*>(sm);
  E* Al = reinterpret_cast<E*>(sm + AB);
  E* Bh = reinterpret_cast<E*>(sm + 2 * AB);
  E* Bl = reinterpret_cast<E*>(sm + 2 * AB + BB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * AB + 2 * BB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcGemmTile tl = tiles[blockIdx.x];
  const TcGemmJob jb = jobs[tl.job];
  const c64* A = static_cast<const c64*>(jb.A);
  const c64* B = static_cast<const c64*>(jb.B);
  c64* Cm = static_cast<c64*>(jb.C);
  const int m0 = tl.tm * TM, n0 = tl.tn * TNC;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, TN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
  uint32_t phase = 0;
  bool ok = true;
  const int nchunks = (jb.K + KC - 1) / KC;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int k0 = ch * KC;
    // A chunk: 128 rows x k-groups of G/2 complex (one 16-byte core-matrix
    // row each); consecutive threads read consecutive pieces of one row
    constexpr int CG = G / 2;   // complex values per group
    for (int e = tid; e < TM * (KC / CG); e += blockDim.x) {
      const int row = e / (KC / CG), kg = e % (KC / CG);
      const int m = m0 + row, k = k0 + CG * kg;
      float x[G];
#pragma unroll
      for (int q = 0; q < CG; ++q) {
        c64 v{0.f, 0.f};
        if (m < jb.M && k + q < jb.K) v = A[(long long)m * jb.lda + k + q];
        x[2 * q] = v.re;
        x[2 * q + 1] = v.im;
      }
      __align__(16) E hx[G], lx[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        hx[q] = F::hi(x[q], split != 0);
        lx[q] = F::lo(x[q], hx[q]);
      }
      *reinterpret_cast<uint4*>(Ah + kg * (A_LBO / sizeof(E)) + row * G) = *reinterpret_cast<const uint4*>(hx);
      if (split)
        *reinterpret_cast<uint4*>(Al + kg * (A_LBO / sizeof(E)) + row * G) = *reinterpret_cast<const uint4*>(lx);
    }
    // Bt chunk: (k, n) pairs of the chunk, 4 real entries each
    for (int e = tid; e < KC * TNC; e += blockDim.x) {
      const int kk = e / TNC, nn = e % TNC;
      const int k = k0 + kk, n = n0 + nn;
      c64 v{0.f, 0.f};
      if (k < jb.K && n < jb.N) v = B[(long long)k * jb.ldb + n];
      const float vals[4] = {v.re, -v.im, v.im, v.re};   // (c, d) = (0,0), (0,1), (1,0), (1,1)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = 2 * nn + (q >> 1), col = 2 * kk + (q & 1);
        const E h = F::hi(vals[q], split != 0);
        put<E, G>(Bh, B_LBO, row, col, h);
        if (split) put<E, G>(Bl, B_LBO, row, col, F::lo(vals[q], h));
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int kk = 0; kk < KR / F::MK; ++kk) {
        // one MMA spans two K-adjacent core matrices
        const uint32_t ao = (uint32_t)(2 * kk) * A_LBO, bo = (uint32_t)(2 * kk) * B_LBO;
        const uint32_t first = (ch == 0 && kk == 0) ? 0u : 1u;
        F::mma(tmem, tc_smem_desc(ah + ao, A_LBO, 128u), tc_smem_desc(bh + bo, B_LBO, 128u), first);
        if (split) {
          F::mma(tmem, tc_smem_desc(ah + ao, A_LBO, 128u), tc_smem_desc(bl + bo, B_LBO, 128u), 1u);
          F::mma(tmem, tc_smem_desc(al + ao, A_LBO, 128u), tc_smem_desc(bh + bo, B_LBO, 128u), 1u);
        }
      }
      tc_commit(bar);
    }
    __syncwarp();
    const bool landed = mbar_wait_bounded(bar, phase, spin);
    phase ^= 1u;
    ok = __syncthreads_and(landed) != 0;
    if (!ok) break;
  }
  if (ok) {
    tc_fence_after();
    uint32_t v0[32], v1[32];
    tc_ld32(tmem + ((uint32_t)(warp * 32) << 16), v0);
    tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, v1);
    const int m = m0 + warp * 32 + lane;
    if (m < jb.M) {
#pragma unroll
      for (int j = 0; j < TNC; ++j) {
        const int n = n0 + j;
        if (n >= jb.N) break;
        const float re = __uint_as_float(j < 16 ? v0[2 * j] : v1[2 * j - 32]);
        const float im = __uint_as_float(j < 16 ? v0[2 * j + 1] : v1[2 * j + 1 - 32]);
        c64& dst = Cm[(long long)m * jb.ldc + n];
        const c64 val{jb.alpha * re, jb.alpha * im};
        dst = jb.beta ? c64{dst.re + val.re, dst.im + val.im} : val;
      }
    }
  } else {
    (void)mbar_wait_bounded(bar, phase ^ 1u, 1LL << 30);
    if (tid == 0) set_status(status, HS_ETIMEOUT, -6, tl.job);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, TN);
}

}  // namespace

int zgemm_tc_launch(const TcGemmJob* d_jobs, const TcGemmTile* d_tiles, int ntiles, int mode, int* status,
                    long long spin, cudaStream_t s) {
  if (ntiles <= 0) return HS_OK;
  const bool bf = mode == 2 || mode == 4;
  const int split = (mode == 3 || mode == 4) ? 1 : 0;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(zgemm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<false>());
    cudaFuncSetAttribute(zgemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<true>());
  });
  note_launch();
  if (bf)
    zgemm_tc_kernel<true><<<ntiles, 128, smem_bytes<true>(), s>>>(d_jobs, d_tiles, split, status, spin);
  else
    zgemm_tc_kernel<false><<<ntiles, 128, smem_bytes<false>(), s>>>(d_jobs, d_tiles, split, status, spin);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

void zgemm_tc_tiles(const std::vector<TcGemmJob>& jobs, int job0, std::vector<TcGemmTile>& tiles) {
  for (int t = 0; t < (int)jobs.size(); ++t)
    for (int tm = 0; tm < (jobs[t].M + TM - 1) / TM; ++tm)
      for (int tn = 0; tn < (jobs[t].N + TNC - 1) / TNC; ++tn) tiles.push_back({job0 + t, tm, tn});
}

int zgemm_tc_batched(const std::vector<TcGemmJob>& jobs, int mode, int* status, long long spin, cudaStream_t s) {
  const bool bf = mode == 2 || mode == 4;
  const int split = (mode == 3 || mode == 4) ? 1 : 0;
  if (jobs.empty()) return HS_OK;
  std::vector<TcGemmTile> tiles;
  for (int t = 0; t < (int)jobs.size(); ++t)
    for (int tm = 0; tm < (jobs[t].M + TM - 1) / TM; ++tm)
      for (int tn = 0; tn < (jobs[t].N + TNC - 1) / TNC; ++tn) tiles.push_back({t, tm, tn});
  TcGemmJob* dj = nullptr;
  TcGemmTile* dt = nullptr;
  HS_CUDA_TRY(cudaMalloc(&dj, jobs.size() * sizeof(TcGemmJob)));
  if (cudaMalloc(&dt, tiles.size() * sizeof(TcGemmTile)) != cudaSuccess) {
    cudaFree(dj);
    return HS_ENOMEM;
  }
  cudaMemcpyAsync(dj, jobs.data(), jobs.size() * sizeof(TcGemmJob), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(TcGemmTile), cudaMemcpyHostToDevice, s);
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(zgemm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<false>());
    cudaFuncSetAttribute(zgemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<true>());
  });
  note_launch();
  if (bf)
    zgemm_tc_kernel<true><<<(int)tiles.size(), 128, smem_bytes<true>(), s>>>(dj, dt, split, status, spin);
  else
    zgemm_tc_kernel<false><<<(int)tiles.size(), 128, smem_bytes<false>(), s>>>(dj, dt, split, status, spin);
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(dj);
  cudaFree(dt);
  if (e != cudaSuccess) return cuda_status(e);
  if (e2 != cudaSuccess) return cuda_status(e2);
  return HS_OK;
}

}  // namespace hs
