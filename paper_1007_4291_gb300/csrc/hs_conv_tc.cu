// Layer 2 of the post-correction (3x3 convolution, 32 -> 32 channels, bias,
// ReLU, bfloat16 out) as an implicit GEMM on the fifth-generation tensor
// cores: D[128 pixels][32 co] = sum over 9 taps and 32 ci of
// A_tap[128 pixels][32 ci] * B_tap[32 ci][32 co], FP32 accumulation in tensor
// memory.
//
// A tile is one run of 128 consecutive pixels along x1 in one image row.  Its
// three input rows (y-1, y, y+1) with one halo column on each side sit in
// shared memory as four channel groups of 8 channels (16 bytes per pixel),
// each group a [3][130] array of 16-byte chunks.  In that layout every
// 8-pixel x 8-channel block is 128 contiguous bytes, i.e. a core matrix of the
// K-major, non-swizzled operand layout, so the operand of tap (ky, kx) is the
// same buffer read from a start address shifted by (ky * 130 + kx) pixels:
// no im2col copy.  Per tile one thread issues 18 MMAs (9 taps x 2 halves of
// K = 16) of shape M = 128, N = 32, K = 16 and commits them to an mbarrier;
// the four warps then read the accumulator rows of their TMEM lane quarter
// (thread = pixel, 32 columns = channels), add the bias, apply ReLU and store
// the pixel's 64 bytes.
#include <algorithm>
#include <cuda_bf16.h>
#include "hs_cnn.cuh"
#include "hs_device.cuh"
#include "hs_tc.cuh"

namespace hs {
namespace {

constexpr int TM = 128;                 // pixels per tile (MMA M)
constexpr int TWP = TM + 2;             // haloed row length
constexpr uint32_t AG = 3 * TWP * 16;   // bytes of one 8-channel group of the A tile
constexpr uint32_t A_BYTES = 4 * AG;    // 24,960
constexpr int KSTEPS = 18;              // 9 taps x 2 halves of 16 channels
constexpr int NC = 32;                  // output channels (MMA N)
constexpr uint32_t B_STEP = 2 * NC * 16;          // bytes of B per K-step
constexpr uint32_t B_BYTES = KSTEPS * B_STEP;     // 18,432
constexpr uint32_t TMEM_COLS = 32;
// Shared memory per CTA: A tile, B operand, mbarrier, TMEM slot, bias; four
// CTAs share an SM (each holds 32 TMEM columns) so that one CTA's loads
// overlap the others' MMAs and epilogues.
constexpr uint32_t SMEM_BYTES = A_BYTES + B_BYTES + 16 + 32 * 4;
constexpr int CTAS_PER_SM = 4;

constexpr uint32_t IDESC = tc_idesc(1u, TM, NC);   // bf16 A and B, FP32 accumulator

// B operand of every K-step from the bf16-rounded FP32 weights W2[tap][ci][co]:
// step s = (tap, half), 16-byte rows (co, 8 consecutive ci), channel group c
// of the half at c * NC * 16, row co at co * 16.
__global__ void pack_w2_kernel(const float* __restrict__ wq, uint4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // (s, c, co)
  if (i >= KSTEPS * 2 * NC) return;
  const int co = i % NC, c = (i / NC) % 2, s = i / (2 * NC);
  const int tap = s >> 1, ci0 = (s & 1) * 16 + c * 8;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __float2bfloat16_rn(wq[CNN_OFF_W2 + (tap * CH + ci0 + q) * CH + co]);
  out[i] = *reinterpret_cast<const uint4*>(v);
}

__global__ void __launch_bounds__(128, CTAS_PER_SM) conv2_tc_kernel(const __nv_bfloat16* __restrict__ x, int n, int R,
                                                        const uint4* __restrict__ wpk, const float* __restrict__ wq,
                                                        __nv_bfloat16* __restrict__ y, int* status, long long spin) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As = sm;
  unsigned char* Bs = sm + A_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + A_BYTES + B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  float* bias = reinterpret_cast<float*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (uint32_t i = tid; i < B_BYTES / 16; i += blockDim.x) reinterpret_cast<uint4*>(Bs)[i] = wpk[i];
  if (tid < NC) bias[tid] = wq[CNN_OFF_W2 + CNN_W2 + tid];
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);

  const int tpr = (n + TM - 1) / TM;
  const long long ntiles = (long long)R * n * tpr;
  uint32_t phase = 0;
  bool ok = true;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int k = (int)(t / ((long long)n * tpr));
    const int rem = (int)(t % ((long long)n * tpr));
    const int row = rem / tpr, x0 = (rem % tpr) * TM;
    const __nv_bfloat16* img = x + (long long)k * n * n * CH;
    // A tile: 3 rows x 130 pixels x 4 channel groups of 16 bytes
    for (int i = tid; i < 3 * TWP * 4; i += blockDim.x) {
      const int g = i & 3, pix = i >> 2;
      const int rr = pix / TWP, cc = pix % TWP;
      const int yy = row + rr - 1, xx = x0 + cc - 1;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (yy >= 0 && yy < n && xx >= 0 && xx < n) v = reinterpret_cast<const uint4*>(img + ((long long)yy * n + xx) * CH)[g];
      *reinterpret_cast<uint4*>(As + g * AG + pix * 16) = v;
    }
    fence_proxy_async_smem();   // the tensor core reads through the async proxy
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int s = 0; s < KSTEPS; ++s) {
        const int tap = s >> 1, h = s & 1, ky = tap / 3, kx = tap % 3;
        const uint64_t ad = tc_smem_desc(a_base + (uint32_t)(2 * h) * AG + (uint32_t)(ky * TWP + kx) * 16u, AG, 128u);
        const uint64_t bd = tc_smem_desc(b_base + (uint32_t)s * B_STEP, NC * 16u, 128u);
        tc_mma_f16(tmem, ad, bd, IDESC, s > 0 ? 1u : 0u);
      }
      tc_commit(bar);
    }
    __syncwarp();
    const bool landed = mbar_wait_bounded(bar, phase, spin);
    phase ^= 1u;
    ok = __syncthreads_and(landed) != 0;
    if (!ok) break;
    tc_fence_after();
    uint32_t v[32];
    tc_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int px = x0 + warp * 32 + lane;
    if (px < n) {
      __align__(16) __nv_bfloat162 o[CH / 2];
#pragma unroll
      for (int c = 0; c < CH / 2; ++c)
        o[c] = __floats2bfloat162_rn(fmaxf(__uint_as_float(v[2 * c]) + bias[2 * c], 0.f),
                                     fmaxf(__uint_as_float(v[2 * c + 1]) + bias[2 * c + 1], 0.f));
      uint4* dst = reinterpret_cast<uint4*>(y + (((long long)k * n + row) * n + px) * CH);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
    }
    tc_fence_before();
    __syncthreads();   // accumulator and A tile free for the next tile
  }
  if (!ok) {
    // the committed MMAs must finish before their accumulator is released
    (void)mbar_wait_bounded(bar, phase ^ 1u, 1LL << 30);
    if (tid == 0) set_status(status, HS_ETIMEOUT, -5, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, TMEM_COLS);
}

}  // namespace

int conv2_tc(Cnn& c, int R, int n, cudaStream_t s) {
  if (!c.w2tc) HS_CUDA_TRY(cudaMalloc(&c.w2tc, B_BYTES));
  if (!c.status) {
    HS_CUDA_TRY(cudaMalloc(&c.status, 4 * sizeof(int)));
    HS_CUDA_TRY(cudaMemset(c.status, 0, 4 * sizeof(int)));
  }
  if (c.w2tc_version != c.t) {
    note_launch();
    pack_w2_kernel<<<(KSTEPS * 2 * NC + 127) / 128, 128, 0, s>>>(c.wq, reinterpret_cast<uint4*>(c.w2tc));
    c.w2tc_version = c.t;
  }
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(conv2_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  });
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (long long)R * n * ((n + TM - 1) / TM);
  const int grid = (int)std::min<long long>(ntiles, (long long)sms * CTAS_PER_SM);
  note_launch();
  conv2_tc_kernel<<<grid, 128, SMEM_BYTES, s>>>(c.h1, n, R, reinterpret_cast<const uint4*>(c.w2tc), c.wq, c.h2,
                                                c.status, 1LL << 30);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_status(e);
}

}  // namespace hs
