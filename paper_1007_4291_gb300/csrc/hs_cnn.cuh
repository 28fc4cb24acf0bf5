// Convolutional post-correction: parameter layout, the network object and
// the launchers shared by hs_cnn.cu, hs_conv_tc.cu and the solver.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "hs_internal.cuh"

namespace hs {

constexpr int CH = 32;                       // hidden channels
constexpr int CNN_W1 = 3 * 3 * 2 * CH;       // W1[3][3][2][32]
constexpr int CNN_W2 = 3 * 3 * CH * CH;      // W2[3][3][32][32]
constexpr int CNN_W3 = 3 * 3 * CH * 2;       // W3[3][3][32][2]
constexpr int CNN_OFF_W1 = 0;                // then b1[32]
constexpr int CNN_OFF_W2 = CNN_W1 + CH;      // then b2[32]
constexpr int CNN_OFF_W3 = CNN_OFF_W2 + CNN_W2 + CH;   // then b3[2]
constexpr int CNN_NPARAM = CNN_OFF_W3 + CNN_W3 + 2;    // 10434

#define HS_TRY_INT(expr) do { int _s = (expr); if (_s != HS_OK) return _s; } while (0)

struct Cnn {
  float* theta = nullptr;   // FP32 master parameters [CNN_NPARAM]
  float* wq = nullptr;      // the same rounded to bfloat16 (stored as float): forward weights
  float* grad = nullptr;    // dL/dtheta
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  int t = 0;                // Adam steps taken
  bool tensor_cores = false; // layer 2 on tcgen05 (else the FP32 reference kernel)
  // workspace, grown on demand
  __nv_bfloat16* h1 = nullptr;   // [R][n][n][32]
  __nv_bfloat16* h2 = nullptr;
  double* sums = nullptr;        // [R] sums of |r|^2, the loss, [R] residual norms, residual loss
  float* dout = nullptr;         // [R][n][n][2]  dL/do
  float* da2 = nullptr;          // [R][n][n][32] dL/da2
  float* da1 = nullptr;          // [R][n][n][32] dL/da1
  void* w2tc = nullptr;          // layer-2 weights in the tensor-core operand layout
  int* status = nullptr;         // device status word of the tensor-core kernel (expired waits)
  void* rbuf = nullptr;          // residual training: c, A c, A conj(d) (complex64, ABI layout)
  int w2tc_version = -1;         // Adam step the packed copy was made from
  size_t cap_px = 0, cap_train = 0;
  int cap_r = 0;
  int reserve(int R, int n);
  int reserve_train(int R, int n);
  ~Cnn();
};

// layer 2 (32 -> 32, bias, ReLU, bf16 out) on the tensor cores: c.h1 -> c.h2
int conv2_tc(Cnn& c, int R, int n, cudaStream_t s);
// z += s N(x / s), s = rms(x), for vectors in the solver's internal layout
// ([point][rhs]) of type HS_C64 or HS_C128; x and z may alias
int cnn_correct(Cnn& c, const void* x, void* z, int type, int R, int n, cudaStream_t s);

}  // namespace hs
