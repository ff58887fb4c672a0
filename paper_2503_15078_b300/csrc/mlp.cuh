// The warm-start network on the device (internal header): layout of its parameters and
// the launchers of its inference and training kernels.
//
// Network: NF = 11 per-contact features (padded to IN = 16) -> three hidden layers of
// H = 128 units with GELU(x) = x Phi(x) -> a linear layer to OUT = 8 outputs, of which the
// first NY = 4 are used. Parameters are one flat FP32 vector in the order W1 (IN x H, row =
// input), b1, W2 (H x H), b2, W3 (H x H), b3, W4 (H x OUT), b4. The tensor-core kernels
// read BF16 copies of the weights (FP32 accumulation); the FP32 vector is the master copy
// that the optimiser updates.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace silg {

constexpr int kMlpNF = 11, kMlpIn = 16, kMlpH = 128, kMlpOut = 8, kMlpNY = 4;
// offsets in the flat parameter vector
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpIn * kMlpH;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH * kMlpH;
constexpr int kOffW4 = kOffB3 + kMlpH;
constexpr int kOffB4 = kOffW4 + kMlpH * kMlpOut;
constexpr int kMlpParams = kOffB4 + kMlpOut;  // 36232

// BF16 weight copies with padded rows (strides chosen so that the fragment loads of the
// eight row groups of a warp fall in distinct shared-memory banks)
constexpr int kLdH = kMlpH + 8;     // 136: rows of 128 values
constexpr int kLdIn = kMlpIn + 8;   // 24: rows of 16 values
constexpr int kLdOut = kMlpOut + 8; // 16: rows of 8 values (W4 row-major)
// row-major [in][out] (training) and transposed [out][in] (inference) sizes, elements
constexpr int kWRowElems = kMlpIn * kLdH + 2 * kMlpH * kLdH + kMlpH * kLdOut;
constexpr int kWTElems = kMlpH * kLdIn + 2 * kMlpH * kLdH + kMlpOut * kLdH;
constexpr int kMlpRows = 64;        // rows (samples) per CTA

// error bit set by a tensor-core inference whose wait gave up (the simulator's timeout bit)
constexpr int kMlpErrTimeout = 4;

struct MlpDev {
  float* theta;            // master parameters (kMlpParams)
  float* adam_m;
  float* adam_v;
  __nv_bfloat16* w_row;    // W1..W4 row-major, padded (training kernel)
  __nv_bfloat16* w_t;      // W1..W4 transposed, padded (inference kernel)
  float* grad;             // kMlpParams
  float* part;             // per-CTA partial gradients (max_ctas x kMlpParams)
  float* part_loss;        // max_ctas
  float* loss;             // 1
  int max_ctas;
  int tc;                  // inference on the 5th-generation tensor cores (tcgen05, TMEM): 1;
                           // warp-level mma.sync: 0
  int* err;                // error word of the inference (kMlpErrTimeout), or null
};

// shared-memory limits of the kernels (per device, before the first launch); 0 on success
int mlp_setup();
// BF16 copies of the master parameters
void mlp_launch_convert(const MlpDev& m, cudaStream_t s);
// Y (n x kMlpOut, FP32) = network(X (n x kMlpIn, FP32)); rows_idx (optional) selects X rows
void mlp_launch_infer(const MlpDev& m, const float* X, int n, float* Y, cudaStream_t s);
// the same for min(*n_dev, n_max) rows, the count read on the device (graph capture)
void mlp_launch_infer_dev(const MlpDev& m, const float* X, const int* n_dev, int n_max, float* Y,
                          cudaStream_t s);
// the tcgen05 inference (k_mlp_tc.cu): its shared-memory limit, and its launch (n_dev
// optional); both inference launchers above dispatch to it when m.tc is set
int mlp_tc_setup();
void mlp_launch_infer_tc(const MlpDev& m, const float* X, int n, const int* n_dev, float* Y,
                         cudaStream_t s);
// gradient of the mean squared error over the batch rows idx[0..n) (all rows if idx is
// null) into m.grad, loss into m.loss; n <= m.max_ctas * kMlpRows
void mlp_launch_gradient(const MlpDev& m, const float* X, const float* T, const int* idx, int n,
                         cudaStream_t s);
// one Adam step (t counts from 1) on the master parameters, then the BF16 copies
void mlp_launch_adam(const MlpDev& m, int t, float lr, cudaStream_t s);

}  // namespace silg
