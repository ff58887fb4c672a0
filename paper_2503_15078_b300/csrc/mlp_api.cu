// C ABI of the warm-start network: creation, parameters, inference and training on the
// device (the kernels are in k_mlp.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "devguard.hpp"
#include "mlp.cuh"
#include "silg.h"

struct sim_mlp_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  silg::MlpDev m{};
  std::vector<void*> allocs;
  int step = 0;  // Adam steps taken
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
    allocs.push_back(p);
    cudaMemsetAsync(p, 0, std::max<size_t>(1, count) * sizeof(T), stream);
    return static_cast<T*>(p);
  }
  ~sim_mlp_s() {
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : allocs) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return SIM_OK;
  if (e == cudaErrorMemoryAllocation) return SIM_ENOMEM;
  return SIM_ECUDA;
}

int finish(sim_mlp_t* n) {
  cudaError_t e = cudaStreamSynchronize(n->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return status_of(e);
}

// features (n x SIM_MLP_FEATURES, host) -> device rows padded to the network's input width
float* upload_features(sim_mlp_t* n, const float* X, int rows, std::vector<void*>& tmp) {
  std::vector<float> h((size_t)rows * silg::kMlpIn, 0.f);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < silg::kMlpNF; ++c) h[(size_t)r * silg::kMlpIn + c] = X[(size_t)r * silg::kMlpNF + c];
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(1, h.size()) * sizeof(float)) != cudaSuccess) return nullptr;
  tmp.push_back(p);
  cudaMemcpyAsync(p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream);
  return static_cast<float*>(p);
}

float* upload(sim_mlp_t* n, const void* src, size_t bytes, std::vector<void*>& tmp) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(1, bytes)) != cudaSuccess) return nullptr;
  tmp.push_back(p);
  if (bytes && src) cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, n->stream);
  return static_cast<float*>(p);
}

void release(sim_mlp_t* n, std::vector<void*>& tmp) {
  cudaStreamSynchronize(n->stream);
  for (void* p : tmp) cudaFree(p);
  tmp.clear();
}

// splitmix64 (Steele, Lea, Flood 2014): the generator of the initial weights and of the
// training order
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

extern "C" {

// the network's device buffers (for sim_set_warmstart)
const silg::MlpDev* silg_mlp_dev(const sim_mlp_t* net, int* device) {
  if (!net) return nullptr;
  if (device) *device = net->device;
  return &net->m;
}

int sim_mlp_create(int32_t device, int32_t max_batch, sim_mlp_t** out) {
  if (!out || max_batch <= 0) return SIM_EINVAL;
  silg::DeviceGuard dg;   // the caller's current device is restored on return
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return SIM_ECUDA;
  if (device < 0 || device >= ndev) return SIM_EINVAL;
  sim_mlp_t* n = new (std::nothrow) sim_mlp_s();
  if (!n) return SIM_ENOMEM;
  try {
    n->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess ||
        silg::mlp_setup() != 0) {
      delete n;
      return SIM_ECUDA;
    }
    silg::MlpDev& m = n->m;
    m.max_ctas = (max_batch + silg::kMlpRows - 1) / silg::kMlpRows;
    m.theta = n->alloc<float>(silg::kMlpParams);
    m.adam_m = n->alloc<float>(silg::kMlpParams);
    m.adam_v = n->alloc<float>(silg::kMlpParams);
    m.w_row = n->alloc<__nv_bfloat16>(silg::kWRowElems);
    m.w_t = n->alloc<__nv_bfloat16>(silg::kWTElems);
    m.grad = n->alloc<float>(silg::kMlpParams);
    m.part = n->alloc<float>((size_t)m.max_ctas * silg::kMlpParams);
    m.part_loss = n->alloc<float>(m.max_ctas);
    m.loss = n->alloc<float>(1);
    m.err = n->alloc<int>(1);
    m.tc = 0;
  } catch (const std::bad_alloc&) {
    delete n;
    return SIM_ENOMEM;
  }
  int st = finish(n);
  if (st != SIM_OK) {
    delete n;
    return st;
  }
  *out = n;
  return SIM_OK;
}

int sim_mlp_set_tensor_cores(sim_mlp_t* n, int32_t kind) {
  if (!n || (kind != SIM_MLP_MMA_SYNC && kind != SIM_MLP_TCGEN05)) return SIM_EINVAL;
  n->m.tc = kind == SIM_MLP_TCGEN05 ? 1 : 0;
  return SIM_OK;
}

void sim_mlp_destroy(sim_mlp_t* n) {
  if (!n) return;
  silg::DeviceGuard dg(n->device);
  delete n;
}

int sim_mlp_set_params(sim_mlp_t* n, const float* theta) {
  if (!n || !theta) return SIM_EINVAL;
  silg::DeviceGuard dg(n->device);
  cudaMemcpyAsync(n->m.theta, theta, sizeof(float) * silg::kMlpParams, cudaMemcpyHostToDevice, n->stream);
  cudaMemsetAsync(n->m.adam_m, 0, sizeof(float) * silg::kMlpParams, n->stream);
  cudaMemsetAsync(n->m.adam_v, 0, sizeof(float) * silg::kMlpParams, n->stream);
  n->step = 0;
  silg::mlp_launch_convert(n->m, n->stream);
  return finish(n);
}

int sim_mlp_init(sim_mlp_t* n, uint64_t seed) {
  if (!n) return SIM_EINVAL;
  // weights uniform in +-sqrt(6 / (fan_in + fan_out)), biases zero; the padded input rows
  // of W1 and output columns of W4 zero
  std::vector<float> th(silg::kMlpParams, 0.f);
  uint64_t s = seed;
  struct L { int off, fi, fo, used_i, used_o; };
  const L layers[] = {{silg::kOffW1, silg::kMlpIn, silg::kMlpH, silg::kMlpNF, silg::kMlpH},
                      {silg::kOffW2, silg::kMlpH, silg::kMlpH, silg::kMlpH, silg::kMlpH},
                      {silg::kOffW3, silg::kMlpH, silg::kMlpH, silg::kMlpH, silg::kMlpH},
                      {silg::kOffW4, silg::kMlpH, silg::kMlpOut, silg::kMlpH, silg::kMlpNY}};
  for (const L& l : layers) {
    const double a = std::sqrt(6.0 / (l.fi + l.fo));
    for (int i = 0; i < l.fi; ++i)
      for (int o = 0; o < l.fo; ++o) {
        const double u = (2.0 * uniform01(s) - 1.0) * a;
        th[l.off + i * l.fo + o] = (i < l.used_i && o < l.used_o) ? (float)u : 0.f;
      }
  }
  return sim_mlp_set_params(n, th.data());
}

int sim_mlp_get_params(const sim_mlp_t* n, float* theta) {
  if (!n || !theta) return SIM_EINVAL;
  silg::DeviceGuard dg(n->device);
  cudaStreamSynchronize(n->stream);
  return status_of(cudaMemcpy(theta, n->m.theta, sizeof(float) * silg::kMlpParams, cudaMemcpyDeviceToHost));
}

int sim_mlp_forward(sim_mlp_t* n, const float* X, int32_t rows, float* Y) {
  if (!n || rows < 0 || (rows > 0 && (!X || !Y))) return SIM_EINVAL;
  if (rows == 0) return SIM_OK;
  silg::DeviceGuard dg(n->device);
  std::vector<void*> tmp;
  float* dx = upload_features(n, X, rows, tmp);
  float* dy = upload(n, nullptr, sizeof(float) * rows * silg::kMlpOut, tmp);
  if (!dx || !dy) {
    release(n, tmp);
    return SIM_ENOMEM;
  }
  silg::mlp_launch_infer(n->m, dx, rows, dy, n->stream);
  std::vector<float> y((size_t)rows * silg::kMlpOut);
  int err = 0;
  cudaMemcpyAsync(y.data(), dy, y.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
  cudaMemcpyAsync(&err, n->m.err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
  cudaMemsetAsync(n->m.err, 0, sizeof(int), n->stream);
  int st = finish(n);
  release(n, tmp);
  if (st != SIM_OK) return st;
  if (err) return SIM_ETIMEOUT;
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < silg::kMlpNY; ++c) Y[(size_t)r * silg::kMlpNY + c] = y[(size_t)r * silg::kMlpOut + c];
  return SIM_OK;
}

int sim_mlp_gradient(sim_mlp_t* n, const float* X, const float* T, int32_t rows, float* grad,
                     float* loss) {
  if (!n || !X || !T || rows <= 0) return SIM_EINVAL;
  if (rows > n->m.max_ctas * silg::kMlpRows) return SIM_ECAPACITY;
  silg::DeviceGuard dg(n->device);
  std::vector<void*> tmp;
  float* dx = upload_features(n, X, rows, tmp);
  float* dt = upload(n, T, sizeof(float) * rows * silg::kMlpNY, tmp);
  if (!dx || !dt) {
    release(n, tmp);
    return SIM_ENOMEM;
  }
  silg::mlp_launch_gradient(n->m, dx, dt, nullptr, rows, n->stream);
  if (grad)
    cudaMemcpyAsync(grad, n->m.grad, sizeof(float) * silg::kMlpParams, cudaMemcpyDeviceToHost, n->stream);
  if (loss) cudaMemcpyAsync(loss, n->m.loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream);
  int st = finish(n);
  release(n, tmp);
  return st;
}

int sim_mlp_train(sim_mlp_t* n, const float* X, const float* T, int32_t rows, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, float* epoch_loss) {
  if (!n || !X || !T || rows <= 0 || epochs < 0 || batch <= 0 || !(lr > 0)) return SIM_EINVAL;
  if (batch > n->m.max_ctas * silg::kMlpRows) return SIM_ECAPACITY;
  silg::DeviceGuard dg(n->device);
  std::vector<void*> tmp;
  float* dx = upload_features(n, X, rows, tmp);
  float* dt = upload(n, T, sizeof(float) * rows * silg::kMlpNY, tmp);
  int* didx = reinterpret_cast<int*>(upload(n, nullptr, sizeof(int) * rows, tmp));
  if (!dx || !dt || !didx) {
    release(n, tmp);
    return SIM_ENOMEM;
  }
  std::vector<int> order(rows);
  uint64_t s = seed;
  for (int e = 0; e < epochs; ++e) {
    // a fresh permutation per epoch (Fisher-Yates with the seeded generator)
    std::iota(order.begin(), order.end(), 0);
    for (int i = rows - 1; i > 0; --i) std::swap(order[i], order[splitmix64(s) % (uint64_t)(i + 1)]);
    cudaMemcpyAsync(didx, order.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, n->stream);
    double lsum = 0;
    int nb = 0;
    for (int b0 = 0; b0 < rows; b0 += batch) {
      const int bn = std::min(batch, rows - b0);
      silg::mlp_launch_gradient(n->m, dx, dt, didx + b0, bn, n->stream);
      silg::mlp_launch_adam(n->m, ++n->step, lr, n->stream);
      if (epoch_loss) {
        float l = 0;
        cudaMemcpyAsync(&l, n->m.loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream);
        cudaStreamSynchronize(n->stream);
        lsum += l;
        ++nb;
      }
    }
    if (epoch_loss) epoch_loss[e] = (float)(lsum / std::max(1, nb));
    // the order array is rewritten next epoch: wait for this epoch's launches
    cudaStreamSynchronize(n->stream);
  }
  int st = finish(n);
  release(n, tmp);
  return st;
}

}  // extern "C"
