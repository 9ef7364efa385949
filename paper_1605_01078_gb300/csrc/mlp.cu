// Learned variant selector: a small MLP (22 -> 64 -> 64 -> 16, FP32, ReLU) that
// predicts, for each of 16 candidates -- classical, 1 or 2 levels of ABC, AB and Naive,
// and 3 levels of ABC, each with the 128x128 or the 64x64 block tile -- the log2 run time of a shape
// as a correction to the analytic performance model's prediction.  Its inputs are
// log2 m, log2 n, log2 k, the dtype and the model's log2 seconds for every candidate
// (which carry the padding of each tile, invisible in the sizes alone).  It stands in
// for the analytic model of Section 4.2 when choosing the implementation: the choice is
// the argmin of model + correction.
//
// Hand-written kernels: forward, loss gradient (forward + reverse mode per sample,
// per-block gradient sums in shared memory, one atomic add per parameter per block),
// Adam, and the single-shape selection used by strassen_select().
//
// Parameter vector (float): [W1 (64x22, row-major), b1 (64), W2 (64x64), b2 (64),
// W3 (16x64), b3 (16)].  Loss: masked mean squared error over measured candidates of
// (network output - (log2 measured seconds - model log2 seconds)).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace sgb {
namespace {

constexpr int kIn = kSelInputs, kH = 64, kOut = kSelCandidates;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kParams = ob3 + kOut;
constexpr int kBlock = 64;  // one thread per hidden unit

// Forward pass of one sample by a block of kH threads; x, h1, h2, z1, z2 in shared
// memory; returns with y[0..kOut) in shared memory.
__device__ void sample_forward(const float* P, const float* x, float* z1, float* h1, float* z2, float* h2,
                               float* y) {
  const int h = threadIdx.x;
  float acc = P[ob1 + h];
  for (int i = 0; i < kIn; ++i) acc += P[oW1 + h * kIn + i] * x[i];
  z1[h] = acc;
  h1[h] = acc > 0.f ? acc : 0.f;
  __syncthreads();
  acc = P[ob2 + h];
  for (int j = 0; j < kH; ++j) acc += P[oW2 + h * kH + j] * h1[j];
  z2[h] = acc;
  h2[h] = acc > 0.f ? acc : 0.f;
  __syncthreads();
  if (h < kOut) {
    float o = P[ob3 + h];
    for (int j = 0; j < kH; ++j) o += P[oW3 + h * kH + j] * h2[j];
    y[h] = o;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBlock) mlp_forward_kernel(const float* __restrict__ params,
                                                             const float* __restrict__ X, int batch,
                                                             float* __restrict__ Y) {
  __shared__ float P[kParams];
  __shared__ float x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], y[kOut];
  for (int i = threadIdx.x; i < kParams; i += kBlock) P[i] = params[i];
  __syncthreads();
  for (int s = blockIdx.x; s < batch; s += gridDim.x) {
    if (threadIdx.x < kIn) x[threadIdx.x] = X[s * kIn + threadIdx.x];
    __syncthreads();
    sample_forward(P, x, z1, h1, z2, h2, y);
    if (threadIdx.x < kOut) Y[s * kOut + threadIdx.x] = y[threadIdx.x];
    __syncthreads();
  }
}

// grad += d loss / d params over the block's samples; loss = sum mask (y - t)^2 * inv.
__global__ void __launch_bounds__(kBlock) mlp_grad_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ X,
                                                          const float* __restrict__ T,
                                                          const float* __restrict__ M, int batch, float inv,
                                                          float* __restrict__ grad) {
  __shared__ float P[kParams];
  __shared__ float G[kParams];
  __shared__ float x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], y[kOut], dy[kOut], dz2[kH];
  const int h = threadIdx.x;
  for (int i = h; i < kParams; i += kBlock) {
    P[i] = params[i];
    G[i] = 0.f;
  }
  __syncthreads();
  for (int s = blockIdx.x; s < batch; s += gridDim.x) {
    if (h < kIn) x[h] = X[s * kIn + h];
    __syncthreads();
    sample_forward(P, x, z1, h1, z2, h2, y);
    if (h < kOut) dy[h] = 2.f * M[s * kOut + h] * (y[h] - T[s * kOut + h]) * inv;
    __syncthreads();
    // layer 3: thread h owns column h of W3 and row h of the hidden state
    float dh2 = 0.f;
    for (int c = 0; c < kOut; ++c) {
      G[oW3 + c * kH + h] += dy[c] * h2[h];
      dh2 += dy[c] * P[oW3 + c * kH + h];
    }
    if (h < kOut) G[ob3 + h] += dy[h];
    const float d2 = z2[h] > 0.f ? dh2 : 0.f;
    dz2[h] = d2;
    __syncthreads();
    // layer 2: row h of W2
    for (int j = 0; j < kH; ++j) G[oW2 + h * kH + j] += d2 * h1[j];
    G[ob2 + h] += d2;
    float dh1 = 0.f;
    for (int r = 0; r < kH; ++r) dh1 += dz2[r] * P[oW2 + r * kH + h];
    const float d1 = z1[h] > 0.f ? dh1 : 0.f;
    for (int i = 0; i < kIn; ++i) G[oW1 + h * kIn + i] += d1 * x[i];
    G[ob1 + h] += d1;
    __syncthreads();
  }
  for (int i = h; i < kParams; i += kBlock) atomicAdd(&grad[i], G[i]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float mi = b1 * m[i] + (1.f - b1) * g[i];
    const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

struct SelectArgs {
  float x[kIn];
  float base[kOut];  // the analytic model's log2 seconds per candidate
  unsigned valid;    // bit c set: candidate c may be chosen
};

__global__ void __launch_bounds__(kBlock) mlp_select_kernel(const float* __restrict__ params,
                                                            const __grid_constant__ SelectArgs a,
                                                            int* __restrict__ out) {
  __shared__ float P[kParams];
  __shared__ float x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], y[kOut];
  for (int i = threadIdx.x; i < kParams; i += kBlock) P[i] = params[i];
  if (threadIdx.x < kIn) x[threadIdx.x] = a.x[threadIdx.x];
  __syncthreads();
  sample_forward(P, x, z1, h1, z2, h2, y);
  if (threadIdx.x == 0) {
    int best = -1;
    float bv = 0.f;
    for (int c = 0; c < kOut; ++c) {
      const float v = a.base[c] + y[c];
      if (((a.valid >> c) & 1u) && (best < 0 || v < bv)) {
        best = c;
        bv = v;
      }
    }
    *out = best;
  }
}

// ---------------------------------------------------------------- selector state

struct ShapeKey {
  int64_t m, n, k;
  int dtype;
  bool operator==(const ShapeKey& o) const { return m == o.m && n == o.n && k == o.k && dtype == o.dtype; }
};
struct ShapeKeyHash {
  size_t operator()(const ShapeKey& s) const {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t v : {(uint64_t)s.m, (uint64_t)s.n, (uint64_t)s.k, (uint64_t)s.dtype}) {
      h ^= v;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

std::mutex g_mlp_mu;
// The loaded network: a host copy, and per device a copy of it (made on the device's
// first selection), the result word and a private stream.
std::vector<float> g_sel_host;
unsigned g_sel_version = 0;  // bumped by every load; device copies of an older version are refreshed
struct SelDevice {
  float* params = nullptr;
  int* out = nullptr;
  cudaStream_t stream = nullptr;
  unsigned version = 0;
};
constexpr int kSelMaxDevices = 64;
SelDevice g_sel_dev[kSelMaxDevices];
unsigned g_sel_dtypes = 0x7u;  // bit d: use the network for dtype d
std::unordered_map<ShapeKey, int, ShapeKeyHash> g_sel_cache[kSelMaxDevices];  // choices per device

// The current device's copy of the network, made or refreshed if needed (may allocate
// and copy); null on failure.
SelDevice* sel_device(int dev) {
  SelDevice& sd = g_sel_dev[dev];
  if (!sd.params) {
    if (cudaMalloc(&sd.params, sizeof(float) * kParams) != cudaSuccess || cudaMalloc(&sd.out, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sd.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    sd.version = 0;
  }
  if (sd.version != g_sel_version) {
    if (cudaMemcpy(sd.params, g_sel_host.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    sd.version = g_sel_version;
  }
  return &sd;
}

int grid_for_batch(int batch) { return batch < 1 ? 1 : (batch < 1024 ? batch : 1024); }

}  // namespace

void selector_candidate(int c, int* levels, int* variant, int* tile) {
  if (c < 2 || c >= 14) {
    *levels = c < 2 ? 0 : 3;
    *variant = STRASSEN_ABC;
    *tile = c < 0 ? 0 : c % 2;
    return;
  }
  const int r = c - 2;
  *levels = 1 + r / 6;
  *variant = (r % 6) / 2;
  *tile = r % 2;
}

bool selector_candidate_valid(int c, int dtype) {
  if (c < 0 || c >= kOut) return false;
  if (dtype == STRASSEN_F64) return true;
  int lv, var, tile;
  selector_candidate(c, &lv, &var, &tile);
  return dtype == STRASSEN_F64_OZ_BF16 && var == STRASSEN_ABC && tile == 0;
}

void selector_features(int64_t m, int64_t n, int64_t k, int dtype, float* x, float* base) {
  x[0] = (float)((std::log2((double)m) - 11.0) / 3.0);
  x[1] = (float)((std::log2((double)n) - 11.0) / 3.0);
  x[2] = (float)((std::log2((double)k) - 11.0) / 3.0);
  x[3] = dtype == 0 ? 1.f : 0.f;
  x[4] = dtype == 1 ? 1.f : 0.f;
  x[5] = dtype == 2 ? 1.f : 0.f;
  for (int c = 0; c < kOut; ++c) {
    int lv, var, tile;
    selector_candidate(c, &lv, &var, &tile);
    // candidates that do not apply to the dtype carry the value of one that does
    if (!selector_candidate_valid(c, dtype)) {
      var = STRASSEN_ABC;
      tile = 0;
    }
    const int64_t mn = std::min(m, std::min(n, k));
    while (lv > 0 && ((int64_t)1 << lv) > mn) --lv;
    const double t = model_seconds_dtype(m, n, k, lv, var, tile, dtype);
    base[c] = (float)std::log2(t > 1e-9 ? t : 1e-9);
    x[6 + c] = (base[c] + 7.f) / 7.f;
  }
}

bool mlp_select(int64_t m, int64_t n, int64_t k, int dtype, int may_launch, int* candidate) {
  std::lock_guard<std::mutex> lock(g_mlp_mu);
  if (g_sel_host.empty() || dtype < 0 || dtype > 2 || !((g_sel_dtypes >> dtype) & 1u)) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSelMaxDevices) {
    cudaGetLastError();
    return false;
  }
  const ShapeKey key{m, n, k, dtype};
  auto& cache = g_sel_cache[dev];
  auto it = cache.find(key);
  if (it != cache.end()) {
    *candidate = it->second;
    return true;
  }
  if (!may_launch) return false;
  SelDevice* sd = sel_device(dev);
  if (!sd) return false;
  SelectArgs a;
  selector_features(m, n, k, dtype, a.x, a.base);
  a.valid = 0;
  for (int c = 0; c < kOut; ++c)
    if (selector_candidate_valid(c, dtype)) a.valid |= 1u << c;
  mlp_select_kernel<<<1, kBlock, 0, sd->stream>>>(sd->params, a, sd->out);
  int host = -1;
  if (cudaMemcpyAsync(&host, sd->out, sizeof(int), cudaMemcpyDeviceToHost, sd->stream) != cudaSuccess ||
      cudaStreamSynchronize(sd->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (host < 0 || host >= kOut) return false;
  if (cache.size() > 100000) cache.clear();
  cache[key] = host;
  *candidate = host;
  return true;
}

}  // namespace sgb

using namespace sgb;

extern "C" {

int strassen_mlp_param_count(void) { return kParams; }

int strassen_mlp_forward(const float* params, const float* X, int batch, float* Y, strassen_stream_t stream) {
  if (batch < 0) return STRASSEN_ERR_ARG;
  if (batch == 0) return STRASSEN_OK;
  if (!params || !X || !Y) return STRASSEN_ERR_NULL;
  mlp_forward_kernel<<<grid_for_batch(batch), kBlock, 0, (cudaStream_t)stream>>>(params, X, batch, Y);
  return cudaGetLastError() == cudaSuccess ? STRASSEN_OK : STRASSEN_ERR_CUDA;
}

int strassen_mlp_loss_grad(const float* params, const float* X, const float* T, const float* mask, int batch,
                           float mask_sum, float* grad, strassen_stream_t stream) {
  if (batch < 0 || !(mask_sum > 0.f)) return STRASSEN_ERR_ARG;
  if (!params || !X || !T || !mask || !grad) return STRASSEN_ERR_NULL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kParams, s) != cudaSuccess) return STRASSEN_ERR_CUDA;
  if (batch == 0) return STRASSEN_OK;
  mlp_grad_kernel<<<grid_for_batch(batch) < 152 ? grid_for_batch(batch) : 152, kBlock, 0, s>>>(
      params, X, T, mask, batch, 1.f / mask_sum, grad);
  return cudaGetLastError() == cudaSuccess ? STRASSEN_OK : STRASSEN_ERR_CUDA;
}

int strassen_mlp_adam(float* params, const float* grad, float* m, float* v, int count, int step, float lr,
                      strassen_stream_t stream) {
  if (count < 0 || step < 1) return STRASSEN_ERR_ARG;
  if (!params || !grad || !m || !v) return STRASSEN_ERR_NULL;
  const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
  adam_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, c1, c2);
  return cudaGetLastError() == cudaSuccess ? STRASSEN_OK : STRASSEN_ERR_CUDA;
}

int strassen_selector_load(const float* params_host, int count) {
  if (count != kParams) return STRASSEN_ERR_ARG;
  if (!params_host) return STRASSEN_ERR_NULL;
  try {
    std::lock_guard<std::mutex> lock(g_mlp_mu);
    g_sel_host.assign(params_host, params_host + kParams);
    ++g_sel_version;
    for (auto& c : g_sel_cache) c.clear();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSelMaxDevices) {
      cudaGetLastError();
      return STRASSEN_ERR_CUDA;
    }
    return sel_device(dev) ? STRASSEN_OK : STRASSEN_ERR_ALLOC;
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
}

int strassen_selector_use(int dtype, int enable) {
  if (dtype < 0 || dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mlp_mu);
  if (enable) g_sel_dtypes |= 1u << dtype;
  else g_sel_dtypes &= ~(1u << dtype);
  for (auto& c : g_sel_cache) c.clear();
  return STRASSEN_OK;
}

int strassen_selector_candidate(int candidate, int* levels, strassen_variant* variant, int* tile_id) {
  if (!levels || !variant || !tile_id) return STRASSEN_ERR_NULL;
  if (candidate < 0 || candidate >= kOut) return STRASSEN_ERR_ARG;
  int lv, var, tile;
  selector_candidate(candidate, &lv, &var, &tile);
  *levels = lv;
  *variant = (strassen_variant)var;
  *tile_id = tile;
  return STRASSEN_OK;
}

int strassen_selector_features(int64_t m, int64_t n, int64_t k, strassen_dtype dtype, float* x, float* base,
                               unsigned* valid) {
  if (!x || !base || !valid) return STRASSEN_ERR_NULL;
  if (m <= 0 || n <= 0 || k <= 0) return STRASSEN_ERR_DIM;
  if ((int)dtype < 0 || (int)dtype > 2) return STRASSEN_ERR_UNSUPPORTED;
  try {
    selector_features(m, n, k, (int)dtype, x, base);
  } catch (...) {
    return STRASSEN_ERR_ALLOC;
  }
  *valid = 0;
  for (int c = 0; c < kOut; ++c)
    if (selector_candidate_valid(c, (int)dtype)) *valid |= 1u << c;
  return STRASSEN_OK;
}

int strassen_selector_clear(void) {
  std::lock_guard<std::mutex> lock(g_mlp_mu);
  int cur = 0;
  const bool have_cur = cudaGetDevice(&cur) == cudaSuccess;
  for (int d = 0; d < kSelMaxDevices; ++d) {
    SelDevice& sd = g_sel_dev[d];
    if (!sd.params) continue;
    if (cudaSetDevice(d) == cudaSuccess) {
      cudaStreamSynchronize(sd.stream);
      cudaFree(sd.params);
      cudaFree(sd.out);
      cudaStreamDestroy(sd.stream);
    }
    sd = SelDevice();
  }
  if (have_cur) cudaSetDevice(cur);
  cudaGetLastError();
  g_sel_host.clear();
  g_sel_dtypes = 0x7u;
  for (auto& c : g_sel_cache) c.clear();
  return STRASSEN_OK;
}

}  // extern "C"
