// Learned prefilter: a small network over the 64 bits of a key (64 -> 128 ->
// 64 -> 1), trained in fp32 on the GPU with fake-quantized weights and a
// straight-through gradient, exported to exact integer arithmetic (int8
// weights and activations, int32 products, ReLU + arithmetic shift +
// saturation, integer threshold), and used in front of a backup blocked
// filter that holds the members the network rejects.
//
// Parameter vector (fp32, kMlpParams entries): W1 [64][128], b1 [128],
// W2 [128][64], b2 [64], W3 [64], b3.
//
// This unit holds the training kernels and the CUDA-core integer model (dp4a:
// four int8 products summed into an int32 per instruction, exact), which also
// serves calibration and compaction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bloomgb.h"
#include "lbf.h"

namespace {

using namespace lbf;
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH1, oW2 = ob1 + kH1, ob2 = oW2 + kH1 * kH2, oW3 = ob2 + kH2,
              ob3 = oW3 + kH2, kMlpParams = ob3 + 1;
static_assert(kMlpParams == BF_MLP_PARAMS, "parameter layout");

// ---------------------------------------------------------------------------
// training (fp32)
// ---------------------------------------------------------------------------
struct TrainWs {
  float* wq;  // fake-quantized W1 | W2 | W3 (same offsets as the parameters)
  float* g;   // gradients (training loop only)
  uint64_t* xb;  // the batch's keys
  float* yb;     // the batch's labels
  float* z1;  // [batch][128]
  float* z2;  // [batch][64]
  float* z3;  // [batch]
  float* d1;  // dZ1 [batch][128]
  float* d2;  // dZ2 [batch][64]
  float* d3;  // dZ3 [batch]
};

__device__ __forceinline__ float bitf(uint64_t key, int i) { return static_cast<float>((key >> i) & 1ull); }

// Fake quantization of one weight tensor per CTA: s = max|W| / 127,
// Wq = s * clamp(round_half_away(W / s), -127, 127).
__global__ void __launch_bounds__(256) k_fakequant(const float* __restrict__ p, float* __restrict__ wq) {
  const int off[3] = {oW1, oW2, oW3};
  const int cnt[3] = {kIn * kH1, kH1 * kH2, kH2};
  const int o = off[blockIdx.x], n = cnt[blockIdx.x];
  __shared__ float red[256];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(p[o + i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  // the rounding decisions are taken in fp64 (the scale and quotient of the
  // fp32 weights), then the quantized weight is stored in fp32
  const double s = red[0] > 0.f ? static_cast<double>(red[0]) / 127.0 : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = static_cast<double>(p[o + i]) / s;
    const double q = copysign(floor(fabs(v) + 0.5), v);
    wq[o + i] = static_cast<float>(fmin(fmax(q, -127.0), 127.0) * s);
  }
}

// sample i of a batch is element ((first + i) mod n) * mult mod n of the
// training set (a permutation of it per n consecutive samples when mult and n
// are coprime)
__global__ void k_gather(const uint64_t* __restrict__ keys, const float* __restrict__ labels, uint64_t n,
                         uint64_t first, uint64_t mult, uint64_t* __restrict__ xb, float* __restrict__ yb,
                         uint32_t batch) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const uint64_t a = (first + b) % n;
  const uint64_t idx = (a * mult) % n;
  xb[b] = keys[idx];
  yb[b] = labels[idx];
}

// forward: one thread per (sample, unit) of a layer
__global__ void k_fwd1(const uint64_t* __restrict__ keys, const float* __restrict__ wq, const float* __restrict__ p,
                       float* __restrict__ z1, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * kH1) return;
  const uint32_t b = t / kH1, j = t % kH1;
  const uint64_t key = keys[b];
  float acc = p[ob1 + j];
  for (int i = 0; i < kIn; ++i) acc += bitf(key, i) * wq[oW1 + i * kH1 + j];
  z1[t] = acc;
}
__global__ void k_fwd2(const float* __restrict__ z1, const float* __restrict__ wq, const float* __restrict__ p,
                       float* __restrict__ z2, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * kH2) return;
  const uint32_t b = t / kH2, j = t % kH2;
  float acc = p[ob2 + j];
  for (int i = 0; i < kH1; ++i) acc += fmaxf(z1[b * kH1 + i], 0.f) * wq[oW2 + i * kH2 + j];
  z2[t] = acc;
}
// logit, loss and dZ3 = (sigmoid(z3) - y) / batch
__global__ void k_fwd3_loss(const float* __restrict__ z2, const float* __restrict__ wq, const float* __restrict__ p,
                            const float* __restrict__ labels, float* __restrict__ z3, float* __restrict__ d3,
                            float* __restrict__ loss, uint32_t batch) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (b < batch) {
    float acc = p[ob3];
    for (int i = 0; i < kH2; ++i) acc += fmaxf(z2[b * kH2 + i], 0.f) * wq[oW3 + i];
    z3[b] = acc;
    const float y = labels[b];
    d3[b] = (1.f / (1.f + expf(-acc)) - y) / static_cast<float>(batch);
    l = (fmaxf(acc, 0.f) - acc * y + log1pf(expf(-fabsf(acc)))) / static_cast<float>(batch);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}
// dZ2 = (dZ3 W3q^T) * [z2 > 0]
__global__ void k_bwd2(const float* __restrict__ d3, const float* __restrict__ z2, const float* __restrict__ wq,
                       float* __restrict__ d2, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * kH2) return;
  const uint32_t b = t / kH2, j = t % kH2;
  d2[t] = z2[t] > 0.f ? d3[b] * wq[oW3 + j] : 0.f;
}
// dZ1 = (dZ2 W2q^T) * [z1 > 0]
__global__ void k_bwd1(const float* __restrict__ d2, const float* __restrict__ z1, const float* __restrict__ wq,
                       float* __restrict__ d1, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch * kH1) return;
  const uint32_t b = t / kH1, i = t % kH1;
  float acc = 0.f;
  if (z1[t] > 0.f)
    for (int j = 0; j < kH2; ++j) acc += d2[b * kH2 + j] * wq[oW2 + i * kH2 + j];
  d1[t] = acc;
}
// weight and bias gradients: one thread per parameter, summing over the batch
// in a fixed order (deterministic)
__global__ void k_wgrad(const TrainWs ws, float* __restrict__ g, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= static_cast<uint32_t>(kMlpParams)) return;
  float acc = 0.f;
  if (t < static_cast<uint32_t>(ob1)) {  // W1[i][j]
    const int i = t / kH1, j = t % kH1;
    for (uint32_t b = 0; b < batch; ++b) acc += bitf(ws.xb[b], i) * ws.d1[b * kH1 + j];
  } else if (t < static_cast<uint32_t>(oW2)) {  // b1[j]
    const int j = t - ob1;
    for (uint32_t b = 0; b < batch; ++b) acc += ws.d1[b * kH1 + j];
  } else if (t < static_cast<uint32_t>(ob2)) {  // W2[i][j]
    const int i = (t - oW2) / kH2, j = (t - oW2) % kH2;
    for (uint32_t b = 0; b < batch; ++b) acc += fmaxf(ws.z1[b * kH1 + i], 0.f) * ws.d2[b * kH2 + j];
  } else if (t < static_cast<uint32_t>(oW3)) {  // b2[j]
    const int j = t - ob2;
    for (uint32_t b = 0; b < batch; ++b) acc += ws.d2[b * kH2 + j];
  } else if (t < static_cast<uint32_t>(ob3)) {  // W3[i]
    const int i = t - oW3;
    for (uint32_t b = 0; b < batch; ++b) acc += fmaxf(ws.z2[b * kH2 + i], 0.f) * ws.d3[b];
  } else {  // b3
    for (uint32_t b = 0; b < batch; ++b) acc += ws.d3[b];
  }
  g[t] = acc;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kMlpParams) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

uint64_t ws_floats(uint32_t batch) {
  const uint64_t par = (kMlpParams + 63) / 64 * 64;
  return 2 * par + static_cast<uint64_t>(batch) * (2 * kH1 + 2 * kH2 + 2 + 3) + 64;
}

TrainWs carve(void* ws, uint32_t batch) {
  const uint64_t par = (kMlpParams + 63) / 64 * 64;
  float* f = static_cast<float*>(ws);
  TrainWs w;
  w.wq = f;
  f += par;
  w.g = f;
  f += par;
  w.xb = reinterpret_cast<uint64_t*>(f);  // 256-byte aligned: par is a multiple of 64 floats
  f += 2 * static_cast<uint64_t>(batch);
  w.yb = f;
  f += (batch + 63) / 64 * 64;
  w.z1 = f; f += static_cast<uint64_t>(batch) * kH1;
  w.z2 = f; f += static_cast<uint64_t>(batch) * kH2;
  w.z3 = f; f += batch;
  w.d1 = f; f += static_cast<uint64_t>(batch) * kH1;
  w.d2 = f; f += static_cast<uint64_t>(batch) * kH2;
  w.d3 = f;
  return w;
}

uint32_t blocks_for(uint64_t n, uint32_t t) { return static_cast<uint32_t>((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// integer model
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dp4a(int a, int b, int c) { return __dp4a(a, b, c); }

// activations of one key: x bytes (0/1) -> h1 (int8 in [0,127]) -> h2 -> score.
// `upto`: 1 = stop after layer 1 (returns max relu(a1)), 2 = after layer 2, 3 = score.
__device__ __forceinline__ long long int_forward(const unsigned char* __restrict__ img, uint64_t key, int upto) {
  const int* w1 = reinterpret_cast<const int*>(img + kImgW1);
  const int* w2 = reinterpret_cast<const int*>(img + kImgW2);
  const int* w3 = reinterpret_cast<const int*>(img + kImgW3);
  const int* b1 = reinterpret_cast<const int*>(img + kImgB1);
  const int* b2 = reinterpret_cast<const int*>(img + kImgB2);
  const int b3 = *reinterpret_cast<const int*>(img + kImgB3);
  const int sh1 = reinterpret_cast<const int*>(img + kImgSh)[0];
  const int sh2 = reinterpret_cast<const int*>(img + kImgSh)[1];
  int x[16];
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const uint32_t nib = static_cast<uint32_t>(key >> (4 * w)) & 0xFu;
    x[w] = static_cast<int>((nib & 1u) | ((nib & 2u) << 7) | ((nib & 4u) << 14) | ((nib & 8u) << 21));
  }
  int h1[32];
  long long top = 0;
#pragma unroll
  for (int j = 0; j < kH1; j += 4) {
    uint32_t packed = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int acc = 0;
#pragma unroll
      for (int w = 0; w < 16; ++w) acc = dp4a(x[w], w1[(j + u) * 16 + w], acc);
      const long long a = static_cast<long long>(acc) + b1[j + u];
      const long long r = a > 0 ? a : 0;
      top = r > top ? r : top;
      const long long h = (r >> sh1) < 127 ? (r >> sh1) : 127;
      packed |= static_cast<uint32_t>(h) << (8 * u);
    }
    h1[j / 4] = static_cast<int>(packed);
  }
  if (upto == 1) return top;
  int h2[16];
  top = 0;
#pragma unroll
  for (int j = 0; j < kH2; j += 4) {
    uint32_t packed = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int acc = 0;
#pragma unroll
      for (int w = 0; w < 32; ++w) acc = dp4a(h1[w], w2[(j + u) * 32 + w], acc);
      const long long a = static_cast<long long>(acc) + b2[j + u];
      const long long r = a > 0 ? a : 0;
      top = r > top ? r : top;
      const long long h = (r >> sh2) < 127 ? (r >> sh2) : 127;
      packed |= static_cast<uint32_t>(h) << (8 * u);
    }
    h2[j / 4] = static_cast<int>(packed);
  }
  if (upto == 2) return top;
  int acc = 0;
#pragma unroll
  for (int w = 0; w < 16; ++w) acc = dp4a(h2[w], w3[w], acc);
  long long sc = static_cast<long long>(acc) + b3;
  sc = sc < INT32_MIN ? INT32_MIN : (sc > INT32_MAX ? INT32_MAX : sc);
  return sc;
}

// mode 0: scores to out32; mode 1: out8[i] |= (score >= tau); mode 2/3: max
// relu activation of layer 1/2 over the keys into *max64 (calibration);
// mode 4: keys whose score is below tau appended to out_keys, their number
// counted in *max64
struct ScoreArgs {
  const unsigned char* img;
  const uint64_t* keys;
  uint64_t n;
  int mode;
  int tau;
  int* out32;
  uint8_t* out8;
  unsigned long long* max64;
  uint64_t* out_keys;
};

__global__ void __launch_bounds__(256, 2) k_int_mlp(const ScoreArgs a) {
  __shared__ __align__(16) unsigned char img[kImgBytes];
  for (int i = threadIdx.x * 4; i < kImgBytes; i += blockDim.x * 4)
    *reinterpret_cast<int*>(img + i) = *reinterpret_cast<const int*>(a.img + i);
  __syncthreads();
  unsigned long long top = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t n_round = (a.n + stride - 1) / stride * stride;  // whole warps reach the ballot
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n_round; i += stride) {
    const bool live = i < a.n;
    const uint64_t key = live ? a.keys[i] : 0;
    if (a.mode == 0) {
      if (live) a.out32[i] = static_cast<int>(int_forward(img, key, 3));
    } else if (a.mode == 1) {
      if (live && int_forward(img, key, 3) >= a.tau) a.out8[i] = 1;
    } else if (a.mode == 4) {
      const bool take = live && int_forward(img, key, 3) < a.tau;
      const unsigned vote = __ballot_sync(0xFFFFFFFFu, take);
      const int lane = threadIdx.x & 31;
      unsigned long long base = 0;
      if (lane == 0 && vote) base = atomicAdd(a.max64, static_cast<unsigned long long>(__popc(vote)));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (take) a.out_keys[base + __popc(vote & ((1u << lane) - 1u))] = key;
    } else if (live) {
      const unsigned long long r = static_cast<unsigned long long>(int_forward(img, key, a.mode == 2 ? 1 : 2));
      top = r > top ? r : top;
    }
  }
  if (a.mode == 2 || a.mode == 3) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, top, o);
      top = v > top ? v : top;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(a.max64, top);
  }
}

double round_half_away(double v) { return v < 0 ? -std::floor(-v + 0.5) : std::floor(v + 0.5); }

double qscale(const float* w, int n) {
  double m = 0;
  for (int i = 0; i < n; ++i) m = std::max(m, std::fabs(static_cast<double>(w[i])));
  return m > 0 ? m / 127.0 : 1.0;
}

int8_t qweight(float w, double s) {
  const double q = round_half_away(static_cast<double>(w) / s);
  return static_cast<int8_t>(std::min(127.0, std::max(-127.0, q)));
}

int32_t qbias(float b, double unit) {
  const double q = round_half_away(static_cast<double>(b) / unit);
  return static_cast<int32_t>(std::min(2147483647.0, std::max(-2147483648.0, q)));
}

int shift_for(unsigned long long r) {
  int sh = 0;
  while ((r >> sh) > 127ull) ++sh;
  return sh;
}

uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bf_status run_int(const unsigned char* d_img, const uint64_t* d_keys, uint64_t n, int mode, int tau, int* out32,
                  uint8_t* out8, unsigned long long* max64, uint64_t* out_keys, cudaStream_t st) {
  if (n == 0) return BF_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>((n + 255) / 256, static_cast<uint64_t>(sms) * 8));
  ScoreArgs a{d_img, d_keys, n, mode, tau, out32, out8, max64, out_keys};
  k_int_mlp<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? BF_OK : BF_ECUDA;
}

// one training step's gradient into g (loss added into *loss if not null)
void launch_grad(const float* p, const uint64_t* keys, const float* labels, uint64_t n, uint64_t first, uint64_t mult,
                 uint32_t batch, float* g, float* loss, const TrainWs& w, cudaStream_t st) {
  k_fakequant<<<3, 256, 0, st>>>(p, w.wq);
  k_gather<<<blocks_for(batch, 256), 256, 0, st>>>(keys, labels, n, first, mult, w.xb, w.yb, batch);
  k_fwd1<<<blocks_for(static_cast<uint64_t>(batch) * kH1, 256), 256, 0, st>>>(w.xb, w.wq, p, w.z1, batch);
  k_fwd2<<<blocks_for(static_cast<uint64_t>(batch) * kH2, 256), 256, 0, st>>>(w.z1, w.wq, p, w.z2, batch);
  k_fwd3_loss<<<blocks_for(batch, 256), 256, 0, st>>>(w.z2, w.wq, p, w.yb, w.z3, w.d3, loss, batch);
  k_bwd2<<<blocks_for(static_cast<uint64_t>(batch) * kH2, 256), 256, 0, st>>>(w.d3, w.z2, w.wq, w.d2, batch);
  k_bwd1<<<blocks_for(static_cast<uint64_t>(batch) * kH1, 256), 256, 0, st>>>(w.d2, w.z1, w.wq, w.d1, batch);
  k_wgrad<<<blocks_for(kMlpParams, 128), 128, 0, st>>>(w, g, batch);
}

bf_status check_sampling(const uint64_t* keys, const float* labels, uint64_t n, uint64_t mult) {
  if (!keys || !labels || n == 0 || n > 0xFFFFFFFFull) return BF_EINVAL;
  if (mult == 0 || mult > 0xFFFFFFFFull) return BF_EINVAL;
  if (n > 1 && gcd64(mult % n, n) != 1) return BF_EINVAL;
  return BF_OK;
}

}  // namespace

namespace lbf {

void image_of(const bf_mlp_int8* m, std::vector<unsigned char>& img) {
  img.assign(kImgBytes, 0);
  for (int j = 0; j < kH1; ++j)
    for (int i = 0; i < kIn; ++i) img[kImgW1 + j * kIn + i] = static_cast<unsigned char>(m->w1[i * kH1 + j]);
  for (int j = 0; j < kH2; ++j)
    for (int i = 0; i < kH1; ++i) img[kImgW2 + j * kH1 + i] = static_cast<unsigned char>(m->w2[i * kH2 + j]);
  for (int i = 0; i < kH2; ++i) img[kImgW3 + i] = static_cast<unsigned char>(m->w3[i]);
  std::memcpy(&img[kImgB1], m->b1, 4 * kH1);
  std::memcpy(&img[kImgB2], m->b2, 4 * kH2);
  std::memcpy(&img[kImgB3], &m->b3, 4);
  std::memcpy(&img[kImgSh], &m->sh1, 4);
  std::memcpy(&img[kImgSh + 4], &m->sh2, 4);
}

}  // namespace lbf

extern "C" {

uint64_t bf_mlp_workspace_bytes(uint32_t batch) { return 4 * ws_floats(batch); }

bf_status bf_mlp_grad(const float* d_params, const uint64_t* d_keys, const float* d_labels, uint64_t n,
                      uint64_t first, uint64_t mult, uint32_t batch, float* d_grads, float* d_loss, void* d_ws,
                      uint64_t ws_bytes, bf_stream_t stream) {
  if (!d_params || !d_grads || !d_ws || batch == 0 || ws_bytes < bf_mlp_workspace_bytes(batch)) return BF_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return BF_EINVAL;
  const bf_status chk = check_sampling(d_keys, d_labels, n, mult);
  if (chk != BF_OK) return chk;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (d_loss && cudaMemsetAsync(d_loss, 0, sizeof(float), st) != cudaSuccess) return BF_ECUDA;
  launch_grad(d_params, d_keys, d_labels, n, first, mult, batch, d_grads, d_loss, carve(d_ws, batch), st);
  return cudaGetLastError() == cudaSuccess ? BF_OK : BF_ECUDA;
}

bf_status bf_mlp_adam(float* d_params, const float* d_grads, float* d_m, float* d_v, uint32_t step, float lr,
                      float beta1, float beta2, float eps, bf_stream_t stream) {
  if (!d_params || !d_grads || !d_m || !d_v || step == 0) return BF_EINVAL;
  const float c1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(step)));
  const float c2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(step)));
  k_adam<<<blocks_for(kMlpParams, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_params, d_grads, d_m,
                                                                                         d_v, lr, beta1, beta2, eps,
                                                                                         c1, c2);
  return cudaGetLastError() == cudaSuccess ? BF_OK : BF_ECUDA;
}

bf_status bf_mlp_train(float* d_params, float* d_m, float* d_v, const uint64_t* d_keys, const float* d_labels,
                       uint64_t n, uint64_t mult, uint32_t batch, uint32_t first_step, uint32_t steps, float lr,
                       float beta1, float beta2, float eps, float* d_loss, void* d_ws, uint64_t ws_bytes,
                       bf_stream_t stream) {
  if (!d_params || !d_m || !d_v || !d_ws || batch == 0 || first_step == 0 ||
      ws_bytes < bf_mlp_workspace_bytes(batch) || reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
    return BF_EINVAL;
  const bf_status chk = check_sampling(d_keys, d_labels, n, mult);
  if (chk != BF_OK) return chk;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (d_loss && cudaMemsetAsync(d_loss, 0, sizeof(float) * steps, st) != cudaSuccess) return BF_ECUDA;
  const TrainWs w = carve(d_ws, batch);
  for (uint32_t s = 0; s < steps; ++s) {
    const uint32_t t = first_step + s;
    launch_grad(d_params, d_keys, d_labels, n, static_cast<uint64_t>(t - 1) * batch % n, mult, batch, w.g,
                d_loss ? d_loss + s : nullptr, w, st);
    const bf_status a = bf_mlp_adam(d_params, w.g, d_m, d_v, t, lr, beta1, beta2, eps, stream);
    if (a != BF_OK) return a;
  }
  return cudaGetLastError() == cudaSuccess ? BF_OK : BF_ECUDA;
}

bf_status bf_mlp_export(const float* h_params, const uint64_t* d_calib, uint64_t n_calib, bf_mlp_int8* out,
                        bf_stream_t stream) {
  if (!h_params || !out || (n_calib && !d_calib)) return BF_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::memset(out, 0, sizeof(*out));
  const double s1 = qscale(h_params + oW1, kIn * kH1), s2 = qscale(h_params + oW2, kH1 * kH2),
               s3 = qscale(h_params + oW3, kH2);
  for (int i = 0; i < kIn * kH1; ++i) out->w1[i] = qweight(h_params[oW1 + i], s1);
  for (int i = 0; i < kH1 * kH2; ++i) out->w2[i] = qweight(h_params[oW2 + i], s2);
  for (int i = 0; i < kH2; ++i) out->w3[i] = qweight(h_params[oW3 + i], s3);
  for (int j = 0; j < kH1; ++j) out->b1[j] = qbias(h_params[ob1 + j], s1);
  // calibration of layer 1 (later layers still zero), then of layer 2
  unsigned char* d_img = nullptr;
  unsigned long long* d_max = nullptr;
  std::vector<unsigned char> img;
  unsigned long long r = 0;
  bf_status s = BF_OK;
  if (cudaMalloc(&d_img, kImgBytes) != cudaSuccess || cudaMalloc(&d_max, 8) != cudaSuccess) {
    cudaGetLastError();
    s = BF_ENOMEM;
  }
  for (int layer = 1; layer <= 2 && s == BF_OK; ++layer) {
    image_of(out, img);
    r = 0;
    if (cudaMemcpyAsync(d_img, img.data(), kImgBytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_max, 0, 8, st) != cudaSuccess) {
      s = BF_ECUDA;
      break;
    }
    s = run_int(d_img, d_calib, n_calib, layer == 1 ? 2 : 3, 0, nullptr, nullptr, d_max, nullptr, st);
    if (s == BF_OK && (cudaMemcpyAsync(&r, d_max, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
      s = BF_ECUDA;
    if (s != BF_OK) break;
    if (layer == 1) {
      out->sh1 = shift_for(r);
      const double u2 = s1 * std::ldexp(1.0, out->sh1) * s2;
      for (int j = 0; j < kH2; ++j) out->b2[j] = qbias(h_params[ob2 + j], u2);
    } else {
      out->sh2 = shift_for(r);
      const double u3 = s1 * std::ldexp(1.0, out->sh1) * s2 * std::ldexp(1.0, out->sh2) * s3;
      out->b3 = qbias(h_params[ob3], u3);
      out->unit = u3;
    }
  }
  if (d_img) cudaFree(d_img);
  if (d_max) cudaFree(d_max);
  return s;
}

bf_status bf_mlp_load(const bf_mlp_int8* m, bf_mlp_model** out) {
  if (!m || !out) return BF_EINVAL;
  *out = nullptr;
  if (m->sh1 < 0 || m->sh1 > 62 || m->sh2 < 0 || m->sh2 > 62) return BF_EINVAL;
  bf_mlp_model* md = new (std::nothrow) bf_mlp_model();
  if (!md) return BF_ENOMEM;
  std::vector<unsigned char> img;
  image_of(m, img);
  cudaGetDevice(&md->device);
  const bool tc = lbf::tc_prepare(m, &md->tc);
  bool ok = cudaMalloc(&md->d_img, kImgBytes) == cudaSuccess && cudaMalloc(&md->d_err, 4) == cudaSuccess &&
            (!tc || cudaMalloc(&md->d_tc, lbf::tc_image_bytes()) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    bf_mlp_free(md);
    return BF_ENOMEM;
  }
  ok = cudaMemcpy(md->d_img, img.data(), kImgBytes, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(md->d_err, 0, 4) == cudaSuccess &&
       (!tc || cudaMemcpy(md->d_tc, md->tc.image.data(), lbf::tc_image_bytes(), cudaMemcpyHostToDevice) == cudaSuccess);
  if (!ok) {
    bf_mlp_free(md);
    return BF_ECUDA;
  }
  *out = md;
  return BF_OK;
}

bf_status bf_mlp_free(bf_mlp_model* m) {
  if (!m) return BF_EINVAL;
  for (int i = 0; i < bf_mlp_model::kDepth; ++i) {
    if (m->pipe[i]) cudaStreamDestroy(m->pipe[i]);
    if (m->ev_done[i]) cudaEventDestroy(m->ev_done[i]);
  }
  if (m->ev_start) cudaEventDestroy(m->ev_start);
  if (m->staging) cudaFree(m->staging);
  if (m->d_img) cudaFree(m->d_img);
  if (m->d_tc) cudaFree(m->d_tc);
  if (m->d_err) cudaFree(m->d_err);
  delete m;
  return BF_OK;
}

bf_status bf_mlp_set_engine(bf_mlp_model* m, int engine) {
  if (!m || engine < BF_MLP_ENGINE_AUTO || engine > BF_MLP_ENGINE_DP4A) return BF_EINVAL;
  if (engine == BF_MLP_ENGINE_TENSOR && !m->d_tc) return BF_EUNSUPPORTED;
  m->engine = engine;
  return BF_OK;
}

bf_status bf_mlp_get_engine(const bf_mlp_model* m, int* engine) {
  if (!m || !engine) return BF_EINVAL;
  *engine = (m->d_tc && m->engine != BF_MLP_ENGINE_DP4A) ? BF_MLP_ENGINE_TENSOR : BF_MLP_ENGINE_DP4A;
  return BF_OK;
}

bf_status bf_mlp_check(const bf_mlp_model* m) {
  if (!m) return BF_EINVAL;
  unsigned int e = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&e, m->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BF_ECUDA;
  return e ? BF_ETIMEDOUT : BF_OK;
}

}  // extern "C"

namespace {

bf_status run_model(const bf_mlp_model* m, const uint64_t* d_keys, uint64_t n, int mode, int tau, int32_t* out32,
                    uint8_t* out8, unsigned long long* count, uint64_t* out_keys, cudaStream_t st) {
  int engine = 0;
  bf_mlp_get_engine(m, &engine);
  if (engine == BF_MLP_ENGINE_TENSOR)
    return lbf::tc_run(m->d_tc, m->tc, d_keys, n, mode, tau, out32, out8, count, out_keys, m->d_err, st) ==
                   cudaSuccess
               ? BF_OK
               : BF_ECUDA;
  return run_int(m->d_img, d_keys, n, mode, tau, out32, out8, count, out_keys, st);
}

}  // namespace

extern "C" {

bf_status bf_mlp_scores(const bf_mlp_model* m, const uint64_t* d_keys, uint64_t n, int32_t* d_scores,
                        bf_stream_t stream) {
  if (!m || (n && (!d_keys || !d_scores))) return BF_EINVAL;
  return run_model(m, d_keys, n, 0, 0, d_scores, nullptr, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_mlp_select_below(const bf_mlp_model* m, int32_t tau, const uint64_t* d_keys, uint64_t n,
                              uint64_t* d_out_keys, uint64_t* d_count, bf_stream_t stream) {
  if (!m || !d_count || (n && (!d_keys || !d_out_keys))) return BF_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st) != cudaSuccess) return BF_ECUDA;
  return run_model(m, d_keys, n, 4, tau, nullptr, nullptr, reinterpret_cast<unsigned long long*>(d_count),
                   d_out_keys, st);
}

bf_status bf_mlp_contains(const bf_mlp_model* m, int32_t tau, const bf_filter* backup, const uint64_t* d_keys,
                          uint64_t n, uint8_t* d_out, bf_stream_t stream) {
  if (!m || !backup || (n && (!d_keys || !d_out))) return BF_EINVAL;
  if (n == 0) return BF_OK;
  int engine = 0;
  bf_mlp_get_engine(m, &engine);
  bf_params bp{};
  void* words = nullptr;
  uint64_t nbytes = 0;
  if (engine == BF_MLP_ENGINE_TENSOR && bf_get_params(backup, &bp) == BF_OK &&
      bf_words(backup, &words, &nbytes) == BF_OK && bp.block_bits == 256 && bp.word_bits == 32 && bp.k == 8 &&
      (bp.groups == 0 || bp.groups == 8) && bp.salts == 0 && reinterpret_cast<uintptr_t>(d_keys) % 8 == 0) {
    // one fused launch: model and backup probe per key
    const lbf::TcBackup tb{static_cast<const uint32_t*>(words), bp.num_blocks, bp.seed};
    return lbf::tc_run(m->d_tc, m->tc, d_keys, n, 5, tau, nullptr, d_out, nullptr, nullptr, m->d_err,
                       reinterpret_cast<cudaStream_t>(stream), &tb) == cudaSuccess
               ? BF_OK
               : BF_ECUDA;
  }
  const bf_status s = bf_contains(backup, d_keys, n, d_out, stream);
  if (s != BF_OK) return s;
  return run_model(m, d_keys, n, 1, tau, nullptr, d_out, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_mlp_contains_host(bf_mlp_model* m, int32_t tau, const bf_filter* backup, const uint64_t* h_keys,
                               uint64_t n, uint8_t* h_out, bf_stream_t stream) {
  if (!m || !backup || (n && (!h_keys || !h_out))) return BF_EINVAL;
  if (n == 0) return BF_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  constexpr uint64_t kChunk = 1ull << 24;
  const uint64_t keys_bytes = kChunk * 8, slot = keys_bytes + kChunk;  // both multiples of 256
  cudaError_t e = cudaSuccess;
  if (!m->staging) {
    if (cudaMalloc(&m->staging, slot * bf_mlp_model::kDepth) != cudaSuccess) {
      cudaGetLastError();
      m->staging = nullptr;
      return BF_ENOMEM;
    }
    m->chunk = kChunk;
    for (int i = 0; i < bf_mlp_model::kDepth; ++i)
      if (cudaStreamCreateWithFlags(&m->pipe[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&m->ev_done[i], cudaEventDisableTiming) != cudaSuccess)
        return BF_ECUDA;
    if (cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming) != cudaSuccess) return BF_ECUDA;
  }
  if ((e = cudaEventRecord(m->ev_start, st)) != cudaSuccess) return BF_ECUDA;
  for (int i = 0; i < bf_mlp_model::kDepth; ++i)
    if (cudaStreamWaitEvent(m->pipe[i], m->ev_start, 0) != cudaSuccess) return BF_ECUDA;
  uint64_t c = 0;
  for (uint64_t lo = 0; lo < n; lo += kChunk, ++c) {
    const uint64_t cnt = std::min(kChunk, n - lo);
    const int k = static_cast<int>(c % bf_mlp_model::kDepth);
    cudaStream_t ps = m->pipe[k];
    char* base = static_cast<char*>(m->staging) + k * slot;
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(base);
    uint8_t* d_out = reinterpret_cast<uint8_t*>(base + keys_bytes);
    if (cudaMemcpyAsync(d_keys, h_keys + lo, cnt * 8, cudaMemcpyHostToDevice, ps) != cudaSuccess) return BF_ECUDA;
    const bf_status s = bf_mlp_contains(m, tau, backup, d_keys, cnt, d_out, reinterpret_cast<bf_stream_t>(ps));
    if (s != BF_OK) return s;
    if (cudaMemcpyAsync(h_out + lo, d_out, cnt, cudaMemcpyDeviceToHost, ps) != cudaSuccess) return BF_ECUDA;
  }
  for (int i = 0; i < bf_mlp_model::kDepth; ++i)
    if (cudaEventRecord(m->ev_done[i], m->pipe[i]) != cudaSuccess || cudaStreamWaitEvent(st, m->ev_done[i], 0) != cudaSuccess)
      return BF_ECUDA;
  return BF_OK;
}

}  // extern "C"
