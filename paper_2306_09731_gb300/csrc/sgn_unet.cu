// sgn_unet.cu - forward, backward and Adam kernels of the periodic U-Net
// (include/sgn_unet.h) that corrects the GMRES starting value of sigma.
//
// Direct convolutions on CUDA cores: the network is small (6e4 parameters on a
// coarse grid of at most 512^2), and every kernel here is far from the cost
// of one matvec of the solver it serves. Activations are stored as T (BF16 or
// FP32), everything else is FP32; sums over pixels (weight gradients, the
// loss) are per-block fixed-order reductions, so results are deterministic.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <new>
#include <string>
#include <vector>

#include "sgn_unet.h"

namespace {

template <typename T>
__device__ __forceinline__ float ldf(const T* p);
template <>
__device__ __forceinline__ float ldf<float>(const float* p) {
  return *p;
}
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename T>
__device__ __forceinline__ T tof(float v);
template <>
__device__ __forceinline__ float tof<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 tof<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

constexpr int TILE = 16;   // output tile side of the 3x3 convolution
constexpr int COT = 8;     // output channels per block

// 3x3 periodic convolution. Forward (TR = false):
//   out[b][co][y][x] = bias[co] + sum_ci sum_k w[co][ci][k] in[b][ci][y+ky-1][x+kx-1]
// Transposed (TR = true, the gradient with respect to the input): the output
// channel is the forward input channel c, the input channel the forward output
// channel o, and the kernel is flipped:
//   out[b][c][y][x] = sum_o sum_k w[o][c][8-k] in[b][o][y+ky-1][x+kx-1]
// (Cw: the forward input-channel count, the row length of w.) H, W are powers
// of two; in and out have batch strides ibs, obs (elements).
template <typename TI, typename TO, bool TR>
__global__ void __launch_bounds__(TILE* TILE) k_conv3(const TI* __restrict__ in, size_t ibs, int Ci, TO* out,
                                                      size_t obs, int Co, const float* __restrict__ w,
                                                      const float* __restrict__ bias, int Cw, int H, int W,
                                                      int relu) {
  __shared__ float tile[TILE + 2][TILE + 2];
  __shared__ float ws[COT][9];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TILE + tx;
  const int tiles_x = (W + TILE - 1) / TILE;
  const int x0 = (blockIdx.x % tiles_x) * TILE, y0 = (blockIdx.x / tiles_x) * TILE;
  const int co0 = blockIdx.y * COT, b = blockIdx.z;
  const size_t HW = (size_t)H * W;
  const TI* inb = in + (size_t)b * ibs;
  float acc[COT];
#pragma unroll
  for (int c = 0; c < COT; ++c) acc[c] = 0.f;
  for (int ci = 0; ci < Ci; ++ci) {
    const TI* src = inb + (size_t)ci * HW;
    for (int i = tid; i < (TILE + 2) * (TILE + 2); i += TILE * TILE) {
      const int ly = i / (TILE + 2), lx = i % (TILE + 2);
      const int gy = (y0 + ly - 1) & (H - 1), gx = (x0 + lx - 1) & (W - 1);
      tile[ly][lx] = ldf(src + (size_t)gy * W + gx);
    }
    if (tid < COT * 9) {
      const int c = tid / 9, k = tid % 9, co = co0 + c;
      float v = 0.f;
      if (co < Co) v = TR ? w[((size_t)ci * Cw + co) * 9 + (8 - k)] : w[((size_t)co * Ci + ci) * 9 + k];
      ws[c][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float v = tile[ty + ky][tx + kx];
#pragma unroll
        for (int c = 0; c < COT; ++c) acc[c] = fmaf(ws[c][ky * 3 + kx], v, acc[c]);
      }
    __syncthreads();
  }
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
#pragma unroll
  for (int c = 0; c < COT; ++c) {
    const int co = co0 + c;
    if (co >= Co) break;
    float v = acc[c] + (bias ? bias[co] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    out[(size_t)b * obs + (size_t)co * HW + (size_t)y * W + x] = tof<TO>(v);
  }
}

// Block sum of K floats in fixed order; thread 0 gets the sums in v.
template <int K>
__device__ __forceinline__ void block_sum(float (&v)[K], float* red /* K * 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
    for (int k = 0; k < K; ++k) red[k * 32 + wid] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < K; ++k) {
      float t = 0.f;
      for (int i = 0; i < nw; ++i) t += red[k * 32 + i];
      v[k] = t;
    }
}

// dw[co][ci][k] = sum_{b,y,x} dp[b][co][y][x] in[b][ci][y+ky-1][x+kx-1];
// db[co] = sum dp[b][co] (blocks with ci = 0). One block per (co, ci).
template <typename TI>
__global__ void __launch_bounds__(256) k_conv3_dw(const TI* __restrict__ in, size_t ibs, int Ci,
                                                  const float* __restrict__ dp, size_t dbs, int Co, int H, int W,
                                                  int B, float* dw, float* db) {
  __shared__ float red[10 * 32];
  const int co = blockIdx.x, ci = blockIdx.y;
  const size_t HW = (size_t)H * W;
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  for (size_t p = threadIdx.x; p < (size_t)B * HW; p += blockDim.x) {
    const int b = (int)(p / HW);
    const int yx = (int)(p % HW), y = yx / W, x = yx % W;
    const float g = dp[(size_t)b * dbs + (size_t)co * HW + yx];
    const TI* src = in + (size_t)b * ibs + (size_t)ci * HW;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int gy = (y + ky - 1) & (H - 1);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) acc[ky * 3 + kx] = fmaf(g, ldf(src + (size_t)gy * W + ((x + kx - 1) & (W - 1))), acc[ky * 3 + kx]);
    }
    acc[9] += g;
  }
  block_sum<10>(acc, red);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 9; ++k) dw[((size_t)co * Ci + ci) * 9 + k] = acc[k];
    if (ci == 0) db[co] = acc[9];
  }
}

// 1x1 convolution C -> 1 (the output layer), FP32 output
template <typename T>
__global__ void k_conv1_fwd(const T* __restrict__ in, size_t ibs, int C, const float* __restrict__ w,
                            const float* __restrict__ bias, float* out, int HW, int B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * HW) return;
  const int b = i / HW, yx = i % HW;
  float v = bias[0];
  for (int c = 0; c < C; ++c) v = fmaf(w[c], ldf(in + (size_t)b * ibs + (size_t)c * HW + yx), v);
  out[i] = v;
}

// gradients of the output layer: dw[c] = sum dout in[c], db = sum dout
// (block c < C: dw[c]; block C: db) and din[c] = w[c] dout masked by in > 0
// (the ReLU of the layer before).
template <typename T>
__global__ void __launch_bounds__(256) k_conv1_dw(const T* __restrict__ in, size_t ibs, int C,
                                                  const float* __restrict__ dout, int HW, int B, float* dw,
                                                  float* db) {
  __shared__ float red[32];
  const int c = blockIdx.x;
  float acc[1] = {0.f};
  for (int i = threadIdx.x; i < B * HW; i += blockDim.x) {
    const int b = i / HW, yx = i % HW;
    acc[0] += dout[i] * (c < C ? ldf(in + (size_t)b * ibs + (size_t)c * HW + yx) : 1.f);
  }
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) {
    if (c < C)
      dw[c] = acc[0];
    else
      db[0] = acc[0];
  }
}

template <typename T>
__global__ void k_conv1_dx_relu(const T* __restrict__ act, size_t abs_, int C, const float* __restrict__ w,
                                const float* __restrict__ dout, float* din, size_t dbs, int HW, int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * HW) return;
  const int b = (int)(i / ((size_t)C * HW));
  const int r = (int)(i % ((size_t)C * HW)), c = r / HW, yx = r % HW;
  const float a = ldf(act + (size_t)b * abs_ + (size_t)c * HW + yx);
  din[(size_t)b * dbs + (size_t)c * HW + yx] = a > 0.f ? w[c] * dout[(size_t)b * HW + yx] : 0.f;
}

// g[b][c][i] = (g (+ extra)) * (act > 0): the ReLU backward, optionally after
// adding a second gradient (the skip connection's)
template <typename T>
__global__ void k_relu_bwd(const T* __restrict__ act, size_t abs_, float* g, size_t gbs,
                           const float* __restrict__ extra, size_t ebs, int C, int HW, int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * HW) return;
  const int b = (int)(i / ((size_t)C * HW));
  const size_t r = i % ((size_t)C * HW);
  float v = g[(size_t)b * gbs + r];
  if (extra) v += extra[(size_t)b * ebs + r];
  g[(size_t)b * gbs + r] = ldf(act + (size_t)b * abs_ + r) > 0.f ? v : 0.f;
}

// 2x2 average pool: out [C][H/2][W/2] from in [C][H][W]
template <typename T>
__global__ void k_pool(const T* __restrict__ in, size_t ibs, T* out, size_t obs, int C, int H, int W, int B) {
  const int h = H / 2, w = W / 2;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * h * w) return;
  const int b = (int)(i / ((size_t)C * h * w));
  const int r = (int)(i % ((size_t)C * h * w)), c = r / (h * w), yx = r % (h * w), y = yx / w, x = yx % w;
  const T* s = in + (size_t)b * ibs + (size_t)c * H * W + (size_t)(2 * y) * W + 2 * x;
  const float v = 0.25f * ((ldf(s) + ldf(s + 1)) + (ldf(s + W) + ldf(s + W + 1)));
  out[(size_t)b * obs + r] = tof<T>(v);
}
// din [C][H][W] = dout [C][H/2][W/2] / 4 at each of the four children
__global__ void k_pool_bwd(const float* __restrict__ dout, size_t obs, float* din, size_t ibs, int C, int H, int W,
                           int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * H * W) return;
  const int b = (int)(i / ((size_t)C * H * W));
  const int r = (int)(i % ((size_t)C * H * W)), c = r / (H * W), yx = r % (H * W), y = yx / W, x = yx % W;
  din[(size_t)b * ibs + r] = 0.25f * dout[(size_t)b * obs + (size_t)c * (H / 2) * (W / 2) + (y / 2) * (W / 2) + x / 2];
}
// nearest 2x upsample: out [C][2H][2W] from in [C][H][W]
template <typename T>
__global__ void k_up(const T* __restrict__ in, size_t ibs, T* out, size_t obs, int C, int H, int W, int B) {
  const int H2 = 2 * H, W2 = 2 * W;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * H2 * W2) return;
  const int b = (int)(i / ((size_t)C * H2 * W2));
  const int r = (int)(i % ((size_t)C * H2 * W2)), c = r / (H2 * W2), yx = r % (H2 * W2), y = yx / W2, x = yx % W2;
  out[(size_t)b * obs + r] = in[(size_t)b * ibs + (size_t)c * H * W + (y / 2) * W + x / 2];
}
// din [C][H][W] = sum of dout over the four children in [C][2H][2W]
__global__ void k_up_bwd(const float* __restrict__ dout, size_t obs, float* din, size_t ibs, int C, int H, int W,
                         int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * C * H * W) return;
  const int b = (int)(i / ((size_t)C * H * W));
  const int r = (int)(i % ((size_t)C * H * W)), c = r / (H * W), yx = r % (H * W), y = yx / W, x = yx % W;
  const float* s = dout + (size_t)b * obs + (size_t)c * 4 * H * W + (size_t)(2 * y) * (2 * W) + 2 * x;
  din[(size_t)b * ibs + r] = (s[0] + s[1]) + (s[2 * W] + s[2 * W + 1]);
}

// dout = 2 (out - target) / n; loss = sum (out - target)^2 / n (one block)
__global__ void __launch_bounds__(1024) k_mse(const float* __restrict__ out, const float* __restrict__ target,
                                              float* dout, int n, double* loss) {
  __shared__ double red[32];
  double acc = 0.0;
  const float s = 2.f / (float)n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = out[i] - target[i];
    dout[i] = s * d;
    acc += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *loss = t / (double)n;
  }
}

__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks_for(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct Layer {
  int Ci, Co, k;
  long long woff, boff;
};

}  // namespace

struct sgn_unet_ctx {
  int n = 0, maxB = 0, bf16 = 1;
  cudaStream_t stream = 0;
  std::vector<Layer> L;
  long long P = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  // activations (element type by bf16) and FP32 gradient buffers
  void *A0 = nullptr, *CAT0 = nullptr, *Q0 = nullptr, *A1 = nullptr, *CAT1 = nullptr, *Q1 = nullptr, *A2 = nullptr,
       *A3 = nullptr, *A4 = nullptr, *A5 = nullptr;
  float *OUT = nullptr, *gOUT = nullptr, *gN16a = nullptr, *gN16b = nullptr, *gN48 = nullptr, *gH32a = nullptr,
        *gH32b = nullptr, *gH64 = nullptr, *gH16 = nullptr, *gQ32a = nullptr, *gQ32b = nullptr;
  const float* lastIn = nullptr;
  int lastB = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

enum { E0 = 0, S0, E1, S1, B0, B1, D1, D0, OUTL, NLAYERS };

struct Fail {
  sgn_status st;
};

#define UCK(...)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess) {                                                                         \
      net->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);                          \
      throw Fail{SGN_ECUDA};                                                                         \
    }                                                                                                \
  } while (0)

void* ualloc(sgn_unet_ctx* net, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    net->err = "cudaMalloc failed";
    throw Fail{SGN_ENOMEM};
  }
  net->allocs.push_back(p);
  return p;
}

// Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases; the output
// layer starts 10x smaller so that the first corrections are small.
void init_params(sgn_unet_ctx* net, unsigned long long seed) {
  std::vector<float> h((size_t)net->P, 0.f);
  unsigned long long s = seed ^ 0x9e3779b97f4a7c15ull;
  auto next = [&]() {  // splitmix64
    s += 0x9e3779b97f4a7c15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) / 9007199254740992.0;  // [0, 1)
  };
  for (size_t li = 0; li < net->L.size(); ++li) {
    const Layer& l = net->L[li];
    const double fan_in = (double)l.Ci * l.k * l.k;
    const double bound = sqrt(6.0 / fan_in) * (li == OUTL ? 0.1 : 1.0);
    const long long nw = (long long)l.Co * l.Ci * l.k * l.k;
    for (long long i = 0; i < nw; ++i) h[(size_t)(l.woff + i)] = (float)((2.0 * next() - 1.0) * bound);
  }
  UCK(cudaMemcpy(net->params, h.data(), sizeof(float) * (size_t)net->P, cudaMemcpyHostToDevice));
  UCK(cudaMemset(net->m, 0, sizeof(float) * (size_t)net->P));
  UCK(cudaMemset(net->v, 0, sizeof(float) * (size_t)net->P));
  UCK(cudaMemset(net->grads, 0, sizeof(float) * (size_t)net->P));
}

template <typename TI, typename TO>
void conv3(sgn_unet_ctx* net, const TI* in, size_t ibs, int li, TO* out, size_t obs, int H, int B, bool relu) {
  const Layer& l = net->L[li];
  dim3 grid(((H + TILE - 1) / TILE) * ((H + TILE - 1) / TILE), (l.Co + COT - 1) / COT, B);
  k_conv3<TI, TO, false><<<grid, dim3(TILE, TILE), 0, net->stream>>>(
      in, ibs, l.Ci, out, obs, l.Co, net->params + l.woff, net->params + l.boff, l.Ci, H, H, relu ? 1 : 0);
  UCK(cudaGetLastError());
}
// gradient with respect to the layer input (channels Ci) from dp (channels Co)
void conv3_dx(sgn_unet_ctx* net, const float* dp, size_t dbs, int li, float* dx, size_t xbs, int H, int B) {
  const Layer& l = net->L[li];
  dim3 grid(((H + TILE - 1) / TILE) * ((H + TILE - 1) / TILE), (l.Ci + COT - 1) / COT, B);
  k_conv3<float, float, true><<<grid, dim3(TILE, TILE), 0, net->stream>>>(
      dp, dbs, l.Co, dx, xbs, l.Ci, net->params + l.woff, nullptr, l.Ci, H, H, 0);
  UCK(cudaGetLastError());
}
template <typename TI>
void conv3_dw(sgn_unet_ctx* net, const TI* in, size_t ibs, const float* dp, size_t dbs, int li, int H, int B) {
  const Layer& l = net->L[li];
  k_conv3_dw<TI><<<dim3(l.Co, l.Ci), 256, 0, net->stream>>>(in, ibs, l.Ci, dp, dbs, l.Co, H, H, B,
                                                             net->grads + l.woff, net->grads + l.boff);
  UCK(cudaGetLastError());
}
template <typename T>
void relu_bwd(sgn_unet_ctx* net, const T* act, size_t abs_, float* g, size_t gbs, const float* extra, size_t ebs,
              int C, int H, int B) {
  const size_t n = (size_t)B * C * H * H;
  k_relu_bwd<T><<<blocks_for(n), 256, 0, net->stream>>>(act, abs_, g, gbs, extra, ebs, C, H * H, B);
  UCK(cudaGetLastError());
}

template <typename T>
void forward_impl(sgn_unet_ctx* net, const float* in, float* out, int B) {
  const int n = net->n, h = n / 2, q = n / 4;
  const size_t N = (size_t)n * n, Hh = (size_t)h * h, Qq = (size_t)q * q;
  T* A0 = (T*)net->A0;
  T* CAT0 = (T*)net->CAT0;
  T* Q0 = (T*)net->Q0;
  T* A1 = (T*)net->A1;
  T* CAT1 = (T*)net->CAT1;
  T* Q1 = (T*)net->Q1;
  T* A2 = (T*)net->A2;
  T* A3 = (T*)net->A3;
  T* A4 = (T*)net->A4;
  T* A5 = (T*)net->A5;
  conv3<float, T>(net, in, 4 * N, E0, A0, 16 * N, n, B, true);
  conv3<T, T>(net, A0, 16 * N, S0, CAT0 + 32 * N, 48 * N, n, B, true);  // s0 -> CAT0[32, 48)
  k_pool<T><<<blocks_for((size_t)B * 16 * Hh), 256, 0, net->stream>>>(CAT0 + 32 * N, 48 * N, Q0, 16 * Hh, 16, n, n, B);
  UCK(cudaGetLastError());
  conv3<T, T>(net, Q0, 16 * Hh, E1, A1, 32 * Hh, h, B, true);
  conv3<T, T>(net, A1, 32 * Hh, S1, CAT1 + 32 * Hh, 64 * Hh, h, B, true);  // s1 -> CAT1[32, 64)
  k_pool<T><<<blocks_for((size_t)B * 32 * Qq), 256, 0, net->stream>>>(CAT1 + 32 * Hh, 64 * Hh, Q1, 32 * Qq, 32, h, h, B);
  UCK(cudaGetLastError());
  conv3<T, T>(net, Q1, 32 * Qq, B0, A2, 32 * Qq, q, B, true);
  conv3<T, T>(net, A2, 32 * Qq, B1, A3, 32 * Qq, q, B, true);
  k_up<T><<<blocks_for((size_t)B * 32 * Hh), 256, 0, net->stream>>>(A3, 32 * Qq, CAT1, 64 * Hh, 32, q, q, B);
  UCK(cudaGetLastError());
  conv3<T, T>(net, CAT1, 64 * Hh, D1, A4, 32 * Hh, h, B, true);
  k_up<T><<<blocks_for((size_t)B * 32 * N), 256, 0, net->stream>>>(A4, 32 * Hh, CAT0, 48 * N, 32, h, h, B);
  UCK(cudaGetLastError());
  conv3<T, T>(net, CAT0, 48 * N, D0, A5, 16 * N, n, B, true);
  const Layer& lo = net->L[OUTL];
  k_conv1_fwd<T><<<blocks_for((size_t)B * N), 256, 0, net->stream>>>(A5, 16 * N, 16, net->params + lo.woff,
                                                                     net->params + lo.boff, net->OUT, (int)N, B);
  UCK(cudaGetLastError());
  if (out) UCK(cudaMemcpyAsync(out, net->OUT, sizeof(float) * B * N, cudaMemcpyDeviceToDevice, net->stream));
}

template <typename T>
void backward_impl(sgn_unet_ctx* net, const float* target, double* loss) {
  const int n = net->n, h = n / 2, q = n / 4, B = net->lastB;
  const size_t N = (size_t)n * n, Hh = (size_t)h * h, Qq = (size_t)q * q;
  T* A0 = (T*)net->A0;
  T* CAT0 = (T*)net->CAT0;
  T* Q0 = (T*)net->Q0;
  T* A1 = (T*)net->A1;
  T* CAT1 = (T*)net->CAT1;
  T* Q1 = (T*)net->Q1;
  T* A2 = (T*)net->A2;
  T* A3 = (T*)net->A3;
  T* A4 = (T*)net->A4;
  T* A5 = (T*)net->A5;
  k_mse<<<1, 1024, 0, net->stream>>>(net->OUT, target, net->gOUT, (int)(B * N), loss);
  UCK(cudaGetLastError());
  // output layer 16 -> 1
  const Layer& lo = net->L[OUTL];
  k_conv1_dw<T><<<17, 256, 0, net->stream>>>(A5, 16 * N, 16, net->gOUT, (int)N, B, net->grads + lo.woff,
                                             net->grads + lo.boff);
  UCK(cudaGetLastError());
  float* dP7 = net->gN16a;  // d(pre-activation of d0), [16] at n
  k_conv1_dx_relu<T><<<blocks_for((size_t)B * 16 * N), 256, 0, net->stream>>>(A5, 16 * N, 16, net->params + lo.woff,
                                                                              net->gOUT, dP7, 16 * N, (int)N, B);
  UCK(cudaGetLastError());
  // d0: 48 -> 16 on CAT0
  conv3_dw<T>(net, CAT0, 48 * N, dP7, 16 * N, D0, n, B);
  float* dCAT0 = net->gN48;
  conv3_dx(net, dP7, 16 * N, D0, dCAT0, 48 * N, n, B);
  // u0: CAT0[0, 32) came from A4 (relu output of d1)
  float* dP6 = net->gH32a;
  k_up_bwd<<<blocks_for((size_t)B * 32 * Hh), 256, 0, net->stream>>>(dCAT0, 48 * N, dP6, 32 * Hh, 32, h, h, B);
  UCK(cudaGetLastError());
  relu_bwd<T>(net, A4, 32 * Hh, dP6, 32 * Hh, nullptr, 0, 32, h, B);
  // d1: 64 -> 32 on CAT1
  conv3_dw<T>(net, CAT1, 64 * Hh, dP6, 32 * Hh, D1, h, B);
  float* dCAT1 = net->gH64;
  conv3_dx(net, dP6, 32 * Hh, D1, dCAT1, 64 * Hh, h, B);
  // u1: CAT1[0, 32) came from A3 (relu output of b1)
  float* dP5 = net->gQ32a;
  k_up_bwd<<<blocks_for((size_t)B * 32 * Qq), 256, 0, net->stream>>>(dCAT1, 64 * Hh, dP5, 32 * Qq, 32, q, q, B);
  UCK(cudaGetLastError());
  relu_bwd<T>(net, A3, 32 * Qq, dP5, 32 * Qq, nullptr, 0, 32, q, B);
  // b1: 32 -> 32 on A2
  conv3_dw<T>(net, A2, 32 * Qq, dP5, 32 * Qq, B1, q, B);
  float* dP4 = net->gQ32b;
  conv3_dx(net, dP5, 32 * Qq, B1, dP4, 32 * Qq, q, B);
  relu_bwd<T>(net, A2, 32 * Qq, dP4, 32 * Qq, nullptr, 0, 32, q, B);
  // b0: 32 -> 32 on Q1
  conv3_dw<T>(net, Q1, 32 * Qq, dP4, 32 * Qq, B0, q, B);
  float* dQ1 = net->gQ32a;
  conv3_dx(net, dP4, 32 * Qq, B0, dQ1, 32 * Qq, q, B);
  // p1: s1 = CAT1[32, 64) gets the pool gradient plus the skip gradient dCAT1[32, 64)
  float* dP3 = net->gH32b;
  k_pool_bwd<<<blocks_for((size_t)B * 32 * Hh), 256, 0, net->stream>>>(dQ1, 32 * Qq, dP3, 32 * Hh, 32, h, h, B);
  UCK(cudaGetLastError());
  relu_bwd<T>(net, CAT1 + 32 * Hh, 64 * Hh, dP3, 32 * Hh, dCAT1 + 32 * Hh, 64 * Hh, 32, h, B);
  // s1: 32 -> 32 on A1
  conv3_dw<T>(net, A1, 32 * Hh, dP3, 32 * Hh, S1, h, B);
  float* dP2 = net->gH32a;
  conv3_dx(net, dP3, 32 * Hh, S1, dP2, 32 * Hh, h, B);
  relu_bwd<T>(net, A1, 32 * Hh, dP2, 32 * Hh, nullptr, 0, 32, h, B);
  // e1: 16 -> 32 on Q0
  conv3_dw<T>(net, Q0, 16 * Hh, dP2, 32 * Hh, E1, h, B);
  float* dQ0 = net->gH16;
  conv3_dx(net, dP2, 32 * Hh, E1, dQ0, 16 * Hh, h, B);
  // p0: s0 = CAT0[32, 48) gets the pool gradient plus dCAT0[32, 48)
  float* dP1 = net->gN16a;
  k_pool_bwd<<<blocks_for((size_t)B * 16 * N), 256, 0, net->stream>>>(dQ0, 16 * Hh, dP1, 16 * N, 16, n, n, B);
  UCK(cudaGetLastError());
  relu_bwd<T>(net, CAT0 + 32 * N, 48 * N, dP1, 16 * N, dCAT0 + 32 * N, 48 * N, 16, n, B);
  // s0: 16 -> 16 on A0
  conv3_dw<T>(net, A0, 16 * N, dP1, 16 * N, S0, n, B);
  float* dP0 = net->gN16b;
  conv3_dx(net, dP1, 16 * N, S0, dP0, 16 * N, n, B);
  relu_bwd<T>(net, A0, 16 * N, dP0, 16 * N, nullptr, 0, 16, n, B);
  // e0: 4 -> 16 on the input
  conv3_dw<float>(net, net->lastIn, 4 * N, dP0, 16 * N, E0, n, B);
}

sgn_status ufail(sgn_unet_ctx* net, sgn_status st, const char* msg) {
  if (net) net->err = msg;
  return st;
}

void ufree(sgn_unet_ctx* net) {
  for (void* p : net->allocs) cudaFree(p);
  net->allocs.clear();
}

}  // namespace

#define UAPI_BEGIN                                                                                 \
  if (!net) return SGN_EINVAL;                                                                     \
  net->err.clear();                                                                                \
  try {
#define UAPI_END                                                                                   \
  }                                                                                                \
  catch (Fail & f) {                                                                               \
    return f.st;                                                                                   \
  }

extern "C" {

sgn_status sgn_unet_create(int n, int max_batch, int act_bf16, unsigned long long seed, sgn_unet_t* out) {
  if (!out) return SGN_EINVAL;
  *out = nullptr;
  if (n < 16 || n > 512 || (n & (n - 1)) != 0 || max_batch < 1 || max_batch > 64) return SGN_EINVAL;
  sgn_unet_ctx* net = new (std::nothrow) sgn_unet_ctx();
  if (!net) return SGN_ENOMEM;
  net->n = n;
  net->maxB = max_batch;
  net->bf16 = act_bf16 ? 1 : 0;
  const int spec[NLAYERS][3] = {{4, 16, 3},  {16, 16, 3}, {16, 32, 3}, {32, 32, 3}, {32, 32, 3},
                                {32, 32, 3}, {64, 32, 3}, {48, 16, 3}, {16, 1, 1}};
  long long off = 0;
  for (int i = 0; i < NLAYERS; ++i) {
    Layer l;
    l.Ci = spec[i][0];
    l.Co = spec[i][1];
    l.k = spec[i][2];
    l.woff = off;
    off += (long long)l.Co * l.Ci * l.k * l.k;
    l.boff = off;
    off += l.Co;
    net->L.push_back(l);
  }
  net->P = off;
  try {
    const size_t B = (size_t)max_batch, N = (size_t)n * n, Hh = N / 4, Qq = N / 16;
    const size_t es = net->bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
    net->params = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->grads = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->m = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->v = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->A0 = ualloc(net, es * B * 16 * N);
    net->CAT0 = ualloc(net, es * B * 48 * N);
    net->Q0 = ualloc(net, es * B * 16 * Hh);
    net->A1 = ualloc(net, es * B * 32 * Hh);
    net->CAT1 = ualloc(net, es * B * 64 * Hh);
    net->Q1 = ualloc(net, es * B * 32 * Qq);
    net->A2 = ualloc(net, es * B * 32 * Qq);
    net->A3 = ualloc(net, es * B * 32 * Qq);
    net->A4 = ualloc(net, es * B * 32 * Hh);
    net->A5 = ualloc(net, es * B * 16 * N);
    net->OUT = (float*)ualloc(net, sizeof(float) * B * N);
    net->gOUT = (float*)ualloc(net, sizeof(float) * B * N);
    net->gN16a = (float*)ualloc(net, sizeof(float) * B * 16 * N);
    net->gN16b = (float*)ualloc(net, sizeof(float) * B * 16 * N);
    net->gN48 = (float*)ualloc(net, sizeof(float) * B * 48 * N);
    net->gH32a = (float*)ualloc(net, sizeof(float) * B * 32 * Hh);
    net->gH32b = (float*)ualloc(net, sizeof(float) * B * 32 * Hh);
    net->gH64 = (float*)ualloc(net, sizeof(float) * B * 64 * Hh);
    net->gH16 = (float*)ualloc(net, sizeof(float) * B * 16 * Hh);
    net->gQ32a = (float*)ualloc(net, sizeof(float) * B * 32 * Qq);
    net->gQ32b = (float*)ualloc(net, sizeof(float) * B * 32 * Qq);
    init_params(net, seed);
    UCK(cudaDeviceSynchronize());
  } catch (Fail& f) {
    ufree(net);
    delete net;
    return f.st;
  }
  *out = net;
  return SGN_OK;
}

sgn_status sgn_unet_destroy(sgn_unet_t net) {
  if (!net) return SGN_EINVAL;
  cudaStreamSynchronize(net->stream);
  ufree(net);
  delete net;
  return SGN_OK;
}

sgn_status sgn_unet_set_stream(sgn_unet_t net, void* s) {
  if (!net) return SGN_EINVAL;
  net->stream = (cudaStream_t)s;
  return SGN_OK;
}

const char* sgn_unet_last_error(sgn_unet_t net) { return net ? net->err.c_str() : ""; }

long long sgn_unet_num_params(sgn_unet_t net) { return net ? net->P : -1; }

int sgn_unet_side(sgn_unet_t net) { return net ? net->n : -1; }

sgn_status sgn_unet_set_params(sgn_unet_t net, const float* p) {
  UAPI_BEGIN
  if (!p) return ufail(net, SGN_EINVAL, "sgn_unet_set_params: NULL");
  UCK(cudaMemcpyAsync(net->params, p, sizeof(float) * (size_t)net->P, cudaMemcpyDeviceToDevice, net->stream));
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_get_params(sgn_unet_t net, float* p) {
  UAPI_BEGIN
  if (!p) return ufail(net, SGN_EINVAL, "sgn_unet_get_params: NULL");
  UCK(cudaMemcpyAsync(p, net->params, sizeof(float) * (size_t)net->P, cudaMemcpyDeviceToDevice, net->stream));
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_get_grads(sgn_unet_t net, float* g) {
  UAPI_BEGIN
  if (!g) return ufail(net, SGN_EINVAL, "sgn_unet_get_grads: NULL");
  UCK(cudaMemcpyAsync(g, net->grads, sizeof(float) * (size_t)net->P, cudaMemcpyDeviceToDevice, net->stream));
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_forward(sgn_unet_t net, const float* in, float* out, int batch) {
  UAPI_BEGIN
  if (!in || batch < 1 || batch > net->maxB) return ufail(net, SGN_EINVAL, "sgn_unet_forward: bad input or batch");
  if (net->bf16)
    forward_impl<__nv_bfloat16>(net, in, out, batch);
  else
    forward_impl<float>(net, in, out, batch);
  net->lastIn = in;
  net->lastB = batch;
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_backward(sgn_unet_t net, const float* target, double* loss_dev) {
  UAPI_BEGIN
  if (!target || net->lastB < 1 || !net->lastIn)
    return ufail(net, SGN_EINVAL, "sgn_unet_backward: no forward pass or NULL target");
  if (net->bf16)
    backward_impl<__nv_bfloat16>(net, target, loss_dev);
  else
    backward_impl<float>(net, target, loss_dev);
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_adam_step(sgn_unet_t net, float lr, float b1, float b2, float eps, int t) {
  UAPI_BEGIN
  if (t < 1) return ufail(net, SGN_EINVAL, "sgn_unet_adam_step: t < 1");
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<blocks_for((size_t)net->P), 256, 0, net->stream>>>(net->params, net->grads, net->m, net->v, net->P, lr,
                                                               b1, b2, eps, c1, c2);
  UCK(cudaGetLastError());
  return SGN_OK;
  UAPI_END
}

}  // extern "C"
