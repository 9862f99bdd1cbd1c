// sgn_unet.cu - the periodic U-Net (include/sgn_unet.h) that corrects the
// GMRES starting value of sigma: any depth and widths.
//
// Training (forward, backward, Adam) runs direct convolutions on CUDA cores in
// NCHW: activations stored as T (BF16 or FP32), everything else FP32; sums over
// pixels (weight gradients, the loss) are per-block fixed-order reductions, so
// results are deterministic. Inference (sgn_unet_infer) runs the 3x3 layers
// after the first as BF16 implicit GEMMs on the tensor cores over NHWC
// activations (sgn_unet_tc.cuh).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <new>
#include <string>
#include <vector>

#include "sgn_unet.h"
#include "sgn_unet_tc.cuh"

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

constexpr int kMaxLevels = 6;

struct Layer {
  int Ci, Co, k;
  long long woff, boff;
  // tensor-core inference (3x3 layers after the first)
  int KC = 0, nkb = 0, smem = 0;
  long long ioff = -1;
  int level = 0;     // resolution level (grid side n / 2^level)
  bool row = false;  // >= 128 pixels per image: the halo-staged row kernel
};


}  // namespace

struct sgn_unet_ctx {
  int n = 0, maxB = 0, bf16 = 1;
  int D = 0, w[kMaxLevels] = {0};
  cudaStream_t stream = 0;
  std::vector<Layer> L;
  long long P = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  // training activations (element type by bf16), NCHW, per level l (grid n / 2^l):
  //   A[l]   w_l channels: e_l's output (l < D-1), b0's output (l = D-1)
  //   CAT[l] w_{l+1} + w_l channels: upsampled level below, then s_l's output (l < D-1)
  //   Q[l]   w_l channels on level l+1's grid: the pooled s_l (l < D-1)
  //   U[l]   w_l channels: d_l's output (l < D-1), b1's output (l = D-1)
  void *A[kMaxLevels] = {}, *CAT[kMaxLevels] = {}, *Q[kMaxLevels] = {}, *U[kMaxLevels] = {};
  float *OUT = nullptr, *gOUT = nullptr;
  // FP32 gradients: two scratch tensors of wmax channels per level, and the
  // concatenation's gradient per level
  float *G[kMaxLevels][2] = {}, *gCAT[kMaxLevels] = {};
  // inference (NHWC BF16): e_l / b0 outputs, s_l outputs, pooled, d_l / b1 outputs
  __nv_bfloat16 *tA[kMaxLevels] = {}, *tS[kMaxLevels] = {}, *tQ[kMaxLevels] = {}, *tU[kMaxLevels] = {};
  __nv_bfloat16* wimg = nullptr;
  unet_tc::WImgTable wtab{};
  int* dev_err = nullptr;
  const float* lastIn = nullptr;
  int lastB = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

// parameter order: e_0, s_0, ..., e_{D-2}, s_{D-2}, b0, b1, d_{D-2}, ..., d_0, out
inline int iE(int l) { return 2 * l; }
inline int iS(int l) { return 2 * l + 1; }
inline int iB0(const sgn_unet_ctx* net) { return 2 * (net->D - 1); }
inline int iB1(const sgn_unet_ctx* net) { return 2 * (net->D - 1) + 1; }
inline int iD(const sgn_unet_ctx* net, int l) { return 2 * net->D + (net->D - 2 - l); }
inline int iOut(const sgn_unet_ctx* net) { return 3 * net->D - 1; }

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
  const int out_layer = iOut(net);
  for (size_t li = 0; li < net->L.size(); ++li) {
    const Layer& l = net->L[li];
    const double fan_in = (double)l.Ci * l.k * l.k;
    const double bound = sqrt(6.0 / fan_in) * ((int)li == out_layer ? 0.1 : 1.0);
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

inline size_t npix(const sgn_unet_ctx* net, int l) { return (size_t)(net->n >> l) * (size_t)(net->n >> l); }

template <typename T>
void forward_impl(sgn_unet_ctx* net, const float* in, float* out, int B) {
  const int D = net->D;
  const int* w = net->w;
  // encoder
  for (int l = 0; l < D - 1; ++l) {
    const int H = net->n >> l;
    const size_t N = npix(net, l), Nq = npix(net, l + 1);
    T* A = (T*)net->A[l];
    T* S = (T*)net->CAT[l] + (size_t)w[l + 1] * N;  // s_l lives in CAT[l] after the upsampled channels
    const size_t cs = (size_t)(w[l + 1] + w[l]) * N;
    if (l == 0)
      conv3<float, T>(net, in, 4 * N, iE(0), A, (size_t)w[0] * N, H, B, true);
    else
      conv3<T, T>(net, (const T*)net->Q[l - 1], (size_t)w[l - 1] * N, iE(l), A, (size_t)w[l] * N, H, B, true);
    conv3<T, T>(net, A, (size_t)w[l] * N, iS(l), S, cs, H, B, true);
    k_pool<T><<<blocks_for((size_t)B * w[l] * Nq), 256, 0, net->stream>>>(S, cs, (T*)net->Q[l], (size_t)w[l] * Nq,
                                                                           w[l], H, H, B);
    UCK(cudaGetLastError());
  }
  // bottleneck
  {
    const int l = D - 1, H = net->n >> l;
    const size_t N = npix(net, l);
    conv3<T, T>(net, (const T*)net->Q[l - 1], (size_t)w[l - 1] * N, iB0(net), (T*)net->A[l], (size_t)w[l] * N, H, B,
                true);
    conv3<T, T>(net, (const T*)net->A[l], (size_t)w[l] * N, iB1(net), (T*)net->U[l], (size_t)w[l] * N, H, B, true);
  }
  // decoder
  for (int l = D - 2; l >= 0; --l) {
    const int H = net->n >> l;
    const size_t N = npix(net, l), Nb = npix(net, l + 1);
    const size_t cs = (size_t)(w[l + 1] + w[l]) * N;
    k_up<T><<<blocks_for((size_t)B * w[l + 1] * N), 256, 0, net->stream>>>(
        (const T*)net->U[l + 1], (size_t)w[l + 1] * Nb, (T*)net->CAT[l], cs, w[l + 1], H / 2, H / 2, B);
    UCK(cudaGetLastError());
    conv3<T, T>(net, (const T*)net->CAT[l], cs, iD(net, l), (T*)net->U[l], (size_t)w[l] * N, H, B, true);
  }
  const Layer& lo = net->L[iOut(net)];
  const size_t N0 = npix(net, 0);
  k_conv1_fwd<T><<<blocks_for((size_t)B * N0), 256, 0, net->stream>>>(
      (const T*)net->U[0], (size_t)w[0] * N0, w[0], net->params + lo.woff, net->params + lo.boff, net->OUT, (int)N0,
      B);
  UCK(cudaGetLastError());
  if (out) UCK(cudaMemcpyAsync(out, net->OUT, sizeof(float) * B * N0, cudaMemcpyDeviceToDevice, net->stream));
}

template <typename T>
void backward_impl(sgn_unet_ctx* net, const float* target, double* loss) {
  const int D = net->D, B = net->lastB;
  const int* w = net->w;
  const size_t N0 = npix(net, 0);
  k_mse<<<1, 1024, 0, net->stream>>>(net->OUT, target, net->gOUT, (int)(B * N0), loss);
  UCK(cudaGetLastError());
  // output layer w_0 -> 1, then the ReLU of d_0
  const Layer& lo = net->L[iOut(net)];
  k_conv1_dw<T><<<w[0] + 1, 256, 0, net->stream>>>((const T*)net->U[0], (size_t)w[0] * N0, w[0], net->gOUT, (int)N0,
                                                   B, net->grads + lo.woff, net->grads + lo.boff);
  UCK(cudaGetLastError());
  k_conv1_dx_relu<T><<<blocks_for((size_t)B * w[0] * N0), 256, 0, net->stream>>>(
      (const T*)net->U[0], (size_t)w[0] * N0, w[0], net->params + lo.woff, net->gOUT, net->G[0][0],
      (size_t)w[0] * N0, (int)N0, B);
  UCK(cudaGetLastError());
  // decoder, from the top level down the U: G[l][0] holds d(pre-activation of d_l)
  for (int l = 0; l < D - 1; ++l) {
    const int H = net->n >> l;
    const size_t N = npix(net, l), Nb = npix(net, l + 1);
    const size_t cs = (size_t)(w[l + 1] + w[l]) * N;
    conv3_dw<T>(net, (const T*)net->CAT[l], cs, net->G[l][0], (size_t)w[l] * N, iD(net, l), H, B);
    conv3_dx(net, net->G[l][0], (size_t)w[l] * N, iD(net, l), net->gCAT[l], cs, H, B);
    // the upsampled channels came from U[l+1] (the ReLU output of d_{l+1} or b1)
    float* g = net->G[l + 1][0];
    k_up_bwd<<<blocks_for((size_t)B * w[l + 1] * Nb), 256, 0, net->stream>>>(net->gCAT[l], cs, g,
                                                                             (size_t)w[l + 1] * Nb, w[l + 1], H / 2,
                                                                             H / 2, B);
    UCK(cudaGetLastError());
    relu_bwd<T>(net, (const T*)net->U[l + 1], (size_t)w[l + 1] * Nb, g, (size_t)w[l + 1] * Nb, nullptr, 0, w[l + 1],
                H / 2, B);
  }
  // bottleneck: G[D-1][0] = d(pre-activation of b1)
  {
    const int l = D - 1, H = net->n >> l;
    const size_t N = npix(net, l);
    const size_t bs = (size_t)w[l] * N;
    conv3_dw<T>(net, (const T*)net->A[l], bs, net->G[l][0], bs, iB1(net), H, B);
    conv3_dx(net, net->G[l][0], bs, iB1(net), net->G[l][1], bs, H, B);
    relu_bwd<T>(net, (const T*)net->A[l], bs, net->G[l][1], bs, nullptr, 0, w[l], H, B);
    conv3_dw<T>(net, (const T*)net->Q[l - 1], (size_t)w[l - 1] * N, net->G[l][1], bs, iB0(net), H, B);
    // d(pooled s_{D-2}) into G[D-1][0]
    conv3_dx(net, net->G[l][1], bs, iB0(net), net->G[l][0], (size_t)w[l - 1] * N, H, B);
  }
  // encoder, back up to the input: G[l+1][0] holds d(Q[l])
  for (int l = D - 2; l >= 0; --l) {
    const int H = net->n >> l;
    const size_t N = npix(net, l), Nq = npix(net, l + 1);
    const size_t cs = (size_t)(w[l + 1] + w[l]) * N, bs = (size_t)w[l] * N;
    float* g0 = net->G[l][0];
    float* g1 = net->G[l][1];
    k_pool_bwd<<<blocks_for((size_t)B * w[l] * N), 256, 0, net->stream>>>(net->G[l + 1][0], (size_t)w[l] * Nq, g0, bs,
                                                                          w[l], H, H, B);
    UCK(cudaGetLastError());
    // s_l also feeds the decoder through the concatenation
    const T* S = (const T*)net->CAT[l] + (size_t)w[l + 1] * N;
    relu_bwd<T>(net, S, cs, g0, bs, net->gCAT[l] + (size_t)w[l + 1] * N, cs, w[l], H, B);
    conv3_dw<T>(net, (const T*)net->A[l], bs, g0, bs, iS(l), H, B);
    conv3_dx(net, g0, bs, iS(l), g1, bs, H, B);
    relu_bwd<T>(net, (const T*)net->A[l], bs, g1, bs, nullptr, 0, w[l], H, B);
    if (l == 0) {
      conv3_dw<float>(net, net->lastIn, 4 * N, g1, bs, iE(0), H, B);
    } else {
      conv3_dw<T>(net, (const T*)net->Q[l - 1], (size_t)w[l - 1] * N, g1, bs, iE(l), H, B);
      conv3_dx(net, g1, bs, iE(l), g0, (size_t)w[l - 1] * N, H, B);
    }
  }
}

// ---------------------------------------------------- tensor-core inference
void tc_conv(sgn_unet_ctx* net, int li, const __nv_bfloat16* src0, int C0, int up0, const __nv_bfloat16* src1,
             int C1, int l, int B, __nv_bfloat16* out, const float* head_w = nullptr, const float* head_b = nullptr,
             float* head_out = nullptr) {
  const Layer& L = net->L[li];
  unet_tc::ConvArgs a{};
  a.src0 = src0;
  a.src1 = src1;
  a.C0 = C0;
  a.C1 = C1;
  a.up0 = up0;
  int lg = 0;
  while ((1 << lg) < (net->n >> l)) ++lg;
  a.lH = a.lW = lg;
  a.npix = B * (int)npix(net, l);
  a.wimg = net->wimg + L.ioff;
  a.bias = net->params + L.boff;
  a.Co = L.Co;
  a.KC = L.KC;
  a.nkb = L.nkb;
  uint32_t cols = 32;
  while ((int)cols < L.Co) cols <<= 1;
  a.tmem_cols = cols;
  a.out = out;
  a.head_w = head_w;
  a.head_b = head_b;
  a.head_out = head_out;
  a.err = net->dev_err;
  const unsigned grid = (unsigned)((a.npix + unet_tc::kM - 1) / unet_tc::kM);
  if (L.row)
    unet_tc::k_conv3_tc_row<<<grid, unet_tc::kThreads, L.smem, net->stream>>>(a);
  else
    unet_tc::k_conv3_tc<<<grid, unet_tc::kThreads, L.smem, net->stream>>>(a);
  UCK(cudaGetLastError());
}

void infer_impl(sgn_unet_ctx* net, const float* in, float* out, int B) {
  const int D = net->D;
  const int* w = net->w;
  {
    const unsigned nb = (unsigned)((net->wtab.total + 255) / 256);
    unet_tc::k_wimg<<<nb, 256, 0, net->stream>>>(net->wtab, net->params, net->wimg);
    UCK(cudaGetLastError());
  }
  int lg0 = 0;
  while ((1 << lg0) < net->n) ++lg0;
  {
    const Layer& L = net->L[iE(0)];
    const int np = B * (int)npix(net, 0);
    unet_tc::k_conv_in_nhwc<<<(np + 127) / 128, 128, sizeof(float) * L.Co * 37, net->stream>>>(
        in, lg0, lg0, np, net->params + L.woff, net->params + L.boff, L.Co, net->tA[0]);
    UCK(cudaGetLastError());
  }
  for (int l = 0; l < D - 1; ++l) {
    if (l > 0) tc_conv(net, iE(l), net->tQ[l - 1], w[l - 1], 0, nullptr, 0, l, B, net->tA[l]);
    tc_conv(net, iS(l), net->tA[l], w[l], 0, nullptr, 0, l, B, net->tS[l]);
    const int nout = B * (int)npix(net, l + 1);
    unet_tc::k_pool_nhwc<<<blocks_for((size_t)nout * (w[l] / 8)), 256, 0, net->stream>>>(
        net->tS[l], lg0 - l, lg0 - l, w[l], nout, net->tQ[l]);
    UCK(cudaGetLastError());
  }
  tc_conv(net, iB0(net), net->tQ[D - 2], w[D - 2], 0, nullptr, 0, D - 1, B, net->tA[D - 1]);
  tc_conv(net, iB1(net), net->tA[D - 1], w[D - 1], 0, nullptr, 0, D - 1, B, net->tU[D - 1]);
  for (int l = D - 2; l >= 1; --l)
    tc_conv(net, iD(net, l), net->tU[l + 1], w[l + 1], 1, net->tS[l], w[l], l, B, net->tU[l]);
  const Layer& lo = net->L[iOut(net)];
  tc_conv(net, iD(net, 0), net->tU[1], w[1], 1, net->tS[0], w[0], 0, B, nullptr, net->params + lo.woff,
          net->params + lo.boff, out);
}

sgn_status ufail(sgn_unet_ctx* net, sgn_status st, const char* msg) {
  if (net) net->err = msg;
  return st;
}

void ufree(sgn_unet_ctx* net) {
  for (void* p : net->allocs) cudaFree(p);
  net->allocs.clear();
}

// channels per K step of a tensor-core layer: the fewest steps per tap whose
// operands fit one shared-memory stage
int pick_kc(int Ci, int Co) {
  for (int nkb = 1; nkb <= Ci / 16; ++nkb) {
    if (Ci % nkb) continue;
    const int kc = Ci / nkb;
    if (kc % 16 || kc > unet_tc::kMaxKC) continue;
    if ((int)unet_tc::stage_bytes(Co, kc) <= unet_tc::kStageMax) return kc;
  }
  return 16;
}

// channels per block of the row kernel: the fewest blocks whose halo and
// weight buffers fit 110 KB (two CTAs per SM), or 200 KB when the layer has
// fewer tiles than the GPU has SMs (one CTA per SM costs nothing there, and
// each block is a step of the tile's dependent chain)
int pick_kc_row(int Ci, int Co, int W, long long tiles) {
  const int budget = (tiles < 148 ? 200 : 110) * 1024;
  for (int nkb = 1; nkb <= Ci / 16; ++nkb) {
    if (Ci % nkb) continue;
    const int kc = Ci / nkb;
    if (kc % 16) continue;
    if ((int)unet_tc::row_smem_bytes(Co, kc, nkb, W) <= budget) return kc;
  }
  return 16;
}

sgn_status create_impl(int n, int max_batch, int act_bf16, unsigned long long seed, int levels, const int* widths,
                       sgn_unet_t* out) {
  if (!out) return SGN_EINVAL;
  *out = nullptr;
  if (levels < 2 || levels > kMaxLevels || !widths) return SGN_EINVAL;
  if (n < 16 || n > 512 || (n & (n - 1)) != 0 || max_batch < 1 || max_batch > 64) return SGN_EINVAL;
  if ((n >> (levels - 1)) < 4) return SGN_EINVAL;
  for (int l = 0; l < levels; ++l)
    if (widths[l] < 16 || widths[l] > 256 || widths[l] % 16 != 0) return SGN_EINVAL;
  // one tensor-core tile of 128 pixels must not need more than 2^31 pixels in all
  if ((long long)max_batch * n * n > (1ll << 30)) return SGN_EINVAL;
  sgn_unet_ctx* net = new (std::nothrow) sgn_unet_ctx();
  if (!net) return SGN_ENOMEM;
  net->n = n;
  net->maxB = max_batch;
  net->bf16 = act_bf16 ? 1 : 0;
  net->D = levels;
  for (int l = 0; l < levels; ++l) net->w[l] = widths[l];
  const int D = levels;
  const int* w = net->w;
  std::vector<int> ci, co, kk, lv;
  auto add = [&](int a, int b, int k, int level) {
    ci.push_back(a);
    co.push_back(b);
    kk.push_back(k);
    lv.push_back(level);
  };
  for (int l = 0; l < D - 1; ++l) {
    add(l == 0 ? 4 : w[l - 1], w[l], 3, l);
    add(w[l], w[l], 3, l);
  }
  add(w[D - 2], w[D - 1], 3, D - 1);
  add(w[D - 1], w[D - 1], 3, D - 1);
  for (int l = D - 2; l >= 0; --l) add(w[l + 1] + w[l], w[l], 3, l);
  add(w[0], 1, 1, 0);
  long long off = 0, ioff = 0;
  int smem_max = 0;
  net->wtab.nl = 0;
  for (size_t i = 0; i < ci.size(); ++i) {
    Layer l;
    l.Ci = ci[i];
    l.Co = co[i];
    l.k = kk[i];
    l.woff = off;
    off += (long long)l.Co * l.Ci * l.k * l.k;
    l.boff = off;
    off += l.Co;
    l.level = lv[i];
    const int side = n >> l.level;
    l.row = side * side >= unet_tc::kM;
    if (l.k == 3 && i > 0) {
      l.KC = l.row ? pick_kc_row(l.Ci, l.Co, side, (long long)max_batch * side * side / unet_tc::kM)
                   : pick_kc(l.Ci, l.Co);
      l.nkb = l.Ci / l.KC;
      l.ioff = ioff;
      unet_tc::WImgLayer& t = net->wtab.l[net->wtab.nl++];
      t.woff = l.woff;
      t.ioff = ioff;
      t.Ci = l.Ci;
      t.Co = l.Co;
      t.KC = l.KC;
      t.nkb = l.nkb;
      t.kb_major = l.row ? 1 : 0;
      ioff += 9ll * l.Ci * l.Co;
      int sm = l.row ? (int)unet_tc::row_smem_bytes(l.Co, l.KC, l.nkb, side)
                     : unet_tc::kStages * (int)unet_tc::stage_bytes(l.Co, l.KC);
      // at most 512 / cols CTAs per SM, so that TMEM is never oversubscribed
      int cols = 32;
      while (cols < l.Co) cols <<= 1;
      const int ctas = 512 / cols;
      const int floor_bytes = 233472 / (ctas + 1) + 1;
      if (sm < floor_bytes) sm = floor_bytes;
      l.smem = sm;
      if (sm > smem_max) smem_max = sm;
    }
    net->L.push_back(l);
  }
  net->wtab.total = ioff;
  net->P = off;
  try {
    const size_t B = (size_t)max_batch;
    const size_t es = net->bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
    const size_t bf = sizeof(__nv_bfloat16);
    int wmax = 4;
    for (int l = 0; l < D; ++l) wmax = w[l] > wmax ? w[l] : wmax;
    net->params = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->grads = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->m = (float*)ualloc(net, sizeof(float) * (size_t)off);
    net->v = (float*)ualloc(net, sizeof(float) * (size_t)off);
    for (int l = 0; l < D; ++l) {
      const size_t N = npix(net, l);
      net->A[l] = ualloc(net, es * B * w[l] * N);
      net->U[l] = ualloc(net, es * B * w[l] * N);
      net->G[l][0] = (float*)ualloc(net, sizeof(float) * B * wmax * N);
      net->G[l][1] = (float*)ualloc(net, sizeof(float) * B * wmax * N);
      net->tA[l] = (__nv_bfloat16*)ualloc(net, bf * B * w[l] * N);
      net->tU[l] = (__nv_bfloat16*)ualloc(net, bf * B * w[l] * N);
      if (l < D - 1) {
        net->CAT[l] = ualloc(net, es * B * (w[l + 1] + w[l]) * N);
        net->Q[l] = ualloc(net, es * B * w[l] * npix(net, l + 1));
        net->gCAT[l] = (float*)ualloc(net, sizeof(float) * B * (w[l + 1] + w[l]) * N);
        net->tS[l] = (__nv_bfloat16*)ualloc(net, bf * B * w[l] * N);
        net->tQ[l] = (__nv_bfloat16*)ualloc(net, bf * B * w[l] * npix(net, l + 1));
      }
    }
    const size_t N0 = npix(net, 0);
    net->OUT = (float*)ualloc(net, sizeof(float) * B * N0);
    net->gOUT = (float*)ualloc(net, sizeof(float) * B * N0);
    net->wimg = (__nv_bfloat16*)ualloc(net, bf * (size_t)(ioff > 0 ? ioff : 1));
    net->dev_err = (int*)ualloc(net, sizeof(int));
    UCK(cudaMemset(net->dev_err, 0, sizeof(int)));
    UCK(cudaFuncSetAttribute(unet_tc::k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
    UCK(cudaFuncSetAttribute(unet_tc::k_conv3_tc_row, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
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
  const int widths[3] = {16, 32, 32};
  return create_impl(n, max_batch, act_bf16, seed, 3, widths, out);
}

sgn_status sgn_unet_create_arch(int n, int max_batch, int act_bf16, unsigned long long seed, int levels,
                                const int* widths, sgn_unet_t* out) {
  return create_impl(n, max_batch, act_bf16, seed, levels, widths, out);
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

int sgn_unet_levels(sgn_unet_t net) { return net ? net->D : -1; }

int sgn_unet_width(sgn_unet_t net, int level) {
  if (!net || level < 0 || level >= net->D) return -1;
  return net->w[level];
}

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

sgn_status sgn_unet_infer(sgn_unet_t net, const float* in, float* out, int batch) {
  UAPI_BEGIN
  if (!in || !out || batch < 1 || batch > net->maxB)
    return ufail(net, SGN_EINVAL, "sgn_unet_infer: bad input, output or batch");
  infer_impl(net, in, out, batch);
  return SGN_OK;
  UAPI_END
}

sgn_status sgn_unet_check(sgn_unet_t net) {
  UAPI_BEGIN
  int h = 0;
  UCK(cudaMemcpyAsync(&h, net->dev_err, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
  UCK(cudaStreamSynchronize(net->stream));
  if (h != 0) {
    UCK(cudaMemsetAsync(net->dev_err, 0, sizeof(int), net->stream));
    return ufail(net, SGN_ECUDA, "sgn_unet_infer: a tensor-core wait ran out (the outputs are not valid)");
  }
  return SGN_OK;
  UAPI_END
}

}  // extern "C"

namespace {

// one tensor-core layer; stall: the self-test's barrier that never completes
sgn_status conv3_tc_run(int batch, int H, int W, const void* src0, int C0, int up0, const void* src1, int C1,
                        const float* weight, const float* bias, int Co, void* out, void* workspace,
                        size_t workspace_bytes, void* stream, int stall) {
  auto pow2 = [](int v) { return v >= 2 && (v & (v - 1)) == 0; };
  const int Ci = C0 + C1;
  if (batch < 1 || !pow2(H) || !pow2(W) || (long long)batch * H * W > (1ll << 30)) return SGN_EINVAL;
  if (up0 && (H < 4 || W < 4)) return SGN_EINVAL;
  if (!src0 || !weight || !bias || !out || !workspace || C0 < 16 || C0 % 16 || C1 < 0 || C1 % 16 ||
      (C1 > 0 && !src1) || Ci > 1024 || Co < 16 || Co > 256 || Co % 16)
    return SGN_EINVAL;
  const size_t img = (size_t)9 * Ci * Co * sizeof(__nv_bfloat16);
  if (workspace_bytes < sgn_conv3_workspace_bytes(C0 + C1, Co) || ((uintptr_t)workspace & 15u)) return SGN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int lH = 0, lW = 0;
  while ((1 << lH) < H) ++lH;
  while ((1 << lW) < W) ++lW;
  const bool row = H * W >= unet_tc::kM;
  const int KC = row ? pick_kc_row(Ci, Co, W, (long long)batch * H * W / unet_tc::kM) : pick_kc(Ci, Co);
  __nv_bfloat16* wimg = (__nv_bfloat16*)workspace;
  int* err = (int*)((char*)workspace + ((img + 15) & ~(size_t)15));
  unet_tc::WImgTable t{};
  t.nl = 1;
  t.l[0].woff = 0;
  t.l[0].ioff = 0;
  t.l[0].Ci = Ci;
  t.l[0].Co = Co;
  t.l[0].KC = KC;
  t.l[0].nkb = Ci / KC;
  t.l[0].kb_major = row ? 1 : 0;
  t.total = 9ll * Ci * Co;
  int cols = 32;
  while (cols < Co) cols <<= 1;
  int sm = row ? (int)unet_tc::row_smem_bytes(Co, KC, Ci / KC, W)
               : unet_tc::kStages * (int)unet_tc::stage_bytes(Co, KC);
  const int floor_bytes = 233472 / (512 / cols + 1) + 1;
  if (sm < floor_bytes) sm = floor_bytes;
  unet_tc::ConvArgs a{};
  a.src0 = (const __nv_bfloat16*)src0;
  a.src1 = (const __nv_bfloat16*)src1;
  a.C0 = C0;
  a.C1 = C1;
  a.up0 = up0 ? 1 : 0;
  a.lH = lH;
  a.lW = lW;
  a.npix = batch * H * W;
  a.wimg = wimg;
  a.bias = bias;
  a.Co = Co;
  a.KC = KC;
  a.nkb = Ci / KC;
  a.tmem_cols = (uint32_t)cols;
  a.out = (__nv_bfloat16*)out;
  a.err = err;
  a.stall = stall;
  if (cudaFuncSetAttribute(row ? (const void*)unet_tc::k_conv3_tc_row : (const void*)unet_tc::k_conv3_tc,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return SGN_ECUDA;
  unet_tc::k_wimg<<<(unsigned)((t.total + 255) / 256), 256, 0, st>>>(t, weight, wimg);
  const unsigned grid = (unsigned)((a.npix + unet_tc::kM - 1) / unet_tc::kM);
  if (row)
    unet_tc::k_conv3_tc_row<<<grid, unet_tc::kThreads, sm, st>>>(a);
  else
    unet_tc::k_conv3_tc<<<grid, unet_tc::kThreads, sm, st>>>(a);
  int h = 0;
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                                              cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || h != 0)
    return SGN_ECUDA;
  return SGN_OK;
}

}  // namespace

extern "C" {

sgn_status sgn_conv3_relu_bf16(int batch, int H, int W, const void* src0, int C0, int up0, const void* src1, int C1,
                               const float* weight, const float* bias, int Co, void* out, void* workspace,
                               size_t workspace_bytes, void* stream) {
  return conv3_tc_run(batch, H, W, src0, C0, up0, src1, C1, weight, bias, Co, out, workspace, workspace_bytes,
                      stream, 0);
}

sgn_status sgn_conv3_wait_selftest(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int C = 16, Co = 16;
  const int shapes[2][2] = {{8, 8}, {4, 128}};  // the gather kernel (64 pixels), the row kernel
  const size_t ws = sgn_conv3_workspace_bytes(C, Co);
  void *src = nullptr, *out = nullptr, *wk = nullptr;
  float *w = nullptr, *bias = nullptr;
  const size_t npix = 4 * 128;
  bool ok = cudaMalloc(&src, npix * C * 2) == cudaSuccess && cudaMalloc(&out, npix * Co * 2) == cudaSuccess &&
            cudaMalloc(&wk, ws) == cudaSuccess && cudaMalloc((void**)&w, sizeof(float) * Co * C * 9) == cudaSuccess &&
            cudaMalloc((void**)&bias, sizeof(float) * Co) == cudaSuccess;
  if (ok)
    ok = cudaMemsetAsync(src, 0, npix * C * 2, st) == cudaSuccess &&
         cudaMemsetAsync(w, 0, sizeof(float) * Co * C * 9, st) == cudaSuccess &&
         cudaMemsetAsync(bias, 0, sizeof(float) * Co, st) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) {
    const int H = shapes[k][0], W = shapes[k][1];
    // the stalled launch must report its run-out wait, and the context must
    // still run the same layer normally afterwards
    ok = conv3_tc_run(1, H, W, src, C, 0, nullptr, 0, w, bias, Co, out, wk, ws, stream, 1) == SGN_ECUDA &&
         cudaGetLastError() == cudaSuccess &&
         conv3_tc_run(1, H, W, src, C, 0, nullptr, 0, w, bias, Co, out, wk, ws, stream, 0) == SGN_OK;
  }
  cudaStreamSynchronize(st);
  cudaFree(src);
  cudaFree(out);
  cudaFree(wk);
  cudaFree(w);
  cudaFree(bias);
  return ok ? SGN_OK : SGN_ECUDA;
}

size_t sgn_conv3_workspace_bytes(int Ci, int Co) {
  if (Ci < 1 || Co < 1) return 0;
  return (((size_t)9 * Ci * Co * sizeof(__nv_bfloat16) + 15) & ~(size_t)15) + 16;
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
