// sgn_unet_tc.cuh - the U-Net's BF16 inference forward on the 5th-generation
// tensor cores (tcgen05), as implicit GEMMs over NHWC activations.
//
// A periodic 3x3 convolution of an NHWC tensor is, per output tile of 128
// pixels, the GEMM D[128][Co] = sum over the nine taps t of
// A_t[128][Ci] B_t[Ci][Co], where row m of A_t holds the Ci channels of the
// input pixel at (y + ty - 1, x + tx - 1) (wrapped) and B_t the weights of tap
// t. One CTA of 128 threads computes one tile:
//   * the accumulator D lives in tensor memory (TMEM lane m = pixel m, one
//     32-bit column per output channel), allocated by warp 0;
//   * the K loop runs over (tap, channel block) steps through three
//     shared-memory stages: the weights of a step arrive by one bulk copy
//     (cp.async.bulk, the copy engine) from a pre-arranged BF16 image, issued
//     one step ahead; the 128 gathered input rows are written by the threads
//     themselves (each thread one pixel, its loads issued one step ahead;
//     wrap-around, nearest upsampling and the channel concatenation of the
//     decoder are folded into this gather);
//   * one thread issues the step's tcgen05.mma instructions (M = 128,
//     N = Co, K = 16 each) and commits them to the stage's mbarrier, which
//     frees the stage for the step three later;
//   * the epilogue reads D back with tcgen05.ld (each warp its 32 lanes),
//     adds the bias, applies the ReLU, rounds to BF16 and stores the NHWC row;
//     for the last layer it also applies the 1x1 output convolution.
// Operands are K-major without swizzling: 8 x 16-byte core matrices, the
// core matrices of one 8-row group along K LBO bytes apart and consecutive
// 8-row groups SBO bytes apart.
//
// Every wait is bounded: a wait that runs out records SGN_TC_WAIT in the
// error word, the CTA waits (bounded again) for what it still has in flight,
// frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace unet_tc {

constexpr int kM = 128;           // output pixels per CTA = TMEM lanes
constexpr int kThreads = 128;     // one thread per pixel row
constexpr int kStageMax = 56 * 1024;
constexpr int kMaxKC = 128;       // channels per K step at most (the gather's registers)
constexpr int kStages = 3;        // shared-memory stages of the K loop
constexpr int SGN_TC_WAIT = 1;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, the
// leading (K-direction) and stride (M/N-direction) byte offsets, all in
// 16-byte units, and the descriptor version 1 at bits 46-48.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major, N / 8 at bits 17-22,
// M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// about a second at most: try_wait suspends the thread between polls
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it)
    if (bar_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b,
                                         unsigned extra_tx = 0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes + extra_tx)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(b))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One convolution launch. The input channels are the concatenation of src0
// (C0 channels, read at (y >> 1, x >> 1) of an H/2 x W/2 grid when up0) and
// src1 (C1 channels, may be 0), both NHWC BF16 with their channel counts as
// row lengths.
struct ConvArgs {
  const __nv_bfloat16* src0;
  const __nv_bfloat16* src1;
  int C0, C1, up0;
  int lH, lW;   // log2 of the output grid (= src1's grid)
  int npix;     // B H W output pixels
  const __nv_bfloat16* wimg;  // [9 * nkb][KC / 8][Co / 8][8][8] BF16 (core-matrix image of each step)
  const float* bias;          // [Co]
  int Co, KC, nkb;
  uint32_t tmem_cols;         // power of two >= max(32, Co)
  __nv_bfloat16* out;         // NHWC [npix][Co], or null with a head
  const float* head_w;        // optional 1x1 head Co -> 1: weights [Co], bias [1]
  const float* head_b;
  float* head_out;            // [npix] FP32
  int* err;
  int stall;                  // self-test only: arm step 0's weight barrier for 16 bytes more
                              // than its copy delivers, so that its waits run out
};

// bytes of one K step's operands in shared memory (A rows, then B)
__host__ __device__ constexpr uint32_t a_bytes(int KC) { return (uint32_t)kM * KC * 2u; }
__host__ __device__ constexpr uint32_t b_bytes(int Co, int KC) { return (uint32_t)Co * KC * 2u; }
__host__ __device__ constexpr uint32_t stage_bytes(int Co, int KC) { return a_bytes(KC) + b_bytes(Co, KC); }

// The epilogue of both kernels, after the last MMA completed: this thread's
// TMEM lane (its pixel) read back 16 columns at a time, bias, ReLU, BF16
// store of the NHWC row; with a head, the 1x1 output convolution of the BF16
// values in FP32. Every thread of the CTA calls it (tcgen05.ld is warp-wide);
// valid: whether the pixel exists (a ragged last tile).
__device__ __forceinline__ void tc_epilogue(const ConvArgs& p, uint32_t tmem, int warp, int pix, bool valid) {
  tc_fence_after();
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  float head = 0.f;
  for (int q = 0; q < p.Co / 16; ++q) {
    float v[16];
    tmem_ld16(lane_addr + (uint32_t)(q * 16), v);
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float a = fmaxf(v[i] + __ldg(p.bias + q * 16 + i), 0.f);
      o[i] = __float2bfloat16_rn(a);
      if (p.head_w) head = fmaf(__ldg(p.head_w + q * 16 + i), __bfloat162float(o[i]), head);
    }
    if (valid && p.out) {
      uint4* dst = reinterpret_cast<uint4*>(p.out + (size_t)pix * p.Co + q * 16);
      dst[0] = reinterpret_cast<const uint4*>(o)[0];
      dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
  }
  if (valid && p.head_w) p.head_out[pix] = head + __ldg(p.head_b);
}

__global__ void __launch_bounds__(kThreads) k_conv3_tc(ConvArgs p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_w[kStages], bar_mma[kStages];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KC = p.KC, Co = p.Co;
  const uint32_t abytes = a_bytes(KC), sbytes = stage_bytes(Co, KC);
  const uint32_t sm0 = smem_addr(sm);

  if (warp == 0) tmem_alloc(&tmem_slot, p.tmem_cols);
  if (tid == 32) {
    for (int i = 0; i < kStages; ++i) {
      bar_init(&bar_w[i], 1);
      bar_init(&bar_mma[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // this thread's pixel: row m = tid of the tile
  const int pix = blockIdx.x * kM + tid;
  const bool valid = pix < p.npix;
  const int W = 1 << p.lW, H = 1 << p.lH;
  const int x = pix & (W - 1), y = (pix >> p.lW) & (H - 1), b = pix >> (p.lW + p.lH);
  const uint32_t idesc = instr_desc_bf16(kM, Co);
  const int nsteps = 9 * p.nkb;

  // this thread's gathered row of one K step: KC / 8 16-byte chunks, loaded
  // one step ahead so that the loads of step s + 1 are in flight while the
  // MMAs of step s are issued and the next buffer is waited for
  uint4 row[kMaxKC / 8];
  auto gather = [&](int step) {
    const int tap = step / p.nkb, kb = step - tap * p.nkb;
    const int yy = (y + tap / 3 - 1) & (H - 1), xx = (x + tap % 3 - 1) & (W - 1);
    const uint4* r0 = reinterpret_cast<const uint4*>(
        p.up0 ? p.src0 + ((((size_t)b << (p.lH + p.lW - 2)) + ((size_t)(yy >> 1) << (p.lW - 1)) + (xx >> 1)) * p.C0)
              : p.src0 + ((((size_t)b << (p.lH + p.lW)) + ((size_t)yy << p.lW) + xx) * p.C0));
    const uint4* r1 = p.src1 ? reinterpret_cast<const uint4*>(
                                   p.src1 + ((((size_t)b << (p.lH + p.lW)) + ((size_t)yy << p.lW) + xx) * p.C1))
                             : r0;
#pragma unroll
    for (int c = 0; c < kMaxKC / 8; ++c) {
      const int ch = kb * KC + 8 * c;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (valid && c < KC / 8) v = ch < p.C0 ? __ldg(r0 + (ch >> 3)) : __ldg(r1 + ((ch - p.C0) >> 3));
      row[c] = v;
    }
  };

  bool ok = true;
  int issued = -1;     // last step whose MMAs were committed (thread 0)
  int copied = -1;     // last step whose weight copy was issued (thread 0)
  int copy_done = -1;  // last step whose weight copy was seen complete (thread 0)
  // step s uses stage s % kStages; its k-th use is phase k of the stage's barriers
  auto stage_of = [](int st) { return st % kStages; };
  auto parity_of = [](int st) { return (unsigned)((st / kStages) & 1); };
  if (tid == 0) {
    bulk_g2s(sm + abytes, p.wimg, b_bytes(Co, KC), &bar_w[0], p.stall ? 16u : 0u);
    copied = 0;
  }
  gather(0);
  for (int s = 0; s < nsteps; ++s) {
    const int buf = stage_of(s);
    // the MMAs of step s - 2 (and so of every earlier step) are done: stage
    // (s + 1) % 3 - last used by step s - 2 - takes step s + 1's weights,
    // stage s % 3 - last used by step s - 3 - step s's rows
    if (s >= 2 && !bar_wait(&bar_mma[stage_of(s - 2)], parity_of(s - 2))) ok = false;
    if (__syncthreads_or(ok ? 0 : 1)) {
      ok = false;
      break;
    }
    unsigned char* A = sm + buf * sbytes;
    if (tid == 0 && s + 1 < nsteps) {
      bulk_g2s(sm + stage_of(s + 1) * sbytes + abytes, p.wimg + (size_t)(s + 1) * Co * KC, b_bytes(Co, KC),
               &bar_w[stage_of(s + 1)]);
      copied = s + 1;
    }
    // A row m = the KC channels [kb KC, (kb + 1) KC) of the tap's pixel
    unsigned char* arow = A + (tid >> 3) * 128 + (tid & 7) * 16;
#pragma unroll
    for (int c = 0; c < kMaxKC / 8; ++c)
      if (c < KC / 8) *reinterpret_cast<uint4*>(arow + (size_t)c * (kM / 8) * 128) = row[c];
    if (s + 1 < nsteps) gather(s + 1);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (!bar_wait(&bar_w[buf], parity_of(s))) {
        ok = false;
      } else {
        copy_done = s;
        tc_fence_after();
        const uint32_t a0 = sm0 + buf * sbytes, b0 = a0 + abytes;
#pragma unroll 1
        for (int j = 0; j < KC / 16; ++j) {
          const uint64_t ad = smem_desc(a0 + (uint32_t)j * 2u * (kM / 8) * 128u, (kM / 8) * 128u, 128u);
          const uint64_t bd = smem_desc(b0 + (uint32_t)j * 2u * (uint32_t)(Co / 8) * 128u, (uint32_t)(Co / 8) * 128u,
                                        128u);
          mma_bf16(tmem, ad, bd, idesc, (s > 0 || j > 0) ? 1 : 0);
        }
        mma_commit(&bar_mma[buf]);
        issued = s;
      }
    }
  }
  if (ok) {
    const int last = nsteps - 1;
    if (!bar_wait(&bar_mma[stage_of(last)], parity_of(last))) ok = false;
  }
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (ok) {
    tc_epilogue(p, tmem, warp, pix, valid);
  } else if (tid == 0) {
    atomicOr(p.err, SGN_TC_WAIT);
    // let what this CTA still has in flight finish before its memory goes
    if (issued >= 0) bar_wait(&bar_mma[stage_of(issued)], parity_of(issued));
    for (int c = copy_done + 1; c <= copied; ++c) bar_wait(&bar_w[stage_of(c)], parity_of(c));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, p.tmem_cols);
}

}  // namespace unet_tc

namespace unet_tc {

// The first layer (4 FP32 NCHW input channels -> Co, ReLU) on CUDA cores: its
// K = 36 is too short for the tensor cores. One thread per pixel; weights
// [Co][4][3][3] and biases in shared memory; BF16 NHWC out, 8 channels per
// 16-byte store.
__global__ void __launch_bounds__(128) k_conv_in_nhwc(const float* __restrict__ x, int lH, int lW, int npix,
                                                      const float* __restrict__ w, const float* __restrict__ bias,
                                                      int Co, __nv_bfloat16* out) {
  extern __shared__ float ws[];  // Co * 36 weights, then Co biases
  for (int i = threadIdx.x; i < Co * 37; i += blockDim.x) ws[i] = i < Co * 36 ? w[i] : bias[i - Co * 36];
  __syncthreads();
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int W = 1 << lW, H = 1 << lH;
  const int xq = pix & (W - 1), yq = (pix >> lW) & (H - 1), b = pix >> (lH + lW);
  float in[36];
#pragma unroll
  for (int ci = 0; ci < 4; ++ci)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = (yq + t / 3 - 1) & (H - 1), xx = (xq + t % 3 - 1) & (W - 1);
      in[ci * 9 + t] = __ldg(x + (((size_t)(b * 4 + ci)) << (lH + lW)) + ((size_t)yy << lW) + xx);
    }
  for (int c8 = 0; c8 < Co / 8; ++c8) {
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float* wr = ws + (c8 * 8 + j) * 36;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 36; ++k) acc = fmaf(wr[k], in[k], acc);
      o[j] = __float2bfloat16_rn(fmaxf(acc + ws[Co * 36 + c8 * 8 + j], 0.f));
    }
    *reinterpret_cast<uint4*>(out + (size_t)pix * Co + c8 * 8) = *reinterpret_cast<const uint4*>(o);
  }
}

// 2x2 average pool of an NHWC BF16 tensor on a 2^lH x 2^lW grid (C channels,
// a multiple of 8): one thread per output pixel and 8-channel group, summed in
// FP32 as (a + b) + (c + d) over the rows 2y, 2y + 1.
__global__ void k_pool_nhwc(const __nv_bfloat16* __restrict__ in, int lH, int lW, int C, int nout,
                            __nv_bfloat16* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int groups = C >> 3;
  if (i >= nout * groups) return;
  const int g = i % groups, op = i / groups;
  const int W2 = 1 << (lW - 1), H2 = 1 << (lH - 1);
  const int ox = op & (W2 - 1), oy = (op >> (lW - 1)) & (H2 - 1), b = op >> (lH + lW - 2);
  const size_t base = ((((size_t)b << (lH + lW)) + ((size_t)(2 * oy) << lW) + 2 * ox) * C) + g * 8;
  const size_t row = (size_t)C << lW;
  __align__(16) __nv_bfloat16 v[4][8];
  *reinterpret_cast<uint4*>(v[0]) = __ldg(reinterpret_cast<const uint4*>(in + base));
  *reinterpret_cast<uint4*>(v[1]) = __ldg(reinterpret_cast<const uint4*>(in + base + C));
  *reinterpret_cast<uint4*>(v[2]) = __ldg(reinterpret_cast<const uint4*>(in + base + row));
  *reinterpret_cast<uint4*>(v[3]) = __ldg(reinterpret_cast<const uint4*>(in + base + row + C));
  __align__(16) __nv_bfloat16 o[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float s = (__bfloat162float(v[0][j]) + __bfloat162float(v[1][j])) +
                    (__bfloat162float(v[2][j]) + __bfloat162float(v[3][j]));
    o[j] = __float2bfloat16_rn(0.25f * s);
  }
  *reinterpret_cast<uint4*>(out + (size_t)op * C + g * 8) = *reinterpret_cast<const uint4*>(o);
}

// BF16 core-matrix images of the 3x3 layers' FP32 weights [Co][Ci][3][3]:
// for step s = tap nkb + kb (kb 9 + tap with kb_major), element (co, k)
// (input channel kb KC + k) at s Co KC + ((k / 8) (Co / 8) + co / 8) 64 +
// (co % 8) 8 + k % 8.
constexpr int kMaxImgLayers = 16;
struct WImgLayer {
  long long woff, ioff;  // FP32 weight offset in the parameters, element offset in the image
  int Ci, Co, KC, nkb;
  int kb_major;          // step order kb 9 + tap (the row kernel) instead of tap nkb + kb
};
struct WImgTable {
  int nl;
  WImgLayer l[kMaxImgLayers];
  long long total;
};

__global__ void k_wimg(WImgTable t, const float* __restrict__ params, __nv_bfloat16* img) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.total) return;
  int li = 0;
  while (li + 1 < t.nl && i >= t.l[li + 1].ioff) ++li;
  const WImgLayer L = t.l[li];
  const long long r = i - L.ioff;
  const int blk = L.Co * L.KC;
  const int step = (int)(r / blk), e = (int)(r % blk);
  const int cg = L.Co >> 3;
  const int c = e / (cg * 64), rem = e % (cg * 64);
  const int co = (rem / 64) * 8 + (rem % 64) / 8, k = c * 8 + (rem & 7);
  const int tap = L.kb_major ? step % 9 : step / L.nkb, kb = L.kb_major ? step / 9 : step % L.nkb;
  const int ci = kb * L.KC + k;
  img[i] = __float2bfloat16_rn(params[L.woff + ((long long)co * L.Ci + ci) * 9 + tap]);
}

}  // namespace unet_tc

namespace unet_tc {

// Grids whose rows hold at least 128 pixels: a tile is 128 consecutive pixels
// of one row, and the input it needs - rows y-1..y+1, columns x0-1..x0+128
// (wrapped) - is staged once per channel block into shared memory as a halo
// [KC/8 chunks][3 x 130 positions][8 channels]. The A operand of tap (dy, dx)
// is then that buffer itself: its 128 rows are the 128 consecutive positions
// from (dy + 1) 130 + dx + 1 on, 16 bytes apart, i.e. a descriptor with
// SBO = 128 and LBO = the chunk stride, started at that offset. The nine
// taps' weights of a channel block arrive by one bulk copy (the image is in
// channel-block-major order for these layers); halo and weights are
// double-buffered across channel blocks, the next block's loaded while the
// current block's MMAs run, and one thread issues a block's 9 KC/16 MMAs back
// to back with one commit.
//
// Rows of fewer than 128 pixels (W < 128, at least 128 pixels per image): a
// tile is the 128 / W whole rows y0.. of one image, and the halo holds three
// copies of rows y0-1 .. y0+128/W, copy kx shifted by kx - 1 columns (wrapped)
// and stored with row stride exactly W. Output pixel m of the tile then reads
// tap (ky, kx) at position m + ky W of copy kx: again 128 consecutive 16-byte
// positions, one descriptor per tap.
constexpr int kHaloPos = 3 * (kM + 2);
// positions per chunk of one halo copy, and the copies
__host__ __device__ constexpr int halo_pos(int W) { return W >= kM ? kHaloPos : kM + 2 * W; }
__host__ __device__ constexpr int halo_copies(int W) { return W >= kM ? 1 : 3; }
__host__ __device__ constexpr uint32_t halo_bytes(int KC, int W) {
  return (uint32_t)halo_copies(W) * halo_pos(W) * KC * 2u;
}
// one buffer of halo + weights per channel block in flight (two when there
// are several blocks)
__host__ __device__ constexpr uint32_t row_smem_bytes(int Co, int KC, int nkb, int W) {
  return (nkb > 1 ? 2u : 1u) * (halo_bytes(KC, W) + 9u * b_bytes(Co, KC));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(kThreads) k_conv3_tc_row(ConvArgs p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_w[2], bar_mma[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KC = p.KC, Co = p.Co, nkb = p.nkb;
  const int W = 1 << p.lW, H = 1 << p.lH;
  const bool wide = W >= kM;
  const int P = halo_pos(W);  // positions of one chunk of one halo copy
  const uint32_t hbytes = halo_bytes(KC, W), wbytes = 9u * b_bytes(Co, KC), bufbytes = hbytes + wbytes;
  const uint32_t sm0 = smem_addr(sm);

  if (warp == 0) tmem_alloc(&tmem_slot, p.tmem_cols);
  if (tid == 32) {
    for (int i = 0; i < 2; ++i) {
      bar_init(&bar_w[i], 1);
      bar_init(&bar_mma[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const int tile = blockIdx.x;
  int x0, y, b;  // wide: the tile's row y and first column x0; narrow: its first row y
  if (wide) {
    const int tiles_row = W >> 7;
    x0 = (tile % tiles_row) << 7;
    y = (tile / tiles_row) & (H - 1);
    b = tile / (tiles_row << p.lH);
  } else {
    const int rows = kM >> p.lW, tiles_img = H / rows;
    x0 = 0;
    y = (tile % tiles_img) * rows;
    b = tile / tiles_img;
  }
  const int pix = tile * kM + tid;
  const uint32_t idesc = instr_desc_bf16(kM, Co);

  // channel block kb's halo (cp.async, piece i = (position, chunk), chunk
  // fastest) and its nine taps' weights (one bulk copy, thread 0) into buffer bf
  auto load_block = [&](int kb, int bf) {
    unsigned char* dst = sm + (size_t)bf * bufbytes;
    if (tid == 0)
      bulk_g2s(dst + hbytes, p.wimg + (size_t)kb * 9 * Co * KC, wbytes, &bar_w[bf], (p.stall && kb == 0) ? 16u : 0u);
    const int chunks = KC >> 3, pieces = halo_copies(W) * P * chunks;
    for (int i = tid; i < pieces; i += kThreads) {
      const int kx = i / (P * chunks), rem = i - kx * P * chunks;
      const int pos = rem / chunks, c = rem - pos * chunks;
      int gy, gx;
      if (wide) {
        const int r = pos / (kM + 2), col = pos - r * (kM + 2);
        gy = (y + r - 1) & (H - 1);
        gx = (x0 + col - 1) & (W - 1);
      } else {
        const int r = pos >> p.lW, xx = pos & (W - 1);
        gy = (y + r - 1) & (H - 1);
        gx = (xx + kx - 1) & (W - 1);
      }
      const int ch = kb * KC + 8 * c;
      const __nv_bfloat16* src;
      if (ch < p.C0) {
        src = p.up0 ? p.src0 + ((((size_t)b << (p.lH + p.lW - 2)) + ((size_t)(gy >> 1) << (p.lW - 1)) + (gx >> 1)) *
                                    p.C0 + ch)
                    : p.src0 + ((((size_t)b << (p.lH + p.lW)) + ((size_t)gy << p.lW) + gx) * p.C0 + ch);
      } else {
        src = p.src1 + ((((size_t)b << (p.lH + p.lW)) + ((size_t)gy << p.lW) + gx) * p.C1 + (ch - p.C0));
      }
      cp_async16(dst + ((size_t)(kx * chunks + c) * P + pos) * 16, src);
    }
  };
  // block kb uses buffer kb & 1; its k-th use is phase k of that buffer's barriers
  auto parity_of = [](int kb) { return (unsigned)((kb >> 1) & 1); };

  // A parity wait tells a phase only from the one before it, so every wait
  // on an mbarrier here is made by thread 0, which sees every commit and every
  // copy in order; the other threads learn the outcome through the block votes.
  bool ok = true;
  int issued = -1, mma_seen = -1, copied = 0, copy_done = -1;
  load_block(0, 0);
  cp_async_commit();
  for (int kb = 0; kb < nkb; ++kb) {
    const int bf = kb & 1;
    const bool pre = kb + 1 < nkb;
    // buffer bf ^ 1 was block kb - 1's: its MMAs must be done
    if (tid == 0 && pre && kb >= 1) {
      if (bar_wait(&bar_mma[(kb - 1) & 1], parity_of(kb - 1)))
        mma_seen = kb - 1;
      else
        ok = false;
    }
    if (__syncthreads_or(ok ? 0 : 1)) {
      ok = false;
      break;
    }
    if (pre) {
      load_block(kb + 1, bf ^ 1);
      if (tid == 0) copied = kb + 1;
    }
    cp_async_commit();
    cp_async_wait1();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (!bar_wait(&bar_w[bf], parity_of(kb))) {
        ok = false;
      } else {
        copy_done = kb;
        tc_fence_after();
        const uint32_t hbase = sm0 + (uint32_t)bf * bufbytes, wbase = hbase + hbytes;
        const uint32_t cstride = (uint32_t)P * 16u;  // bytes between chunks of a copy (LBO)
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap % 3;
          const uint32_t a0 =
              hbase + (wide ? (uint32_t)((ky * (kM + 2) + kx) * 16)
                            : (uint32_t)kx * (uint32_t)(KC >> 3) * cstride + (uint32_t)(ky * W * 16));
          const uint32_t b0 = wbase + (uint32_t)tap * b_bytes(Co, KC);
#pragma unroll 1
          for (int j = 0; j < KC / 16; ++j) {
            const uint64_t ad = smem_desc(a0 + (uint32_t)j * 2u * cstride, cstride, 128u);
            const uint64_t bd = smem_desc(b0 + (uint32_t)j * 2u * (uint32_t)(Co / 8) * 128u,
                                          (uint32_t)(Co / 8) * 128u, 128u);
            mma_bf16(tmem, ad, bd, idesc, (kb > 0 || tap > 0 || j > 0) ? 1 : 0);
          }
        }
        mma_commit(&bar_mma[bf]);
        issued = kb;
      }
    }
  }
  // the last block's commit (the one before it was seen before its buffer was refilled)
  if (ok && tid == 0) {
    if (bar_wait(&bar_mma[(nkb - 1) & 1], parity_of(nkb - 1)))
      mma_seen = nkb - 1;
    else
      ok = false;
  }
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (ok) {
    tc_epilogue(p, tmem, warp, pix, true);
  } else if (tid == 0) {
    atomicOr(p.err, SGN_TC_WAIT);
    // drain in order what this CTA still has in flight
    for (int k = mma_seen + 1; k <= issued; ++k)
      if (!bar_wait(&bar_mma[k & 1], parity_of(k))) break;
    for (int k = copy_done + 1; k <= copied; ++k) bar_wait(&bar_w[k & 1], parity_of(k));
  }
  cp_async_wait0();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, p.tmem_cols);
}

}  // namespace unet_tc
