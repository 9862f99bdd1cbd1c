// fft_core.cuh - shared-memory Stockham FFT building blocks for sm_103a.
//
// The spectral method of Section 3 needs many 1D transforms of power-of-two
// length N (8..4096) along x (rows) and y (columns). One transform is done by
// a group of T = N/8 threads. Thread t of the group keeps the elements
// t + s*T (s = 0..7) in registers, both before and after the transform
// ("thread-strided natural order"), so the last stage of an inverse transform
// hands its outputs straight to the first stage of a forward transform.
//
// Stages are radix-8 (Stockham autosort), with one radix-2 or radix-4 stage
// when log2 N is not a multiple of 3: last in plan 0, first in plan 1 (where
// it needs no twiddles and every radix-8 stage does); sgn_autotune picks the
// plan per pass. In a stage of radix Rs < 8 a thread
// runs 8/Rs butterflies; butterfly q of thread t has index j = t + q*T and its
// inputs j + r*N/Rs are exactly the thread's slots q + r*(8/Rs), so every stage
// reads the same thread-strided slots. Between stages data goes through shared
// memory at an index that keeps every stage bank-conflict free: FP64 (16-byte
// elements) pads, p + (p >> 3); FP32 (8-byte elements) XOR-swizzles within
// aligned groups of 16 elements (one transform per buffer) or 8 elements
// (several interleaved columns), see sidx().
//
// Twiddles W_N^k = exp(-2 pi i k / N) come from a table in global memory
// (L1-resident) laid out by stage: the stage of sub-transform length
// Ns = 2^lNs and radix R reads its R - 1 twiddle rows W_{R Ns}^{jm r}
// (r = 1..R-1, jm = 0..Ns-1) at offset 2^lNs - 8 of the table, row r - 1
// holding jm = 0..Ns-1 contiguously. The threads of a warp take consecutive jm,
// so one twiddle load touches one or two cache lines instead of up to one line
// per thread (the W_N^{jm r} entries of a flat table lie 2^(lN-lNs-3) r
// entries apart). staged_exponent() gives the k of each entry. A table holds
// plan 0's rows in entries [0, N) and plan 1's in [N, 2N) (in plan 1 the stage
// of lNs starts at N + 2^lNs - 2^rem, rem = lN mod 3). The inverse transform
// uses the conjugates. No transform scales its output.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgn {

template <typename T>
struct __align__(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ cpx<T> scl(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by +i / -i
template <typename T>
__device__ __forceinline__ cpx<T> mul_i(cpx<T> a) { return mk(-a.y, a.x); }
template <typename T>
__device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) { return mk(a.y, -a.x); }
// multiply by (i*k) for a real k
template <typename T>
__device__ __forceinline__ cpx<T> mul_ik(cpx<T> a, T k) { return mk(-a.y * k, a.x * k); }

template <typename T>
__device__ __forceinline__ cpx<T> ldg(const cpx<T>* p);
template <>
__device__ __forceinline__ cpx<double> ldg(const cpx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ cpx<float> ldg(const cpx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}

// read-only scalar load (wavenumbers, M^-1); the double-float type overloads it
template <typename T>
__device__ __forceinline__ T ldr(const T* p) {
  return __ldg(p);
}

// Shared-memory slot of element p of a transform whose buffer interleaves
// 2^lcs columns. 16-byte elements: a quarter-warp phase touches 8 elements, and
// one pad slot every 8 keeps the stride-8 writes of the first stage, the
// 64a + b writes of the second and consecutive reads on distinct banks. 8-byte
// elements: a half-warp phase touches 16; within each aligned group of 16 the
// slot is XOR-ed with (g & 7) | (bit 2 of g) << 3, g = p >> 4, which separates
// the stride-8 writes (low three bits cycle over 8 groups) and the 64a + b
// writes (bit 3 flips between groups g and g + 4). With 2 or more interleaved
// columns only p mod 8 selects the bank pair, so the XOR uses (p >> 3) & 7.
template <typename T>
__device__ __forceinline__ int sidx(int p, int lcs);
template <>
__device__ __forceinline__ int sidx<double>(int p, int lcs) {
  return (p + (p >> 3)) << lcs;
}
template <>
__device__ __forceinline__ int sidx<float>(int p, int lcs) {
  if (lcs == 0) {
    const int g = p >> 4;
    return p ^ ((g & 7) | (((g >> 2) & 1) << 3));
  }
  return (p ^ ((p >> 3) & 7)) << lcs;
}
// shared-memory elements needed by one transform of length N (either layout)
__host__ __device__ constexpr int smem_elems(int N) { return N + (N >> 3); }
// element types whose exchange buffers need no padding (their sidx swizzles
// within aligned groups instead): the double-float passes, see dfloat.cuh
template <typename T>
struct unpadded_smem {
  static constexpr bool value = false;
};
template <typename T>
__host__ __device__ constexpr int smem_elems_of(int N) {
  return unpadded_smem<T>::value ? N : smem_elems(N);
}

// Exponent k of entry i of the staged twiddle table of a length-2^lN
// transform (the entry is W_N^k), or -1 past the last stage's rows. The
// radix-8 stages have lNs = 3, 6, ..., then one radix-2 or radix-4 stage when
// 3 does not divide lN (the stage plan of fft_regs); the stage of lNs starts at
// 2^lNs - 8 and holds (R - 1) rows of 2^lNs entries. Fewer than N entries in all.
__host__ __device__ inline int staged_exponent(int i, int lN, int plan = 0) {
  const int n8 = lN / 3, rem = lN - 3 * n8;
  if (plan && rem) {
    // plan 1: the radix-2^rem stage first (no twiddles), then radix-8 stages
    // at lNs = rem, rem + 3, ..., lN - 3, the stage of lNs at 2^lNs - 2^rem
    for (int lNs = rem; lNs <= lN - 3; lNs += 3) {
      const int Ns = 1 << lNs, off = Ns - (1 << rem);
      if (i < off) return -1;
      if (i < off + 7 * Ns) {
        const int q = i - off;
        return ((q & (Ns - 1)) * (q / Ns + 1)) << (lN - lNs - 3);
      }
    }
    return -1;
  }
  for (int lNs = 3;; lNs += 3) {
    const bool tail = lNs == 3 * n8;  // the radix-2 or radix-4 stage, if any
    if (lNs > 3 * n8 || (tail && rem == 0)) return -1;
    const int lr = tail ? rem : 3;
    const int Ns = 1 << lNs, off = Ns - 8;
    if (i < off) return -1;
    if (i < off + ((1 << lr) - 1) * Ns) {
      const int q = i - off;
      return ((q & (Ns - 1)) * (q / Ns + 1)) << (lN - lNs - lr);
    }
  }
}

// ---------------------------------------------------------------- butterflies
// Forward transforms use W = exp(-2 pi i / n); INV uses exp(+2 pi i / n).

template <bool INV, typename T>
__device__ __forceinline__ cpx<T> rot_quarter(cpx<T> a) {  // times W_4
  return INV ? mul_i(a) : mul_mi(a);
}

template <bool INV, typename T>
__device__ __forceinline__ void bfly2(cpx<T>& a, cpx<T>& b) {
  cpx<T> t = a - b;
  a = a + b;
  b = t;
}

// 4-point DFT in place: X[m] = sum_n x[n] W4^{nm}
template <bool INV, typename T>
__device__ __forceinline__ void bfly4(cpx<T>& x0, cpx<T>& x1, cpx<T>& x2, cpx<T>& x3) {
  cpx<T> t0 = x0 + x2, t1 = x0 - x2;
  cpx<T> t2 = x1 + x3, t3 = rot_quarter<INV>(x1 - x3);
  x0 = t0 + t2;
  x2 = t0 - t2;
  x1 = t1 + t3;
  x3 = t1 - t3;
}

// 8-point DFT in place, decimation in frequency: the even outputs are the
// 4-point DFT of x[n] + x[n+4], the odd outputs that of (x[n] - x[n+4]) W8^n.
template <bool INV, typename T>
__device__ __forceinline__ void bfly8(cpx<T>* x) {
  const T h = (T)0.70710678118654752440084436210484903928;
  cpx<T> a0 = x[0] + x[4], a1 = x[1] + x[5], a2 = x[2] + x[6], a3 = x[3] + x[7];
  cpx<T> b0 = x[0] - x[4], b1 = x[1] - x[5], b2 = x[2] - x[6], b3 = x[3] - x[7];
  if (!INV) {
    b1 = mk((b1.x + b1.y) * h, (b1.y - b1.x) * h);    // (1 - i)/sqrt2
    b2 = mul_mi(b2);                                   // -i
    b3 = mk((b3.y - b3.x) * h, -(b3.x + b3.y) * h);   // (-1 - i)/sqrt2
  } else {
    b1 = mk((b1.x - b1.y) * h, (b1.x + b1.y) * h);    // (1 + i)/sqrt2
    b2 = mul_i(b2);                                    // +i
    b3 = mk(-(b3.x + b3.y) * h, (b3.x - b3.y) * h);   // (-1 + i)/sqrt2
  }
  bfly4<INV>(a0, a1, a2, a3);
  bfly4<INV>(b0, b1, b2, b3);
  x[0] = a0; x[2] = a1; x[4] = a2; x[6] = a3;
  x[1] = b0; x[3] = b1; x[5] = b2; x[7] = b3;
}

// ---------------------------------------------------------------- one stage
// Radix-RS stage of a length-N Stockham FFT, sub-transform length Ns = 2^lNs.
// v: the thread's 8 slots (inputs). If LAST, outputs return in v (same slot
// map); otherwise they go to sm at padded positions.
template <bool INV, int RS, bool LAST, typename T>
__device__ __forceinline__ void fft_stage(cpx<T> (&v)[8], cpx<T>* sm, const cpx<T>* __restrict__ tw,
                                          int t, int lN, int lNs, int lcs) {
  constexpr int LRS = (RS == 8) ? 3 : (RS == 4 ? 2 : 1);
  constexpr int NB = 8 / RS;
  const int T_ = 1 << (lN - 3);
  const int Ns = 1 << lNs;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = t + q * T_;
    const int jm = j & (Ns - 1);
    cpx<T> xs[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) xs[r] = v[q + r * NB];
    if (lNs > 0) {
      cpx<T> w[RS];
      // this stage's rows of the staged table: entry (r - 1) * Ns + jm is W^{jm r}
      const cpx<T>* tws = tw + (Ns - 8) + jm;
      if (sizeof(T) == 4 && RS >= 4) {
        // FP32: three table loads and products for the rest (the L1 pipe, not
        // the FMA pipe, limits the FP32 passes); FP64 loads all (FP64 products
        // cost more than loads on this part)
        w[1] = ldg(tws);
        w[2] = ldg(tws + Ns);
        w[3] = cmul(w[1], w[2]);
        if (RS == 8) {
          w[4] = ldg(tws + 3 * Ns);
          w[5] = cmul(w[1], w[4]);
          w[6] = cmul(w[2], w[4]);
          w[7] = cmul(w[3], w[4]);
        }
      } else {
#pragma unroll
        for (int r = 1; r < RS; ++r) w[r] = ldg(tws + (r - 1) * Ns);
      }
#pragma unroll
      for (int r = 1; r < RS; ++r) xs[r] = INV ? cmulc(xs[r], w[r]) : cmul(xs[r], w[r]);
    }
    if (RS == 8) bfly8<INV>(xs);
    if (RS == 4) bfly4<INV>(xs[0], xs[1], xs[2], xs[3]);
    if (RS == 2) bfly2<INV>(xs[0], xs[1]);
    if (LAST) {
#pragma unroll
      for (int r = 0; r < RS; ++r) v[q + r * NB] = xs[r];
    } else {
      const int base = ((j >> lNs) << (lNs + LRS)) + jm;
#pragma unroll
      for (int r = 0; r < RS; ++r) sm[sidx<T>(base + r * Ns, lcs)] = xs[r];
    }
  }
}

// Slot s of thread t is element t + s*T_; element p lives at sm[sidx(p, lcs)]
// (lcs = log2 of the interleave factor when several columns share a buffer).
template <typename T>
__device__ __forceinline__ void load_slots(cpx<T> (&v)[8], const cpx<T>* sm, int t, int T_, int lcs) {
#pragma unroll
  for (int s = 0; s < 8; ++s) v[s] = sm[sidx<T>(t + s * T_, lcs)];
}
template <typename T>
__device__ __forceinline__ void store_slots(const cpx<T> (&v)[8], cpx<T>* sm, int t, int T_, int lcs) {
#pragma unroll
  for (int s = 0; s < 8; ++s) sm[sidx<T>(t + s * T_, lcs)] = v[s];
}

// Full transform of length N = 2^lN (lN >= 3) held in v (thread-strided
// natural order in and out). sm: this transform's shared buffer of
// smem_elems(N) elements at stride 2^lcs. sm must be free on entry and is free
// again on exit. Contains __syncthreads(): every thread of the block must call
// it with the same lN (threads of idle groups work on valid dummy data).
// plan (0 or 1): where the radix-2 or radix-4 stage goes (see the top of
// the file); tw is the table of both plans.
template <bool INV, typename T>
__device__ __forceinline__ void fft_regs(cpx<T> (&v)[8], cpx<T>* sm, const cpx<T>* __restrict__ tw,
                                         int t, int lN, int lcs = 0, int plan = 0) {
  const int T_ = 1 << (lN - 3);
  const int n8 = lN / 3;        // radix-8 stages
  const int rem = lN - 3 * n8;  // 0, 1 or 2 -> extra stage of radix 1 (none), 2, 4
  if (plan && rem) {
    // plan 1's rows start at N; fft_stage reads stage lNs at (2^lNs - 8), so
    // shift the base by 8 - 2^rem
    const cpx<T>* tw1 = tw + (1 << lN) + 8 - (1 << rem);
    if (rem == 1)
      fft_stage<INV, 2, false>(v, sm, tw1, t, lN, 0, lcs);
    else
      fft_stage<INV, 4, false>(v, sm, tw1, t, lN, 0, lcs);
    __syncthreads();
    load_slots(v, sm, t, T_, lcs);
    __syncthreads();
    int lNs = rem;
    for (int st = 0; st < n8; ++st) {
      if (st == n8 - 1) {
        fft_stage<INV, 8, true>(v, sm, tw1, t, lN, lNs, lcs);
      } else {
        fft_stage<INV, 8, false>(v, sm, tw1, t, lN, lNs, lcs);
        __syncthreads();
        load_slots(v, sm, t, T_, lcs);
        __syncthreads();
      }
      lNs += 3;
    }
    return;
  }
  int lNs = 0;
  for (int st = 0; st < n8; ++st) {
    const bool last = (st == n8 - 1) && rem == 0;
    if (last) {
      fft_stage<INV, 8, true>(v, sm, tw, t, lN, lNs, lcs);
    } else {
      fft_stage<INV, 8, false>(v, sm, tw, t, lN, lNs, lcs);
      __syncthreads();
      load_slots(v, sm, t, T_, lcs);
      __syncthreads();
    }
    lNs += 3;
  }
  if (rem == 1) fft_stage<INV, 2, true>(v, sm, tw, t, lN, lNs, lcs);
  if (rem == 2) fft_stage<INV, 4, true>(v, sm, tw, t, lN, lNs, lcs);
}

}  // namespace sgn
