// vec_common.cuh - device helpers for kernels that sweep whole half spectra.
#pragma once
#include "sgn_internal.h"

namespace sgn {

// Flat walk over the Ny*ldS entries of a half spectrum with the column (and
// row) carried along, so that no per-entry division is needed. With (k, K)
// the thread takes every K-th of its grid-stride entries starting at the k-th
// (K interleaved walkers keep K entries' loads in flight per iteration);
// stride = K * thread count, cstep = stride % ldS, rstep = stride / ldS.
struct Walk {
  size_t e, n, stride;
  int row, col, ldS, cstep, rstep;
  __device__ __forceinline__ Walk(const Geom& G, int k = 0, int K = 1) {
    ldS = G.ldS;
    n = (size_t)G.Ny * ldS;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    stride = nthreads * (size_t)K;
    e = (size_t)blockIdx.x * blockDim.x + threadIdx.x + (size_t)k * nthreads;
    row = (int)(e / ldS);
    col = (int)(e - (size_t)row * ldS);
    cstep = (int)(stride % ldS);
    rstep = (int)(stride / ldS);
  }
  __device__ __forceinline__ bool ok() const { return e < n; }
  __device__ __forceinline__ void next() {
    e += stride;
    col += cstep;
    row += rstep;
    if (col >= ldS) {
      col -= ldS;
      row += 1;
    }
  }
};

// Parseval weight of a half-spectrum column: 1 on kx = 0 and kx = Nx/2, 2 on
// the columns in between, 0 on padding columns.
template <typename A = double>
__device__ __forceinline__ A col_weight_k(const Geom& G, int col) {
  return (col == 0 || col == (G.Nx >> 1)) ? (A)1 : (col < G.Nxh ? (A)2 : (A)0);
}

template <typename T>
__device__ __forceinline__ double wdot(cpx<T> a, cpx<T> b) {
  return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}

// Sum v over the block; result valid on thread 0. red: >= 32 doubles.
__device__ __forceinline__ double block_reduce(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
  __syncthreads();
  return tot;
}

// True (in every thread) in the block that finishes last; it then sees every
// other block's partials. Resets the counter for the next launch. wrote: this
// thread stored a partial; only those stores need the fence before the ticket.
__device__ __forceinline__ bool last_block(unsigned* counter, bool wrote = true) {
  __shared__ int s_last;
  if (wrote) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y;
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == total - 1) ? 1 : 0;
    if (s_last) *counter = 0u;
  }
  __syncthreads();
  return s_last != 0;
}

}  // namespace sgn
