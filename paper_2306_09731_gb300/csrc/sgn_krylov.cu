// sgn_krylov.cu - GMRES building blocks on spectral vectors (Section 3;
// Saad & Schultz's GMRES with left preconditioning).
//
// Krylov vectors are half spectra [Ny][ldS] of real fields. Their inner
// product is the Parseval-weighted sum  <a, b> = sum w(kx) Re(conj(a) b),
// w = 1 on the kx = 0 and kx = Nx/2 columns and 2 elsewhere, which equals
// Nx*Ny times the Euclidean inner product of the physical fields; relative
// residuals are therefore the same as for unknowns in physical space.
//
// Orthogonalisation is classical Gram-Schmidt with selective
// reorthogonalisation (the DGKS test): one pass forms all dot products and
// |w|^2, one pass applies w -= sum h_i V_i and forms |w'|^2; a second
// (dots, update) pair runs only when |w'|^2 < |w|^2 / 2, decided on the device
// (the second-pass kernels are gated by a device flag). All reductions
// accumulate in FP64, per block with warp shuffles, then over the NBLK block
// partials in a fixed order (deterministic). On a GB300 these BLAS-1 kernels
// are FP64-issue bound, not HBM bound (4 DFMA per 16-byte entry against an
// FP64:HBM balance below 1 DFMA per byte), so each entry's Parseval weight is
// folded into w once rather than into every dot product.
#include <math.h>

#include "sgn_internal.h"
#include "vec_common.cuh"

namespace sgn {

// Givens update of column j of the Hessenberg matrix (one thread): the column
// from the two Gram-Schmidt passes and |w|, previous rotations, a new rotation
// zeroing H[j+1][j], and the residual estimate |g_{j+1}| into the readback.
__device__ void givens_step(GmresDev* st, int j, GmresReadback* rb, const int* flags) {
  const int ld = MAXM + 1;
  double* Hj = st->H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) Hj[i] = st->h1[i] + st->h2[i];
  const double hn = sqrt(st->nrm2);
  Hj[j + 1] = hn;
  st->hnext = hn;
  st->inv_hnext = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double a = Hj[i], b = Hj[i + 1];
    Hj[i] = st->cs[i] * a + st->sn[i] * b;
    Hj[i + 1] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double d = hypot(Hj[j], Hj[j + 1]);
  const double c = d > 0.0 ? Hj[j] / d : 1.0;
  const double s = d > 0.0 ? Hj[j + 1] / d : 0.0;
  st->cs[j] = c;
  st->sn[j] = s;
  Hj[j] = d;
  Hj[j + 1] = 0.0;
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->res = fabs(st->g[j + 1]);
  rb->res = st->res;
  rb->hnext = hn;
  rb->flags = flags ? *flags : 0;
}

// True (in every thread) in the block that finishes last; it then sees every
// other block's partials. Resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ int s_last;
  __threadfence();
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

// Fixed-order sum over the NBLK block partials of one slot (valid on thread 0).
__device__ __forceinline__ double reduce_slot(const double* partials, int slot, double* red) {
  double v = 0.0;
  for (int b = threadIdx.x; b < NBLK; b += blockDim.x) v += __ldcg(partials + (size_t)slot * NBLK + b);
  return block_reduce(v, red);
}

// Per-thread accumulation type: FP64 vectors accumulate in FP64; FP32 vectors
// (the inner solve of precision 1) form products and each thread's running
// sum over its few entries (about 7 at 2048^2) in FP32 and hand the partial
// sum to the FP64 warp/block/grid reduction. On a GB300 (FP64:FP32 = 1:58) a
// per-entry FP64 conversion and DFMA would cost as much as for FP64 vectors.
template <typename T>
struct Acc {
  typedef double type;
};
template <>
struct Acc<float> {
  typedef float type;
};

constexpr int DOT_CHUNK = 4;  // dot products per block row of the grid (blockIdx.y)

// partials[i * NBLK + b] = block b's share of <V_i, w> for the chunk
// i = 4*blockIdx.y .. +3 (i < nv); chunk 0 also writes |w|^2 to slot nv.
// Four accumulators keep registers low enough for 4 blocks per SM: the
// kernel is latency bound at lower occupancy.
// gate (may be null): the kernel does nothing unless *gate != 0.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_dots(Geom G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                                                 double* partials, const int* gate, double* out,
                                                 unsigned* counter) {
  typedef typename Acc<T>::type A;
  if (gate && *gate == 0) return;
  __shared__ double red[32];
  const int i0 = blockIdx.y * DOT_CHUNK;
  const int nc = min(DOT_CHUNK, nv - i0);
  A acc[DOT_CHUNK];
#pragma unroll
  for (int i = 0; i < DOT_CHUNK; ++i) acc[i] = (A)0;
  A nrm = (A)0;
  const cpx<T>* Vc = V + (size_t)i0 * vstride;
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<T> we = w[it.e];
    const A wt = col_weight_k<A>(G, it.col);
    const A wx = wt * (A)we.x, wy = wt * (A)we.y;
    cpx<T> v[DOT_CHUNK];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i)
      if (i < nc) v[i] = Vc[i * vstride + it.e];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i)
      if (i < nc) acc[i] += wx * (A)v[i].x + wy * (A)v[i].y;
    nrm += wx * (A)we.x + wy * (A)we.y;
  }
#pragma unroll
  for (int i = 0; i < DOT_CHUNK; ++i) {
    if (i < nc) {
      const double tot = block_reduce((double)acc[i], red);
      if (threadIdx.x == 0) partials[(size_t)(i0 + i) * NBLK + blockIdx.x] = tot;
    }
  }
  if (blockIdx.y == 0) {
    const double tot = block_reduce((double)nrm, red);
    if (threadIdx.x == 0) partials[(size_t)nv * NBLK + blockIdx.x] = tot;
  }
  // the last block combines all partials: out[i] = <V_i, w>, out[nv] = |w|^2
  if (last_block(counter)) {
    for (int i = 0; i <= nv; ++i) {
      const double tot = reduce_slot(partials, i, red);
      if (threadIdx.x == 0) out[i] = tot;
    }
  }
}

// w -= sum_i coef[i] V_i (i < nv) and |w_new|^2 into slot 0. Gated like k_dots.
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_update(Geom G, const cpx<T>* V, size_t vstride, int nv,
                                                    const double* __restrict__ coef, cpx<T>* w, double* partials,
                                                    const int* gate, GmresDev* st, int j, int pass,
                                                    unsigned* counter, GmresReadback* rb, const int* flags) {
  typedef typename Acc<T>::type A;
  if (gate && *gate == 0) return;
  __shared__ double red[32];
  __shared__ A cf[MAXV];
  if (threadIdx.x < MAXV) cf[threadIdx.x] = (A)(threadIdx.x < nv ? coef[threadIdx.x] : 0.0);
  __syncthreads();
  A nrm = (A)0;
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<T> we = w[it.e];
    A zx = (A)we.x, zy = (A)we.y;
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      const cpx<T> v0 = V[(size_t)(i + 0) * vstride + it.e], v1 = V[(size_t)(i + 1) * vstride + it.e];
      const cpx<T> v2 = V[(size_t)(i + 2) * vstride + it.e], v3 = V[(size_t)(i + 3) * vstride + it.e];
      zx -= cf[i] * (A)v0.x + cf[i + 1] * (A)v1.x + cf[i + 2] * (A)v2.x + cf[i + 3] * (A)v3.x;
      zy -= cf[i] * (A)v0.y + cf[i + 1] * (A)v1.y + cf[i + 2] * (A)v2.y + cf[i + 3] * (A)v3.y;
    }
    for (; i < nv; ++i) {
      const cpx<T> v0 = V[(size_t)i * vstride + it.e];
      zx -= cf[i] * (A)v0.x;
      zy -= cf[i] * (A)v0.y;
    }
    const cpx<T> z = mk((T)zx, (T)zy);
    w[it.e] = z;
    const A wt = col_weight_k<A>(G, it.col);
    nrm += wt * ((A)z.x * (A)z.x + (A)z.y * (A)z.y);
  }
  const double tot = block_reduce((double)nrm, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  // the last block: |w'|^2, then (first pass) the DGKS test, and the Givens
  // step once the orthogonalisation is final. pass: 1 first pass with the DGKS
  // test, 2 second pass, 3 single pass (no reorthogonalisation)
  if (last_block(counter)) {
    const double n2 = reduce_slot(partials, 0, red);
    if (threadIdx.x == 0) {
      st->nrm2 = n2;
      bool final_pass = (pass == 2);
      if (pass == 1 || pass == 3) {
        // pass 3: first pass of an Arnoldi step that never reorthogonalises
        const int need = (pass == 1 && n2 < 0.5 * st->h1[nv]) ? 1 : 0;
        st->reorth = need;
        if (!need) {
          for (int i = 0; i <= MAXV; ++i) st->h2[i] = 0.0;
          final_pass = true;
        }
      }
      if (final_pass) givens_step(st, j, rb, flags);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(Geom G, const cpx<T>* c, const cpx<T>* w, cpx<T>* r,
                                                  double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<T> z = c[it.e] - w[it.e];
    r[it.e] = z;
    acc += col_weight_k(G, it.col) * wdot(z, z);
  }
  const double tot = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename TI, typename TO>
__global__ void k_scale(Geom G, const cpx<TI>* x, const double* factor, int invert, cpx<TO>* y) {
  // arithmetic in the wider of the two types (FP32 when both are FP32)
  typedef typename Acc<decltype(TI() * TO())>::type A;
  const double f0 = *factor;
  const A f = (A)(invert ? 1.0 / f0 : f0);
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<TI> v = x[it.e];
    y[it.e] = mk((TO)((A)v.x * f), (TO)((A)v.y * f));
  }
}

// The combination sum_i coef[i] V_i is formed in V's accumulation type (FP32
// for the inner corrections of precision 1, whose relative accuracy only has
// to match the FP32 basis) and added to x in x's type.
template <typename TV, typename TX>
__global__ void k_axpy_multi(Geom G, const cpx<TV>* V, size_t vstride, int nv, const double* __restrict__ coef,
                             cpx<TX>* x) {
  typedef typename Acc<TV>::type A;
  __shared__ A cf[MAXV];
  if (threadIdx.x < MAXV) cf[threadIdx.x] = (A)(threadIdx.x < nv ? coef[threadIdx.x] : 0.0);
  __syncthreads();
  for (Walk it(G); it.ok(); it.next()) {
    A dx = (A)0, dy = (A)0;
    for (int i = 0; i < nv; ++i) {
      const cpx<TV> v = V[(size_t)i * vstride + it.e];
      dx += cf[i] * (A)v.x;
      dy += cf[i] * (A)v.y;
    }
    const cpx<TX> xv = x[it.e];
    x[it.e] = mk((TX)(xv.x + (TX)dx), (TX)(xv.y + (TX)dy));
  }
}

// y = a x + b y (FP64 arithmetic); the extrapolated GMRES start
template <typename T>
__global__ void k_axpby(Geom G, double a, const cpx<T>* x, double b, cpx<T>* y) {
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<T> u = x[it.e], v = y[it.e];
    y[it.e] = mk((T)(a * (double)u.x + b * (double)v.x), (T)(a * (double)u.y + b * (double)v.y));
  }
}

template <typename T>
__global__ void k_zero(Geom G, cpx<T>* x) {
  for (Walk it(G); it.ok(); it.next()) x[it.e] = mk((T)0, (T)0);
}

// out[i] = sum_b partials[i*NBLK + b] (fixed order), i < n. Gated.
__global__ void k_reduce(const double* partials, int n, double* out, int sqrt_out, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[32];
  for (int i = 0; i < n; ++i) {
    double v = 0.0;
    for (int b = threadIdx.x; b < NBLK; b += blockDim.x) v += partials[(size_t)i * NBLK + b];
    const double tot = block_reduce(v, red);
    if (threadIdx.x == 0) out[i] = sqrt_out ? sqrt(tot) : tot;
  }
}

// DGKS test after the first Gram-Schmidt pass: reorthogonalise when the
// update removed more than half of |w|^2 (|w'| < |w|/sqrt 2); otherwise the
// second-pass coefficients are zero.
__global__ void k_reorth_decide(GmresDev* st, int nv) {
  if (threadIdx.x != 0) return;
  const double nw = st->h1[nv];
  const int need = (st->nrm2 < 0.5 * nw) ? 1 : 0;
  st->reorth = need;
  if (!need)
    for (int i = 0; i < MAXV; ++i) st->h2[i] = 0.0;
}

// ---------------------------------------------------------- scalar kernels

// g = (beta, 0, ...), the start of a GMRES cycle
__global__ void k_gmres_start(GmresDev* st, const double* beta) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i <= MAXM; ++i) st->g[i] = 0.0;
  st->g[0] = *beta;
  st->res = *beta;
}

// Column j of the Hessenberg matrix from the two CGS passes and the norm,
// previous rotations applied, new rotation zeroing H[j+1][j], residual
// estimate |g_{j+1}|.
__global__ void k_givens(GmresDev* st, int j, GmresReadback* rb, const int* flags) {
  if (threadIdx.x != 0) return;
  givens_step(st, j, rb, flags);
}

// y = H(0:k,0:k)^{-1} g(0:k) by back substitution
__global__ void k_backsolve(GmresDev* st, int k) {
  if (threadIdx.x != 0) return;
  const int ld = MAXM + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int l = i + 1; l < k; ++l) s -= st->H[i + (size_t)l * ld] * st->y[l];
    st->y[i] = s / st->H[i + (size_t)i * ld];
  }
}

__global__ void k_readback_scalar(const double* x, const int* flags, GmresReadback* rb) {
  if (threadIdx.x != 0) return;
  rb->scalar = *x;
  rb->flags = flags ? *flags : 0;
}

// ----------------------------------------------------------- invariants

// partials[q*NBLK + b], q = mass, px, py, energy (Section 2.3)
__global__ void __launch_bounds__(256) k_invariant_sums(Geom G, const double* h, const double* vx,
                                                        const double* vy, const double* sig, const double* sx,
                                                        const double* sy, double g, double* partials) {
  __shared__ double red[32];
  double m = 0.0, px = 0.0, py = 0.0, en = 0.0;
  const size_t n = G.nphys();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double hv = h[i], r = 1.0 / hv;
    const double ux = vx[i] - sx[i] * r, uy = vy[i] - sy[i] * r;
    const double s = sig[i];
    m += hv - 1.0;
    px += hv * ux;
    py += hv * uy;
    en += 0.5 * hv * (ux * ux + uy * uy) + 1.5 * s * s * r * r * r + 0.5 * g * (hv - 1.0) * (hv - 1.0);
  }
  double vals[4] = {m, px, py, en};
  for (int q = 0; q < 4; ++q) {
    const double tot = block_reduce(vals[q], red);
    if (threadIdx.x == 0) partials[(size_t)q * NBLK + blockIdx.x] = tot;
  }
}

// ------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_dots(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                        double* partials, const int* gate, double* out, unsigned* counter, const Exec& ex) {
  dim3 grid(NBLK, (nv + DOT_CHUNK - 1) / DOT_CHUNK);
  if (grid.y == 0) grid.y = 1;
  ex.begin(PK_KRYLOV);
  k_dots<T><<<grid, 256, 0, ex.s>>>(G, V, vstride, nv, w, partials, gate, out, counter);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cgs_update(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const double* coef,
                              cpx<T>* w, double* partials, const int* gate, GmresDev* st, int j, int pass,
                              unsigned* counter, GmresReadback* rb, const int* flags, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_cgs_update<T><<<NBLK, 256, 0, ex.s>>>(G, V, vstride, nv, coef, w, partials, gate, st, j, pass, counter, rb,
                                         flags);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_residual(const Geom& G, const cpx<T>* c, const cpx<T>* w, cpx<T>* r, double* partials,
                            const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_residual<T><<<NBLK, 256, 0, ex.s>>>(G, c, w, r, partials);
  ex.end();
  return cudaGetLastError();
}
template <typename TI, typename TO>
cudaError_t launch_scale(const Geom& G, const cpx<TI>* x, const double* factor, bool invert, cpx<TO>* y,
                         const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_scale<TI, TO><<<NBLK, 256, 0, ex.s>>>(G, x, factor, invert ? 1 : 0, y);
  ex.end();
  return cudaGetLastError();
}
template <typename TV, typename TX>
cudaError_t launch_axpy_multi(const Geom& G, const cpx<TV>* V, size_t vstride, int nv, const double* coef,
                              cpx<TX>* x, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_axpy_multi<TV, TX><<<NBLK, 256, 0, ex.s>>>(G, V, vstride, nv, coef, x);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_zero(const Geom& G, cpx<T>* x, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_zero<T><<<NBLK, 256, 0, ex.s>>>(G, x);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(const Geom& G, double a, const cpx<T>* x, double b, cpx<T>* y, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_axpby<T><<<NBLK, 256, 0, ex.s>>>(G, a, x, b, y);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partials, int n, double* out, bool sqrt_out, const int* gate,
                          const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_reduce<<<1, 256, 0, ex.s>>>(partials, n, out, sqrt_out ? 1 : 0, gate);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_reorth_decide(GmresDev* st, int nv, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_reorth_decide<<<1, 32, 0, ex.s>>>(st, nv);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_gmres_start(GmresDev* st, const double* beta, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_gmres_start<<<1, 32, 0, ex.s>>>(st, beta);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_givens(GmresDev* st, int j, GmresReadback* rb_dev, const int* flags, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_givens<<<1, 32, 0, ex.s>>>(st, j, rb_dev, flags);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_backsolve(GmresDev* st, int k, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_backsolve<<<1, 32, 0, ex.s>>>(st, k);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_readback_scalar(const double* x, const int* flags, GmresReadback* rb_dev, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_readback_scalar<<<1, 32, 0, ex.s>>>(x, flags, rb_dev);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_invariant_sums(const Geom& G, const double* h, const double* vx, const double* vy,
                                  const double* sig, const double* sx, const double* sy, double g,
                                  double* partials, const Exec& ex) {
  ex.begin(PK_IO);
  k_invariant_sums<<<NBLK, 256, 0, ex.s>>>(G, h, vx, vy, sig, sx, sy, g, partials);
  ex.end();
  return cudaGetLastError();
}

#define SGN_KRYLOV_INST(T)                                                                                   \
  template cudaError_t launch_dots<T>(const Geom&, const cpx<T>*, size_t, int, const cpx<T>*, double*,       \
                                      const int*, double*, unsigned*, const Exec&);                         \
  template cudaError_t launch_cgs_update<T>(const Geom&, const cpx<T>*, size_t, int, const double*, cpx<T>*, \
                                            double*, const int*, GmresDev*, int, int, unsigned*,            \
                                            GmresReadback*, const int*, const Exec&);                       \
  template cudaError_t launch_residual<T>(const Geom&, const cpx<T>*, const cpx<T>*, cpx<T>*, double*,       \
                                          const Exec&);                                                     \
  template cudaError_t launch_zero<T>(const Geom&, cpx<T>*, const Exec&);                                   \
  template cudaError_t launch_axpby<T>(const Geom&, double, const cpx<T>*, double, cpx<T>*, const Exec&);

SGN_KRYLOV_INST(double)
SGN_KRYLOV_INST(float)
template cudaError_t launch_scale<double, double>(const Geom&, const cpx<double>*, const double*, bool,
                                                  cpx<double>*, const Exec&);
template cudaError_t launch_scale<double, float>(const Geom&, const cpx<double>*, const double*, bool,
                                                 cpx<float>*, const Exec&);
template cudaError_t launch_scale<float, float>(const Geom&, const cpx<float>*, const double*, bool,
                                                cpx<float>*, const Exec&);
template cudaError_t launch_axpy_multi<double, double>(const Geom&, const cpx<double>*, size_t, int,
                                                       const double*, cpx<double>*, const Exec&);
template cudaError_t launch_axpy_multi<float, double>(const Geom&, const cpx<float>*, size_t, int,
                                                      const double*, cpx<double>*, const Exec&);

}  // namespace sgn
