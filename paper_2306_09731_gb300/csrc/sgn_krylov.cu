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
// folded into w once rather than into every dot product. The Gram-Schmidt
// pair runs one wave of KBLK blocks (4 per SM). The FP32 basis of the inner
// solve is kept unnormalised, V_i = s_i X_i with the scales s_i on the device,
// so no pass rescales a vector (k_cgs_update writes X_{j+1} itself).
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

// Fixed-order sum over the first nblk block partials of one slot (slot
// stride NBLK; valid on thread 0).
__device__ __forceinline__ double reduce_slot(const double* partials, int slot, double* red, int nblk = NBLK) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += __ldcg(partials + (size_t)slot * NBLK + b);
  return block_reduce(v, red);
}

// Blocks of the Gram-Schmidt sweeps: one wave at four 256-thread blocks per
// SM (a sweep is ~7 entries a thread at 2048^2 with NBLK blocks, and the
// block reductions and the last block's sum over the partials are a fixed
// cost per block)
constexpr int KBLK = 608;

// out[s] = sum of the first nblk partials of slot s (slot stride NBLK),
// s < nslots, one warp per slot:
// each lane keeps 8 loads in flight over its lane-strided share, then a
// shuffle tree. The order is fixed, so the sums are deterministic. Up to
// blockDim/32 slots finish in one round (the slot-by-slot block reduction
// took one dependent load chain and two barriers per slot).
__device__ __forceinline__ void reduce_slots(const double* partials, int nslots, double* out, int nblk = NBLK) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s = warp; s < nslots; s += nw) {
    const double* p = partials + (size_t)s * NBLK;
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 0.0;
    for (int b = lane; b < nblk; b += 32 * 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int bb = b + 32 * u;
        if (bb < nblk) a[u] += __ldcg(p + bb);
      }
    }
    double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[s] = v;
  }
}

// Block sums of K values with one barrier: thread k (< K) returns the sum of
// value k. Each warp sums in the accumulation type A (FP32 for the FP32
// vectors: an FP64 shuffle tree costs more FP64-pipe time than the sweep
// itself on this part), then the warp sums are added in FP64 in a fixed order.
// red: K * 32 doubles of shared memory.
template <int K, typename A>
__device__ __forceinline__ double block_reduce_multi(A (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[k * 32 + wid] = (double)v[k];
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < K)
    for (int i = 0; i < nw; ++i) t += red[threadIdx.x * 32 + i];
  return t;
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

constexpr int DOT_CHUNK = 4;  // dot products per sweep of a block's entries

// partials[i * NBLK + b] = block b's share of <V_i, w> (i < nv) and
// partials[nv * NBLK + b] its share of |w|^2. Each block runs over the basis in
// chunks of four vectors (one sweep of its entries per chunk; at the usual
// cycle lengths one chunk), so the grid does not depend on nv: graph mode reads
// nv from the device. Four accumulators keep registers low enough for 4 blocks
// per SM.
// gate (may be null): the kernel does nothing unless *gate != 0.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_dots(Geom G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                                                 double* partials, const int* gate, double* out,
                                                 unsigned* counter, const int* jdev, const double* vscl) {
  typedef typename Acc<T>::type A;
  if (gate && *gate == 0) return;
  if (jdev) nv = *jdev + 1;
  __shared__ double red[(DOT_CHUNK + 1) * 32];
  for (int i0 = 0; i0 < nv; i0 += DOT_CHUNK) {
    const int nc = min(DOT_CHUNK, nv - i0);
    const bool chunk0 = i0 == 0;
    A acc[DOT_CHUNK];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i) acc[i] = (A)0;
    A nrm = (A)0;
    const cpx<T>* Vc = V + (size_t)i0 * vstride;
    // two interleaved walkers: both entries' loads issue before any use
    for (Walk a(G, 0, 2), b(G, 1, 2); a.ok(); a.next(), b.next()) {
      const bool bok = b.ok();
      const size_t eb = bok ? b.e : a.e;
      const cpx<T> wa = w[a.e], wb = w[eb];
      cpx<T> va[DOT_CHUNK], vb[DOT_CHUNK];
#pragma unroll
      for (int i = 0; i < DOT_CHUNK; ++i)
        if (i < nc) {
          va[i] = Vc[i * vstride + a.e];
          vb[i] = Vc[i * vstride + eb];
        }
      const A ta = col_weight_k<A>(G, a.col), tb = bok ? col_weight_k<A>(G, b.col) : (A)0;
      const A ax = ta * (A)wa.x, ay = ta * (A)wa.y, bx = tb * (A)wb.x, by = tb * (A)wb.y;
#pragma unroll
      for (int i = 0; i < DOT_CHUNK; ++i)
        if (i < nc) acc[i] += (ax * (A)va[i].x + ay * (A)va[i].y) + (bx * (A)vb[i].x + by * (A)vb[i].y);
      if (chunk0) nrm += (ax * (A)wa.x + ay * (A)wa.y) + (bx * (A)wb.x + by * (A)wb.y);
    }
    // thread i < DOT_CHUNK holds <V_{i0+i}, w>, thread DOT_CHUNK |w|^2
    A vals[DOT_CHUNK + 1];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i) vals[i] = acc[i];
    vals[DOT_CHUNK] = nrm;
    const double tot = block_reduce_multi<DOT_CHUNK + 1>(vals, red);
    if (threadIdx.x < DOT_CHUNK && (int)threadIdx.x < nc)
      partials[(size_t)(i0 + threadIdx.x) * NBLK + blockIdx.x] = tot;
    if (threadIdx.x == DOT_CHUNK && chunk0) partials[(size_t)nv * NBLK + blockIdx.x] = tot;
    __syncthreads();  // red is reused by the next chunk
  }
  // the last block combines all partials: out[i] = <V_i, w>, out[nv] = |w|^2
  if (last_block(counter, threadIdx.x <= DOT_CHUNK)) {
    reduce_slots(partials, nv + 1, out, gridDim.x);
    // scaled basis (vscl): V_i = s_i X_i and w = s_j w~ for the stored X_i and
    // the matvec of X_j: <V_i, w> = s_i s_j <X_i, w~>, |w|^2 = s_j^2 |w~|^2
    if (vscl) {
      __syncthreads();
      if ((int)threadIdx.x <= nv) {
        const double sj = vscl[nv - 1];
        out[threadIdx.x] *= ((int)threadIdx.x < nv ? vscl[threadIdx.x] : sj) * sj;
      }
    }
  }
}

// w -= sum_i coef[i] V_i (i < nv) and |w_new|^2 into slot 0. Gated like k_dots.
// After the final Givens step of Arnoldi step j (graph mode): count the matvec,
// record the residual estimate, and keep the Arnoldi loop running unless the
// cycle is done (the eager host loop's test).
__device__ __forceinline__ void ctl_step(GmresDev* st, int j, const GraphCtl& ctl) {
  st->its += 1;
  st->tot_its += 1;
  st->k = j + 1;
  st->j = j + 1;
  st->res_in = st->res;
  const bool stop = !(st->res > st->inner_target) || st->its >= ctl.maxit || !(st->hnext > 0.0) ||
                    st->k >= ctl.m || st->res != st->res;
  cudaGraphSetConditional(ctl.h_step, stop ? 0u : 1u);
}

// scaled (FP32 inner solve): the basis is stored unnormalised, V_i = s_i X_i
// (s = st->vscl) and w holds w~ = A X_j; the kernel writes X_{j+1} = w~ -
// sum_i (h_i s_i / s_j) X_i = w' / s_j straight into slot j+1 of V (no scaling
// pass), |w'|^2 = s_j^2 |X_{j+1}|^2, and s_{j+1} = s_j / |w'|.
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_update(Geom G, const cpx<T>* V, size_t vstride, int nv,
                                                    const double* __restrict__ coef, cpx<T>* w, double* partials,
                                                    const int* gate, GmresDev* st, int j, int pass,
                                                    unsigned* counter, GmresReadback* rb, const int* flags,
                                                    const int* jdev, GraphCtl ctl, int scaled) {
  typedef typename Acc<T>::type A;
  if (gate && *gate == 0) return;
  if (jdev) {
    j = *jdev;
    nv = j + 1;
  }
  __shared__ double red[32];
  __shared__ A cf[MAXV + 4];
  if (threadIdx.x < MAXV + 4) {
    double c = threadIdx.x < nv ? coef[threadIdx.x] : 0.0;
    if (scaled && threadIdx.x < nv) c *= st->vscl[threadIdx.x] / st->vscl[j];
    cf[threadIdx.x] = (A)c;
  }
  __syncthreads();
  cpx<T>* wout = scaled ? const_cast<cpx<T>*>(V) + (size_t)(j + 1) * vstride : w;
  A nrm = (A)0;
  // two interleaved walkers; four basis vectors per round with predicated
  // loads rather than a remainder loop, so that a round's loads (8 entries)
  // are in flight together
  for (Walk a(G, 0, 2), b(G, 1, 2); a.ok(); a.next(), b.next()) {
    const bool bok = b.ok();
    const size_t eb = bok ? b.e : a.e;
    const cpx<T> wa = w[a.e], wb = w[eb];
    A zax = (A)wa.x, zay = (A)wa.y, zbx = (A)wb.x, zby = (A)wb.y;
    for (int i = 0; i < nv; i += 4) {
      cpx<T> va[4], vb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = i + u < nv;
        va[u] = in ? V[(size_t)(i + u) * vstride + a.e] : mk((T)0, (T)0);
        vb[u] = in ? V[(size_t)(i + u) * vstride + eb] : mk((T)0, (T)0);
      }
      zax -= (cf[i] * (A)va[0].x + cf[i + 1] * (A)va[1].x) + (cf[i + 2] * (A)va[2].x + cf[i + 3] * (A)va[3].x);
      zay -= (cf[i] * (A)va[0].y + cf[i + 1] * (A)va[1].y) + (cf[i + 2] * (A)va[2].y + cf[i + 3] * (A)va[3].y);
      zbx -= (cf[i] * (A)vb[0].x + cf[i + 1] * (A)vb[1].x) + (cf[i + 2] * (A)vb[2].x + cf[i + 3] * (A)vb[3].x);
      zby -= (cf[i] * (A)vb[0].y + cf[i + 1] * (A)vb[1].y) + (cf[i + 2] * (A)vb[2].y + cf[i + 3] * (A)vb[3].y);
    }
    const cpx<T> za = mk((T)zax, (T)zay), zb = mk((T)zbx, (T)zby);
    wout[a.e] = za;
    nrm += col_weight_k<A>(G, a.col) * ((A)za.x * (A)za.x + (A)za.y * (A)za.y);
    if (bok) {
      wout[b.e] = zb;
      nrm += col_weight_k<A>(G, b.col) * ((A)zb.x * (A)zb.x + (A)zb.y * (A)zb.y);
    }
  }
  A one[1] = {nrm};
  const double tot = block_reduce_multi<1>(one, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  // the last block: |w'|^2, then (first pass) the DGKS test, and the Givens
  // step once the orthogonalisation is final. pass: 1 first pass with the DGKS
  // test, 2 second pass, 3 single pass (no reorthogonalisation)
  if (last_block(counter, threadIdx.x == 0)) {
    const double n2 = reduce_slot(partials, 0, red, gridDim.x);
    if (threadIdx.x == 0) {
      st->nrm2 = scaled ? n2 * st->vscl[j] * st->vscl[j] : n2;
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
      // graph mode: the Arnoldi loop continues only if the final pass re-arms it
      if (ctl.enabled) cudaGraphSetConditional(ctl.h_step, 0u);
      if (final_pass) {
        givens_step(st, j, rb, flags);
        if (scaled) st->vscl[j + 1] = st->hnext > 0.0 ? st->vscl[j] / st->hnext : 0.0;
        if (ctl.enabled) ctl_step(st, j, ctl);
      }
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
__global__ void k_scale(Geom G, const cpx<TI>* x, const double* factor, int invert, cpx<TO>* y, const int* ysel,
                        size_t ystride) {
  if (ysel) y += (size_t)(*ysel) * ystride;
  // arithmetic in the output type: an FP32 result (the inner basis) is
  // scaled in FP32 after the conversion, which stays off the FP64 pipe
  const double f0 = *factor;
  const TO f = (TO)(invert ? 1.0 / f0 : f0);
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<TI> v = x[it.e];
    y[it.e] = mk(cvt<TO>(v.x) * f, cvt<TO>(v.y) * f);
  }
}

// The combination sum_i coef[i] V_i is formed in V's accumulation type (FP32
// for the inner corrections of precision 1, whose relative accuracy only has
// to match the FP32 basis) and added to x in x's type.
template <typename TV, typename TX>
__global__ void k_axpy_multi(Geom G, const cpx<TV>* V, size_t vstride, int nv, const double* __restrict__ coef,
                             cpx<TX>* x, const int* ndev, const double* vscl) {
  typedef typename Acc<TV>::type A;
  if (ndev) nv = *ndev;
  if (nv <= 0) return;
  __shared__ A cf[MAXV];
  // scaled basis (vscl): V_i = s_i X_i
  if (threadIdx.x < MAXV)
    cf[threadIdx.x] = (A)(threadIdx.x < nv ? coef[threadIdx.x] * (vscl ? vscl[threadIdx.x] : 1.0) : 0.0);
  __syncthreads();
  for (Walk it(G); it.ok(); it.next()) {
    A dx = (A)0, dy = (A)0;
    for (int i = 0; i < nv; ++i) {
      const cpx<TV> v = V[(size_t)i * vstride + it.e];
      dx += cf[i] * (A)v.x;
      dy += cf[i] * (A)v.y;
    }
    const cpx<TX> xv = x[it.e];
    x[it.e] = mk(xv.x + cvt<TX>(dx), xv.y + cvt<TX>(dy));
  }
}

// y = a x + b y (FP64 arithmetic); the extrapolated GMRES start
template <typename T>
__global__ void k_axpby(Geom G, double a, const cpx<T>* x, double b, cpx<T>* y, const int* gate,
                        const int* gate2) {
  if ((gate && *gate == 0) || (gate2 && *gate2 == 0)) return;
  for (Walk it(G); it.ok(); it.next()) {
    const cpx<T> u = x[it.e], v = y[it.e];
    y[it.e] = mk((T)(a * (double)u.x + b * (double)v.x), (T)(a * (double)u.y + b * (double)v.y));
  }
}

template <typename T>
__global__ void k_copy_gated(Geom G, const cpx<T>* x, cpx<T>* y, const int* gate) {
  if (*gate == 0) return;
  for (Walk it(G); it.ok(); it.next()) y[it.e] = x[it.e];
}

template <typename T>
__global__ void k_zero(Geom G, cpx<T>* x, const int* gate) {
  if (gate && *gate == 0) return;
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

// ---------------------------------------------------------- scalar kernels

// g = (beta, 0, ...), the start of a GMRES cycle
__global__ void k_gmres_start(GmresDev* st, const double* beta) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i <= MAXM; ++i) st->g[i] = 0.0;
  st->g[0] = *beta;
  st->res = *beta;
  st->vscl[0] = 1.0;
}

// y = H(0:k,0:k)^{-1} g(0:k) by back substitution
__global__ void k_backsolve(GmresDev* st, int k, const int* kdev) {
  if (threadIdx.x != 0) return;
  if (kdev) k = *kdev;
  const int ld = MAXM + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int l = i + 1; l < k; ++l) s -= st->H[i + (size_t)l * ld] * st->y[l];
    st->y[i] = s / st->H[i + (size_t)i * ld];
  }
}

// ---------------------------------------------------- graph-mode control
// One thread each. They make on the device the decisions the eager host loop
// makes after its stream synchronisations.

// end of a solve: its statistics
__device__ void ctl_finish(GmresDev* st, bool conv, double relres) {
  st->conv = conv ? 1 : 0;
  if (!conv) st->notconv = 1;
  st->last_relres = relres;
  st->last_its = st->its;
  st->max_its = max(st->max_its, st->its);
}

// after c = M^-1 b and |c|: a zero right-hand side gives sigma = 0 and no cycle
__global__ void k_ctl_begin(GmresDev* st, const double* cnorm_d, GraphCtl ctl) {
  if (threadIdx.x != 0) return;
  const double cn = *cnorm_d;
  st->cnorm = cn;
  st->target = ctl.tol * cn;
  st->its = 0;
  st->sweeps = 0;
  st->k = 0;
  st->j = 0;
  st->zero_sigma = (cn == 0.0) ? 1 : 0;
  st->tot_solves += 1;
  if (cn == 0.0) ctl_finish(st, true, 0.0);
  cudaGraphSetConditional(ctl.h_sweep, cn == 0.0 ? 0u : 1u);
}

// after the residual beta of a restart cycle / refinement sweep: stop, or
// start a cycle on V_0 = r / beta
__global__ void k_ctl_sweep(GmresDev* st, const double* beta_d, GraphCtl ctl) {
  if (threadIdx.x != 0) return;
  const double beta = *beta_d;
  st->beta = beta;
  st->k = 0;
  st->j = 0;
  st->vscl[0] = 1.0;
  st->sweeps += 1;
  st->tot_sweeps += 1;
  const bool done = !(beta > st->target);
  // every cycle takes at least one Arnoldi step, so its bounds the sweeps;
  // the second test only guards the loop itself
  const bool capped = st->its >= ctl.maxit || st->sweeps > ctl.maxit + 1;
  if (done || capped) {
    ctl_finish(st, done && beta == beta, beta / st->cnorm);
    cudaGraphSetConditional(ctl.h_sweep, 0u);
    cudaGraphSetConditional(ctl.h_step, 0u);
    return;
  }
  st->inner_target = ctl.mixed ? fmax(0.5 * st->target, kInnerRel * beta) : st->target;
  for (int i = 0; i <= MAXM; ++i) st->g[i] = 0.0;
  st->g[0] = beta;
  st->res = beta;
  st->res_in = beta;
  cudaGraphSetConditional(ctl.h_step, 1u);
}

// after a cycle's update sigma += V y: converged (mixed precision: only when
// the FP32 estimate can be trusted), NaN, or another cycle / sweep
__global__ void k_ctl_after(GmresDev* st, GraphCtl ctl) {
  if (threadIdx.x != 0) return;
  if (st->k == 0) return;  // the sweep stopped before the cycle
  const double r = st->res_in;
  if (r != r) {
    ctl_finish(st, false, r);
    cudaGraphSetConditional(ctl.h_sweep, 0u);
    return;
  }
  const bool conv = ctl.mixed ? (r <= st->target && kFp32Trust * st->beta <= 0.5 * st->target) : (r <= st->target);
  if (conv) {
    ctl_finish(st, true, r / st->cnorm);
    cudaGraphSetConditional(ctl.h_sweep, 0u);
  }
}

__global__ void k_set_int(int* p, int v) {
  if (threadIdx.x == 0) *p = v;
}

// Polynomial start across steps. With a fixed dt, the sigma that stage s
// solves for is a smooth function of the step's start time, so the values of
// the last steps at equal spacing predict the next by the polynomial through
// them: Newton's backward differences give 3, -3, 1 (quadratic, 3 steps) and
// 4, -6, 4, -1 (cubic, 4 steps), with error O(dt^3) and O(dt^4) against the
// O(dt^2) of the linear extrapolation inside a step. Slot (q, s) of the ring
// is ring + (4 q + s - 1) vs; hist->head is the slot q of the current step.
__device__ __forceinline__ const cpx<double>* ext_slot(const cpx<double>* ring, size_t vs, int q, int s) {
  return ring + (size_t)(4 * (q & 3) + s - 1) * vs;
}

__global__ void k_ext_start(Geom G, const cpx<double>* ring, size_t vs, int s, const ExtHist* hist,
                            cpx<double>* sig) {
  const int lv = hist->levels;
  if (lv < 3) return;
  const int head = hist->head;
  const cpx<double>* p0 = ext_slot(ring, vs, head - 1, s);
  const cpx<double>* p1 = ext_slot(ring, vs, head - 2, s);
  const cpx<double>* p2 = ext_slot(ring, vs, head - 3, s);
  if (lv >= 4) {
    const cpx<double>* p3 = ext_slot(ring, vs, head - 4, s);
    for (Walk it(G); it.ok(); it.next()) {
      const cpx<double> a = p0[it.e], b = p1[it.e], c = p2[it.e], d = p3[it.e];
      sig[it.e] = mk(4.0 * a.x - 6.0 * b.x + 4.0 * c.x - d.x, 4.0 * a.y - 6.0 * b.y + 4.0 * c.y - d.y);
    }
  } else {
    for (Walk it(G); it.ok(); it.next()) {
      const cpx<double> a = p0[it.e], b = p1[it.e], c = p2[it.e];
      sig[it.e] = mk(3.0 * (a.x - b.x) + c.x, 3.0 * (a.y - b.y) + c.y);
    }
  }
}

__global__ void k_ext_store(Geom G, const cpx<double>* sig, cpx<double>* ring, size_t vs, int s,
                            const ExtHist* hist) {
  cpx<double>* dst = ring + (size_t)(4 * (hist->head & 3) + s - 1) * vs;
  for (Walk it(G); it.ok(); it.next()) dst[it.e] = sig[it.e];
}

// end of a step: its slot becomes the newest level
__global__ void k_ext_advance(ExtHist* hist) {
  if (threadIdx.x == 0) {
    hist->head = (hist->head + 1) & 3;
    hist->levels = min(hist->levels + 1, 4);
    hist->full = hist->levels >= 4 ? 1 : 0;
    hist->lin = hist->levels < 3 ? 1 : 0;
  }
}

// start of a call: keep the levels only if *flag (the call continues the
// trajectory the handle returned last)
__global__ void k_ext_keep(ExtHist* hist, const int* flag) {
  if (threadIdx.x == 0 && *flag == 0) {
    hist->levels = 0;
    hist->full = 0;
    hist->lin = 1;
  }
}

// *flag = 1 when every component of the three spectra b is within rel * max|a|
// of a's (a: the state the handle returned last, b: a call's input state),
// else 0 (NaN counts as a difference). The maxima are taken on the bit
// patterns of |b - a| and |a|: for non-negative doubles the patterns order
// as the values do (a NaN's sorts above infinity, so it wins the maximum and
// fails the final test), so only the subtractions use the FP64 pipe. Block
// maxima in partials, combined by the last block.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(256) k_same_state(Geom G, const cpx<double>* a0, const cpx<double>* a1,
                                                    const cpx<double>* a2, const cpx<double>* b0,
                                                    const cpx<double>* b1, const cpx<double>* b2, double rel,
                                                    double* partials, unsigned* counter, int* flag) {
  __shared__ unsigned long long red[2][32];
  const cpx<double>* A[3] = {a0, a1, a2};
  const cpx<double>* B[3] = {b0, b1, b2};
  unsigned long long md = 0ull, ma = 0ull;
  for (Walk it(G); it.ok(); it.next()) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const cpx<double> a = A[f][it.e], b = B[f][it.e];
      const unsigned long long dx = abs_bits(b.x - a.x), dy = abs_bits(b.y - a.y);
      const unsigned long long ax = abs_bits(a.x), ay = abs_bits(a.y);
      md = dx > md ? dx : md;
      md = dy > md ? dy : md;
      ma = ax > ma ? ax : ma;
      ma = ay > ma ? ay : ma;
    }
  }
  md = warp_max_u64(md);
  ma = warp_max_u64(ma);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  if (lane == 0) {
    red[0][wid] = md;
    red[1][wid] = ma;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) {
      md = red[0][i] > md ? red[0][i] : md;
      ma = red[1][i] > ma ? red[1][i] : ma;
    }
    partials[blockIdx.x] = __longlong_as_double((long long)md);
    partials[NBLK + blockIdx.x] = __longlong_as_double((long long)ma);
  }
  if (last_block(counter, threadIdx.x == 0)) {
    // every thread of the last block takes a share of the block maxima
    unsigned long long D = 0ull, M = 0ull;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      const unsigned long long d = (unsigned long long)__double_as_longlong(__ldcg(partials + b));
      const unsigned long long m = (unsigned long long)__double_as_longlong(__ldcg(partials + NBLK + b));
      D = d > D ? d : D;
      M = m > M ? m : M;
    }
    D = warp_max_u64(D);
    M = warp_max_u64(M);
    __syncthreads();
    if (lane == 0) {
      red[0][wid] = D;
      red[1][wid] = M;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < nw; ++i) {
        D = red[0][i] > D ? red[0][i] : D;
        M = red[1][i] > M ? red[1][i] : M;
      }
      const double dd = __longlong_as_double((long long)D), mm = __longlong_as_double((long long)M);
      *flag = (mm > 0.0 && dd <= rel * mm) ? 1 : 0;
    }
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
                        double* partials, const int* gate, double* out, unsigned* counter, const Exec& ex,
                        const int* jdev, const double* vscl) {
  ex.begin(PK_KRYLOV);
  k_dots<T><<<KBLK, 256, 0, ex.s>>>(G, V, vstride, nv, w, partials, gate, out, counter, jdev, vscl);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cgs_update(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const double* coef,
                              cpx<T>* w, double* partials, const int* gate, GmresDev* st, int j, int pass,
                              unsigned* counter, GmresReadback* rb, const int* flags, const Exec& ex,
                              const int* jdev, const GraphCtl* ctl, bool scaled) {
  GraphCtl c{};
  if (ctl) c = *ctl;
  ex.begin(PK_KRYLOV);
  k_cgs_update<T><<<KBLK, 256, 0, ex.s>>>(G, V, vstride, nv, coef, w, partials, gate, st, j, pass, counter, rb,
                                         flags, jdev, c, scaled ? 1 : 0);
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
                         const Exec& ex, const int* ysel, size_t ystride) {
  ex.begin(PK_KRYLOV);
  k_scale<TI, TO><<<NBLK, 256, 0, ex.s>>>(G, x, factor, invert ? 1 : 0, y, ysel, ystride);
  ex.end();
  return cudaGetLastError();
}
template <typename TV, typename TX>
cudaError_t launch_axpy_multi(const Geom& G, const cpx<TV>* V, size_t vstride, int nv, const double* coef,
                              cpx<TX>* x, const Exec& ex, const int* ndev, const double* vscl) {
  ex.begin(PK_KRYLOV);
  k_axpy_multi<TV, TX><<<NBLK, 256, 0, ex.s>>>(G, V, vstride, nv, coef, x, ndev, vscl);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_zero(const Geom& G, cpx<T>* x, const Exec& ex, const int* gate) {
  ex.begin(PK_KRYLOV);
  k_zero<T><<<NBLK, 256, 0, ex.s>>>(G, x, gate);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(const Geom& G, double a, const cpx<T>* x, double b, cpx<T>* y, const Exec& ex,
                         const int* gate, const int* gate2) {
  ex.begin(PK_KRYLOV);
  k_axpby<T><<<NBLK, 256, 0, ex.s>>>(G, a, x, b, y, gate, gate2);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_copy_gated(const Geom& G, const cpx<T>* x, cpx<T>* y, const int* gate, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_copy_gated<T><<<NBLK, 256, 0, ex.s>>>(G, x, y, gate);
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
cudaError_t launch_gmres_start(GmresDev* st, const double* beta, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_gmres_start<<<1, 32, 0, ex.s>>>(st, beta);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_backsolve(GmresDev* st, int k, const Exec& ex, const int* kdev) {
  ex.begin(PK_KRYLOV);
  k_backsolve<<<1, 32, 0, ex.s>>>(st, k, kdev);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ctl_begin(GmresDev* st, const double* cnorm, GraphCtl ctl, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ctl_begin<<<1, 32, 0, ex.s>>>(st, cnorm, ctl);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ctl_sweep(GmresDev* st, const double* beta, GraphCtl ctl, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ctl_sweep<<<1, 32, 0, ex.s>>>(st, beta, ctl);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ctl_after(GmresDev* st, GraphCtl ctl, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ctl_after<<<1, 32, 0, ex.s>>>(st, ctl);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_same_state(const Geom& G, const cpx<double>* const* a, const cpx<double>* const* b, double rel,
                              double* partials, unsigned* counter, int* flag, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_same_state<<<NBLK, 256, 0, ex.s>>>(G, a[0], a[1], a[2], b[0], b[1], b[2], rel, partials, counter, flag);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_set_int<<<1, 32, 0, ex.s>>>(p, v);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_ext_start(const Geom& G, const cpx<double>* ring, int s, const ExtHist* hist, cpx<double>* sig,
                             const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ext_start<<<NBLK, 256, 0, ex.s>>>(G, ring, G.nspec(), s, hist, sig);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ext_store(const Geom& G, const cpx<double>* sig, cpx<double>* ring, int s, const ExtHist* hist,
                             const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ext_store<<<NBLK, 256, 0, ex.s>>>(G, sig, ring, G.nspec(), s, hist);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ext_advance(ExtHist* hist, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ext_advance<<<1, 32, 0, ex.s>>>(hist);
  ex.end();
  return cudaGetLastError();
}
cudaError_t launch_ext_keep(ExtHist* hist, const int* flag, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_ext_keep<<<1, 32, 0, ex.s>>>(hist, flag);
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
                                      const int*, double*, unsigned*, const Exec&, const int*,              \
                                      const double*);                                                      \
  template cudaError_t launch_cgs_update<T>(const Geom&, const cpx<T>*, size_t, int, const double*, cpx<T>*, \
                                            double*, const int*, GmresDev*, int, int, unsigned*,            \
                                            GmresReadback*, const int*, const Exec&, const int*,            \
                                            const GraphCtl*, bool);                                         \
  template cudaError_t launch_residual<T>(const Geom&, const cpx<T>*, const cpx<T>*, cpx<T>*, double*,       \
                                          const Exec&);                                                     \
  template cudaError_t launch_zero<T>(const Geom&, cpx<T>*, const Exec&, const int*);                       \
  template cudaError_t launch_axpby<T>(const Geom&, double, const cpx<T>*, double, cpx<T>*, const Exec&,     \
                                       const int*, const int*);                                               \
  template cudaError_t launch_copy_gated<T>(const Geom&, const cpx<T>*, cpx<T>*, const int*, const Exec&);

SGN_KRYLOV_INST(double)
SGN_KRYLOV_INST(float)
template cudaError_t launch_scale<double, double>(const Geom&, const cpx<double>*, const double*, bool,
                                                  cpx<double>*, const Exec&, const int*, size_t);
template cudaError_t launch_scale<double, float>(const Geom&, const cpx<double>*, const double*, bool,
                                                 cpx<float>*, const Exec&, const int*, size_t);
template cudaError_t launch_scale<float, float>(const Geom&, const cpx<float>*, const double*, bool,
                                                cpx<float>*, const Exec&, const int*, size_t);
template cudaError_t launch_axpy_multi<double, double>(const Geom&, const cpx<double>*, size_t, int,
                                                       const double*, cpx<double>*, const Exec&, const int*,
                                                       const double*);
template cudaError_t launch_axpy_multi<float, double>(const Geom&, const cpx<float>*, size_t, int,
                                                      const double*, cpx<double>*, const Exec&, const int*,
                                                      const double*);

}  // namespace sgn
