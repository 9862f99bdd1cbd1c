// sgn_krylov.cu - GMRES building blocks on spectral vectors (Section 3;
// Saad & Schultz's GMRES with left preconditioning).
//
// Krylov vectors are half spectra [Ny][ldS] of real fields. Their inner
// product is the Parseval-weighted sum  <a, b> = sum w(kx) Re(conj(a) b),
// w = 1 on the kx = 0 and kx = Nx/2 columns and 2 elsewhere, which equals
// Nx*Ny times the Euclidean inner product of the physical fields; relative
// residuals are therefore the same as for unknowns in physical space.
//
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): one pass
// forms all dot products, and each update pass w -= sum h_i V_i also forms the
// dot products (or the norm) of the updated vector in the same sweep. All
// reductions accumulate in FP64, per block with warp shuffles, then over the
// RED_BLOCKS block partials in a fixed order (deterministic).
#include <math.h>

#include "sgn_internal.h"

namespace sgn {

__device__ __forceinline__ double col_weight_k(const Geom& G, int col) {
  return (col == 0 || col == (G.Nx >> 1)) ? 1.0 : 2.0;
}

template <typename T>
__device__ __forceinline__ double wdot(cpx<T> a, cpx<T> b) {
  return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}

// Sum v over the block into red (one slot per warp); result valid on thread 0.
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

// partials[i * RED_BLOCKS + block] = sum over the block's rows of <V_i, w>
template <typename T>
__global__ void __launch_bounds__(256) k_dots(Geom G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                                              double* partials) {
  __shared__ double red[32];
  double acc[MAXV];
#pragma unroll
  for (int i = 0; i < MAXV; ++i) acc[i] = 0.0;
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x) {
    for (int col = threadIdx.x; col < G.Nxh; col += blockDim.x) {
      const size_t e = (size_t)row * G.ldS + col;
      const double wt = col_weight_k(G, col);
      const cpx<T> we = w[e];
#pragma unroll
      for (int i = 0; i < MAXV; ++i)
        if (i < nv) acc[i] += wt * wdot(V[i * vstride + e], we);
    }
  }
#pragma unroll
  for (int i = 0; i < MAXV; ++i) {
    if (i < nv) {
      const double tot = block_reduce(acc[i], red);
      if (threadIdx.x == 0) partials[(size_t)i * RED_BLOCKS + blockIdx.x] = tot;
    }
  }
}

// w -= sum_i coef[i] V_i, then either the dots <V_i, w_new> (i < nv) and
// |w_new|^2 (slot nv), or only |w_new|^2 (slot 0).
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_update(Geom G, const cpx<T>* V, size_t vstride, int nv,
                                                    const double* __restrict__ coef, cpx<T>* w, double* partials,
                                                    int want_dots) {
  __shared__ double red[32];
  __shared__ double cf[MAXV];
  if (threadIdx.x < MAXV) cf[threadIdx.x] = threadIdx.x < nv ? coef[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[MAXV + 1];
#pragma unroll
  for (int i = 0; i <= MAXV; ++i) acc[i] = 0.0;
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x) {
    for (int col = threadIdx.x; col < G.Nxh; col += blockDim.x) {
      const size_t e = (size_t)row * G.ldS + col;
      const double wt = col_weight_k(G, col);
      double zx = (double)w[e].x, zy = (double)w[e].y;
#pragma unroll
      for (int i = 0; i < MAXV; ++i) {
        if (i < nv) {
          const cpx<T> v = V[i * vstride + e];
          zx -= cf[i] * (double)v.x;
          zy -= cf[i] * (double)v.y;
        }
      }
      const cpx<T> z = mk((T)zx, (T)zy);
      w[e] = z;
      if (want_dots) {
#pragma unroll
        for (int i = 0; i < MAXV; ++i)
          if (i < nv) acc[i] += wt * wdot(V[i * vstride + e], z);
      }
      acc[MAXV] += wt * wdot(z, z);
    }
  }
  if (want_dots) {
#pragma unroll
    for (int i = 0; i < MAXV; ++i) {
      if (i < nv) {
        const double tot = block_reduce(acc[i], red);
        if (threadIdx.x == 0) partials[(size_t)i * RED_BLOCKS + blockIdx.x] = tot;
      }
    }
  }
  const double tot = block_reduce(acc[MAXV], red);
  if (threadIdx.x == 0) partials[(size_t)(want_dots ? nv : 0) * RED_BLOCKS + blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(Geom G, const cpx<T>* c, const cpx<T>* w, cpx<T>* r,
                                                  double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x) {
    for (int col = threadIdx.x; col < G.Nxh; col += blockDim.x) {
      const size_t e = (size_t)row * G.ldS + col;
      const cpx<T> z = c[e] - w[e];
      r[e] = z;
      acc += col_weight_k(G, col) * wdot(z, z);
    }
  }
  const double tot = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scale(Geom G, const cpx<T>* x, const double* factor, int invert, cpx<T>* y) {
  const double f0 = *factor;
  const T f = (T)(invert ? 1.0 / f0 : f0);
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x)
    for (int col = threadIdx.x; col < G.Nxh; col += blockDim.x) {
      const size_t e = (size_t)row * G.ldS + col;
      y[e] = scl(x[e], f);
    }
}

template <typename T>
__global__ void k_axpy_multi(Geom G, const cpx<T>* V, size_t vstride, int nv, const double* __restrict__ coef,
                             cpx<T>* x) {
  __shared__ double cf[MAXV];
  if (threadIdx.x < MAXV) cf[threadIdx.x] = threadIdx.x < nv ? coef[threadIdx.x] : 0.0;
  __syncthreads();
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x)
    for (int col = threadIdx.x; col < G.Nxh; col += blockDim.x) {
      const size_t e = (size_t)row * G.ldS + col;
      double zx = (double)x[e].x, zy = (double)x[e].y;
      for (int i = 0; i < nv; ++i) {
        const cpx<T> v = V[i * vstride + e];
        zx += cf[i] * (double)v.x;
        zy += cf[i] * (double)v.y;
      }
      x[e] = mk((T)zx, (T)zy);
    }
}

template <typename T>
__global__ void k_zero(Geom G, cpx<T>* x) {
  for (int row = blockIdx.x; row < G.Ny; row += gridDim.x)
    for (int col = threadIdx.x; col < G.ldS; col += blockDim.x) x[(size_t)row * G.ldS + col] = mk((T)0, (T)0);
}

// out[i] = sum_b partials[i*RED_BLOCKS + b] (fixed order), i < n
__global__ void k_reduce(const double* partials, int n, double* out, int sqrt_out) {
  __shared__ double red[32];
  for (int i = 0; i < n; ++i) {
    double v = 0.0;
    for (int b = threadIdx.x; b < RED_BLOCKS; b += blockDim.x) v += partials[(size_t)i * RED_BLOCKS + b];
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
}

// Column j of the Hessenberg matrix from the two CGS passes and the norm,
// previous rotations applied, new rotation zeroing H[j+1][j], residual
// estimate |g_{j+1}|.
__global__ void k_givens(GmresDev* st, int j, GmresReadback* rb, const int* flags) {
  if (threadIdx.x != 0) return;
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

// partials[q*RED_BLOCKS + b], q = mass, px, py, energy (Section 2.3)
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
    if (threadIdx.x == 0) partials[(size_t)q * RED_BLOCKS + blockIdx.x] = tot;
  }
}

// ------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_dots(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                        double* partials, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_dots<T><<<RED_BLOCKS, 256, 0, ex.s>>>(G, V, vstride, nv, w, partials);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cgs_update(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const double* coef,
                              cpx<T>* w, double* partials, bool want_dots, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_cgs_update<T><<<RED_BLOCKS, 256, 0, ex.s>>>(G, V, vstride, nv, coef, w, partials, want_dots ? 1 : 0);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_residual(const Geom& G, const cpx<T>* c, const cpx<T>* w, cpx<T>* r, double* partials,
                            const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_residual<T><<<RED_BLOCKS, 256, 0, ex.s>>>(G, c, w, r, partials);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale(const Geom& G, const cpx<T>* x, const double* factor, bool invert, cpx<T>* y,
                         const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_scale<T><<<RED_BLOCKS * 2, 256, 0, ex.s>>>(G, x, factor, invert ? 1 : 0, y);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_axpy_multi(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const double* coef,
                              cpx<T>* x, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_axpy_multi<T><<<RED_BLOCKS * 2, 256, 0, ex.s>>>(G, V, vstride, nv, coef, x);
  ex.end();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_zero(const Geom& G, cpx<T>* x, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_zero<T><<<RED_BLOCKS * 2, 256, 0, ex.s>>>(G, x);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partials, int n, double* out, bool sqrt_out, const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_reduce<<<1, 256, 0, ex.s>>>(partials, n, out, sqrt_out ? 1 : 0);
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
  k_invariant_sums<<<RED_BLOCKS, 256, 0, ex.s>>>(G, h, vx, vy, sig, sx, sy, g, partials);
  ex.end();
  return cudaGetLastError();
}

#define SGN_KRYLOV_INST(T)                                                                                   \
  template cudaError_t launch_dots<T>(const Geom&, const cpx<T>*, size_t, int, const cpx<T>*, double*,       \
                                      const Exec&);                                                         \
  template cudaError_t launch_cgs_update<T>(const Geom&, const cpx<T>*, size_t, int, const double*, cpx<T>*, \
                                            double*, bool, const Exec&);                                    \
  template cudaError_t launch_residual<T>(const Geom&, const cpx<T>*, const cpx<T>*, cpx<T>*, double*,       \
                                          const Exec&);                                                     \
  template cudaError_t launch_scale<T>(const Geom&, const cpx<T>*, const double*, bool, cpx<T>*,            \
                                       const Exec&);                                                        \
  template cudaError_t launch_axpy_multi<T>(const Geom&, const cpx<T>*, size_t, int, const double*, cpx<T>*, \
                                            const Exec&);                                                   \
  template cudaError_t launch_zero<T>(const Geom&, cpx<T>*, const Exec&);

SGN_KRYLOV_INST(double)

}  // namespace sgn
