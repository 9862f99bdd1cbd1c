// sgn_diag.cu - the monitoring quantities of the paper's experiments.
//
// Sections 4.1 and 4.2 test line solitary waves against transverse
// perturbations by the L-infinity norm of h and where it is reached, by the speed of the
// solitary wave of Eq. (sol) with that crest, and by the difference between
// the computed state and that solitary wave; Section 3 reads resolution from
// the decay of the DFT coefficients. Each quantity is a grid-wide max: one
// sweep, per-block results, and the last block to finish combines them in a
// fixed order (max and the lowest index of a tie are order-free anyway).
#include <math.h>

#include "sgn_internal.h"
#include "vec_common.cuh"

namespace sgn {

namespace {

constexpr int DIAG_THREADS = 256;

// (value, index) order of the crest search: larger value first, NaN above
// every number, the lower flat index on ties
__device__ __forceinline__ bool crest_before(double a, long long ia, double b, long long ib) {
  const bool na = a != a, nb = b != b;
  if (na != nb) return na;
  if (na) return ia < ib;
  return a > b || (a == b && ia < ib);
}

// max that keeps a NaN
__device__ __forceinline__ double nanmax(double a, double b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

__device__ __forceinline__ void warp_crest(double& v, long long& i) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (crest_before(v2, i2, v, i)) {
      v = v2;
      i = i2;
    }
  }
}

__device__ __forceinline__ double warp_nanmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block max of K values (thread 0 returns them in m)
template <int K>
__device__ __forceinline__ void block_nanmax(double (&m)[K], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) m[k] = warp_nanmax(m[k]);
  if (lane == 0)
    for (int k = 0; k < K; ++k) red[k * 32 + wid] = m[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < K; ++k) {
      double t = red[k * 32];
      for (int w = 1; w < nw; ++w) t = nanmax(t, red[k * 32 + w]);
      m[k] = t;
    }
  __syncthreads();
}

// x coordinate of column j, as the grid is defined (x_j = -L/2 + L j / N)
__device__ __forceinline__ double xcoord(const Geom& G, int j) { return -0.5 * G.Lx + G.Lx * (double)j / (double)G.Nx; }

}  // namespace

// partials: [0, NBLK) crest values, [NBLK, 2 NBLK) their indices (exact in a
// double below 2^53), [2 NBLK, 3 NBLK) max |vy|
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_max(Geom G, const double* __restrict__ h,
                                                           const double* __restrict__ vy, double* partials,
                                                           unsigned* counter, DiagDev* d) {
  __shared__ double rv[32], rvy[32];
  __shared__ long long ri[32];
  const size_t n = G.nphys();
  double best = -INFINITY, my = 0.0;
  long long bi = (long long)n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double v = h[e];
    if (crest_before(v, (long long)e, best, bi)) {
      best = v;
      bi = (long long)e;
    }
    my = nanmax(my, fabs(vy[e]));
  }
  warp_crest(best, bi);
  my = warp_nanmax(my);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    rv[wid] = best;
    ri[wid] = bi;
    rvy[wid] = my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      if (crest_before(rv[w], ri[w], best, bi)) {
        best = rv[w];
        bi = ri[w];
      }
      my = nanmax(my, rvy[w]);
    }
    partials[blockIdx.x] = best;
    partials[NBLK + blockIdx.x] = (double)bi;
    partials[2 * NBLK + blockIdx.x] = my;
  }
  if (last_block(counter, threadIdx.x == 0) && threadIdx.x == 0) {
    double b = __ldcg(partials);
    long long ib = (long long)__ldcg(partials + NBLK);
    double m = __ldcg(partials + 2 * NBLK);
    for (int k = 1; k < (int)gridDim.x; ++k) {
      const double v = __ldcg(partials + k);
      const long long iv = (long long)__ldcg(partials + NBLK + k);
      if (crest_before(v, iv, b, ib)) {
        b = v;
        ib = iv;
      }
      m = nanmax(m, __ldcg(partials + 2 * NBLK + k));
    }
    d->h_max = b;
    d->i_max = ib;
    d->max_vy = m;
  }
}

// Line solitary wave of Eq. (sol), h_inf = 1, crest 1 + a at xi = 0:
//   h = 1 + a sech^2(kappa xi), kappa^2 = 3a / (4 (1 + a)), c^2 = g (1 + a),
//   v = c - (c/h) (1 + (h^2)''/6),  (h^2)'' = 2 (h'^2 + h h'').
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_soliton(Geom G, const double* __restrict__ h,
                                                               const double* __restrict__ vx, double g,
                                                               double* partials, unsigned* counter, DiagDev* d) {
  __shared__ double red[2 * 32];
  const double hm = d->h_max;
  const int js = (int)(d->i_max % G.Nx);
  const double xs = xcoord(G, js);
  const double a = hm - 1.0;
  const double c = sqrt(g * hm);
  const double kap = sqrt(3.0 * a / (4.0 * hm));
  const bool ok = a > 0.0;
  const size_t n = G.nphys();
  double m[2] = {0.0, 0.0};
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % (size_t)G.Nx);
    double xi = xcoord(G, j) - xs;
    if (xi >= 0.5 * G.Lx) xi -= G.Lx;
    if (xi < -0.5 * G.Lx) xi += G.Lx;
    const double T = tanh(kap * xi);
    const double S = 1.0 - T * T;
    const double S1 = -2.0 * kap * S * T;
    const double S2 = kap * kap * (4.0 * S - 6.0 * S * S);
    const double hc = 1.0 + a * S;
    const double h1 = a * S1, h2 = a * S2;
    const double q2 = 2.0 * (h1 * h1 + hc * h2);
    const double vc = c - (c / hc) * (1.0 + q2 / 6.0);
    m[0] = nanmax(m[0], fabs(h[e] - hc));
    m[1] = nanmax(m[1], fabs(vx[e] - vc));
  }
  block_nanmax<2>(m, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = m[0];
    partials[NBLK + blockIdx.x] = m[1];
  }
  if (last_block(counter, threadIdx.x == 0) && threadIdx.x == 0) {
    double r0 = __ldcg(partials), r1 = __ldcg(partials + NBLK);
    for (int k = 1; k < (int)gridDim.x; ++k) {
      r0 = nanmax(r0, __ldcg(partials + k));
      r1 = nanmax(r1, __ldcg(partials + NBLK + k));
    }
    d->dev_h = ok ? r0 : __longlong_as_double(0x7ff8000000000000ll);
    d->dev_vx = ok ? r1 : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Outer band of the half spectrum: column m_x = col (0..Nx/2, standing also
// for -m_x), row m_y = row or row - Ny; in the band when 16|m| >= 7N in x or y.
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_tail(Geom G, const cpx<double>* __restrict__ s0,
                                                            const cpx<double>* __restrict__ s1,
                                                            const cpx<double>* __restrict__ s2, double* partials,
                                                            unsigned* counter, DiagDev* d) {
  __shared__ double red[3 * 32];
  double m[3] = {0.0, 0.0, 0.0};
  for (Walk it(G); it.ok(); it.next()) {
    if (it.col >= G.Nxh) continue;
    const int my = it.row <= (G.Ny >> 1) ? it.row : G.Ny - it.row;
    if (!(16 * it.col >= 7 * G.Nx || 16 * my >= 7 * G.Ny)) continue;
    const cpx<double> a = s0[it.e], b = s1[it.e], c = s2[it.e];
    m[0] = nanmax(m[0], hypot(a.x, a.y));
    m[1] = nanmax(m[1], hypot(b.x, b.y));
    m[2] = nanmax(m[2], hypot(c.x, c.y));
  }
  block_nanmax<3>(m, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) partials[k * NBLK + blockIdx.x] = m[k];
  if (last_block(counter, threadIdx.x == 0) && threadIdx.x == 0) {
    const double inv = 1.0 / (double)G.nphys();
    for (int k = 0; k < 3; ++k) {
      double r = __ldcg(partials + k * NBLK);
      for (int b = 1; b < (int)gridDim.x; ++b) r = nanmax(r, __ldcg(partials + k * NBLK + b));
      d->tail[k] = r * inv;
    }
  }
}

cudaError_t launch_diag_max(const Geom& G, const double* h, const double* vy, double* partials, unsigned* counter,
                            DiagDev* d, const Exec& ex) {
  ex.begin(PK_IO);
  k_diag_max<<<NBLK, DIAG_THREADS, 0, ex.s>>>(G, h, vy, partials, counter, d);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_diag_soliton(const Geom& G, const double* h, const double* vx, double g, double* partials,
                                unsigned* counter, DiagDev* d, const Exec& ex) {
  ex.begin(PK_IO);
  k_diag_soliton<<<NBLK, DIAG_THREADS, 0, ex.s>>>(G, h, vx, g, partials, counter, d);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_diag_tail(const Geom& G, const cpx<double>* s0, const cpx<double>* s1, const cpx<double>* s2,
                             double* partials, unsigned* counter, DiagDev* d, const Exec& ex) {
  ex.begin(PK_IO);
  k_diag_tail<<<NBLK, DIAG_THREADS, 0, ex.s>>>(G, s0, s1, s2, partials, counter, d);
  ex.end();
  return cudaGetLastError();
}

}  // namespace sgn
