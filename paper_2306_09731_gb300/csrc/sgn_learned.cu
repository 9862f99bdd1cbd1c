// sgn_learned.cu - the coarse-grid transfer of the learned GMRES start.
//
// The network of the learned start works on an n x n coarse grid. Its inputs
// are band-limited samples of fine fields, and its output goes back as the
// same Fourier modes of sigma's spectrum:
//   restriction  f_c[i] = (1/N) sum_{|m| < n/2} F[m] e^{2 pi i m.i / n}
//                (the fine field's low modes evaluated at every (N/n)-th
//                point; F the unnormalised DFT of the fine field, N = Nx Ny);
//   prolongation F[m] += s (N / n^2) sum_i f_c[i] e^{-2 pi i m.i / n}, |m| < n/2
//                (the band-limited field with samples s f_c).
// Both are separable truncated DFTs, done directly: O(n^3) work, about 1e6
// multiply-adds per field at n = 128, against ~1e9 of one solver matvec.
// FP32 arithmetic (the network itself is BF16) with FP64 fine spectra.
#include <math.h>

#include "sgn_internal.h"

namespace sgn {

namespace {

// e^{2 pi i t / n} for t < n
__global__ void k_coarse_twiddles(int n, float2* tw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  float s, c;
  sincospif(2.0f * (float)t / (float)n, &s, &c);
  tw[t] = make_float2(c, s);
}

__device__ __forceinline__ int band_row(int m, int Ny) { return m >= 0 ? m : Ny + m; }

// Y[f][iy][kx] = sum_{|m| < n/2} X_f[row(m)][kx] e^{2 pi i m iy / n}, kx < n/2
__global__ void k_restrict_y(Geom G, CoarseIn in, int n, const float2* __restrict__ tw, float2* Y) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y, f = blockIdx.z;
  if (kx >= n / 2) return;
  const cpx<double>* X = in.spec[f];
  float re = 0.f, im = 0.f;
  for (int m = -(n / 2 - 1); m <= n / 2 - 1; ++m) {
    const cpx<double> x = X[(size_t)band_row(m, G.Ny) * G.ldS + kx];
    const float2 w = tw[((m * iy) % n + n) % n];
    const float xr = (float)x.x, xi = (float)x.y;
    re += xr * w.x - xi * w.y;
    im += xr * w.y + xi * w.x;
  }
  Y[((size_t)f * n + iy) * (n / 2) + kx] = make_float2(re, im);
}

// out_f[iy][ix] = scale_f (1/N (Re Y[iy][0] + 2 sum_{kx=1}^{n/2-1} Re(Y[iy][kx] e^{2 pi i kx ix / n}))
//                           + shift_f)
__global__ void k_restrict_x(Geom G, CoarseIn in, int n, const float2* __restrict__ tw,
                             const float2* __restrict__ Y) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y, f = blockIdx.z;
  if (ix >= n) return;
  const float2* y = Y + ((size_t)f * n + iy) * (n / 2);
  float acc = 0.f;
  for (int kx = 1; kx < n / 2; ++kx) {
    const float2 v = y[kx], w = tw[(kx * ix) % n];
    acc += v.x * w.x - v.y * w.y;
  }
  const float val = (y[0].x + 2.f * acc) * (float)(1.0 / (double)G.nphys());
  in.out[f][(size_t)iy * n + ix] = in.scale[f] * (val + in.shift[f]);
}

// Z[iy][kx] = sum_ix fc[iy][ix] e^{-2 pi i kx ix / n}, kx < n/2
__global__ void k_prolong_x(const float* __restrict__ fc, int n, const float2* __restrict__ tw, float2* Z) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (kx >= n / 2) return;
  float re = 0.f, im = 0.f;
  for (int ix = 0; ix < n; ++ix) {
    const float v = fc[(size_t)iy * n + ix];
    const float2 w = tw[(kx * ix) % n];
    re += v * w.x;
    im -= v * w.y;
  }
  Z[(size_t)iy * (n / 2) + kx] = make_float2(re, im);
}

// X[row(m)][kx] += s (N / n^2) sum_iy Z[iy][kx] e^{-2 pi i m iy / n}, |m| < n/2
__global__ void k_prolong_y(Geom G, const float2* __restrict__ Z, int n, const float2* __restrict__ tw,
                            const double* scale, double sconst, const int* gate, cpx<double>* X) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, mi = blockIdx.y;  // m = mi - (n/2 - 1)
  if (kx >= n / 2 || (gate && *gate == 0)) return;
  const int m = mi - (n / 2 - 1);
  float re = 0.f, im = 0.f;
  for (int iy = 0; iy < n; ++iy) {
    const float2 z = Z[(size_t)iy * (n / 2) + kx];
    const float2 w = tw[((m * iy) % n + n) % n];
    // z * conj(w)
    re += z.x * w.x + z.y * w.y;
    im += z.y * w.x - z.x * w.y;
  }
  const double s = (scale ? *scale : 1.0) * sconst * (double)G.nphys() / ((double)n * (double)n);
  cpx<double>* x = X + (size_t)band_row(m, G.Ny) * G.ldS + kx;
  x->x += s * (double)re;
  x->y += s * (double)im;
}

}  // namespace

cudaError_t launch_coarse_twiddles(int n, float2* tw, const Exec& ex) {
  k_coarse_twiddles<<<(n + 127) / 128, 128, 0, ex.s>>>(n, tw);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Geom& G, const CoarseIn& in, int nf, int n, const float2* tw, float2* Y,
                            const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_restrict_y<<<dim3((n / 2 + 63) / 64, n, nf), 64, 0, ex.s>>>(G, in, n, tw, Y);
  ex.end();
  ex.begin(PK_KRYLOV);
  k_restrict_x<<<dim3((n + 63) / 64, n, nf), 64, 0, ex.s>>>(G, in, n, tw, Y);
  ex.end();
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(const Geom& G, const float* fc, int n, const float2* tw, float2* Z,
                               const double* scale, double sconst, cpx<double>* X, const Exec& ex,
                               const int* gate) {
  ex.begin(PK_KRYLOV);
  k_prolong_x<<<dim3((n / 2 + 63) / 64, n), 64, 0, ex.s>>>(fc, n, tw, Z);
  ex.end();
  ex.begin(PK_KRYLOV);
  k_prolong_y<<<dim3((n / 2 + 63) / 64, n - 1), 64, 0, ex.s>>>(G, Z, n, tw, scale, sconst, gate, X);
  ex.end();
  return cudaGetLastError();
}

}  // namespace sgn
