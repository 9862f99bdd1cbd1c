// sgn_noalloc.cu - sgn_elliptic_apply without any device allocation.
//
// Some callers cannot allocate device memory: a host application whose own
// pool or caching allocator already holds the GPU's memory budget (a fresh
// cudaMalloc would fail, or would force that pool to release and re-reserve
// memory), a plugin inside a framework that must not allocate behind the
// framework's back, and latency-sensitive loops that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree. For them this file
// offers L[sigma] with every intermediate (twiddle and wavenumber tables, the
// coefficient fields, four half spectra) placed in one file-scope __device__
// array of SGN_NOALLOC_MAX_POINTS grid points' worth of storage (about 4 MB),
// which every GPU that loads the library holds until the process exits.
//
// The kernels are the ones sgn_elliptic_apply uses; only the buffers differ.
// In host code g_noalloc_scratch is a host-side stand-in, not a device
// address, so every call asks the runtime for the array's device address on
// the current device with cudaGetSymbolAddress (a table lookup once the
// module is loaded; the first call on a device loads it, which is why that
// first call should come before any stream capture). Nothing is cached on the
// host: calls from several host threads share no host state but the
// per-thread error message, and a context torn down by cudaDeviceReset leaves
// no stale address behind.
#include <math.h>
#include <stdio.h>

#include <string>

#include "sgn.h"
#include "sgn_internal.h"

using namespace sgn;

// message slot read by sgn_last_error(NULL), one per host thread
extern thread_local std::string g_create_error;

namespace {
constexpr size_t kScratchBytes = (size_t)4 << 20;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

sgn_status noalloc_fail(sgn_status st, const std::string& msg) {
  g_create_error = "sgn_elliptic_apply_noalloc: " + msg;
  return st;
}
}  // namespace

// Scratch shared by every call on a device; its contents persist between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Twiddles W_N^k = exp(-2 pi i k/N) in the staged layout of the transforms
// (entry i is W_N^staged_exponent(i)) and the wavenumbers (Nyquist set to 0).
__global__ void k_noalloc_tables(int Nx, int Ny, int lNx, int lNy, double Lx, double Ly, cpx<double>* twx,
                                 cpx<double>* twy, double* kx, double* ky) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double two_pi = 6.283185307179586476925286766559;
  double s = 0.0, c = 0.0;
  if (i < Nx) {
    const int k = staged_exponent(i, lNx);
    if (k >= 0) sincospi(2.0 * (double)k / (double)Nx, &s, &c);
    twx[i] = mk(c, -s);
  }
  if (i < Ny) {
    const int k = staged_exponent(i, lNy);
    s = c = 0.0;
    if (k >= 0) sincospi(2.0 * (double)k / (double)Ny, &s, &c);
    twy[i] = mk(c, -s);
    const int m = i < Ny / 2 ? i : i - Ny;
    ky[i] = (i == Ny / 2) ? 0.0 : two_pi * (double)m / Ly;
  }
  if (i <= Nx / 2) kx[i] = (i == Nx / 2) ? 0.0 : two_pi * (double)i / Lx;
}

extern "C" sgn_status sgn_elliptic_apply_noalloc(int Nx, int Ny, double Lx, double Ly, const double* h,
                                                 const double* sigma, double* out, void* cuda_stream) {
  if (!h || !sigma || !out) return noalloc_fail(SGN_EINVAL, "NULL field pointer");
  if (!is_pow2(Nx) || !is_pow2(Ny) || Nx < 8 || Ny < 8 || Nx > 4096 || Ny > 4096)
    return noalloc_fail(SGN_EINVAL, "Nx, Ny must be powers of two in [8, 4096]");
  if ((long long)Nx * Ny > SGN_NOALLOC_MAX_POINTS)
    return noalloc_fail(SGN_EINVAL, "grid of " + std::to_string(Nx) + " x " + std::to_string(Ny) +
                                        " points exceeds the allocation-free limit of " +
                                        std::to_string(SGN_NOALLOC_MAX_POINTS) + " points");
  if (!(Lx > 0.0) || !(Ly > 0.0) || !isfinite(Lx) || !isfinite(Ly))
    return noalloc_fail(SGN_EINVAL, "Lx, Ly must be positive and finite");

  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // the static array's address on the current device (looked up on every
  // call: no host-side cache to race on or to go stale)
  void* scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess || !scratch)
    return noalloc_fail(SGN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // the shared-memory opt-in of the transform kernels (per device; cheap to repeat)
  init_kernel_attributes<double>();

  Geom G{};
  G.Nx = Nx;
  G.Ny = Ny;
  G.lNx = log2i(Nx);
  G.lNy = log2i(Ny);
  G.Nxh = Nx / 2 + 1;
  G.ldS = G.Nxh;
  G.Lx = Lx;
  G.Ly = Ly;

  // carve the scratch: tables, coefficient fields, flags, four half spectra
  unsigned char* base = static_cast<unsigned char*>(scratch);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off = align256(off + bytes);
    return p;
  };
  Tables<double> tb{};
  tb.twx = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * Nx));
  tb.twy = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * Ny));
  tb.kx = reinterpret_cast<double*>(take(sizeof(double) * G.Nxh));
  tb.ky = reinterpret_cast<double*>(take(sizeof(double) * Ny));
  double* hh = reinterpret_cast<double*>(take(sizeof(double) * G.nphys()));
  double* cr = reinterpret_cast<double*>(take(sizeof(double) * G.nphys()));
  double* cc = reinterpret_cast<double*>(take(sizeof(double) * G.nphys()));
  int* flags = reinterpret_cast<int*>(take(sizeof(int)));
  cpx<double>* sig = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * G.nspec()));
  cpx<double>* w = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * G.nspec()));
  cpx<double>* tmp[2];
  tmp[0] = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * G.nspec()));
  tmp[1] = reinterpret_cast<cpx<double>*>(take(sizeof(cpx<double>) * G.nspec()));
  if (off > kScratchBytes) return noalloc_fail(SGN_EINVAL, "scratch layout exceeds the static array");

  const Exec ex{stream, nullptr};
  const int tn = (Nx > Ny ? Nx : Ny);
  k_noalloc_tables<<<(tn + 255) / 256, 256, 0, stream>>>(Nx, Ny, G.lNx, G.lNy, Lx, Ly, tb.twx, tb.twy, tb.kx,
                                                          tb.ky);
  e = cudaGetLastError();
  // the flags keep the previous call's value: clear them first
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = launch_coef_phys<double>(G, h, hh, cr, cc, flags, CoefCopy{}, ex);
  const double* fin[1] = {sigma};
  cpx<double>* sg[1] = {sig};
  if (e == cudaSuccess) e = launch_x_r2c<double>(G, tb, fin, 1, sg, ex);
  if (e == cudaSuccess) e = launch_y_fft<double>(G, tb, false, (const cpx<double>* const*)sg, nullptr, 1, sg, ex);
  if (e == cudaSuccess) e = launch_matvec<double>(G, tb, sig, cr, cc, w, tmp, false, ex);
  const cpx<double>* win[1] = {w};
  if (e == cudaSuccess) e = launch_y_fft<double>(G, tb, true, win, nullptr, 1, tmp, ex);
  double* o[1] = {out};
  if (e == cudaSuccess)
    e = launch_x_c2r<double>(G, tb, (const cpx<double>* const*)tmp, nullptr, 1, o, 1.0 / (double)G.nphys(), ex);
  int hflags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return noalloc_fail(SGN_ECUDA, cudaGetErrorString(e));
  if (hflags & FLAG_NONFINITE) return noalloc_fail(SGN_ENONFINITE, "non-finite depth h");
  if (hflags & FLAG_CAVITATION) return noalloc_fail(SGN_ECAVITATION, "cavitation: h <= 0 somewhere");
  return SGN_OK;
}
