// sgn_internal.h - host-side interface between the C-ABI layer and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "dfloat.cuh"
#include "fft_core.cuh"

namespace sgn {

// Upper bound of the GMRES restart length (Krylov basis of MAXM+1 vectors).
constexpr int MAXM = 32;
constexpr int MAXV = MAXM + 1;
// Blocks of the vector and reduction kernels (8 per SM of a GB300's 152).
constexpr int NBLK = 1216;

// Grid geometry. Spectra are stored row-major [Ny][ldS] complex, row ky holds
// kx = 0..Nx/2 (R2C half storage along x); ldS >= Nxh.
struct Geom {
  int Nx, Ny, lNx, lNy, Nxh, ldS;
  double Lx, Ly;
  __host__ __device__ size_t nphys() const { return (size_t)Nx * Ny; }
  __host__ __device__ size_t nspec() const { return (size_t)Ny * ldS; }
};

// Device flags raised by the coefficient pass (OR-ed bits); FLAG_WAIT: a
// y-pass gave up waiting for its tensor copies (a bounded wait ran out).
enum : int { FLAG_CAVITATION = 1, FLAG_NONFINITE = 2, FLAG_WAIT = 4 };

// Launch shapes of the transform passes picked by sgn_autotune: threads per
// block of each pass, per arithmetic (0 = the built-in choice). A y-pass block
// of t threads transforms t / (Ny/8) columns, an x-pass block t / (Nx/8) row
// pairs; the shape changes no arithmetic, only how the work is tiled.
enum TunePass : int { TP_MV_YINV = 0, TP_MV_YFWD, TP_RHS_YINV, TP_RHS_YFWD, TP_MV_X, TP_RHS_X, TP_COUNT };
enum TuneType : int { TT_F32 = 0, TT_F64, TT_DFL, TT_COUNT };
struct Tune {
  int tpb[TT_COUNT][TP_COUNT];
  int plan[TT_COUNT][TP_COUNT];  // radix plan of each pass's transforms (0 or 1)
};
template <typename T>
constexpr int tune_type() {
  return sizeof(T) == 4 ? TT_F32 : (std::is_same<T, double>::value ? TT_F64 : TT_DFL);
}

// Tensor maps of the FP32 matvec y-passes (built when a handle is made):
// v: the Krylov basis as a [nvec][Ny][2 ldS] FP32 tensor, t0, t1: the two
// y-forward inputs as [1][Ny][2 ldS]; the boxes are [1][rows][2 C], C the
// columns of one block. ok = 0: the passes load their inputs with plain and
// cp.async loads instead.
struct MvTma {
  CUtensorMap v, t0, t1;
  const void* vbase;
  const void* t0base;
  const void* t1base;
  size_t vs;
  int nvec;
  int cinv, cfwd;  // columns per block the boxes were made for
  int ok;
  int* flags;
};
// Builds the maps for the basis V (nvec vectors) and tmp[0], tmp[1], for the
// y-pass shapes of tune (may be null: built-in shapes); returns false (ok = 0)
// if the driver's encoder is unavailable or refuses them.
bool make_mv_tma(const Geom& G, const void* V, int nvec, const void* t0, const void* t1, int* flags,
                 const Tune* tune, MvTma* out);
// Threads per block of a pass: the built-in choice and the candidates the
// autotuner tries (powers of two, whole columns or row pairs, within the
// kernel's launch bound), for arithmetic `type` (TuneType).
int pass_default_threads(const Geom& G, int type, int pass);
int pass_candidates(const Geom& G, int type, int pass, int* out, int max_out);

// Epilogue modes of the RHS y-forward pass (the RK4 stage update, Section 3).
enum RkMode : int {
  RK_STORE_K = 0,  // write K = (h_t, vx_t, vy_t) spectra
  RK_STAGE1 = 1,   // acc = K;       U_s = U_n + dt/2 K
  RK_STAGE2 = 2,   // acc += 2K;     U_s = U_n + dt/2 K
  RK_STAGE3 = 3,   // acc += 2K;     U_s = U_n + dt K
  RK_FINAL = 4     // U_n += dt/6 (acc + K), then the Krasny filter if on
};

// Per-precision device tables.
template <typename T>
struct Tables {
  cpx<T>* twx = nullptr;  // W_Nx^k, k < Nx
  cpx<T>* twy = nullptr;  // W_Ny^k, k < Ny
  T* kx = nullptr;        // 2 pi m / Lx, m = 0..Nx/2, Nyquist 0   [Nxh]
  T* ky = nullptr;        // 2 pi m / Ly, m = 0..Ny/2-1, -Ny/2..-1, Nyquist 0 [Ny]
  T* minv = nullptr;      // 1 / (3 + kx^2 + ky^2) per half-spectrum entry [Ny][ldS] (FP64, double-float)
};

// GMRES scalars that live on the device (Hessenberg, rotations, residual).
struct GmresDev {
  double H[(MAXM + 1) * MAXM];  // column-major, H[i + j*(MAXM+1)]
  double cs[MAXM], sn[MAXM], g[MAXM + 1], y[MAXM];
  double h1[MAXV + 1], h2[MAXV + 1];  // Gram-Schmidt passes; slot nv holds |w|^2
  // FP32 inner solve: basis vector i is stored unnormalised, V_i = vscl[i] X_i
  // (the orthogonalised vector of step i-1, written straight into its slot)
  double vscl[MAXV + 1];
  double nrm2;                // squared norm of the orthogonalised vector
  int reorth;                 // second pass needed (DGKS test)
  int pad_;
  double hnext, inv_hnext;    // H[j+1][j] and its inverse
  double res;                 // |g_{j+1}|
  // device-side control of graph mode (see GraphCtl): the solve's state and
  // counters that the host reads after a graph launch
  double cnorm, target, beta, res_in, inner_target;
  int j;             // next Arnoldi step of the current cycle
  int k;             // Arnoldi steps completed in the current cycle
  int its;           // matvecs of the current solve
  int conv;          // current solve converged
  int zero_sigma;    // right-hand side is zero: sigma = 0
  int have_s3;       // extrapolated start: sigma of stage 3 is available
  int notconv;       // some solve since the last reset missed the tolerance
  int sweeps;        // residual evaluations of the current solve
  int last_its, max_its;
  int pad2_;
  long long tot_its, tot_sweeps, tot_solves;
  double last_relres;
};

// Mixed precision (precision = 1): the inner FP32 GMRES stops once it has
// reduced its residual estimate by kInnerRel (below that the FP32 estimate
// stops tracking the true residual), and its estimate is trusted as the final
// FP64 residual only when kFp32Trust * beta, a bound on the gap between the
// FP32 estimate and the true residual for a sweep that started at residual
// beta, is below half the tolerance. Otherwise the next sweep recomputes the
// residual in FP64.
constexpr double kInnerRel = 1e-6;
constexpr double kFp32Trust = 1e-5;

// Constants and conditional-node handles of the graph-mode GMRES control.
struct GraphCtl {
  unsigned long long h_sweep;  // WHILE over restart cycles / refinement sweeps
  unsigned long long h_step;   // WHILE over the Arnoldi steps of a cycle
  double tol;
  int m, maxit, mixed, enabled;
};

// What the host reads back after each Arnoldi step.
struct GmresReadback {
  double res;
  double hnext;
  double scalar;  // generic scalar (a norm) for other sync points
  int flags;
  int pad;
};

// ------------------------------------------------------------ profiling
// Kernel classes timed with CUDA events when profiling is on.
enum ProfKind : int {
  PK_COEF = 0,     // y-inverse + x-pass of h (coefficients of Eq. (sigmav))
  PK_MV_YINV,      // matvec: y-inverse of sigma_hat, i ky sigma_hat
  PK_MV_X,         // matvec: fused x-pass
  PK_MV_YFWD,      // matvec: y-forward + preconditioner
  PK_RHS_YINV,     // RHS: y-inverse of vx, vy, sigma, i ky sigma
  PK_RHS_X,        // RHS: fused x-pass
  PK_RHS_YFWD,     // RHS: y-forward + RK4 update
  PK_KRYLOV,       // GMRES vector kernels and reductions
  PK_IO,           // physical <-> spectral conversions at call boundaries
  PK_REF_YINV,     // FP64 refinement matvec of precision 1: y-inverse
  PK_REF_X,        //   fused x-pass
  PK_REF_YFWD,     //   y-forward + M^-1
  PK_RK,           // RK4 stage update (flat, after the RHS y-forward)
  PK_COUNT
};

struct Prof {
  static constexpr int POOL = 512;
  bool on = false;
  bool ready = false;
  cudaEvent_t ev[2 * POOL];
  int kind[POOL];
  int n = 0;
  double ms[PK_COUNT] = {};
  long long cnt[PK_COUNT] = {};
  long long launches = 0;  // every kernel the library launched (profiling or not)

  void init() {
    if (ready) return;
    for (int i = 0; i < 2 * POOL; ++i) cudaEventCreate(&ev[i]);
    ready = true;
  }
  void destroy() {
    if (!ready) return;
    for (int i = 0; i < 2 * POOL; ++i) cudaEventDestroy(ev[i]);
    ready = false;
  }
  // accumulates every recorded pair; waits for the last one
  void harvest() {
    if (!ready || n == 0) return;
    cudaEventSynchronize(ev[2 * n - 1]);
    for (int i = 0; i < n; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
        ms[kind[i]] += t;
        cnt[kind[i]] += 1;
      }
    }
    n = 0;
  }
  void reset() {
    n = 0;
    for (int k = 0; k < PK_COUNT; ++k) {
      ms[k] = 0.0;
      cnt[k] = 0;
    }
    launches = 0;
  }
};

// Where and how a launcher enqueues: the stream, and the profiler (may be null).
struct Exec {
  cudaStream_t s;
  Prof* p;
  int kind_override = -1;  // time every launch of this call under one class
  bool refine = false;     // matvec passes count as the FP64 refinement classes
  const Tune* tune = nullptr;
  int tpb(int type, int pass) const { return tune ? tune->tpb[type][pass] : 0; }
  int plan(int type, int pass) const { return tune ? tune->plan[type][pass] : 0; }
  void begin(int k, int nlaunch = 1) const {
    if (!p) return;
    if (kind_override >= 0) k = kind_override;
    if (refine && k >= PK_MV_YINV && k <= PK_MV_YFWD) k += PK_REF_YINV - PK_MV_YINV;
    p->launches += nlaunch;
    if (!p->on || !p->ready) return;
    if (p->n == Prof::POOL) p->harvest();
    p->kind[p->n] = k;
    cudaEventRecord(p->ev[2 * p->n], s);
  }
  void end() const {
    if (!p || !p->on || !p->ready) return;
    cudaEventRecord(p->ev[2 * p->n + 1], s);
    p->n += 1;
  }
};

// ------------------------------------------------------------ launchers
// All launchers enqueue on ex.s and return cudaGetLastError().

template <typename T>
void init_kernel_attributes();

// physical rows -> x-spectral half rows (R2C along x), nf fields
template <typename T>
cudaError_t launch_x_r2c(const Geom& G, const Tables<T>& tb, const double* const* f, int nf,
                         cpx<T>* const* out, const Exec& ex);
// x-spectral half rows (times i kx if deriv) -> physical rows, times scale
template <typename T>
cudaError_t launch_x_c2r(const Geom& G, const Tables<T>& tb, const cpx<T>* const* in, const int* deriv,
                         int nf, double* const* out, double scale, const Exec& ex);
// column transforms of nf spectra (in place allowed); inverse may pre-multiply by i ky
template <typename T>
cudaError_t launch_y_fft(const Geom& G, const Tables<T>& tb, bool inverse, const cpx<T>* const* in,
                         const int* deriv, int nf, cpx<T>* const* out, const Exec& ex);

// Optional FP32 copies of the coefficient fields (all null: none written).
struct CoefCopy {
  float* h = nullptr;
  float* cr = nullptr;
  float* cc = nullptr;
};

// coefficient pass: from Hy = y-inverse of h_hat, write h - 1, cr = 0.5/(N h), cc = 1.5/(N h^3)
template <typename T>
cudaError_t launch_coef_x(const Geom& G, const Tables<T>& tb, const cpx<T>* Hy, T* h, T* cr, T* cc,
                          int* flags, const CoefCopy& cp, const Exec& ex);
// the same three arrays straight from a physical h (float64)
template <typename T>
cudaError_t launch_coef_phys(const Geom& G, const double* hphys, T* h, T* cr, T* cc, int* flags,
                             const CoefCopy& cp, const Exec& ex);

// matvec w = M^-1 L sigma (precond) or L sigma (!precond), spectral in/out.
// tmp: 4 spectra of scratch (S, Sy, C, By).
// jsel (may be null): the input is sig + (*jsel) * jstride (graph mode: the
// Arnoldi step index lives on the device)
// tma (may be null; FP32): tensor maps of V and tmp[0..1]; used when sig lies
// in V (sig = V + j vs, or V with jsel) and tmp is the maps' pair.
template <typename T>
cudaError_t launch_matvec(const Geom& G, const Tables<T>& tb, const cpx<T>* sig, const T* cr, const T* cc,
                          cpx<T>* w, cpx<T>* const* tmp, bool precond, const Exec& ex,
                          const int* jsel = nullptr, size_t jstride = 0, const MvTma* tma = nullptr);

// the same with sigma_hat and w stored in S and the passes in T (the
// double-float refinement matvec: T = dfl, S = double)
template <typename T, typename S>
cudaError_t launch_matvec_io(const Geom& G, const Tables<T>& tb, const cpx<S>* sig, const T* cr, const T* cc,
                             cpx<S>* w, cpx<T>* const* tmp, bool precond, const Exec& ex,
                             const int* jsel = nullptr, size_t jstride = 0);
// y-inverse of one FP64 half spectrum into the pass type T
template <typename T>
cudaError_t launch_y_inv64(const Geom& G, const Tables<T>& tb, const cpx<double>* in, cpx<T>* out, const Exec& ex);
// y-forward of one half spectrum of type T, stored as FP64
template <typename T>
cudaError_t launch_y_fwd64(const Geom& G, const Tables<T>& tb, const cpx<T>* in, cpx<double>* out, const Exec& ex);
void init_kernel_attributes_df();
// the part of it for precision 3's double-float right-hand side (its own unit)
void init_kernel_attributes_df_rhs();

// RHS of one stage from state U (3 spectra), sigma_hat, h, cr; K goes through
// the RK epilogue. tmp: 4 spectra. Writes b_hat of the next stage state.
struct RkArgs {
  int mode;
  double dt;
  int dealias;
  int krasny;
  double krasny_thr;
  double g;
};
// Arguments of the RK4 stage-update kernel.
template <typename T, typename S>
struct RkK {
  const cpx<T>* K[3];
  cpx<S>* Un[3];
  cpx<S>* Unext[3];
  cpx<S>* acc[3];
  cpx<S>* b;
  const S* kxs;
  const S* kys;
  // stage state and sigma_hat of the right-hand side (its linear part, added
  // by the update when the passes run in FP32)
  const cpx<S>* Y[3];
  const cpx<S>* sig;
  RkArgs rk;
};

// T: compute type of the passes (tmp, h, cr); S: storage type of the state,
// sigma_hat and b_hat (FP64 in both modes).
template <typename T, typename S>
cudaError_t launch_rhs(const Geom& G, const Tables<T>& tb, const Tables<S>& tbs, cpx<S>* const* U,
                       const cpx<S>* sig, const T* h, const T* cr, cpx<T>* const* tmp, cpx<S>* const* Un,
                       cpx<S>* const* Unext, cpx<S>* const* acc, cpx<S>* bhat, const RkArgs& rk,
                       const Exec& ex);

// b_hat = -(i kx vx_hat + i ky vy_hat)
template <typename T>
cudaError_t launch_spec_div(const Geom& G, const Tables<T>& tb, const cpx<T>* vx, const cpx<T>* vy,
                            cpx<T>* b, const Exec& ex);
// project the kx = 0 and kx = Nx/2 columns onto their Hermitian part (in place)
template <typename T>
cudaError_t launch_hermitian_fix(const Geom& G, cpx<T>* x, const Exec& ex);
// out = M^-1 in (spectral), and the weighted squared norm into partials
template <typename T>
cudaError_t launch_precond(const Geom& G, const Tables<T>& tb, const cpx<T>* in, cpx<T>* out,
                           double* partials, const Exec& ex);

// ---- Krylov vector kernels (spectral vectors, Parseval-weighted inner product)
// out[i] = <V_i, w> (i < nv) and out[nv] = |w|^2, reduced by the last block
// to finish; gate: run only if *gate != 0 (may be null). counter: a zeroed
// device word private to this call site (left zeroed).
// jdev (may be null): nv = *jdev + 1 read on the device (graph mode); nv is then
// the largest value it can take (for the grid size).
template <typename T>
cudaError_t launch_dots(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const cpx<T>* w,
                        double* partials, const int* gate, double* out, unsigned* counter, const Exec& ex,
                        const int* jdev = nullptr, const double* vscl = nullptr);
// Gram-Schmidt update w -= sum_i coef[i] V_i of Arnoldi step j; the last block
// stores |w'|^2, takes the DGKS decision (pass 1) and runs the Givens step once
// the orthogonalisation is final (pass 1 without reorthogonalisation, pass 2,
// or pass 3 = a single pass that never reorthogonalises).
// jdev (may be null): j and nv = j + 1 read on the device; ctl.enabled: after
// the Givens step the last block advances the graph-mode control (its, k, j,
// the Arnoldi loop condition).
template <typename T>
cudaError_t launch_cgs_update(const Geom& G, const cpx<T>* V, size_t vstride, int nv, const double* coef,
                              cpx<T>* w, double* partials, const int* gate, GmresDev* st, int j, int pass,
                              unsigned* counter, GmresReadback* rb, const int* flags, const Exec& ex,
                              const int* jdev = nullptr, const GraphCtl* ctl = nullptr, bool scaled = false);
// r = c - w, and partial squared norm of r
template <typename T>
cudaError_t launch_residual(const Geom& G, const cpx<T>* c, const cpx<T>* w, cpx<T>* r, double* partials,
                            const Exec& ex);
// y = x * f, f = *factor or 1 / *factor (device scalar); may change precision.
// ysel (may be null): y += (*ysel) * ystride (graph mode).
template <typename TI, typename TO>
cudaError_t launch_scale(const Geom& G, const cpx<TI>* x, const double* factor, bool invert, cpx<TO>* y,
                         const Exec& ex, const int* ysel = nullptr, size_t ystride = 0);
// x += sum_i coef[i] V_i (V in TV, x in TX); ndev (may be null): nv = *ndev
template <typename TV, typename TX>
cudaError_t launch_axpy_multi(const Geom& G, const cpx<TV>* V, size_t vstride, int nv, const double* coef,
                              cpx<TX>* x, const Exec& ex, const int* ndev = nullptr, const double* vscl = nullptr);
// x = 0; gate (may be null): only if *gate != 0
template <typename T>
cudaError_t launch_zero(const Geom& G, cpx<T>* x, const Exec& ex, const int* gate = nullptr);
// y = a x + b y; gate, gate2 (may be null): only if *gate != 0 and *gate2 != 0
template <typename T>
cudaError_t launch_axpby(const Geom& G, double a, const cpx<T>* x, double b, cpx<T>* y, const Exec& ex,
                         const int* gate = nullptr, const int* gate2 = nullptr);
// y = x over the spectral entries, only if *gate != 0 (gate not null)
template <typename T>
cudaError_t launch_copy_gated(const Geom& G, const cpx<T>* x, cpx<T>* y, const int* gate, const Exec& ex);

// reduce partials[b][0..n) over blocks into out[0..n); if sqrt_out, take sqrt
cudaError_t launch_reduce(const double* partials, int n, double* out, bool sqrt_out, const int* gate,
                          const Exec& ex);
// GMRES scalar kernels (one thread)
cudaError_t launch_gmres_start(GmresDev* st, const double* beta, const Exec& ex);
cudaError_t launch_backsolve(GmresDev* st, int k, const Exec& ex, const int* kdev = nullptr);
// graph-mode control kernels (one thread); see csrc/sgn_krylov.cu
cudaError_t launch_ctl_begin(GmresDev* st, const double* cnorm, GraphCtl ctl, const Exec& ex);
cudaError_t launch_ctl_sweep(GmresDev* st, const double* beta, GraphCtl ctl, const Exec& ex);
cudaError_t launch_ctl_after(GmresDev* st, GraphCtl ctl, const Exec& ex);
cudaError_t launch_set_int(int* p, int v, const Exec& ex);
// Polynomial start across steps (guess = 3): the ring holds each RK4 stage's
// solved sigma over the last 4 steps, slot (q, s) at ring + (4 q + s - 1) *
// nspec, q in 0..3, s in 1..4 (see sgn_krylov.cu).
struct ExtHist {
  int levels;  // steps held, 0..4
  int head;    // slot q of the step being taken
  int full;    // 1 while levels == 4 (the cubic start): the learned start's gate
  int lin;     // 1 while levels < 3: guess 2's linear start (and its copies) still apply
};
// sigma = the quadratic (levels 3) or cubic (levels 4) extrapolation of stage
// s from the ring; with fewer levels sigma is left as it is
cudaError_t launch_ext_start(const Geom& G, const cpx<double>* ring, int s, const ExtHist* hist, cpx<double>* sig,
                             const Exec& ex);
// ring slot (head, s) = sigma
cudaError_t launch_ext_store(const Geom& G, const cpx<double>* sig, cpx<double>* ring, int s, const ExtHist* hist,
                             const Exec& ex);
// after a step's last stage: head advances, levels += 1 (at most 4), full =
// (levels == 4), lin = (levels < 3)
cudaError_t launch_ext_advance(ExtHist* hist, const Exec& ex);
// levels = full = 0 and lin = 1 unless *flag
cudaError_t launch_ext_keep(ExtHist* hist, const int* flag, const Exec& ex);
// *flag = 1 if the three spectra b equal a within rel * max|a| (see sgn_krylov.cu)
cudaError_t launch_same_state(const Geom& G, const cpx<double>* const* a, const cpx<double>* const* b, double rel,
                              double* partials, unsigned* counter, int* flag, const Exec& ex);
cudaError_t launch_readback_scalar(const double* x, const int* flags, GmresReadback* rb_dev, const Exec& ex);

// invariants: physical pointwise sums (mass, px, py, energy) -> partials[4][NBLK]
cudaError_t launch_invariant_sums(const Geom& G, const double* h, const double* vx, const double* vy,
                                  const double* sig, const double* sx, const double* sy, double g,
                                  double* partials, const Exec& ex);

// ------------------------------------------------------------ diagnostics
// Device results of the monitoring pass (sgn_diagnostics).
struct DiagDev {
  double h_max;
  long long i_max;
  double max_vy;
  double dev_h, dev_vx;
  double tail[3];
};
// max of h with its lowest index and max |vy|; partials: 3 * NBLK doubles
cudaError_t launch_diag_max(const Geom& G, const double* h, const double* vy, double* partials, unsigned* counter,
                            DiagDev* d, const Exec& ex);
// deviation from the line solitary wave of speed sqrt(g h_max) at the crest
cudaError_t launch_diag_soliton(const Geom& G, const double* h, const double* vx, double g, double* partials,
                                unsigned* counter, DiagDev* d, const Exec& ex);
// outer-band maximum of three FP64 half spectra, divided by Nx Ny
cudaError_t launch_diag_tail(const Geom& G, const cpx<double>* s0, const cpx<double>* s1, const cpx<double>* s2,
                             double* partials, unsigned* counter, DiagDev* d, const Exec& ex);

// ------------------------------------------------------- learned start
// Restriction of up to 5 FP64 half spectra to n x n coarse samples:
// out[f] = scale[f] * (band-limited sample + shift[f]).
struct CoarseIn {
  const cpx<double>* spec[5];
  float* out[5];
  float scale[5];
  float shift[5];
};
// tw[t] = e^{2 pi i t / n}, t < n (FP32)
cudaError_t launch_coarse_twiddles(int n, float2* tw, const Exec& ex);
// Y: scratch of nf * n * n/2 float2
cudaError_t launch_restrict(const Geom& G, const CoarseIn& in, int nf, int n, const float2* tw, float2* Y,
                            const Exec& ex);
// X += (*scale if scale else 1) * sconst * prolongation(fc); Z: scratch n * n/2 float2;
// nothing is added when gate is set and *gate == 0
cudaError_t launch_prolong_add(const Geom& G, const float* fc, int n, const float2* tw, float2* Z,
                               const double* scale, double sconst, cpx<double>* X, const Exec& ex,
                               const int* gate = nullptr);

}  // namespace sgn
