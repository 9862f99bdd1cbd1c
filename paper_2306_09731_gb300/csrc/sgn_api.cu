// sgn_api.cu - C ABI (include/sgn.h) and host orchestration of the SGN hot path.
//
// The handle owns every device buffer. The RK4 state lives in spectral form
// (half spectra of h, vx, vy) between steps; sigma_hat is the GMRES warm start
// carried from stage to stage and step to step (Section 3: each solve
// starts from the previous solve's sigma; opt.guess 2 and 3 extrapolate it in
// time instead). One stage is:
//   coefficients  h, 1/(2N h), 3/(2N h^3) from h_hat        (y-inverse + x-pass)
//   GMRES         L sigma = b, b_hat = -(i kx vx + i ky vy) (Eq. (sigmav))
//   RHS + update  K = (h_t, v_t) and the RK4 stage update  (3 fused passes and
//                 the update, which adds K's linear part when the passes are FP32)
// By default the GMRES loop runs on the host: each Arnoldi step enqueues its
// kernels and reads back one residual estimate (one stream synchronisation per
// step). With opt.graph = 1 one RK4 step is a CUDA graph instead: the restart
// cycles and Arnoldi steps are conditional WHILE nodes, and one-thread control
// kernels take the host loop's decisions on the device.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "sgn.h"
#include "sgn_internal.h"
#include "sgn_unet.h"

using namespace sgn;

typedef cpx<double> C64;
typedef cpx<float> C32;
typedef cpx<dfl> CDF;


struct sgn_ctx {
  Geom G{};
  double g = 1.0;
  sgn_options opt{};
  cudaStream_t stream = 0;
  int device = 0;
  Tables<double> tb{};
  C64* Un[3] = {};
  C64* Us[3] = {};
  C64* acc[3] = {};
  C64* sig = nullptr;
  C64* bh = nullptr;
  C64* cvec = nullptr;
  C64* w = nullptr;
  C64* tmp[4] = {};
  C64* V = nullptr;
  double* h = nullptr;
  double* cr = nullptr;
  double* cc = nullptr;
  // mixed precision (precision = 1 and 2)
  Tables<float> tb32{};
  C32* V32 = nullptr;
  C32* w32 = nullptr;
  C32* tmp32[4] = {};
  float* h32 = nullptr;
  float* cr32 = nullptr;
  float* cc32 = nullptr;
  C64* r64 = nullptr;
  // precision 2: double-float tables and matvec coefficients
  Tables<dfl> tbd{};
  dfl* crd = nullptr;
  dfl* ccd = nullptr;
  dfl* hd = nullptr;  // precision 3: h - 1 in double-float for the RHS
  // extrapolated GMRES start (guess = 2): sigma of stage 1 of this step and
  // of stage 3 of the previous step, as half spectra
  C64* sig_s1 = nullptr;
  C64* sig_s3 = nullptr;
  bool have_s3 = false;
  // polynomial start across steps (guess = 3): 4 steps x 4 stages of sigma
  C64* ext_ring = nullptr;
  ExtHist* ext = nullptr;
  // The extrapolation history across calls: hist_ok after an RK4 call with
  // guess 2 or 3 (cleared by every other call), hist_keep its value when the
  // current call began, hist_dt that call's dt.
  bool hist_ok = false, hist_keep = false;
  double hist_dt = 0.0;
  double* phys[4] = {};  // staging for sgn_rk4_step_host / derivatives (lazy)
  double* partials = nullptr;
  double* scal = nullptr;  // small device scalars
  GmresDev* gst = nullptr;
  GmresReadback* rb_dev = nullptr;
  GmresReadback* rb_host = nullptr;  // pinned
  double* inv_host = nullptr;        // pinned, 4 doubles
  int* flags = nullptr;
  unsigned* counters = nullptr;  // last-block reduction tickets (zeroed, self-resetting)
  Prof prof;
  // graph mode (opt.graph = 1): one RK4 step as an instantiated graph
  cudaStream_t cap = nullptr;  // private stream the step is captured on
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  double graph_dt = 0.0;
  // kernels per step outside the loops, per restart cycle / sweep, per Arnoldi step
  long long graph_fixed = 0, graph_per_sweep = 0, graph_per_step = 0;
  GmresDev* gst_host = nullptr;  // pinned
  DiagDev* diag = nullptr;       // sgn_diagnostics results (lazy)
  // learned start (sgn_set_learned_guess)
  sgn_unet_t net = nullptr;
  int ln = 0;
  float in_scale[4] = {1.f, 1.f, 1.f, 1.f};
  float out_scale = 1.f;
  int tau_pow = 1;
  float2* ltw = nullptr;  // e^{2 pi i t / ln}
  float2* lY = nullptr;   // restriction / prolongation scratch
  float* lin = nullptr;   // network input [4][ln][ln]
  float* lout = nullptr;  // network output [ln][ln]
  // recording of training samples (sgn_record_learned)
  float* rec_buf = nullptr;
  int rec_n = 0, rec_cap = 0, rec_count = 0, rec_tau_pow = 1;
  bool rec_stage = false;  // the current stage is being recorded
  int ext_lv = 0;          // host copy of ext->levels in the host-driven loop
  float2* rtw = nullptr;
  float2* rY = nullptr;
  C64* sig_fb = nullptr;  // sigma_start of the recorded stage
  // sgn_coarse_sample / sgn_coarse_embed scratch
  int cn = 0;
  float2* ctw = nullptr;
  float2* cY = nullptr;
  DiagDev* diag_host = nullptr;  // pinned
  std::vector<cudaGraph_t> sweep_bodies, step_bodies;  // owned by their conditional nodes
  bool trace = false;  // SGN_TRACE=1: one stderr line per mixed-precision sweep
  // tensor maps of the FP32 matvec y-passes (precisions 1, 2); SGN_TMA=0
  // loads their inputs with plain and cp.async loads instead
  MvTma mvt{};
  // sgn_rk4_step_host: copy stream and its events (made on first use)
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev[9] = {};
  Tune tune{};  // launch shapes picked by sgn_autotune (0: built-in)
  std::vector<void*> allocs;
  std::string err;
  sgn_stats stats{};
};

// message of the last failing handle-less call (sgn_create, sgn_elliptic_apply_noalloc),
// one per host thread, like errno
thread_local std::string g_create_error;

namespace {

struct Fail {
  sgn_status st;
};

#define CK(...)                                                                                   \
  do {                                                                                            \
    cudaError_t e_ = (__VA_ARGS__);                                                               \
    if (e_ != cudaSuccess) {                                                                      \
      ctx->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);                       \
      throw Fail{SGN_ECUDA};                                                                      \
    }                                                                                             \
  } while (0)

sgn_status fail(sgn_ctx* ctx, sgn_status st, const std::string& msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_create_error = msg;
  return st;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// cos and sin of 2 pi k / n by reduction to the first octant (n power of 2).
void cos_sin_2pi(long k, long n, double* c, double* s) {
  k %= n;
  if (k < 0) k += n;
  const long q = k / (n / 4), kr = k % (n / 4);
  const double two_pi = 6.283185307179586476925286766559;
  double c0, s0;
  if (kr <= n / 8) {
    c0 = cos(two_pi * (double)kr / (double)n);
    s0 = sin(two_pi * (double)kr / (double)n);
  } else {
    const long m = n / 4 - kr;
    c0 = sin(two_pi * (double)m / (double)n);
    s0 = cos(two_pi * (double)m / (double)n);
  }
  switch (q) {
    case 0: *c = c0; *s = s0; break;
    case 1: *c = -s0; *s = c0; break;
    case 2: *c = -c0; *s = -s0; break;
    default: *c = s0; *s = -c0; break;
  }
}

// Every device buffer starts zeroed, so the padding column of the spectra is
// zero in every buffer that no pass writes there.
template <typename P>
P* dalloc(sgn_ctx* ctx, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(P));
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    throw Fail{SGN_ENOMEM};
  }
  ctx->allocs.push_back(p);
  e = cudaMemset(p, 0, count * sizeof(P));
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string("cudaMemset: ") + cudaGetErrorString(e);
    throw Fail{SGN_ECUDA};
  }
  return static_cast<P*>(p);
}

void free_graph(sgn_ctx* ctx) {
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  ctx->sweep_bodies.clear();
  ctx->step_bodies.clear();
}

void free_all(sgn_ctx* ctx) {
  free_graph(ctx);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  ctx->cap = nullptr;
  if (ctx->io_stream) {
    cudaStreamSynchronize(ctx->io_stream);
    cudaStreamDestroy(ctx->io_stream);
    for (int i = 0; i < 9; ++i)
      if (ctx->io_ev[i]) cudaEventDestroy(ctx->io_ev[i]);
  }
  ctx->io_stream = nullptr;
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  if (ctx->rb_host) cudaFreeHost(ctx->rb_host);
  if (ctx->inv_host) cudaFreeHost(ctx->inv_host);
  if (ctx->gst_host) cudaFreeHost(ctx->gst_host);
  if (ctx->diag_host) cudaFreeHost(ctx->diag_host);
  ctx->diag_host = nullptr;
  ctx->rb_host = nullptr;
  ctx->inv_host = nullptr;
  ctx->gst_host = nullptr;
}

// W_N^k = exp(-2 pi i k/N) in the staged layout of the transforms: entry i
// of [0, N) holds W_N^staged_exponent(i) for radix plan 0, entry N + i that
// of plan 1 (unused entries are zero)
std::vector<C64> staged_twiddles(int N, int lN) {
  std::vector<C64> t(2 * (size_t)N);
  for (int plan = 0; plan < 2; ++plan)
    for (int i = 0; i < N; ++i) {
      const int k = staged_exponent(i, lN, plan);
      double c = 0.0, s = 0.0;
      if (k >= 0) cos_sin_2pi(k, N, &c, &s);
      t[(size_t)plan * N + i].x = c;
      t[(size_t)plan * N + i].y = -s;
    }
  return t;
}

void build_tables(sgn_ctx* ctx) {
  const Geom& G = ctx->G;
  const std::vector<C64> tx = staged_twiddles(G.Nx, G.lNx), ty = staged_twiddles(G.Ny, G.lNy);
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> kx(G.Nxh), ky(G.Ny);
  for (int k = 0; k < G.Nxh; ++k) kx[k] = (k == G.Nx / 2) ? 0.0 : two_pi * k / G.Lx;
  for (int k = 0; k < G.Ny; ++k) {
    const int m = k < G.Ny / 2 ? k : k - G.Ny;
    ky[k] = (k == G.Ny / 2) ? 0.0 : two_pi * m / G.Ly;
  }
  // M^-1 = 1/(3 + kx^2 + ky^2) for the FP64 passes (Section 3 preconditioner)
  std::vector<double> minv((size_t)G.Ny * G.ldS, 0.0);
  for (int r = 0; r < G.Ny; ++r)
    for (int c = 0; c < G.Nxh; ++c) minv[(size_t)r * G.ldS + c] = 1.0 / (3.0 + kx[c] * kx[c] + ky[r] * ky[r]);
  ctx->tb.minv = dalloc<double>(ctx, minv.size());
  CK(cudaMemcpy(ctx->tb.minv, minv.data(), minv.size() * sizeof(double), cudaMemcpyHostToDevice));
  ctx->tb.twx = dalloc<C64>(ctx, 2 * (size_t)G.Nx);
  ctx->tb.twy = dalloc<C64>(ctx, 2 * (size_t)G.Ny);
  ctx->tb.kx = dalloc<double>(ctx, G.Nxh);
  ctx->tb.ky = dalloc<double>(ctx, G.Ny);
  CK(cudaMemcpy(ctx->tb.twx, tx.data(), tx.size() * sizeof(C64), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->tb.twy, ty.data(), ty.size() * sizeof(C64), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->tb.kx, kx.data(), G.Nxh * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->tb.ky, ky.data(), G.Ny * sizeof(double), cudaMemcpyHostToDevice));
  if (ctx->opt.precision >= 2) {
    // double-float copies: nearest FP32 pair of each FP64 entry
    std::vector<CDF> dx(tx.size()), dy(ty.size());
    for (size_t k = 0; k < tx.size(); ++k) dx[k] = CDF{dfl(tx[k].x), dfl(tx[k].y)};
    for (size_t k = 0; k < ty.size(); ++k) dy[k] = CDF{dfl(ty[k].x), dfl(ty[k].y)};
    std::vector<dfl> kxd(kx.begin(), kx.end()), kyd(ky.begin(), ky.end()), md(minv.begin(), minv.end());
    ctx->tbd.twx = dalloc<CDF>(ctx, dx.size());
    ctx->tbd.twy = dalloc<CDF>(ctx, dy.size());
    ctx->tbd.kx = dalloc<dfl>(ctx, G.Nxh);
    ctx->tbd.ky = dalloc<dfl>(ctx, G.Ny);
    ctx->tbd.minv = dalloc<dfl>(ctx, md.size());
    CK(cudaMemcpy(ctx->tbd.twx, dx.data(), dx.size() * sizeof(CDF), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tbd.twy, dy.data(), dy.size() * sizeof(CDF), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tbd.kx, kxd.data(), G.Nxh * sizeof(dfl), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tbd.ky, kyd.data(), G.Ny * sizeof(dfl), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tbd.minv, md.data(), md.size() * sizeof(dfl), cudaMemcpyHostToDevice));
  }
  if (ctx->opt.precision >= 1) {
    std::vector<C32> fx(tx.size()), fy(ty.size());
    for (size_t k = 0; k < tx.size(); ++k) fx[k] = C32{(float)tx[k].x, (float)tx[k].y};
    for (size_t k = 0; k < ty.size(); ++k) fy[k] = C32{(float)ty[k].x, (float)ty[k].y};
    std::vector<float> kxf(kx.begin(), kx.end()), kyf(ky.begin(), ky.end());
    ctx->tb32.twx = dalloc<C32>(ctx, fx.size());
    ctx->tb32.twy = dalloc<C32>(ctx, fy.size());
    ctx->tb32.kx = dalloc<float>(ctx, G.Nxh);
    ctx->tb32.ky = dalloc<float>(ctx, G.Ny);
    CK(cudaMemcpy(ctx->tb32.twx, fx.data(), fx.size() * sizeof(C32), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tb32.twy, fy.data(), fy.size() * sizeof(C32), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tb32.kx, kxf.data(), G.Nxh * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tb32.ky, kyf.data(), G.Ny * sizeof(float), cudaMemcpyHostToDevice));
  }
}

CoefCopy coef_copy(sgn_ctx* ctx) {
  CoefCopy cp;
  if (ctx->opt.precision >= 1) {
    cp.h = ctx->h32;
    cp.cr = ctx->cr32;
    cp.cc = ctx->cc32;
  }
  return cp;
}

Exec EX(sgn_ctx* ctx, int kind_override = -1) {
  Exec e{ctx->stream, &ctx->prof};
  e.kind_override = kind_override;
  e.tune = &ctx->tune;
  return e;
}

// launches of the refinement residual of precision 1 and 2
Exec EX_REFINE(sgn_ctx* ctx) {
  Exec e = EX(ctx);
  e.refine = true;
  return e;
}

CDF* const* tmp_df(sgn_ctx* ctx) { return reinterpret_cast<CDF* const*>(ctx->tmp); }

// w = [M^-1] L sigma_hat in the handle's refinement arithmetic: double-float
// for precision 2, FP64 otherwise
void refine_matvec(sgn_ctx* ctx, bool precond, const Exec& ex) {
  if (ctx->opt.precision >= 2)
    CK((launch_matvec_io<dfl, double>(ctx->G, ctx->tbd, ctx->sig, ctx->crd, ctx->ccd, ctx->w, tmp_df(ctx), precond,
                                      ex)));
  else
    CK(launch_matvec<double>(ctx->G, ctx->tb, ctx->sig, ctx->cr, ctx->cc, ctx->w, ctx->tmp, precond, ex));
}

// coefficient fields from a physical depth h
void coef_phys(sgn_ctx* ctx, const double* h) {
  if (ctx->opt.precision >= 2)
    CK(launch_coef_phys<dfl>(ctx->G, h, ctx->hd, ctx->crd, ctx->ccd, ctx->flags, coef_copy(ctx), EX(ctx)));
  else
    CK(launch_coef_phys<double>(ctx->G, h, ctx->h, ctx->cr, ctx->cc, ctx->flags, coef_copy(ctx), EX(ctx)));
}

// ------------------------------------------------------------ transforms

void fwd2(sgn_ctx* ctx, const double* const* f, int nf, C64* const* out) {
  CK(launch_x_r2c<double>(ctx->G, ctx->tb, f, nf, out, EX(ctx)));
  CK(launch_y_fft<double>(ctx->G, ctx->tb, false, (const C64* const*)out, nullptr, nf, out, EX(ctx)));
}

// physical out[i] = inverse 2D transform of (i kx)^dx (i ky)^dy in[i]; uses tmp[0..nf)
void inv2(sgn_ctx* ctx, const C64* const* in, const int* dx, const int* dy, int nf, double* const* out) {
  CK(launch_y_fft<double>(ctx->G, ctx->tb, true, in, dy, nf, ctx->tmp, EX(ctx)));
  CK(launch_x_c2r<double>(ctx->G, ctx->tb, (const C64* const*)ctx->tmp, dx, nf, out,
                          1.0 / (double)ctx->G.nphys(), EX(ctx)));
}

// Host-buffer calls: per-field copies on a copy stream, overlapped with the
// per-field transforms on the handle's stream (field i's transform waits only
// for its own host-to-device copy; field i's device-to-host copy starts as
// soon as its inverse transform is done).
struct HostIO {
  cudaStream_t cs;
  cudaEvent_t in[4], out[4];
  double* host[4];
  size_t bytes;
};

// One field to and from spectral space in double-float arithmetic (the state
// conversions of precision 2: 2^-48 relative rounding per transform, far
// below the FP32 bulk's, at about a third of the FP64 passes' time)
void fwd1_df(sgn_ctx* ctx, const double* f, C64* out) {
  CDF* scratch = tmp_df(ctx)[0];
  CK(launch_x_r2c<dfl>(ctx->G, ctx->tbd, &f, 1, &scratch, EX(ctx)));
  CK(launch_y_fwd64<dfl>(ctx->G, ctx->tbd, scratch, out, EX(ctx)));
}
void inv1_df(sgn_ctx* ctx, const C64* in, double* out) {
  CDF* scratch = tmp_df(ctx)[0];
  CK(launch_y_inv64<dfl>(ctx->G, ctx->tbd, in, scratch, EX(ctx)));
  const CDF* sc = scratch;
  CK(launch_x_c2r<dfl>(ctx->G, ctx->tbd, &sc, nullptr, 1, &out, 1.0 / (double)ctx->G.nphys(), EX(ctx)));
}

// (h, vx, vy) -> Un, sigma -> sig (spectral); io may be null
void fwd_state(sgn_ctx* ctx, const double* const* f, const HostIO* io) {
  const bool df = ctx->opt.precision >= 2;
  if (!io && !df) {
    fwd2(ctx, f, 3, ctx->Un);
    fwd2(ctx, f + 3, 1, &ctx->sig);
    return;
  }
  C64* dst[4] = {ctx->Un[0], ctx->Un[1], ctx->Un[2], ctx->sig};
  for (int i = 0; i < 4; ++i) {
    if (io) CK(cudaStreamWaitEvent(ctx->stream, io->in[i], 0));
    if (df)
      fwd1_df(ctx, f[i], dst[i]);
    else
      fwd2(ctx, f + i, 1, dst + i);
  }
}

// Un -> (h, vx, vy), sig -> sigma (physical); with io, each field is copied to
// io->host[i] on the copy stream once it is ready
void inv_state(sgn_ctx* ctx, double* const* o, const HostIO* io) {
  const bool df = ctx->opt.precision >= 2;
  if (!io && !df) {
    inv2(ctx, (const C64* const*)ctx->Un, nullptr, nullptr, 3, o);
    inv2(ctx, (const C64* const*)&ctx->sig, nullptr, nullptr, 1, o + 3);
    return;
  }
  const C64* src[4] = {ctx->Un[0], ctx->Un[1], ctx->Un[2], ctx->sig};
  for (int i = 0; i < 4; ++i) {
    if (df)
      inv1_df(ctx, src[i], o[i]);
    else
      inv2(ctx, src + i, nullptr, nullptr, 1, o + i);
    if (!io) continue;
    CK(cudaEventRecord(io->out[i], ctx->stream));
    CK(cudaStreamWaitEvent(io->cs, io->out[i], 0));
    CK(cudaMemcpyAsync(io->host[i], o[i], io->bytes, cudaMemcpyDeviceToHost, io->cs));
  }
}

void sync_read(sgn_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->rb_host, ctx->rb_dev, sizeof(GmresReadback), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->prof.on) ctx->prof.harvest();
}

void check_flags(sgn_ctx* ctx, int flags) {
  if (flags & FLAG_NONFINITE) {
    ctx->err = "non-finite depth h";
    throw Fail{SGN_ENONFINITE};
  }
  if (flags & FLAG_CAVITATION) {
    ctx->err = "cavitation: h <= 0 somewhere";
    throw Fail{SGN_ECAVITATION};
  }
  if (flags & FLAG_WAIT) {
    ctx->err = "a y-pass stopped waiting for its tensor copies (bounded wait ran out)";
    throw Fail{SGN_ECUDA};
  }
}

// coefficient fields from the spectral depth h_hat
void coef_from_spectral(sgn_ctx* ctx, const C64* hh) {
  if (ctx->opt.precision >= 2) {
    CK(launch_y_inv64<dfl>(ctx->G, ctx->tbd, hh, tmp_df(ctx)[0], EX(ctx, PK_COEF)));
    CK(launch_coef_x<dfl>(ctx->G, ctx->tbd, tmp_df(ctx)[0], ctx->hd, ctx->crd, ctx->ccd, ctx->flags,
                          coef_copy(ctx), EX(ctx)));
    return;
  }
  CK(launch_y_fft<double>(ctx->G, ctx->tb, true, &hh, nullptr, 1, ctx->tmp, EX(ctx, PK_COEF)));
  CK(launch_coef_x<double>(ctx->G, ctx->tb, ctx->tmp[0], ctx->h, ctx->cr, ctx->cc, ctx->flags, coef_copy(ctx),
                            EX(ctx)));
}

// One Arnoldi step of the inner or outer GMRES on the basis V (type T):
// w = A V_j, classical Gram-Schmidt with DGKS reorthogonalisation, Givens.
// Returns the residual estimate and H[j+1][j] through the readback.
template <typename T>
void arnoldi_step(sgn_ctx* ctx, const Tables<T>& tb, const T* cr, const T* cc, cpx<T>* V, cpx<T>* w,
                  cpx<T>* const* tmp, int j) {
  const Geom& G = ctx->G;
  const size_t vs = G.nspec();
  const int nv = j + 1;
  CK(launch_matvec<T>(G, tb, V + (size_t)j * vs, cr, cc, w, tmp, true, EX(ctx), nullptr, 0, &ctx->mvt));
  const int* gate = &ctx->gst->reorth;
  unsigned* cnt = ctx->counters;
  // FP64 Arnoldi (the plain path and nothing else) reorthogonalises by the DGKS
  // test; the FP32 inner solve of precision 1 runs one classical Gram-Schmidt
  // pass: it only has to reduce its residual by 1e-6 and the FP64 refinement
  // checks the result (measured: same iteration and refinement counts, 4% faster)
  const bool dgks = sizeof(T) == 8;
  // the FP32 basis is stored unnormalised (GmresDev::vscl): the update writes
  // the next basis vector itself, with no scaling pass
  const double* vscl = dgks ? nullptr : ctx->gst->vscl;
  CK(launch_dots<T>(G, V, vs, nv, w, ctx->partials, nullptr, ctx->gst->h1, cnt + 0, EX(ctx), nullptr, vscl));
  CK(launch_cgs_update<T>(G, V, vs, nv, ctx->gst->h1, w, ctx->partials, nullptr, ctx->gst, j, dgks ? 1 : 3,
                          cnt + 1, ctx->rb_dev, ctx->flags, EX(ctx), nullptr, nullptr, !dgks));
  if (dgks) {
    CK(launch_dots<T>(G, V, vs, nv, w, ctx->partials, gate, ctx->gst->h2, cnt + 2, EX(ctx)));
    CK(launch_cgs_update<T>(G, V, vs, nv, ctx->gst->h2, w, ctx->partials, gate, ctx->gst, j, 2, cnt + 3,
                            ctx->rb_dev, ctx->flags, EX(ctx)));
  }
  sync_read(ctx);
}

// --------------------------------------------------------------- GMRES
// Left-preconditioned restarted GMRES on A = M^-1 L, c = M^-1 b (Section 3).
// Uses ctx->h/cr/cc, ctx->bh (b_hat); ctx->sig is the guess and the result.
// Returns true if converged.
bool gmres_fp64(sgn_ctx* ctx, int* iters_out, double* relres_out) {
  const Geom& G = ctx->G;
  cudaStream_t s = ctx->stream;
  const int m = ctx->opt.restart;
  const size_t vs = G.nspec();
  double* cnorm_d = ctx->scal + 0;
  double* beta_d = ctx->scal + 1;
  CK(launch_hermitian_fix<double>(G, ctx->bh, EX(ctx)));
  CK(launch_precond<double>(G, ctx->tb, ctx->bh, ctx->cvec, ctx->partials, EX(ctx)));
  CK(launch_reduce(ctx->partials, 1, cnorm_d, true, nullptr, EX(ctx)));
  CK(launch_readback_scalar(cnorm_d, ctx->flags, ctx->rb_dev, EX(ctx)));
  sync_read(ctx);
  check_flags(ctx, ctx->rb_host->flags);
  const double cnorm = ctx->rb_host->scalar;
  ctx->stats.solves++;
  if (cnorm == 0.0) {
    CK(launch_zero<double>(G, ctx->sig, EX(ctx)));
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    ctx->stats.last_iters = 0;
    ctx->stats.last_relres = 0.0;
    return true;
  }
  const double target = ctx->opt.tol * cnorm;
  int its = 0;
  bool conv = false;
  double res = 0.0;
  C64* const V = ctx->V;
  for (;;) {
    CK(launch_matvec<double>(G, ctx->tb, ctx->sig, ctx->cr, ctx->cc, ctx->w, ctx->tmp, true, EX(ctx)));
    CK(launch_residual<double>(G, ctx->cvec, ctx->w, V, ctx->partials, EX(ctx)));
    CK(launch_reduce(ctx->partials, 1, beta_d, true, nullptr, EX(ctx)));
    CK(launch_readback_scalar(beta_d, ctx->flags, ctx->rb_dev, EX(ctx)));
    sync_read(ctx);
    check_flags(ctx, ctx->rb_host->flags);
    const double beta = ctx->rb_host->scalar;
    res = beta;
    if (!(beta > target)) {
      conv = !(beta != beta);
      break;
    }
    if (its >= ctx->opt.maxit) break;
    CK(launch_scale<double, double>(G, V, beta_d, true, V, EX(ctx)));
    CK(launch_gmres_start(ctx->gst, beta_d, EX(ctx)));
    int k = 0;
    for (int j = 0; j < m; ++j) {
      arnoldi_step<double>(ctx, ctx->tb, ctx->cr, ctx->cc, V, ctx->w, ctx->tmp, j);
      ++its;
      res = ctx->rb_host->res;
      const double hnext = ctx->rb_host->hnext;
      k = j + 1;
      if (res <= target || its >= ctx->opt.maxit || !(hnext > 0.0) || res != res) break;
      if (j + 1 < m) CK(launch_scale<double, double>(G, ctx->w, &ctx->gst->hnext, true, V + (size_t)(j + 1) * vs, EX(ctx)));
    }
    CK(launch_backsolve(ctx->gst, k, EX(ctx)));
    CK(launch_axpy_multi<double, double>(G, V, vs, k, ctx->gst->y, ctx->sig, EX(ctx)));
    if (res <= target) {
      conv = true;
      break;
    }
    if (res != res) break;
  }
  ctx->stats.matvecs += its;
  if (its > ctx->stats.max_iters) ctx->stats.max_iters = its;
  ctx->stats.last_iters = its;
  ctx->stats.last_relres = res / cnorm;
  if (iters_out) *iters_out = its;
  if (relres_out) *relres_out = res / cnorm;
  return conv;
}

// Mixed-precision GMRES (precision = 1), iterative refinement: each sweep
// computes the residual r = c - A sigma with the FP64 matvec, then solves the
// correction equation A d = r by GMRES with FP32 matvecs and FP32 Krylov
// vectors (FP64 dot products, Givens rotations and sigma += d). The
// tolerance test is the FP64 one of gmres_fp64.
bool gmres_mixed(sgn_ctx* ctx, int* iters_out, double* relres_out) {
  const Geom& G = ctx->G;
  const int m = ctx->opt.restart;
  const size_t vs = G.nspec();
  double* cnorm_d = ctx->scal + 0;
  double* beta_d = ctx->scal + 1;
  CK(launch_hermitian_fix<double>(G, ctx->bh, EX(ctx)));
  CK(launch_precond<double>(G, ctx->tb, ctx->bh, ctx->cvec, ctx->partials, EX(ctx)));
  CK(launch_reduce(ctx->partials, 1, cnorm_d, true, nullptr, EX(ctx)));
  CK(launch_readback_scalar(cnorm_d, ctx->flags, ctx->rb_dev, EX(ctx)));
  sync_read(ctx);
  check_flags(ctx, ctx->rb_host->flags);
  const double cnorm = ctx->rb_host->scalar;
  ctx->stats.solves++;
  if (cnorm == 0.0) {
    CK(launch_zero<double>(G, ctx->sig, EX(ctx)));
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    ctx->stats.last_iters = 0;
    ctx->stats.last_relres = 0.0;
    return true;
  }
  const double target = ctx->opt.tol * cnorm;
  int its = 0;
  bool conv = false;
  double res = 0.0;
  for (;;) {
    refine_matvec(ctx, true, EX_REFINE(ctx));
    CK(launch_residual<double>(G, ctx->cvec, ctx->w, ctx->r64, ctx->partials, EX(ctx)));
    CK(launch_reduce(ctx->partials, 1, beta_d, true, nullptr, EX(ctx)));
    CK(launch_readback_scalar(beta_d, ctx->flags, ctx->rb_dev, EX(ctx)));
    sync_read(ctx);
    check_flags(ctx, ctx->rb_host->flags);
    ctx->stats.refinements++;
    const double beta = ctx->rb_host->scalar;
    res = beta;
    if (!(beta > target)) {
      conv = !(beta != beta);
      break;
    }
    if (its >= ctx->opt.maxit) break;
    C32* const V = ctx->V32;
    CK(launch_scale<double, float>(G, ctx->r64, beta_d, true, V, EX(ctx)));
    CK(launch_gmres_start(ctx->gst, beta_d, EX(ctx)));
    const double inner_target = fmax(0.5 * target, kInnerRel * beta);
    double res_in = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      arnoldi_step<float>(ctx, ctx->tb32, ctx->cr32, ctx->cc32, V, ctx->w32, ctx->tmp32, j);
      check_flags(ctx, ctx->rb_host->flags);
      ++its;
      res_in = ctx->rb_host->res;
      const double hnext = ctx->rb_host->hnext;
      k = j + 1;
      if (res_in <= inner_target || its >= ctx->opt.maxit || !(hnext > 0.0) || res_in != res_in) break;
    }
    CK(launch_backsolve(ctx->gst, k, EX(ctx)));
    CK(launch_axpy_multi<float, double>(G, V, vs, k, ctx->gst->y, ctx->sig, EX(ctx), nullptr, ctx->gst->vscl));
    if (ctx->trace)
      fprintf(stderr, "[sgn] mixed sweep: beta/|c| %.3e, inner its %d, inner estimate/|c| %.3e, total its %d\n",
              beta / cnorm, k, res_in / cnorm, its);
    if (res_in != res_in) {
      res = res_in;
      break;
    }
    if (res_in <= target && kFp32Trust * beta <= 0.5 * target) {
      res = res_in;
      conv = true;
      break;
    }
  }
  ctx->stats.matvecs += its;
  if (its > ctx->stats.max_iters) ctx->stats.max_iters = its;
  ctx->stats.last_iters = its;
  ctx->stats.last_relres = res / cnorm;
  if (iters_out) *iters_out = its;
  if (relres_out) *relres_out = res / cnorm;
  return conv;
}

bool gmres(sgn_ctx* ctx, int* iters_out, double* relres_out) {
  return ctx->opt.precision >= 1 ? gmres_mixed(ctx, iters_out, relres_out) : gmres_fp64(ctx, iters_out, relres_out);
}

// ------------------------------------------------------- learned start
// Kernels one network forward pass launches (13) for the launch count.
// kernels of one sgn_unet_infer: the weight image, the first layer, two per
// level above the bottleneck (s_l and its pool), e_l for 0 < l < D-1, b0, b1
// and D-1 decoder layers
int unet_launches(sgn_unet_t net) { return 4 * sgn_unet_levels(net) - 1; }

double learned_tau(int pw, double dt) { return pw == 0 ? 1.0 : (pw == 1 ? 0.5 * dt : 0.25 * dt * dt); }

// Stages 2 and 4 (every stage with guess 3), after the start of opt.guess:
// record the coarse inputs (and keep sigma_start) and/or add the network's
// correction to sigma_hat.
void learned_pre(sgn_ctx* ctx, C64* const* U, int mode, double dt, bool graph = false) {
  ctx->rec_stage = false;
  const bool poly = ctx->opt.guess == 3;
  if (mode == RK_STORE_K || (!poly && mode != RK_STAGE2 && mode != RK_FINAL)) return;
  // with the extrapolated start, stage 2 of a call's first step has no
  // stage-3 history and starts from sigma_1 instead, and the polynomial start
  // is cubic only once the ring holds 4 steps: starts of another kind, left
  // alone (graph mode tests the device flags)
  const bool s2_plain = ctx->opt.guess == 2 && mode == RK_STAGE2;
  if (s2_plain && !graph && !ctx->have_s3) return;
  if (poly && !graph && ctx->ext_lv < 4) return;
  const Geom& G = ctx->G;
  if (ctx->rec_buf && ctx->rec_count < ctx->rec_cap) {
    const int n = ctx->rec_n;
    const size_t nn = (size_t)n * n;
    float* slot = ctx->rec_buf + (size_t)ctx->rec_count * 5 * nn;
    CoarseIn ci{};
    for (int f = 0; f < 4; ++f) {
      ci.spec[f] = f < 3 ? U[f] : ctx->sig;
      ci.out[f] = slot + f * nn;
      ci.scale[f] = 1.f;
      ci.shift[f] = f == 0 ? -1.f : 0.f;
    }
    CK(launch_restrict(G, ci, 4, n, ctx->rtw, ctx->rY, EX(ctx)));
    CK(cudaMemcpyAsync(ctx->sig_fb, ctx->sig, G.nspec() * sizeof(C64), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->rec_stage = true;
  }
  if (ctx->net) {
    const int n = ctx->ln;
    const size_t nn = (size_t)n * n;
    CoarseIn ci{};
    for (int f = 0; f < 4; ++f) {
      ci.spec[f] = f < 3 ? U[f] : ctx->sig;
      ci.out[f] = ctx->lin + f * nn;
      ci.scale[f] = ctx->in_scale[f];
      ci.shift[f] = f == 0 ? -1.f : 0.f;
    }
    CK(launch_restrict(G, ci, 4, n, ctx->ltw, ctx->lY, EX(ctx)));
    sgn_unet_set_stream(ctx->net, ctx->stream);
    const sgn_status st = sgn_unet_infer(ctx->net, ctx->lin, ctx->lout, 1);
    if (st != SGN_OK) {
      ctx->err = std::string("learned start: ") + sgn_unet_last_error(ctx->net);
      throw Fail{st};
    }
    ctx->prof.launches += unet_launches(ctx->net);
    const int* gate = !graph ? nullptr : (poly ? &ctx->ext->full : (s2_plain ? &ctx->gst->have_s3 : nullptr));
    CK(launch_prolong_add(G, ctx->lout, n, ctx->ltw, ctx->lY, nullptr,
                          (double)ctx->out_scale * learned_tau(ctx->tau_pow, dt), ctx->sig, EX(ctx), gate));
  }
}

// after the solve of a recorded stage: target (sigma_solved - sigma_start) / tau
void learned_post(sgn_ctx* ctx, double dt) {
  if (!ctx->rec_stage) return;
  const Geom& G = ctx->G;
  const int n = ctx->rec_n;
  const size_t nn = (size_t)n * n;
  float* slot = ctx->rec_buf + (size_t)ctx->rec_count * 5 * nn;
  CK(cudaMemcpyAsync(ctx->tmp[0], ctx->sig, G.nspec() * sizeof(C64), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(launch_axpby<double>(G, -1.0, ctx->sig_fb, 1.0, ctx->tmp[0], EX(ctx)));
  CoarseIn ci{};
  ci.spec[0] = ctx->tmp[0];
  ci.out[0] = slot + 4 * nn;
  ci.scale[0] = (float)(1.0 / learned_tau(ctx->rec_tau_pow, dt));
  CK(launch_restrict(G, ci, 1, n, ctx->rtw, ctx->rY, EX(ctx)));
  ctx->rec_count += 1;
  ctx->rec_stage = false;
}

// coarse scratch for side n: twiddles and 5 * n * n/2 complex values
void coarse_alloc(sgn_ctx* ctx, int n, float2** tw, float2** Y) {
  *tw = dalloc<float2>(ctx, n);
  *Y = dalloc<float2>(ctx, (size_t)5 * n * (n / 2));
  CK(launch_coarse_twiddles(n, *tw, EX(ctx)));
}

// RHS of state U (K into the RK epilogue) in the handle's arithmetic: FP64
// (precision 0), FP32 (1, 2) or double-float (3)
void launch_rhs_ctx(sgn_ctx* ctx, C64* const* U, C64* bnext, const RkArgs& rk) {
  if (ctx->opt.precision == 3)
    CK((launch_rhs<dfl, double>(ctx->G, ctx->tbd, ctx->tb, U, ctx->sig, ctx->hd, ctx->crd, tmp_df(ctx), ctx->Un,
                                ctx->Us, ctx->acc, bnext, rk, EX(ctx))));
  else if (ctx->opt.precision >= 1)
    CK((launch_rhs<float, double>(ctx->G, ctx->tb32, ctx->tb, U, ctx->sig, ctx->h32, ctx->cr32, ctx->tmp32, ctx->Un,
                                  ctx->Us, ctx->acc, bnext, rk, EX(ctx))));
  else
    CK((launch_rhs<double, double>(ctx->G, ctx->tb, ctx->tb, U, ctx->sig, ctx->h, ctx->cr, ctx->tmp, ctx->Un,
                                   ctx->Us, ctx->acc, bnext, rk, EX(ctx))));
}

// one RK4 stage (s = 1..4) or a plain RHS evaluation (mode RK_STORE_K)
bool stage(sgn_ctx* ctx, int mode, double dt) {
  C64* const* U = (mode == RK_STAGE1 || mode == RK_STORE_K) ? ctx->Un : ctx->Us;
  coef_from_spectral(ctx, U[0]);
  if (ctx->opt.guess == 1) CK(launch_zero<double>(ctx->G, ctx->sig, EX(ctx)));
  // guess 3 falls back on guess 2's start (and needs its copies) only while
  // its ring holds fewer than 3 steps
  const bool lin2 = ctx->opt.guess == 2 || (ctx->opt.guess == 3 && ctx->ext_lv < 3);
  if (lin2) {
    // linear extrapolation in time over the stage times t, t+dt/2, t+dt/2, t+dt:
    // stage 2 from sigma(t) and the previous step's sigma(t - dt/2),
    // stage 4 from sigma(t + dt/2) and sigma(t)
    if (mode == RK_STAGE2 && ctx->have_s3) CK(launch_axpby<double>(ctx->G, -1.0, ctx->sig_s3, 2.0, ctx->sig, EX(ctx)));
    if (mode == RK_FINAL) CK(launch_axpby<double>(ctx->G, -1.0, ctx->sig_s1, 2.0, ctx->sig, EX(ctx)));
  }
  const bool ext = ctx->opt.guess == 3 && mode != RK_STORE_K;
  if (ext) CK(launch_ext_start(ctx->G, ctx->ext_ring, mode, ctx->ext, ctx->sig, EX(ctx)));
  learned_pre(ctx, U, mode, dt);
  const bool conv = gmres(ctx, nullptr, nullptr);
  learned_post(ctx, dt);
  if (ctx->opt.guess >= 2) {
    const size_t bytes = ctx->G.nspec() * sizeof(C64);
    if (mode == RK_STAGE1 && lin2)
      CK(cudaMemcpyAsync(ctx->sig_s1, ctx->sig, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (mode == RK_STAGE3) {
      if (lin2) CK(cudaMemcpyAsync(ctx->sig_s3, ctx->sig, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      ctx->have_s3 = true;
    }
  }
  if (ext) {
    CK(launch_ext_store(ctx->G, ctx->sig, ctx->ext_ring, mode, ctx->ext, EX(ctx)));
    if (mode == RK_FINAL) {
      CK(launch_ext_advance(ctx->ext, EX(ctx)));
      ctx->ext_lv = ctx->ext_lv < 4 ? ctx->ext_lv + 1 : 4;
    }
  }
  RkArgs rk{};
  rk.mode = mode;
  rk.dt = dt;
  rk.dealias = ctx->opt.dealias;
  rk.krasny = ctx->opt.krasny;
  rk.krasny_thr = ctx->opt.krasny_thr;
  rk.g = ctx->g;
  C64* bnext = mode == RK_STORE_K ? nullptr : ctx->bh;
  launch_rhs_ctx(ctx, U, bnext, rk);
  return conv;
}

void reset_flags(sgn_ctx* ctx) { CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->stream)); }

void ensure_phys(sgn_ctx* ctx) {
  if (ctx->phys[0]) return;
  for (int i = 0; i < 4; ++i) ctx->phys[i] = dalloc<double>(ctx, ctx->G.nphys());
}

// The extrapolated starts (guess 2 and 3) carry sigma from one step to the
// next: stage 3's (guess 2) and every stage's of the last 4 steps (guess 3). A call that continues the trajectory the handle's last RK4 call
// returned (same dt, and an input state equal to that output within 1e-8 of
// the largest coefficient: the conversions' round trip, and the
// anti-Hermitian remainder that FP32 increments leave in the kx = 0 and Nyquist
// columns and the real output drops, ~1e-10) keeps that history, so its first
// step extrapolates too; any other input starts without it. The history only
// chooses GMRES's starting value: every solve still meets opt.tol.
// continues_history() saves the last output state (Un) before the
// call's conversions overwrite it; same_state_flag() compares and writes the
// device flag gst->have_s3.
bool continues_history(sgn_ctx* ctx, double dt) {
  if (ctx->opt.guess < 2 || !ctx->hist_keep || dt != ctx->hist_dt) return false;
  const size_t bytes = ctx->G.nspec() * sizeof(C64);
  for (int f = 0; f < 3; ++f)
    CK(cudaMemcpyAsync(ctx->acc[f], ctx->Un[f], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return true;
}
void same_state_flag(sgn_ctx* ctx) {
  const C64* a[3] = {ctx->acc[0], ctx->acc[1], ctx->acc[2]};
  const C64* b[3] = {ctx->Un[0], ctx->Un[1], ctx->Un[2]};
  CK(launch_same_state(ctx->G, a, b, 1e-8, ctx->partials, ctx->counters + 6, &ctx->gst->have_s3, EX(ctx)));
}
// guess = 3: the ring's steps stay only when the call continues the trajectory
// (cont, and the device flag same_state_flag() wrote)
void ext_history(sgn_ctx* ctx, bool cont) {
  if (ctx->opt.guess != 3) return;
  if (cont) {
    CK(launch_ext_keep(ctx->ext, &ctx->gst->have_s3, EX(ctx)));
  } else {
    CK(launch_set_int(&ctx->ext->levels, 0, EX(ctx)));
    CK(launch_set_int(&ctx->ext->full, 0, EX(ctx)));
    CK(launch_set_int(&ctx->ext->lin, 1, EX(ctx)));
  }
}

void rk4_device(sgn_ctx* ctx, double* h, double* vx, double* vy, double* sigma, double dt, int nsteps,
                bool* conv_all, const HostIO* io = nullptr) {
  const double* f4[4] = {h, vx, vy, sigma};
  reset_flags(ctx);
  const bool cont = continues_history(ctx, dt);
  fwd_state(ctx, f4, io);
  CK(launch_spec_div<double>(ctx->G, ctx->tb, ctx->Un[1], ctx->Un[2], ctx->bh, EX(ctx)));
  ctx->have_s3 = false;
  if (cont) same_state_flag(ctx);
  ext_history(ctx, cont);
  if (cont) {
    int keep = 0;
    CK(cudaMemcpyAsync(&keep, &ctx->gst->have_s3, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_s3 = keep != 0;
  }
  if (!(cont && ctx->have_s3)) ctx->ext_lv = 0;
  bool conv = true;
  for (int n = 0; n < nsteps; ++n) {
    conv &= stage(ctx, RK_STAGE1, dt);
    conv &= stage(ctx, RK_STAGE2, dt);
    conv &= stage(ctx, RK_STAGE3, dt);
    conv &= stage(ctx, RK_FINAL, dt);
  }
  double* o4[4] = {h, vx, vy, sigma};
  inv_state(ctx, o4, io);
  *conv_all = conv;
  ctx->hist_ok = ctx->opt.guess >= 2;
  ctx->hist_dt = dt;
}


// ------------------------------------------------------------ graph mode
// One RK4 step as a CUDA graph. Straight-line work is stream-captured into
// the graph; each GMRES solve becomes
//   ... c = M^-1 b, |c|, k_ctl_begin, [sigma = 0 if c = 0]
//   WHILE (h_sweep) {                       restart cycle / refinement sweep
//     A sigma (FP64), r = c - A sigma, |r|, k_ctl_sweep, V_0 = r/|r|
//     WHILE (h_step) { Arnoldi step j (j read from the device), V_{j+1} }
//     y = H^-1 g, sigma += V y, k_ctl_after
//   }
// where the Givens step of the last Gram-Schmidt kernel and the control
// kernels set the two conditions with the tests of gmres_fp64 / gmres_mixed.

// Captures stretches of launches on ctx->cap into graph g after the nodes in
// tail, and appends conditional WHILE nodes.
struct GraphSeg {
  sgn_ctx* ctx;
  cudaGraph_t g;
  std::vector<cudaGraphNode_t> tail;

  void open() {
    CK(cudaStreamBeginCaptureToGraph(ctx->cap, g, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(),
                                     cudaStreamCaptureModeThreadLocal));
  }
  void close() {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(ctx->cap, &cs, nullptr, nullptr, &deps, nullptr, &nd));
    std::vector<cudaGraphNode_t> t(deps, deps + nd);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(ctx->cap, &out));
    tail = t;
  }
  cudaGraphConditionalHandle handle() {
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    return h;
  }
  // WHILE node after the tail; returns its body graph
  cudaGraph_t add_while(cudaGraphConditionalHandle h) {
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(), &p));
    tail.assign(1, node);
    return p.conditional.phGraph_out[0];
  }
};

// Kernels enqueued by f (counted through the profiler's launch counter).
template <typename F>
long long count_launches(sgn_ctx* ctx, F&& f) {
  const long long before = ctx->prof.launches;
  f();
  const long long n = ctx->prof.launches - before;
  ctx->prof.launches = before;
  return n;
}

// One Arnoldi step with device-side j: the body of the inner WHILE node.
template <typename T>
void graph_arnoldi(sgn_ctx* ctx, const Tables<T>& tb, const T* cr, const T* cc, cpx<T>* V, cpx<T>* w,
                   cpx<T>* const* tmp, const GraphCtl& ctl) {
  const Geom& G = ctx->G;
  const size_t vs = G.nspec();
  const int m = ctx->opt.restart;
  const int* jd = &ctx->gst->j;
  const int* gate = &ctx->gst->reorth;
  unsigned* cnt = ctx->counters;
  const bool dgks = sizeof(T) == 8;
  const double* vscl = dgks ? nullptr : ctx->gst->vscl;
  CK(launch_matvec<T>(G, tb, V, cr, cc, w, tmp, true, EX(ctx), jd, vs, &ctx->mvt));
  CK(launch_dots<T>(G, V, vs, m, w, ctx->partials, nullptr, ctx->gst->h1, cnt + 0, EX(ctx), jd, vscl));
  CK(launch_cgs_update<T>(G, V, vs, m, ctx->gst->h1, w, ctx->partials, nullptr, ctx->gst, 0, dgks ? 1 : 3, cnt + 1,
                          ctx->rb_dev, ctx->flags, EX(ctx), jd, &ctl, !dgks));
  if (dgks) {
    CK(launch_dots<T>(G, V, vs, m, w, ctx->partials, gate, ctx->gst->h2, cnt + 2, EX(ctx), jd));
    CK(launch_cgs_update<T>(G, V, vs, m, ctx->gst->h2, w, ctx->partials, gate, ctx->gst, 0, 2, cnt + 3,
                            ctx->rb_dev, ctx->flags, EX(ctx), jd, &ctl));
  }
  // FP64: V_{j+1} = w / H[j+1][j]; j has already advanced (index m is the
  // spare slot). FP32: the update stored the unnormalised V_{j+1} itself.
  if (dgks) CK(launch_scale<T, T>(G, w, &ctx->gst->hnext, true, V, EX(ctx), jd, vs));
}

// One GMRES solve (FP64 or mixed) appended to the top-level segment.
void graph_gmres(sgn_ctx* ctx, GraphSeg& top) {
  const Geom& G = ctx->G;
  const bool mixed = ctx->opt.precision >= 1;
  const size_t vs = G.nspec();
  double* cnorm_d = ctx->scal + 0;
  double* beta_d = ctx->scal + 1;
  GraphCtl ctl{};
  ctl.tol = ctx->opt.tol;
  ctl.m = ctx->opt.restart;
  ctl.maxit = ctx->opt.maxit;
  ctl.mixed = mixed ? 1 : 0;
  ctl.enabled = 1;
  // the handle is made while no capture into the graph is open
  top.close();
  ctl.h_sweep = top.handle();
  top.open();
  long long fixed = count_launches(ctx, [&] {
    CK(launch_hermitian_fix<double>(G, ctx->bh, EX(ctx)));
    CK(launch_precond<double>(G, ctx->tb, ctx->bh, ctx->cvec, ctx->partials, EX(ctx)));
    CK(launch_reduce(ctx->partials, 1, cnorm_d, true, nullptr, EX(ctx)));
    CK(launch_ctl_begin(ctx->gst, cnorm_d, ctl, EX(ctx)));
    CK(launch_zero<double>(G, ctx->sig, EX(ctx), &ctx->gst->zero_sigma));
  });
  top.close();
  GraphSeg sweep{ctx, top.add_while(ctl.h_sweep), {}};
  ctl.h_step = sweep.handle();
  sweep.open();
  long long per_sweep = count_launches(ctx, [&] {
    refine_matvec(ctx, true, EX(ctx));
    C64* r = mixed ? ctx->r64 : ctx->V;
    CK(launch_residual<double>(G, ctx->cvec, ctx->w, r, ctx->partials, EX(ctx)));
    CK(launch_reduce(ctx->partials, 1, beta_d, true, nullptr, EX(ctx)));
    CK(launch_ctl_sweep(ctx->gst, beta_d, ctl, EX(ctx)));
    if (mixed)
      CK((launch_scale<double, float>(G, r, beta_d, true, ctx->V32, EX(ctx))));
    else
      CK((launch_scale<double, double>(G, r, beta_d, true, ctx->V, EX(ctx))));
  });
  sweep.close();
  ctx->sweep_bodies.push_back(sweep.g);
  GraphSeg step{ctx, sweep.add_while(ctl.h_step), {}};
  ctx->step_bodies.push_back(step.g);
  step.open();
  long long per_step = count_launches(ctx, [&] {
    if (mixed)
      graph_arnoldi<float>(ctx, ctx->tb32, ctx->cr32, ctx->cc32, ctx->V32, ctx->w32, ctx->tmp32, ctl);
    else
      graph_arnoldi<double>(ctx, ctx->tb, ctx->cr, ctx->cc, ctx->V, ctx->w, ctx->tmp, ctl);
  });
  step.close();
  sweep.open();
  per_sweep += count_launches(ctx, [&] {
    CK(launch_backsolve(ctx->gst, 0, EX(ctx), &ctx->gst->k));
    if (mixed)
      CK((launch_axpy_multi<float, double>(G, ctx->V32, vs, 0, ctx->gst->y, ctx->sig, EX(ctx), &ctx->gst->k,
                                           ctx->gst->vscl)));
    else
      CK((launch_axpy_multi<double, double>(G, ctx->V, vs, 0, ctx->gst->y, ctx->sig, EX(ctx), &ctx->gst->k)));
    CK(launch_ctl_after(ctx->gst, ctl, EX(ctx)));
  });
  sweep.close();
  top.open();
  ctx->graph_fixed += fixed;
  ctx->graph_per_sweep = per_sweep;
  ctx->graph_per_step = per_step;
}

// One RK4 stage appended to the top-level segment (open on entry and exit).
void graph_stage(sgn_ctx* ctx, GraphSeg& top, int mode, double dt) {
  C64* const* U = mode == RK_STAGE1 ? ctx->Un : ctx->Us;
  const size_t bytes = ctx->G.nspec() * sizeof(C64);
  ctx->graph_fixed += count_launches(ctx, [&] {
    coef_from_spectral(ctx, U[0]);
    if (ctx->opt.guess == 1) CK(launch_zero<double>(ctx->G, ctx->sig, EX(ctx)));
    // guess 3: guess 2's start and copies only while the ring holds < 3 steps
    const int* lin = ctx->opt.guess == 3 ? &ctx->ext->lin : nullptr;
    if (ctx->opt.guess >= 2) {
      if (mode == RK_STAGE2)
        CK(launch_axpby<double>(ctx->G, -1.0, ctx->sig_s3, 2.0, ctx->sig, EX(ctx), &ctx->gst->have_s3, lin));
      if (mode == RK_FINAL) CK(launch_axpby<double>(ctx->G, -1.0, ctx->sig_s1, 2.0, ctx->sig, EX(ctx), lin));
    }
    if (ctx->opt.guess == 3) CK(launch_ext_start(ctx->G, ctx->ext_ring, mode, ctx->ext, ctx->sig, EX(ctx)));
    learned_pre(ctx, U, mode, dt, true);  // no recording in graph mode (sgn_record_learned refuses it)
  });
  graph_gmres(ctx, top);
  ctx->graph_fixed += count_launches(ctx, [&] {
    if (ctx->opt.guess >= 2) {
      const int* lin = ctx->opt.guess == 3 ? &ctx->ext->lin : nullptr;
      auto keep = [&](C64* dst) {
        if (lin)
          CK(launch_copy_gated<double>(ctx->G, ctx->sig, dst, lin, EX(ctx)));
        else
          CK(cudaMemcpyAsync(dst, ctx->sig, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      };
      if (mode == RK_STAGE1) keep(ctx->sig_s1);
      if (mode == RK_STAGE3) {
        keep(ctx->sig_s3);
        CK(launch_set_int(&ctx->gst->have_s3, 1, EX(ctx)));
      }
    }
    if (ctx->opt.guess == 3) {
      CK(launch_ext_store(ctx->G, ctx->sig, ctx->ext_ring, mode, ctx->ext, EX(ctx)));
      if (mode == RK_FINAL) CK(launch_ext_advance(ctx->ext, EX(ctx)));
    }
    RkArgs rk{};
    rk.mode = mode;
    rk.dt = dt;
    rk.dealias = ctx->opt.dealias;
    rk.krasny = ctx->opt.krasny;
    rk.krasny_thr = ctx->opt.krasny_thr;
    rk.g = ctx->g;
    launch_rhs_ctx(ctx, U, ctx->bh, rk);
  });
}

// Kernel and conditional nodes of a graph (not of its bodies).
void count_nodes(sgn_ctx* ctx, cudaGraph_t g, long long* kernels, long long* conds, long long* others) {
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) CK(cudaGraphGetNodes(g, nodes.data(), &n));
  *kernels = *conds = *others = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel)
      ++*kernels;
    else if (t == cudaGraphNodeTypeConditional)
      ++*conds;
    else
      ++*others;
  }
}

// The loops end only through their control kernels, so before the first
// launch the built graph is checked against what was enqueued: four WHILE
// nodes at the top, each sweep body holding its kernels (k_ctl_sweep and
// k_ctl_after among them) and one nested WHILE node, each Arnoldi body its
// kernels (the Gram-Schmidt kernel with the Givens controller among them).
void check_step_graph(sgn_ctx* ctx) {
  long long k, c, o;
  count_nodes(ctx, ctx->step_graph, &k, &c, &o);
  bool ok = c == 4 && ctx->sweep_bodies.size() == 4 && ctx->step_bodies.size() == 4;
  for (size_t i = 0; ok && i < ctx->sweep_bodies.size(); ++i) {
    count_nodes(ctx, ctx->sweep_bodies[i], &k, &c, &o);
    ok = k == ctx->graph_per_sweep && c == 1 && o == 0;
    if (!ok) break;
    count_nodes(ctx, ctx->step_bodies[i], &k, &c, &o);
    ok = k == ctx->graph_per_step && c == 0 && o == 0;
  }
  if (!ok) {
    ctx->err = "graph mode: the captured step graph does not have the expected loop structure";
    throw Fail{SGN_ECUDA};
  }
}

// Builds and instantiates the step graph for time step dt. Every launch goes
// to ctx->cap while it is built (ctx->stream is swapped and restored) with
// profiling off, so the Exec of each launcher only counts kernels.
void build_step_graph(sgn_ctx* ctx, double dt) {
  free_graph(ctx);
  if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
  if (!ctx->gst_host) CK(cudaMallocHost((void**)&ctx->gst_host, sizeof(GmresDev)));
  CK(cudaGraphCreate(&ctx->step_graph, 0));
  const cudaStream_t saved = ctx->stream;
  const bool prof_on = ctx->prof.on;
  ctx->stream = ctx->cap;
  ctx->prof.on = false;
  ctx->graph_fixed = 0;
  GraphSeg top{ctx, ctx->step_graph, {}};
  try {
    top.open();
    graph_stage(ctx, top, RK_STAGE1, dt);
    graph_stage(ctx, top, RK_STAGE2, dt);
    graph_stage(ctx, top, RK_STAGE3, dt);
    graph_stage(ctx, top, RK_FINAL, dt);
    top.close();
    check_step_graph(ctx);
    CK(cudaGraphInstantiate(&ctx->step_exec, ctx->step_graph, 0));
  } catch (Fail&) {
    // end whichever segment was capturing (the top level or a WHILE body):
    // the graph it returns belongs to the step graph and goes with it below
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(ctx->cap, &junk);
    }
    cudaGetLastError();
    ctx->stream = saved;
    ctx->prof.on = prof_on;
    if (ctx->net) sgn_unet_set_stream(ctx->net, ctx->stream);
    free_graph(ctx);
    throw;
  }
  ctx->stream = saved;
  ctx->prof.on = prof_on;
  if (ctx->net) sgn_unet_set_stream(ctx->net, ctx->stream);
  ctx->graph_dt = dt;
}

// rk4_device with each step replayed from the step graph. The GMRES
// statistics and the depth flags are read once, after the last step.
// Graph-mode steps in two halves: everything up to the asynchronous readback
// of the device statistics, then (after a synchronisation) their harvest. A
// batch of handles enqueues all members first and harvests after, so that the
// members' work overlaps on their streams.
void rk4_graph_enqueue(sgn_ctx* ctx, double* h, double* vx, double* vy, double* sigma, double dt, int nsteps,
                       const HostIO* io = nullptr) {
  if (!ctx->step_exec || ctx->graph_dt != dt) build_step_graph(ctx, dt);
  const double* f4[4] = {h, vx, vy, sigma};
  reset_flags(ctx);
  CK(cudaMemsetAsync(ctx->gst, 0, sizeof(GmresDev), ctx->stream));
  const bool cont = continues_history(ctx, dt);
  fwd_state(ctx, f4, io);
  if (cont) same_state_flag(ctx);
  ext_history(ctx, cont);
  ctx->hist_dt = dt;
  CK(launch_spec_div<double>(ctx->G, ctx->tb, ctx->Un[1], ctx->Un[2], ctx->bh, EX(ctx)));
  for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(ctx->step_exec, ctx->stream));
  double* o4[4] = {h, vx, vy, sigma};
  inv_state(ctx, o4, io);
  CK(cudaMemcpyAsync(ctx->gst_host, ctx->gst, sizeof(GmresDev), cudaMemcpyDeviceToHost, ctx->stream));
  CK(launch_readback_scalar(ctx->scal, ctx->flags, ctx->rb_dev, EX(ctx)));
  CK(cudaMemcpyAsync(ctx->rb_host, ctx->rb_dev, sizeof(GmresReadback), cudaMemcpyDeviceToHost, ctx->stream));
}

void rk4_graph_finish(sgn_ctx* ctx, int nsteps, bool* conv_all) {
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->prof.on) ctx->prof.harvest();
  const GmresDev& st = *ctx->gst_host;
  ctx->stats.solves += (int)st.tot_solves;
  ctx->stats.matvecs += st.tot_its;
  if (ctx->opt.precision >= 1) ctx->stats.refinements += st.tot_sweeps;
  if (st.max_its > ctx->stats.max_iters) ctx->stats.max_iters = st.max_its;
  ctx->stats.last_iters = st.last_its;
  ctx->stats.last_relres = st.last_relres;
  ctx->prof.launches += (long long)nsteps * ctx->graph_fixed + st.tot_sweeps * ctx->graph_per_sweep +
                        st.tot_its * ctx->graph_per_step;
  check_flags(ctx, ctx->rb_host->flags);
  *conv_all = st.notconv == 0;
  ctx->hist_ok = ctx->opt.guess >= 2;
}

void rk4_device_graph(sgn_ctx* ctx, double* h, double* vx, double* vy, double* sigma, double dt, int nsteps,
                      bool* conv_all, const HostIO* io = nullptr) {
  rk4_graph_enqueue(ctx, h, vx, vy, sigma, dt, nsteps, io);
  rk4_graph_finish(ctx, nsteps, conv_all);
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

void sgn_default_options(sgn_options* o) {
  if (!o) return;
  o->precision = 0;
  o->restart = 20;
  o->maxit = 1000;
  o->tol = 1e-10;
  o->krasny = 0;
  o->krasny_thr = 1e-12;
  o->dealias = 0;
  o->guess = 0;
  o->graph = 0;
}

sgn_status sgn_create(int Nx, int Ny, double Lx, double Ly, double g, const sgn_options* opt, sgn_t* out) {
  if (!out) return fail(nullptr, SGN_EINVAL, "sgn_create: out is NULL");
  *out = nullptr;
  if (!pow2(Nx) || !pow2(Ny) || Nx < 8 || Ny < 8 || Nx > 4096 || Ny > 4096)
    return fail(nullptr, SGN_EINVAL, "sgn_create: Nx, Ny must be powers of two in [8, 4096]");
  if (!(Lx > 0.0) || !(Ly > 0.0) || !isfinite(Lx) || !isfinite(Ly) || !isfinite(g))
    return fail(nullptr, SGN_EINVAL, "sgn_create: Lx, Ly must be positive and finite, g finite");
  sgn_options o;
  sgn_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < 0 || o.precision > 3)
    return fail(nullptr, SGN_EINVAL,
                "sgn_create: precision must be 0 (FP64), 1 (FP32 + FP64 refinement), 2 (FP32 + double-float "
                "refinement) or 3 (precision 2 with a double-float right-hand side)");
  if (o.restart < 1 || o.restart > MAXM) return fail(nullptr, SGN_EINVAL, "sgn_create: restart must be in [1, 32]");
  if (o.maxit < 1 || !(o.tol >= 0.0) || !(o.krasny_thr >= 0.0) || o.guess < 0 || o.guess > 3 ||
      (o.graph != 0 && o.graph != 1))
    return fail(nullptr, SGN_EINVAL, "sgn_create: bad maxit, tol, krasny_thr, guess or graph");
  sgn_ctx* ctx = new (std::nothrow) sgn_ctx();
  if (!ctx) return fail(nullptr, SGN_ENOMEM, "sgn_create: host allocation failed");
  ctx->opt = o;
  ctx->g = g;
  {
    const char* tr = getenv("SGN_TRACE");
    ctx->trace = tr && tr[0] == '1';
  }
  Geom& G = ctx->G;
  G.Nx = Nx;
  G.Ny = Ny;
  G.lNx = ilog2(Nx);
  G.lNy = ilog2(Ny);
  G.Nxh = Nx / 2 + 1;
  // rows padded to an even count of entries: 16-byte row strides for the
  // FP32 spectra, as the tensor copies of the y-passes require (the padding
  // column is zero in every spectrum and has Parseval weight 0)
  G.ldS = G.Nxh + (G.Nxh & 1);
  G.Lx = Lx;
  G.Ly = Ly;
  try {
    CK(cudaGetDevice(&ctx->device));
    init_kernel_attributes<double>();
    if (o.precision >= 1) init_kernel_attributes<float>();
    if (o.precision >= 2) init_kernel_attributes_df();
    build_tables(ctx);
    const size_t ns = G.nspec();
    for (int f = 0; f < 3; ++f) {
      ctx->Un[f] = dalloc<C64>(ctx, ns);
      ctx->Us[f] = dalloc<C64>(ctx, ns);
      ctx->acc[f] = dalloc<C64>(ctx, ns);
    }
    ctx->sig = dalloc<C64>(ctx, ns);
    if (o.guess >= 2) {
      ctx->sig_s1 = dalloc<C64>(ctx, ns);
      ctx->sig_s3 = dalloc<C64>(ctx, ns);
    }
    if (o.guess == 3) {
      ctx->ext_ring = dalloc<C64>(ctx, 16 * ns);
      ctx->ext = dalloc<ExtHist>(ctx, 1);
      const ExtHist h0{0, 0, 0, 1};
      CK(cudaMemcpy(ctx->ext, &h0, sizeof(h0), cudaMemcpyHostToDevice));
    }
    ctx->bh = dalloc<C64>(ctx, ns);
    ctx->cvec = dalloc<C64>(ctx, ns);
    ctx->w = dalloc<C64>(ctx, ns);
    for (int i = 0; i < 4; ++i) ctx->tmp[i] = dalloc<C64>(ctx, ns);
    if (o.precision >= 2) {
      ctx->crd = dalloc<dfl>(ctx, G.nphys());
      ctx->ccd = dalloc<dfl>(ctx, G.nphys());
    }
    if (o.precision == 3) ctx->hd = dalloc<dfl>(ctx, G.nphys());
    if (o.precision >= 1) {
      ctx->V32 = dalloc<C32>(ctx, ns * (size_t)(o.restart + 1));
      ctx->w32 = dalloc<C32>(ctx, ns);
      for (int i = 0; i < 4; ++i) ctx->tmp32[i] = dalloc<C32>(ctx, ns);
      ctx->h32 = dalloc<float>(ctx, G.nphys());
      ctx->cr32 = dalloc<float>(ctx, G.nphys());
      ctx->cc32 = dalloc<float>(ctx, G.nphys());
      ctx->r64 = dalloc<C64>(ctx, ns);
    } else {
      ctx->V = dalloc<C64>(ctx, ns * (size_t)(o.restart + 1));
    }
    ctx->h = dalloc<double>(ctx, G.nphys());
    ctx->cr = dalloc<double>(ctx, G.nphys());
    ctx->cc = dalloc<double>(ctx, G.nphys());
    ctx->partials = dalloc<double>(ctx, (size_t)(MAXV + 2) * NBLK);
    ctx->scal = dalloc<double>(ctx, 16);
    ctx->gst = dalloc<GmresDev>(ctx, 1);
    ctx->rb_dev = dalloc<GmresReadback>(ctx, 1);
    ctx->flags = dalloc<int>(ctx, 1);
    ctx->counters = dalloc<unsigned>(ctx, 8);
    CK(cudaMemset(ctx->counters, 0, 8 * sizeof(unsigned)));
    if (o.precision >= 1) {
      const char* tv = getenv("SGN_TMA");
      if (!(tv && tv[0] == '0'))
        make_mv_tma(G, ctx->V32, o.restart + 1, ctx->tmp32[0], ctx->tmp32[1], ctx->flags, &ctx->tune, &ctx->mvt);
    }
    CK(cudaMallocHost((void**)&ctx->rb_host, sizeof(GmresReadback)));
    CK(cudaMallocHost((void**)&ctx->inv_host, 4 * sizeof(double)));
    CK(cudaMemset(ctx->flags, 0, sizeof(int)));
    CK(cudaMemset(ctx->gst, 0, sizeof(GmresDev)));
    // spectra are zero-initialised so padding never holds garbage
    for (int f = 0; f < 3; ++f) {
      CK(cudaMemset(ctx->Un[f], 0, ns * sizeof(C64)));
      CK(cudaMemset(ctx->Us[f], 0, ns * sizeof(C64)));
      CK(cudaMemset(ctx->acc[f], 0, ns * sizeof(C64)));
    }
    CK(cudaMemset(ctx->sig, 0, ns * sizeof(C64)));
    CK(cudaDeviceSynchronize());
  } catch (Fail& f) {
    g_create_error = ctx->err;
    free_all(ctx);
    delete ctx;
    return f.st;
  }
  *out = ctx;
  return SGN_OK;
}

sgn_status sgn_destroy(sgn_t ctx) {
  if (!ctx) return SGN_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  ctx->prof.destroy();
  free_all(ctx);
  delete ctx;
  return SGN_OK;
}

sgn_status sgn_set_stream(sgn_t ctx, void* stream) {
  if (!ctx) return SGN_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return SGN_OK;
}

const char* sgn_last_error(sgn_t ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

sgn_status sgn_set_profiling(sgn_t ctx, int on) {
  if (!ctx) return SGN_EINVAL;
  if (on) {
    ctx->prof.init();
    ctx->prof.reset();
  } else {
    ctx->prof.harvest();
  }
  ctx->prof.on = on != 0;
  return SGN_OK;
}

sgn_status sgn_get_profile(sgn_t ctx, double* ms, long long* counts, int n, long long* launches) {
  if (!ctx) return SGN_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  ctx->prof.harvest();
  for (int k = 0; k < n && k < PK_COUNT; ++k) {
    if (ms) ms[k] = ctx->prof.ms[k];
    if (counts) counts[k] = ctx->prof.cnt[k];
  }
  if (launches) *launches = ctx->prof.launches;
  return SGN_OK;
}

sgn_status sgn_get_stats(sgn_t ctx, sgn_stats* out) {
  if (!ctx || !out) return SGN_EINVAL;
  *out = ctx->stats;
  return SGN_OK;
}

#define API_BEGIN                                                                                  \
  if (!ctx) return SGN_EINVAL;                                                                     \
  ctx->err.clear();                                                                                \
  ctx->hist_keep = ctx->hist_ok;                                                                   \
  ctx->hist_ok = false;                                                                            \
  try {
#define API_END                                                                                    \
  }                                                                                                \
  catch (Fail & f) {                                                                               \
    return f.st;                                                                                   \
  }

sgn_status sgn_spectral_derivative(sgn_t ctx, const double* f, double* fx, double* fy) {
  API_BEGIN
  if (!f) return fail(ctx, SGN_EINVAL, "sgn_spectral_derivative: f is NULL");
  const double* fi[1] = {f};
  fwd2(ctx, fi, 1, &ctx->w);
  const C64* in[1] = {ctx->w};
  if (fx) {
    int dx[1] = {1}, dy[1] = {0};
    double* o[1] = {fx};
    inv2(ctx, in, dx, dy, 1, o);
  }
  if (fy) {
    int dx[1] = {0}, dy[1] = {1};
    double* o[1] = {fy};
    inv2(ctx, in, dx, dy, 1, o);
  }
  return SGN_OK;
  API_END
}

sgn_status sgn_fft2_r2c(sgn_t ctx, const double* f, double* fhat) {
  API_BEGIN
  if (!f || !fhat) return fail(ctx, SGN_EINVAL, "sgn_fft2_r2c: NULL pointer");
  const double* fi[1] = {f};
  fwd2(ctx, fi, 1, &ctx->w);
  const Geom& G = ctx->G;
  CK(cudaMemcpy2DAsync(fhat, G.Nxh * sizeof(C64), ctx->w, G.ldS * sizeof(C64), G.Nxh * sizeof(C64), G.Ny,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  return SGN_OK;
  API_END
}

sgn_status sgn_fft2_c2r(sgn_t ctx, const double* fhat, double* f) {
  API_BEGIN
  if (!f || !fhat) return fail(ctx, SGN_EINVAL, "sgn_fft2_c2r: NULL pointer");
  const Geom& G = ctx->G;
  CK(cudaMemcpy2DAsync(ctx->w, G.ldS * sizeof(C64), fhat, G.Nxh * sizeof(C64), G.Nxh * sizeof(C64), G.Ny,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  const C64* in[1] = {ctx->w};
  double* o[1] = {f};
  inv2(ctx, in, nullptr, nullptr, 1, o);
  return SGN_OK;
  API_END
}

sgn_status sgn_elliptic_apply(sgn_t ctx, const double* h, const double* sigma, double* out) {
  API_BEGIN
  if (!h || !sigma || !out) return fail(ctx, SGN_EINVAL, "sgn_elliptic_apply: NULL pointer");
  reset_flags(ctx);
  coef_phys(ctx, h);
  const double* fi[1] = {sigma};
  fwd2(ctx, fi, 1, &ctx->sig);
  refine_matvec(ctx, false, EX(ctx));
  const C64* in[1] = {ctx->w};
  double* o[1] = {out};
  inv2(ctx, in, nullptr, nullptr, 1, o);
  CK(launch_readback_scalar(ctx->scal, ctx->flags, ctx->rb_dev, EX(ctx)));
  sync_read(ctx);
  check_flags(ctx, ctx->rb_host->flags);
  return SGN_OK;
  API_END
}

sgn_status sgn_gmres_solve(sgn_t ctx, const double* h, const double* b, double* sigma, int* iters,
                           double* relres) {
  API_BEGIN
  if (!h || !b || !sigma) return fail(ctx, SGN_EINVAL, "sgn_gmres_solve: NULL pointer");
  reset_flags(ctx);
  coef_phys(ctx, h);
  const double* fb[1] = {b};
  fwd2(ctx, fb, 1, &ctx->bh);
  const double* fs[1] = {sigma};
  fwd2(ctx, fs, 1, &ctx->sig);
  const bool conv = gmres(ctx, iters, relres);
  const C64* in[1] = {ctx->sig};
  double* o[1] = {sigma};
  inv2(ctx, in, nullptr, nullptr, 1, o);
  CK(cudaStreamSynchronize(ctx->stream));
  if (!conv) return fail(ctx, SGN_ENOTCONV, "GMRES reached maxit before the tolerance");
  return SGN_OK;
  API_END
}

sgn_status sgn_rhs(sgn_t ctx, const double* h, const double* vx, const double* vy, double* sigma, double* ht,
                   double* vxt, double* vyt) {
  API_BEGIN
  if (!h || !vx || !vy || !sigma || !ht || !vxt || !vyt) return fail(ctx, SGN_EINVAL, "sgn_rhs: NULL pointer");
  reset_flags(ctx);
  const double* f3[3] = {h, vx, vy};
  fwd2(ctx, f3, 3, ctx->Un);
  const double* fs[1] = {sigma};
  fwd2(ctx, fs, 1, &ctx->sig);
  CK(launch_spec_div<double>(ctx->G, ctx->tb, ctx->Un[1], ctx->Un[2], ctx->bh, EX(ctx)));
  const bool conv = stage(ctx, RK_STORE_K, 0.0);
  double* o3[3] = {ht, vxt, vyt};
  inv2(ctx, (const C64* const*)ctx->acc, nullptr, nullptr, 3, o3);
  double* os[1] = {sigma};
  inv2(ctx, (const C64* const*)&ctx->sig, nullptr, nullptr, 1, os);
  CK(cudaStreamSynchronize(ctx->stream));
  if (!conv) return fail(ctx, SGN_ENOTCONV, "GMRES reached maxit before the tolerance");
  return SGN_OK;
  API_END
}

sgn_status sgn_rk4_step(sgn_t ctx, double* h, double* vx, double* vy, double* sigma, double dt, int nsteps) {
  API_BEGIN
  if (!h || !vx || !vy || !sigma) return fail(ctx, SGN_EINVAL, "sgn_rk4_step: NULL pointer");
  if (nsteps < 0 || !isfinite(dt)) return fail(ctx, SGN_EINVAL, "sgn_rk4_step: bad dt or nsteps");
  if (nsteps == 0) return SGN_OK;
  bool conv = true;
  if (ctx->opt.graph && !ctx->prof.on)
    rk4_device_graph(ctx, h, vx, vy, sigma, dt, nsteps, &conv);
  else
    rk4_device(ctx, h, vx, vy, sigma, dt, nsteps, &conv);
  CK(cudaStreamSynchronize(ctx->stream));
  if (!conv) return fail(ctx, SGN_ENOTCONV, "GMRES reached maxit in at least one stage");
  return SGN_OK;
  API_END
}

sgn_status sgn_rk4_step_batch(sgn_t* ctxs, int count, double* const* h, double* const* vx, double* const* vy,
                              double* const* sigma, double dt, int nsteps, sgn_status* status) {
  if (!ctxs || count < 1 || !h || !vx || !vy || !sigma || nsteps < 0 || !isfinite(dt)) return SGN_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !h[i] || !vx[i] || !vy[i] || !sigma[i]) return SGN_EINVAL;
    if (status) status[i] = SGN_OK;
  }
  if (nsteps == 0) return SGN_OK;
  // phase 1: enqueue every member (graph-mode members without a host wait;
  // host-loop members run to completion here)
  std::vector<sgn_status> st(count, SGN_OK);
  std::vector<char> pending(count, 0);
  for (int i = 0; i < count; ++i) {
    sgn_t ctx = ctxs[i];
    ctx->err.clear();
    ctx->hist_keep = ctx->hist_ok;
    ctx->hist_ok = false;
    try {
      if (ctx->opt.graph && !ctx->prof.on) {
        rk4_graph_enqueue(ctx, h[i], vx[i], vy[i], sigma[i], dt, nsteps);
        pending[i] = 1;
      } else {
        bool conv = true;
        rk4_device(ctx, h[i], vx[i], vy[i], sigma[i], dt, nsteps, &conv);
        CK(cudaStreamSynchronize(ctx->stream));
        if (!conv) st[i] = fail(ctx, SGN_ENOTCONV, "GMRES reached maxit in at least one stage");
      }
    } catch (Fail& f) {
      st[i] = f.st;
    }
  }
  // phase 2: wait for and harvest the graph-mode members
  for (int i = 0; i < count; ++i) {
    if (!pending[i]) continue;
    sgn_t ctx = ctxs[i];
    try {
      bool conv = true;
      rk4_graph_finish(ctx, nsteps, &conv);
      if (!conv) st[i] = fail(ctx, SGN_ENOTCONV, "GMRES reached maxit in at least one stage");
    } catch (Fail& f) {
      st[i] = f.st;
    }
  }
  sgn_status first = SGN_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (first == SGN_OK && st[i] != SGN_OK) first = st[i];
  }
  return first;
}

sgn_status sgn_rk4_step_host(sgn_t ctx, double* h, double* vx, double* vy, double* sigma, double dt,
                             int nsteps) {
  API_BEGIN
  if (!h || !vx || !vy || !sigma) return fail(ctx, SGN_EINVAL, "sgn_rk4_step_host: NULL pointer");
  if (nsteps < 0 || !isfinite(dt)) return fail(ctx, SGN_EINVAL, "sgn_rk4_step_host: bad dt or nsteps");
  ensure_phys(ctx);
  const size_t bytes = ctx->G.nphys() * sizeof(double);
  double* hv[4] = {h, vx, vy, sigma};
  if (nsteps == 0) {
    for (int i = 0; i < 4; ++i) CK(cudaMemcpyAsync(ctx->phys[i], hv[i], bytes, cudaMemcpyHostToDevice, ctx->stream));
    for (int i = 0; i < 4; ++i) CK(cudaMemcpyAsync(hv[i], ctx->phys[i], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SGN_OK;
  }
  if (!ctx->io_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 9; ++i) CK(cudaEventCreateWithFlags(&ctx->io_ev[i], cudaEventDisableTiming));
  }
  HostIO io{};
  io.cs = ctx->io_stream;
  io.bytes = bytes;
  for (int i = 0; i < 4; ++i) {
    io.in[i] = ctx->io_ev[i];
    io.out[i] = ctx->io_ev[4 + i];
    io.host[i] = hv[i];
  }
  // the copies follow whatever the handle's stream holds already; whatever
  // happens below, no copy into the caller's buffers outlives the call
  struct IoSync {
    cudaStream_t s;
    ~IoSync() { cudaStreamSynchronize(s); }
  } io_sync{io.cs};
  CK(cudaEventRecord(ctx->io_ev[8], ctx->stream));
  CK(cudaStreamWaitEvent(io.cs, ctx->io_ev[8], 0));
  for (int i = 0; i < 4; ++i) {
    CK(cudaMemcpyAsync(ctx->phys[i], hv[i], bytes, cudaMemcpyHostToDevice, io.cs));
    CK(cudaEventRecord(io.in[i], io.cs));
  }
  bool conv = true;
  if (ctx->opt.graph && !ctx->prof.on)
    rk4_device_graph(ctx, ctx->phys[0], ctx->phys[1], ctx->phys[2], ctx->phys[3], dt, nsteps, &conv, &io);
  else
    rk4_device(ctx, ctx->phys[0], ctx->phys[1], ctx->phys[2], ctx->phys[3], dt, nsteps, &conv, &io);
  CK(cudaStreamSynchronize(io.cs));
  CK(cudaStreamSynchronize(ctx->stream));
  if (!conv) return fail(ctx, SGN_ENOTCONV, "GMRES reached maxit in at least one stage");
  return SGN_OK;
  API_END
}

static bool coarse_side_ok(const sgn_ctx* ctx, int n) {
  return n >= 16 && (n & (n - 1)) == 0 && n <= ctx->G.Nx && n <= ctx->G.Ny;
}

sgn_status sgn_set_learned_guess(sgn_t ctx, void* net, int n, const float in_scale[4], float out_scale,
                                 int tau_power) {
  API_BEGIN
  // the captured step graph contains the network (or not): rebuild it
  free_graph(ctx);
  if (!net) {
    ctx->net = nullptr;
    return SGN_OK;
  }
  sgn_unet_t u = static_cast<sgn_unet_t>(net);
  if (!coarse_side_ok(ctx, n) || sgn_unet_side(u) != n)
    return fail(ctx, SGN_EINVAL, "sgn_set_learned_guess: n must be a power of two in [16, min(Nx, Ny)] and the "
                                 "network's side");
  if (!in_scale || !isfinite(out_scale) || tau_power < 0 || tau_power > 2)
    return fail(ctx, SGN_EINVAL, "sgn_set_learned_guess: bad in_scale, out_scale or tau_power");
  if (ctx->ln != n) {
    coarse_alloc(ctx, n, &ctx->ltw, &ctx->lY);
    ctx->lin = dalloc<float>(ctx, (size_t)4 * n * n);
    ctx->lout = dalloc<float>(ctx, (size_t)n * n);
    ctx->ln = n;
  }
  for (int f = 0; f < 4; ++f) ctx->in_scale[f] = in_scale[f];
  ctx->out_scale = out_scale;
  ctx->tau_pow = tau_power;
  ctx->net = u;
  CK(cudaStreamSynchronize(ctx->stream));
  return SGN_OK;
  API_END
}

sgn_status sgn_record_learned(sgn_t ctx, int n, float* buf, int capacity, int tau_power) {
  API_BEGIN
  if (!buf) {
    ctx->rec_buf = nullptr;
    return SGN_OK;
  }
  if (ctx->opt.graph) return fail(ctx, SGN_EINVAL, "sgn_record_learned: needs the host-driven loop (graph = 0)");
  if (!coarse_side_ok(ctx, n) || capacity < 1 || tau_power < 0 || tau_power > 2)
    return fail(ctx, SGN_EINVAL, "sgn_record_learned: bad n, capacity or tau_power");
  if (ctx->rec_n != n) {
    coarse_alloc(ctx, n, &ctx->rtw, &ctx->rY);
    ctx->rec_n = n;
  }
  if (!ctx->sig_fb) ctx->sig_fb = dalloc<C64>(ctx, ctx->G.nspec());
  ctx->rec_buf = buf;
  ctx->rec_cap = capacity;
  ctx->rec_count = 0;
  ctx->rec_tau_pow = tau_power;
  return SGN_OK;
  API_END
}

sgn_status sgn_recorded_count(sgn_t ctx, int* count) {
  if (!ctx || !count) return SGN_EINVAL;
  *count = ctx->rec_count;
  return SGN_OK;
}

sgn_status sgn_coarse_sample(sgn_t ctx, const double* f, int n, float* out) {
  API_BEGIN
  if (!f || !out || !coarse_side_ok(ctx, n)) return fail(ctx, SGN_EINVAL, "sgn_coarse_sample: bad argument");
  if (ctx->cn != n) {
    coarse_alloc(ctx, n, &ctx->ctw, &ctx->cY);
    ctx->cn = n;
  }
  const float2* tw = ctx->ctw;
  float2* Y = ctx->cY;
  const double* fi[1] = {f};
  fwd2(ctx, fi, 1, &ctx->w);
  CoarseIn ci{};
  ci.spec[0] = ctx->w;
  ci.out[0] = out;
  ci.scale[0] = 1.f;
  CK(launch_restrict(ctx->G, ci, 1, n, tw, Y, EX(ctx)));
  CK(cudaStreamSynchronize(ctx->stream));
  return SGN_OK;
  API_END
}

sgn_status sgn_coarse_embed(sgn_t ctx, const float* fc, int n, double scale, double* f) {
  API_BEGIN
  if (!f || !fc || !coarse_side_ok(ctx, n) || !isfinite(scale))
    return fail(ctx, SGN_EINVAL, "sgn_coarse_embed: bad argument");
  if (ctx->cn != n) {
    coarse_alloc(ctx, n, &ctx->ctw, &ctx->cY);
    ctx->cn = n;
  }
  const float2* tw = ctx->ctw;
  float2* Y = ctx->cY;
  const double* fi[1] = {f};
  fwd2(ctx, fi, 1, &ctx->w);
  CK(launch_prolong_add(ctx->G, fc, n, tw, Y, nullptr, scale, ctx->w, EX(ctx)));
  const C64* in[1] = {ctx->w};
  double* o[1] = {f};
  inv2(ctx, in, nullptr, nullptr, 1, o);
  CK(cudaStreamSynchronize(ctx->stream));
  return SGN_OK;
  API_END
}

sgn_status sgn_diagnostics(sgn_t ctx, const double* h, const double* vx, const double* vy, sgn_diag* out) {
  API_BEGIN
  if (!h || !vx || !vy || !out) return fail(ctx, SGN_EINVAL, "sgn_diagnostics: NULL pointer");
  if (!ctx->diag) {
    ctx->diag = dalloc<DiagDev>(ctx, 1);
    CK(cudaMallocHost((void**)&ctx->diag_host, sizeof(DiagDev)));
  }
  const Geom& G = ctx->G;
  unsigned* cnt = ctx->counters + 7;  // the three passes run in order on one stream
  CK(launch_diag_max(G, h, vy, ctx->partials, cnt, ctx->diag, EX(ctx)));
  CK(launch_diag_soliton(G, h, vx, ctx->g, ctx->partials, cnt, ctx->diag, EX(ctx)));
  const double* f3[3] = {h, vx, vy};
  fwd2(ctx, f3, 3, ctx->tmp);
  CK(launch_diag_tail(G, ctx->tmp[0], ctx->tmp[1], ctx->tmp[2], ctx->partials, cnt, ctx->diag, EX(ctx)));
  CK(cudaMemcpyAsync(ctx->diag_host, ctx->diag, sizeof(DiagDev), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->prof.on) ctx->prof.harvest();
  const DiagDev& d = *ctx->diag_host;
  out->h_max = d.h_max;
  out->i_max = d.i_max;
  const long long jx = d.i_max % G.Nx, jy = d.i_max / G.Nx;
  out->x_s = -0.5 * G.Lx + G.Lx * (double)jx / (double)G.Nx;
  out->y_s = -0.5 * G.Ly + G.Ly * (double)jy / (double)G.Ny;
  out->c_fit = sqrt(ctx->g * d.h_max);
  out->dev_h = d.dev_h;
  out->dev_vx = d.dev_vx;
  out->max_vy = d.max_vy;
  for (int k = 0; k < 3; ++k) out->tail[k] = d.tail[k];
  return SGN_OK;
  API_END
}

// ------------------------------------------------------------- autotuning
namespace {

// One timed operation of the autotuner: the FP32, FP64 or double-float matvec
// or the RHS, on the handle's scratch.
void tune_run(sgn_ctx* ctx, int op) {
  const Geom& G = ctx->G;
  switch (op) {
    case 0:  // FP32 matvec (inner solve of precisions 1, 2)
      CK(launch_matvec<float>(G, ctx->tb32, ctx->V32, ctx->cr32, ctx->cc32, ctx->w32, ctx->tmp32, true, EX(ctx),
                              nullptr, 0, &ctx->mvt));
      break;
    case 1:  // FP64 matvec of precision 0 (Arnoldi and residual)
      CK(launch_matvec<double>(G, ctx->tb, ctx->V, ctx->cr, ctx->cc, ctx->w, ctx->tmp, true, EX(ctx)));
      break;
    case 2:  // refinement matvec of precisions 1 (FP64) and 2 (double-float)
      refine_matvec(ctx, true, EX_REFINE(ctx));
      break;
    default: {  // one RHS evaluation (K into the RK accumulator, scratch between steps)
      RkArgs rk{};
      rk.mode = RK_STORE_K;
      rk.g = ctx->g;
      launch_rhs_ctx(ctx, ctx->Un, nullptr, rk);
    }
  }
}

// Average launch time (us) of profiling class cls over reps runs of op, after
// one untimed run.
constexpr double kTuneMargin = 0.02;

double tune_time(sgn_ctx* ctx, int op, int cls, int reps) {
  ctx->prof.on = false;
  tune_run(ctx, op);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.reset();
  ctx->prof.on = true;
  for (int r = 0; r < reps; ++r) tune_run(ctx, op);
  ctx->prof.harvest();
  ctx->prof.on = false;
  const long long c = ctx->prof.cnt[cls];
  return c > 0 ? 1e3 * ctx->prof.ms[cls] / (double)c : 1e30;
}

}  // namespace

sgn_status sgn_autotune(sgn_t ctx, int reps, sgn_tuning* out) {
  API_BEGIN
  if (reps < 1 || reps > 100) return fail(ctx, SGN_EINVAL, "sgn_autotune: reps must be in [1, 100]");
  const Geom& G = ctx->G;
  const int prec = ctx->opt.precision;
  CK(cudaStreamSynchronize(ctx->stream));
  free_graph(ctx);  // a captured step keeps the shapes it was captured with
  ctx->prof.init();
  const bool was_on = ctx->prof.on;
  const long long launches0 = ctx->prof.launches;
  ctx->prof.harvest();
  sgn_tuning res{};
  // (op, arithmetic, the passes it times with their profiling classes)
  struct Job {
    int op, type;
    int pass[3], cls[3];
  };
  std::vector<Job> jobs;
  if (prec >= 1) {
    jobs.push_back({0, TT_F32, {TP_MV_YINV, TP_MV_X, TP_MV_YFWD}, {PK_MV_YINV, PK_MV_X, PK_MV_YFWD}});
    jobs.push_back({2, prec >= 2 ? TT_DFL : TT_F64, {TP_MV_YINV, TP_MV_X, TP_MV_YFWD},
                    {PK_REF_YINV, PK_REF_X, PK_REF_YFWD}});
    jobs.push_back({3, prec == 3 ? TT_DFL : TT_F32, {TP_RHS_YINV, TP_RHS_X, TP_RHS_YFWD},
                    {PK_RHS_YINV, PK_RHS_X, PK_RHS_YFWD}});
  } else {
    jobs.push_back({1, TT_F64, {TP_MV_YINV, TP_MV_X, TP_MV_YFWD}, {PK_MV_YINV, PK_MV_X, PK_MV_YFWD}});
    jobs.push_back({3, TT_F64, {TP_RHS_YINV, TP_RHS_X, TP_RHS_YFWD}, {PK_RHS_YINV, PK_RHS_X, PK_RHS_YFWD}});
  }
  auto remap = [&]() {
    if (prec >= 1 && ctx->mvt.ok)
      make_mv_tma(G, ctx->V32, ctx->opt.restart + 1, ctx->tmp32[0], ctx->tmp32[1], ctx->flags, &ctx->tune,
                  &ctx->mvt);
  };
  for (const Job& jb : jobs) {
    for (int k = 0; k < 3; ++k) {
      const int ps = jb.pass[k], ty = jb.type;
      const int def = pass_default_threads(G, ty, ps);
      int cand[16];
      const int nc = pass_candidates(G, ty, ps, cand, 16);
      ctx->tune.tpb[ty][ps] = def;
      ctx->tune.plan[ty][ps] = 0;
      remap();
      const double t_def = tune_time(ctx, jb.op, jb.cls[k], reps);
      int best = def;
      double t_best = t_def;
      // a candidate replaces the built-in shape or plan only when it is at
      // least kTuneMargin faster: timings of one pass repeat to ~1%, and a
      // pick made on noise can lose more than that in the running step
      for (int c = 0; c < nc; ++c) {
        if (cand[c] == def) continue;
        ctx->tune.tpb[ty][ps] = cand[c];
        remap();
        const double t = tune_time(ctx, jb.op, jb.cls[k], reps);
        if (t < (1.0 - kTuneMargin) * t_best) {
          t_best = t;
          best = cand[c];
        }
      }
      ctx->tune.tpb[ty][ps] = best;
      remap();
      // the radix plan of the pass's axis, at the picked shape (one plan when
      // 3 divides log2 of the length)
      const int lN = (ps == TP_MV_X || ps == TP_RHS_X) ? G.lNx : G.lNy;
      int plan = 0;
      if (lN % 3 != 0) {
        ctx->tune.plan[ty][ps] = 1;
        const double t = tune_time(ctx, jb.op, jb.cls[k], reps);
        if (t < (1.0 - kTuneMargin) * t_best) {
          t_best = t;
          plan = 1;
        }
        ctx->tune.plan[ty][ps] = plan;
      }
      res.threads[ty][ps] = best;
      res.default_threads[ty][ps] = def;
      res.plan[ty][ps] = plan;
      res.us_default[ty][ps] = (float)t_def;
      res.us_tuned[ty][ps] = (float)t_best;
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.reset();
  ctx->prof.launches = launches0;
  ctx->prof.on = was_on;
  if (out) *out = res;
  return SGN_OK;
  API_END
}

sgn_status sgn_set_tuning(sgn_t ctx, const sgn_tuning* t) {
  API_BEGIN
  if (!t) return fail(ctx, SGN_EINVAL, "sgn_set_tuning: NULL tuning");
  const Geom& G = ctx->G;
  Tune nt{};
  for (int ty = 0; ty < TT_COUNT; ++ty)
    for (int ps = 0; ps < TP_COUNT; ++ps) {
      const int th = t->threads[ty][ps], pl = t->plan[ty][ps];
      if (pl != 0 && pl != 1) return fail(ctx, SGN_EINVAL, "sgn_set_tuning: a plan is not 0 or 1");
      if (th != 0) {
        int cand[16];
        const int nc = pass_candidates(G, ty, ps, cand, 16);
        bool ok = th == pass_default_threads(G, ty, ps);
        for (int c = 0; c < nc && !ok; ++c) ok = cand[c] == th;
        if (!ok) return fail(ctx, SGN_EINVAL, "sgn_set_tuning: a thread count is not a shape of its pass");
      }
      nt.tpb[ty][ps] = th;
      nt.plan[ty][ps] = pl;
    }
  CK(cudaStreamSynchronize(ctx->stream));
  free_graph(ctx);  // a captured step keeps the shapes it was captured with
  ctx->tune = nt;
  if (ctx->opt.precision >= 1 && ctx->mvt.ok)
    make_mv_tma(G, ctx->V32, ctx->opt.restart + 1, ctx->tmp32[0], ctx->tmp32[1], ctx->flags, &ctx->tune,
                &ctx->mvt);
  return SGN_OK;
  API_END
}

sgn_status sgn_invariants(sgn_t ctx, const double* h, const double* vx, const double* vy, const double* sigma,
                          double out[4]) {
  API_BEGIN
  if (!h || !vx || !vy || !sigma || !out) return fail(ctx, SGN_EINVAL, "sgn_invariants: NULL pointer");
  ensure_phys(ctx);
  const double* fs[1] = {sigma};
  fwd2(ctx, fs, 1, &ctx->w);
  const C64* in[2] = {ctx->w, ctx->w};
  int dx[2] = {1, 0}, dy[2] = {0, 1};
  double* o[2] = {ctx->phys[0], ctx->phys[1]};
  inv2(ctx, in, dx, dy, 2, o);
  CK(launch_invariant_sums(ctx->G, h, vx, vy, sigma, ctx->phys[0], ctx->phys[1], ctx->g, ctx->partials,
                           EX(ctx)));
  CK(launch_reduce(ctx->partials, 4, ctx->scal + 4, false, nullptr, EX(ctx)));
  CK(cudaMemcpyAsync(ctx->inv_host, ctx->scal + 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double dA = ctx->G.Lx * ctx->G.Ly / (double)ctx->G.nphys();
  for (int q = 0; q < 4; ++q) out[q] = ctx->inv_host[q] * dA;
  return SGN_OK;
  API_END
}

}  // extern "C"
