/*
 * sgn.h - C ABI of the GB300 (sm_103a) 2D Serre-Green-Naghdi hot path.
 *
 * Method: Gavrilyuk & Klein, "Numerical study of the Serre-Green-Naghdi
 * equations in 2D" (arXiv 2306.09731). The library integrates the potential
 * form of SGN in the variables (h, v = grad phi):
 *     h_t = -div(h u),  u = v - grad(sigma)/h                  Section 2.2, Eq. (1)
 *     v_t = -grad( |v|^2/2 - |grad sigma|^2/(2h^2) + g h - 9 sigma^2/(2h^4) )
 *                                                             Section 3 (v-form of Eq. (2))
 *     L[sigma] = 3 sigma/h^3 - div(grad sigma / h) = -div v    Section 3, Eq. (sigmav)
 * by Fourier collocation on a periodic box, left-preconditioned restarted GMRES
 * with M = 3 + kx^2 + ky^2 for sigma, and classic RK4 in time (Section 3).
 *
 * Conventions shared by every call:
 *  - Grid: Nx x Ny points, both powers of two with 8 <= N <= 4096. Lx, Ly are
 *    FULL periods (the paper's 2*pi*L_x); the box is [-Lx/2, Lx/2) x [-Ly/2, Ly/2)
 *    and x_j = -Lx/2 + j*Lx/Nx. h_inf = 1.
 *  - Field pointers are DEVICE pointers (except the *_host variants) to real
 *    float64 arrays laid out row-major [Ny][Nx], x fastest, 8-byte aligned,
 *    not aliasing each other unless stated. The caller owns them.
 *  - Wavenumbers k = 2*pi*m/L; the Nyquist wavenumber is set to 0 in every i*k
 *    multiplier and in M, so M equals L exactly at h = 1.
 *  - Calls are enqueued on the handle's stream (sgn_set_stream; default: the
 *    legacy default stream). Calls that run GMRES synchronise that stream once
 *    per GMRES iteration to read the convergence test.
 *  - Every call returns a status; on failure sgn_last_error() gives a message.
 *    A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef SGN_H
#define SGN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgn_ctx* sgn_t;

typedef enum {
  SGN_OK = 0,
  SGN_EINVAL = 1,       /* bad argument: null pointer, size, option */
  SGN_ENOTCONV = 2,     /* GMRES hit maxit; the best iterate is still returned */
  SGN_ECAVITATION = 3,  /* h <= 0 somewhere (the paper assumes h > 0, Section 1) */
  SGN_ENONFINITE = 4,   /* NaN or Inf in h */
  SGN_ECUDA = 5,        /* a CUDA runtime error; see sgn_last_error */
  SGN_ENOMEM = 6        /* device allocation failed in sgn_create */
} sgn_status;

typedef struct {
  int precision;      /* 0 = FP64 throughout; 1 = FP32 transforms, pointwise work and
                         inner GMRES, with FP64 state, dot products, Givens and an
                         FP64 refinement residual (same FP64 tolerance test); the
                         FP32 passes form only the right-hand side's part nonlinear
                         in the state, and the RK update adds the linear part
                         (-i k.v - |k|^2 sigma in h_t, -i k g h in v_t) in FP64;
                         2 = as 1, but the refinement residual's matvec and the
                         coefficient pass run in double-float arithmetic (a value is
                         the sum of two FP32 numbers: 48-bit significand, FP32
                         exponent range, so 1/h^3 must stay below ~3e38); the
                         tolerance test is unchanged;
                         3 = as 2, with the right-hand side of the RK4 stages (its
                         transforms, products and the K spectra) in double-float as
                         well: only the inner GMRES runs in FP32, so the trajectory
                         follows the FP64 one to its own rounding (for long runs
                         whose small modes grow, where the FP32 rounding of the
                         nonlinear part would seed them); also converts the state in
                         double-float */
  int restart;        /* GMRES restart length m, 1..32 (default 20) */
  int maxit;          /* cap on GMRES matvecs per solve, all cycles (default 1000) */
  double tol;         /* stop when ||M^-1(b - L sigma)||_2 <= tol ||M^-1 b||_2 (default 1e-10) */
  int krasny;         /* 1: Krasny filter after every RK4 step (Section 3); default 0 */
  double krasny_thr;  /* zero DFT coefficients with |c|/(Nx*Ny) < thr (default 1e-12) */
  int dealias;        /* 1: 2/3-rule mask on the RHS spectra (not in the paper); default 0 */
  int guess;          /* GMRES start: 0 = the last computed sigma (Section 3), 1 = zero,
                         2 = linear extrapolation in time inside sgn_rk4_step (stage 2 from
                         sigma(t) and the previous step's sigma(t - dt/2), stage 4 from
                         sigma(t + dt/2) and sigma(t)); the previous step's sigma is kept
                         from the handle's last RK4 call when the new call has the same dt
                         and its input state is that call's output (within 1e-8 of the
                         largest Fourier coefficient); every solve still meets tol;
                         3 = guess 2 until the handle has solved 3 steps of the
                         trajectory, then each stage starts from the polynomial in time
                         through the same stage's sigma of the last 3 (quadratic) or 4
                         (cubic) steps: O(dt^3) / O(dt^4) against guess 2's O(dt^2)
                         (with the FP32 right-hand side of precisions 1 and 2 the
                         rounding noise of the stage states bounds that gain, and near
                         rest it is gone);
                         it keeps 16 spectra of history (16 * Ny * (Nx/2 + 2) complex
                         doubles), carried across calls by guess 2's rule */
  int graph;          /* 1: sgn_rk4_step and sgn_rk4_step_host run each RK4 step as one
                         CUDA graph whose GMRES loops are conditional WHILE nodes driven
                         by device-side tests (no host synchronisation inside the call;
                         cavitation and non-finite h are reported when the call ends);
                         the graph is built on the first call and rebuilt when dt
                         changes. 0 (default): the host-driven loop, one stream
                         synchronisation per Arnoldi step. Profiling (sgn_set_profiling)
                         always takes the host-driven loop. */
} sgn_options;

/* Fills *opt with the defaults listed above. */
void sgn_default_options(sgn_options* opt);

/* Creates a handle for an Nx x Ny grid of full periods Lx x Ly and gravity g.
 * Allocates every device buffer the calls need (twiddle tables, spectra,
 * the Krylov basis of restart+1 vectors) on the current device. opt may be
 * NULL for the defaults. Returns SGN_EINVAL for unsupported sizes, SGN_ENOMEM
 * if allocation fails. */
sgn_status sgn_create(int Nx, int Ny, double Lx, double Ly, double g,
                      const sgn_options* opt, sgn_t* out);

/* Frees the handle and its device memory (after synchronising its stream). */
sgn_status sgn_destroy(sgn_t ctx);

/* Sets the CUDA stream (a cudaStream_t passed as void*) for later calls. */
sgn_status sgn_set_stream(sgn_t ctx, void* cuda_stream);

/* Spectral derivatives of a real field (Section 3, g_x ~ i k_x g):
 * fx = d f/dx, fy = d f/dy. Either output may be NULL. */
sgn_status sgn_spectral_derivative(sgn_t ctx, const double* f, double* fx, double* fy);

/* 2D real-to-complex DFT (unnormalised, e^{-i k x}): f [Ny][Nx] real ->
 * fhat [Ny][Nx/2+1] complex, stored as interleaved (re, im) float64 pairs,
 * i.e. 2*Ny*(Nx/2+1) doubles. Row ky holds kx = 0..Nx/2. */
sgn_status sgn_fft2_r2c(sgn_t ctx, const double* f, double* fhat);

/* Inverse of sgn_fft2_r2c including the 1/(Nx*Ny) factor. The imaginary parts
 * of the kx = 0 and kx = Nx/2 entries after the y-transform are ignored. */
sgn_status sgn_fft2_c2r(sgn_t ctx, const double* fhat, double* f);

/* out = L[sigma] = 3 sigma/h^3 - d/dx(sigma_x/h) - d/dy(sigma_y/h)
 * (Section 3, Eq. (sigmav)), unpreconditioned, in the arithmetic of the
 * handle's refinement residual (double-float for precision 2, else FP64).
 * Returns SGN_ECAVITATION / SGN_ENONFINITE if h is not positive and finite. */
sgn_status sgn_elliptic_apply(sgn_t ctx, const double* h, const double* sigma, double* out);

/* Solves L[sigma] = b by left-preconditioned restarted GMRES (Section 3;
 * Saad & Schultz), sigma_inout is the initial guess on entry and the solution
 * on exit. iters (may be NULL) receives the matvec count; relres (may be NULL)
 * the final estimate of ||M^-1 r|| / ||M^-1 b||. SGN_ENOTCONV if maxit is hit. */
sgn_status sgn_gmres_solve(sgn_t ctx, const double* h, const double* b,
                           double* sigma_inout, int* iters, double* relres);

/* One evaluation of the right-hand side (Section 2.2 Eq. (1), Section 3):
 * solves Eq. (sigmav) for sigma from the guess in sigma_inout (written back),
 * then ht = -div(h u), vxt, vyt = -grad F. With dealias = 1 the outputs are
 * 2/3-masked. */
sgn_status sgn_rhs(sgn_t ctx, const double* h, const double* vx, const double* vy,
                   double* sigma_inout, double* ht, double* vxt, double* vyt);

/* Advances (h, vx, vy) in place by nsteps classic RK4 steps of size dt
 * (Section 3). Each stage's GMRES starts from the last computed sigma
 * (sigma_inout on entry, the stage-4 sigma of the last step on exit). The
 * state is held in spectral form between steps; the Krasny filter, when on,
 * runs after every step. */
sgn_status sgn_rk4_step(sgn_t ctx, double* h, double* vx, double* vy,
                        double* sigma_inout, double dt, int nsteps);

/* sgn_rk4_step on HOST arrays (pageable or pinned): copies the four fields
 * to the device, steps, and copies them back before returning. */
sgn_status sgn_rk4_step_host(sgn_t ctx, double* h, double* vx, double* vy,
                             double* sigma_inout, double dt, int nsteps);

/* Conserved quantities (Section 2.3, Eqs. (total_mass), (total_momentum),
 * (total_energy)) by the rectangle rule with u = v - grad(sigma)/h:
 * out[0] = mass sum(h - 1) dA, out[1..2] = momentum sum(h u) dA,
 * out[3] = energy sum(h|u|^2/2 + 3 sigma^2/(2h^3) + g(h-1)^2/2) dA.
 * out is a HOST array of 4 doubles; the call synchronises the stream. */
sgn_status sgn_invariants(sgn_t ctx, const double* h, const double* vx,
                          const double* vy, const double* sigma, double out[4]);

/* Statistics of the last GMRES-using call: total matvecs, number of solves,
 * the largest iteration count of one solve and the last relative residual. */
typedef struct {
  long long matvecs;      /* Arnoldi matvecs (FP32 ones in precision 1) */
  int solves;
  int max_iters;
  double last_relres;
  int last_iters;
  long long refinements;  /* FP64 residual evaluations of precision 1 */
} sgn_stats;
sgn_status sgn_get_stats(sgn_t ctx, sgn_stats* out);

/* Per-kernel-class timing with CUDA events on the handle's stream (off by
 * default). Classes, in order: 0 coefficients of Eq. (sigmav) from h_hat,
 * 1-3 the matvec passes (y-inverse, fused x-pass, y-forward + M^-1),
 * 4-6 the RHS passes (y-inverse, fused x-pass, y-forward + RK4 update),
 * 7 GMRES vector kernels and reductions, 8 conversions at call boundaries,
 * 9-11 the FP64 refinement matvec passes of precision 1 (the matvec classes
 * 1-3 then count only its FP32 inner matvecs), 12 the RK4 stage update.
 * sgn_set_profiling(ctx, 1) clears the counters; sgn_get_profile fills up to n
 * entries of ms (summed milliseconds) and counts (timed launches) and
 * *launches with the number of kernels launched since the last clear. */
#define SGN_PROFILE_CLASSES 13
sgn_status sgn_set_profiling(sgn_t ctx, int on);
sgn_status sgn_get_profile(sgn_t ctx, double* ms, long long* counts, int n, long long* launches);

/* Allocation-free L[sigma]. The paper has no counterpart: this exists for
 * callers that cannot allocate device memory, e.g. a host application whose
 * own pool or caching allocator already holds the GPU's memory budget, a
 * plugin that must not allocate behind its framework's back, or a
 * latency-sensitive loop that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree.
 * Computes out = L[sigma] exactly as sgn_elliptic_apply does (same kernels,
 * device field pointers in the same layout), without a handle: every
 * intermediate lives in one static device array sized for
 * SGN_NOALLOC_MAX_POINTS grid points (about 4 MB), held on every GPU that
 * loads the library until the process exits. The call allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).
 *  - Nx, Ny: powers of two in [8, 4096] as for sgn_create, with
 *    Nx*Ny <= SGN_NOALLOC_MAX_POINTS (so 4096 x 16 and 16 x 4096 are the
 *    longest axes). Any other size, or a NULL pointer, returns SGN_EINVAL
 *    with a message in sgn_last_error(NULL).
 *  - Every call looks up the static array's address on the current device
 *    (cudaGetSymbolAddress); the first call on a device also loads the
 *    library's device code there, so make that first call before any stream
 *    capture. No host-side state is cached, so calls from several host
 *    threads share nothing on the host but sgn_last_error(NULL), which is kept
 *    per host thread.
 *  - Every call uses the same array and leaves its contents behind: calls
 *    that overlap on the GPU (other streams, other host threads) race. Calls
 *    on one stream, one after another, are safe.
 *  - Enqueued on cuda_stream (a cudaStream_t, NULL for the legacy default
 *    stream); the call synchronises that stream before returning its status
 *    (SGN_ECAVITATION / SGN_ENONFINITE as in sgn_elliptic_apply). */
#define SGN_NOALLOC_MAX_POINTS 65536
sgn_status sgn_elliptic_apply_noalloc(int Nx, int Ny, double Lx, double Ly,
                                      const double* h, const double* sigma, double* out,
                                      void* cuda_stream);

/* Message for the last failing call on ctx. With ctx NULL: the message of
 * the last failing handle-less call (sgn_create, sgn_elliptic_apply_noalloc)
 * made by the calling host thread (one slot per thread, like errno). */
const char* sgn_last_error(sgn_t ctx);

/* Ensembles: count independent problems, each with its own handle
 * (its own grid size, options and stream, set with sgn_set_stream), advanced
 * by nsteps RK4 steps each, like sgn_rk4_step on h[i], vx[i], vy[i],
 * sigma[i]. Members created with graph = 1 are all enqueued on their streams
 * before any is waited for, so members on distinct streams run concurrently on
 * the GPU; members with graph = 0 run one after another (their GMRES loop
 * synchronises). status (may be NULL) receives each member's status; the
 * return value is SGN_OK or the first failing member's status. Results are
 * those of sgn_rk4_step on each member. */
sgn_status sgn_rk4_step_batch(sgn_t* ctxs, int count, double* const* h, double* const* vx, double* const* vy,
                              double* const* sigma, double dt, int nsteps, sgn_status* status);

/* ------------------------------------------------------------------------
 * Monitoring quantities of the paper's experiments (Sections 3 and 4):
 *   h_max, i_max, x_s, y_s  L-infinity norm of h and the grid point where it is
 *                           reached (lowest flat index y*Nx + x on ties; NaN
 *                           counts as largest), x_j = -Lx/2 + j Lx/Nx as in
 *                           sgn_create (Section 4.1 locates the crest this way)
 *   c_fit                   sqrt(g h_max): the speed of the line solitary wave
 *                           of Eq. (sol) whose crest is h_max (h_inf = 1;
 *                           Section 4.2 fits c from the maximum this way)
 *   dev_h, dev_vx           max |h - h_c|, max |vx - v_c| over the grid, h_c and
 *                           v_c of Eq. (sol) with speed c_fit centred at x_s,
 *                           nearest periodic image in x; NaN if h_max <= 1
 *   max_vy                  max |vy| (zero for a line solitary wave)
 *   tail[3]                 max |DFT coefficient| / (Nx Ny) of h, vx, vy over
 *                           the outermost modes, 16 |m_x| >= 7 Nx or
 *                           16 |m_y| >= 7 Ny (the decay of the DFT
 *                           coefficients that Section 3 reads as resolution)
 * h, vx, vy: device float64 [Ny][Nx], read only. Uses the handle's scratch
 * spectra; synchronises the handle's stream. */
typedef struct {
  double h_max;
  long long i_max;
  double x_s, y_s;
  double c_fit;
  double dev_h, dev_vx;
  double max_vy;
  double tail[3];
} sgn_diag;

sgn_status sgn_diagnostics(sgn_t ctx, const double* h, const double* vx, const double* vy, sgn_diag* out);

/* ------------------------------------------------------------------------
 * Launch shapes of the transform passes. Every 2D transform of Section 3's
 * spectral derivatives runs as an x-pass over row pairs and a y-pass over
 * column tiles. How many columns one y-pass block transforms (row pairs for
 * an x-pass) trades the width of its memory accesses against the number of
 * blocks, and the best choice depends on the grid and the arithmetic: a 256^2
 * grid has 129 columns, which the built-in 4096-point-sized tiles spread over
 * a handful of blocks. sgn_autotune times every candidate shape of every pass
 * the handle runs (threads per block: powers of two, whole columns or row
 * pairs, up to each kernel's launch bound), `reps` launches each after one
 * untimed launch, on the handle's own buffers, and keeps the fastest (a shape
 * or plan other than the built-in one only when it is at least 2% faster, so
 * that timing noise does not decide); later
 * calls of the handle use those shapes. Shapes change no formula: FP64 and
 * double-float results are bitwise identical to those of the built-in shapes;
 * an FP32 pass whose picked shape differs from the built-in one runs the
 * kernel compiled for runtime lengths, whose FP32 rounding may differ in the
 * last bit (multiply-adds fused differently), and every solve still meets
 * opt.tol.
 * Each transform of length 2^l with l not a multiple of 3 has a radix-2 or
 * radix-4 stage beside its radix-8 stages; the tuner also times the radix plan
 * of every pass at its picked shape: plan 0 runs that stage last, plan 1 first
 * (it then needs no twiddles and every radix-8 stage does). Plans change the
 * rounding of a pass (FP64 and double-float results then differ from the
 * built-in plan's in the last bits; every solve still meets opt.tol).
 * out (may be NULL): per arithmetic [type] (0 FP32, 1 FP64, 2 double-float)
 * and pass [pass] (0 matvec y-inverse, 1 matvec y-forward, 2 RHS y-inverse,
 * 3 RHS y-forward, 4 matvec x-pass, 5 RHS x-pass): threads per block chosen
 * and built in, the radix plan chosen, and the average launch time of the
 * built-in and the chosen configuration in microseconds; 0 threads for the
 * passes the handle's precision does not run.
 * Overwrites the handle's scratch spectra (not the warm start of sigma);
 * synchronises the handle's stream; call it between steps. reps in [1, 100],
 * else SGN_EINVAL. */
typedef struct {
  int threads[3][6];
  int default_threads[3][6];
  float us_tuned[3][6];
  float us_default[3][6];
  int plan[3][6];
} sgn_tuning;

sgn_status sgn_autotune(sgn_t ctx, int reps, sgn_tuning* out);

/* Applies a tuning (threads and plan of each pass, as sgn_autotune returns
 * it, e.g. saved from an earlier run on the same grid) without timing
 * anything: threads 0 keeps a pass's built-in shape, any other value must be
 * one of the shapes sgn_autotune considers for that pass (SGN_EINVAL
 * otherwise, and for a plan other than 0 or 1); the other fields are ignored.
 * Synchronises the handle's stream; captured step graphs are rebuilt. */
sgn_status sgn_set_tuning(sgn_t ctx, const sgn_tuning* t);

/* ------------------------------------------------------------------------
 * Learned GMRES start. Section 3 starts GMRES from the last computed
 * sigma; a network (include/sgn_unet.h) can correct that start. At RK4 stages
 * 2 and 4 (the stages whose state moved by O(dt) since the fallback's; with
 * guess = 3 at every stage, once the polynomial start is cubic), after the
 * start chosen by opt.guess, the library forms on an n x n coarse grid
 *   in = (in_scale[0] (h - 1), in_scale[1] vx, in_scale[2] vy,
 *         in_scale[3] sigma_start)
 * as band-limited samples of the stage state (the Fourier modes |m_x|, |m_y|
 * < n/2 evaluated at every (N/n)-th grid point), runs the network on it and
 * adds out_scale * tau * net(in), tau = (dt/2)^tau_power, to the same modes of
 * sigma's spectrum (with guess = 2, not at stage 2 of a call's first step,
 * which has no extrapolation history; with guess = 3, not before the handle
 * has solved 4 steps of the trajectory). The network runs as sgn_unet_infer
 * (BF16 on the tensor cores) on the handle's stream (it is re-pointed there).
 * Every solve still meets opt.tol. n must be a power of two in
 * [16, min(Nx, Ny)] and equal to the network's side; net = NULL detaches. */
sgn_status sgn_set_learned_guess(sgn_t ctx, void* net, int n, const float in_scale[4], float out_scale,
                                 int tau_power);

/* Records training samples for the learned start: during sgn_rk4_step and
 * sgn_rk4_step_host with the host-driven loop (graph = 0; SGN_EINVAL
 * otherwise), each stage the learned start corrects appends to buf (device float32, capacity
 * samples of [5][n][n]) the four coarse inputs above without in_scale (channels
 * 0-3, sigma_start taken before any learned correction) and the coarse target
 * (sigma_solved - sigma_start) / tau (channel 4). Recording stops silently when
 * buf is full; buf = NULL stops it. sgn_recorded_count returns the number of
 * samples written since the last sgn_record_learned call. */
sgn_status sgn_record_learned(sgn_t ctx, int n, float* buf, int capacity, int tau_power);
sgn_status sgn_recorded_count(sgn_t ctx, int* count);

/* The restriction and prolongation of the learned start, on physical fields:
 * sgn_coarse_sample: out [n][n] (device float32) = the modes |m_x|, |m_y| < n/2
 * of f (device float64 [Ny][Nx]) evaluated at the grid points (j Nx/n, i Ny/n);
 * sgn_coarse_embed: f += the band-limited field whose samples at those points
 * are scale * fc (fc device float32 [n][n]; its modes |m| < n/2 only). */
sgn_status sgn_coarse_sample(sgn_t ctx, const double* f, int n, float* out);
sgn_status sgn_coarse_embed(sgn_t ctx, const float* fc, int n, double scale, double* f);

#ifdef __cplusplus
}
#endif
#endif /* SGN_H */
