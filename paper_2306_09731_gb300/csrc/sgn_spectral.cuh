// sgn_spectral.cuh - spectral passes of the SGN hot path (Section 3).
//
// Templates only (plus a few host functions, each compiled in one unit): the
// kernels are instantiated per arithmetic in sgn_spectral.cu (FP64 and the
// shared host code), sgn_spectral_f32.cu and sgn_spectral_df.cu, which the
// build compiles in parallel.
//
// Every 2D transform is split into an x-pass over row PAIRS and a y-pass over
// column tiles of the half spectrum [Ny][ldS]:
//  * x-pass: rows y0 = 2p, y1 = 2p+1 travel together as one complex signal
//    z = f(y0) + i f(y1). An inverse x-transform of two half spectra is one
//    complex inverse FFT of length Nx; a forward one is a complex FFT followed by
//    the split F0 = Z + conj(Z(-k)), F1 = -i (Z - conj(Z(-k))) (each 2x the
//    half-spectrum of a real row).
//  * y-pass: C neighbouring kx columns per block, interleaved in shared memory.
// The pointwise work of the method is fused into these passes:
//  * matvec (Eq. (sigmav) preconditioned): y-inverse of sigma_hat and i ky
//    sigma_hat; x-pass forms sigma, sigma_x, sigma_y, a = 3 sigma/h^3,
//    b = grad(sigma)/h, forward x and the combination a - i kx bx; y-forward,
//    minus i ky by, times 1/(3 + kx^2 + ky^2).
//  * RHS (Eq. (1) and the v-form of Eq. (2)): y-inverse of vx, vy, sigma,
//    i ky sigma; x-pass forms q = h v - grad sigma (= h u) and
//    F = |v|^2/2 - |grad sigma|^2/(2h^2) + g h - 9 sigma^2/(2 h^4), forward x;
//    y-forward with -i k combinations and the RK4 stage update. In FP32 the
//    passes form only the part of q and F that is nonlinear in the state, and
//    the update adds the linear part from the FP64 spectra (rhs_lin_split).
#pragma once
#include <math.h>

#include <type_traits>

#include "sgn_internal.h"
#include "vec_common.cuh"

namespace sgn {

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ cpx<T> ld(const cpx<T>* p) {
  return *p;
}

// Packed full-length spectrum of two real rows from their half spectra:
// Z[k] = G0[k] + i G1[k], G = (deriv ? i kx : 1) * S, extended by Hermitian
// symmetry for k > N/2; the kx = 0 and kx = N/2 entries are taken real (the
// C2R convention).
template <typename T>
__device__ __forceinline__ void load_packed(cpx<T> (&v)[8], const cpx<T>* S0, const cpx<T>* S1, bool deriv,
                                            const T* __restrict__ kx, int t, int lN) {
  const int N = 1 << lN, T_ = N >> 3, half = N >> 1;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int k = t + s * T_;
    const int kk = (k <= half) ? k : N - k;
    cpx<T> A = ld(S0 + kk), B = ld(S1 + kk);
    if (deriv) {
      const T kv = ldr(kx + kk);
      A = mul_ik(A, kv);
      B = mul_ik(B, kv);
    }
    if (kk == 0 || kk == half) {
      A.y = (T)0;
      B.y = (T)0;
    }
    if (k > half) {
      A.y = -A.y;
      B.y = -B.y;
    }
    v[s] = mk(A.x - B.y, A.y + B.x);
  }
}

// After a forward FFT of z = f0 + i f1 held in v: writes v to sm, syncs, and
// returns for the thread's half-spectrum indices k = t + s*T_ (s < 4, plus
// k = N/2 on t == 0) the values 2*F0[k] and 2*F1[k]. Leaves sm in use: the
// caller syncs before reusing it.
template <typename T>
__device__ __forceinline__ void split_pair(const cpx<T> (&v)[8], cpx<T>* sm, int t, int lN, cpx<T> (&f0)[5],
                                           cpx<T> (&f1)[5]) {
  const int N = 1 << lN, T_ = N >> 3;
  store_slots(v, sm, t, T_, 0);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int k = t + s * T_;
    const cpx<T> P = v[s];
    const cpx<T> Q = conjg(sm[sidx<T>((N - k) & (N - 1), 0)]);
    f0[s] = P + Q;
    f1[s] = mul_mi(P - Q);
  }
}

__device__ __forceinline__ bool split_owns(int s, int t) { return s < 4 || t == 0; }

// Block layout of the x-pass: P row pairs per block, T_ = Nx/8 threads each.
struct XLayout {
  int t, grp, pair, y0, y1;
  bool valid;
};
// LN > 0: the row length 2^LN is a compile-time constant (the common sizes of
// the FP32 passes), so the stage loops unroll and every index shift folds; 0:
// read it from G.
template <int LN = 0>
__device__ __forceinline__ XLayout x_layout(const Geom& G) {
  XLayout L;
  const int lT = (LN > 0 ? LN : G.lNx) - 3;
  L.grp = threadIdx.x >> lT;
  L.t = threadIdx.x & ((1 << lT) - 1);
  const int P = blockDim.x >> lT;
  int pair = blockIdx.x * P + L.grp;
  L.valid = pair < (G.Ny >> 1);
  if (!L.valid) pair = (G.Ny >> 1) - 1;
  L.pair = pair;
  L.y0 = 2 * pair;
  L.y1 = L.y0 + 1;
  return L;
}

template <typename T>
__device__ __forceinline__ cpx<T>* x_smem(const Geom& G, int grp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  return reinterpret_cast<cpx<T>*>(smraw) + grp * smem_elems_of<T>(G.Nx);
}

// ------------------------------------------------------------ plain x-passes

// FP64 values into and out of a pass's type (double-float: exact split and
// bit placement, no FP64-pipe arithmetic)
template <typename T>
__device__ __forceinline__ T from_f64(double x) {
  if constexpr (std::is_same<T, dfl>::value)
    return dfl_from_f64(x);
  else
    return (T)x;
}
template <typename T>
__device__ __forceinline__ double to_f64(T x) {
  if constexpr (std::is_same<T, dfl>::value)
    return dfl_to_f64(x);
  else
    return (double)x;
}

template <typename T>
struct XR2CArgs {
  const double* f[4];
  cpx<T>* out[4];
};

template <typename T>
__global__ void k_x_r2c(Geom G, const cpx<T>* __restrict__ tw, XR2CArgs<T> a) {
  const XLayout L = x_layout(G);
  cpx<T>* sm = x_smem<T>(G, L.grp);
  const int N = G.Nx, T_ = N >> 3;
  const double* f = a.f[blockIdx.y];
  cpx<T> v[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    v[s] = mk(from_f64<T>(f[(size_t)L.y0 * N + x]), from_f64<T>(f[(size_t)L.y1 * N + x]));
  }
  fft_regs<false>(v, sm, tw, L.t, G.lNx);
  cpx<T> f0[5], f1[5];
  split_pair(v, sm, L.t, G.lNx, f0, f1);
  if (!L.valid) return;
  cpx<T>* o = a.out[blockIdx.y];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (!split_owns(s, L.t)) continue;
    const int k = L.t + s * T_;
    o[(size_t)L.y0 * G.ldS + k] = scl(f0[s], (T)0.5f);
    o[(size_t)L.y1 * G.ldS + k] = scl(f1[s], (T)0.5f);
  }
}

template <typename T>
struct XC2RArgs {
  const cpx<T>* in[4];
  double* out[4];
  int deriv[4];
};

template <typename T>
__global__ void k_x_c2r(Geom G, const cpx<T>* __restrict__ tw, const T* __restrict__ kx, XC2RArgs<T> a,
                        double scale) {
  const XLayout L = x_layout(G);
  cpx<T>* sm = x_smem<T>(G, L.grp);
  const int N = G.Nx, T_ = N >> 3;
  const int fi = blockIdx.y;
  cpx<T> v[8];
  load_packed(v, a.in[fi] + (size_t)L.y0 * G.ldS, a.in[fi] + (size_t)L.y1 * G.ldS, a.deriv[fi] != 0, kx,
              L.t, G.lNx);
  fft_regs<true>(v, sm, tw, L.t, G.lNx);
  if (!L.valid) return;
  double* o = a.out[fi];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    o[(size_t)L.y0 * N + x] = to_f64<T>(v[s].x) * scale;
    o[(size_t)L.y1 * N + x] = to_f64<T>(v[s].y) * scale;
  }
}

// ------------------------------------------------------ coefficient passes

// 1/h in FP64 by the Newton-Raphson iteration r <- r + r (1 - h r) from an FP32
// reciprocal seed: each step squares the relative error (1e-7 -> 1e-14 ->
// rounding), for a handful of FMAs instead of a full FP64 division, which costs
// about 25 FP64 instructions on a part with a 1:58 FP64:FP32 rate. Depths
// outside the FP32 range take the plain division.
__device__ __forceinline__ double recip_nr(double h) {
  if (!(h > 1e-30 && h < 1e30)) return 1.0 / h;
  double r = (double)(1.0f / (float)h);
  double e = fma(-h, r, 1.0);
  r = fma(r, e, r);
  e = fma(-h, r, 1.0);
  return fma(r, e, r);
}

template <typename T>
__device__ __forceinline__ void coef_point(double hv, double invN, T* h, T* cr, T* cc, size_t i, int* flags,
                                           const CoefCopy& cp) {
  if (!isfinite(hv)) {
    atomicOr(flags, FLAG_NONFINITE);
  } else if (!(hv > 0.0)) {
    atomicOr(flags, FLAG_CAVITATION);
  }
  const double r = recip_nr(hv);
  const double vr = 0.5 * invN * r, vc = 1.5 * invN * r * r * r;
  h[i] = (T)(hv - 1.0);  // the depth anomaly h - h_inf (exact in FP64 near h = 1)
  cr[i] = (T)vr;
  cc[i] = (T)vc;
  if (cp.h) {
    cp.h[i] = (float)(hv - 1.0);
    cp.cr[i] = (float)vr;
    cp.cc[i] = (float)vc;
  }
}

// The same three coefficients in double-float (precision 2): 1/h by one Newton
// step from the FP32 reciprocal (see recip), the factors 1/(2N) and 3/(2N) as
// exact power-of-two scalings and one product by 1.5; h is the depth in FP32
// range (1/h^3 must not overflow). The FP32 copies are the high parts. h may be
// null (the refinement matvec reads only cr and cc).
__device__ __forceinline__ void coef_point_df(dfl hv, float invN, dfl* h, dfl* cr, dfl* cc, size_t i, int* flags,
                                              const CoefCopy& cp) {
  // the transforms leave their sums unnormalised: the FP32 copies, the sign
  // and the finiteness test need hi to be the nearest FP32 value (near h = 1,
  // an unnormalised hi is off by a few ulps of 1, all of it in h - 1)
  hv = renorm(hv);
  if (!isfinite(hv.hi)) {
    atomicOr(flags, FLAG_NONFINITE);
  } else if (!(hv.hi > 0.0f)) {
    atomicOr(flags, FLAG_CAVITATION);
  }
  const dfl r = recip(hv);
  const dfl vr = scale_pow2(r, 0.5f * invN);
  const dfl vc = scale_pow2(mul_f((r * r) * r, 1.5f), invN);
  const dfl a = renorm(hv - dfl(1.0f));
  if (h) h[i] = a;
  cr[i] = vr;
  cc[i] = vc;
  if (cp.h) {
    cp.h[i] = a.hi;
    cp.cr[i] = vr.hi;
    cp.cc[i] = vc.hi;
  }
}

// Hy = y-inverse of h_hat; x-inverse gives N*h. Writes the anomaly h - 1,
// cr = 0.5/(N h) and cc = 1.5/(N h^3): the coefficients of Eq. (sigmav) with
// the factor 1/(2N) of the matvec's packed transforms folded in.
template <typename T>
__global__ void k_coef_x(Geom G, const cpx<T>* __restrict__ tw, const T* __restrict__ kx, const cpx<T>* Hy,
                         T* h, T* cr, T* cc, int* flags, CoefCopy cp) {
  const XLayout L = x_layout(G);
  cpx<T>* sm = x_smem<T>(G, L.grp);
  const int N = G.Nx, T_ = N >> 3;
  cpx<T> v[8];
  load_packed(v, Hy + (size_t)L.y0 * G.ldS, Hy + (size_t)L.y1 * G.ldS, false, kx, L.t, G.lNx);
  fft_regs<true>(v, sm, tw, L.t, G.lNx);
  if (!L.valid) return;
  const double invN = 1.0 / (double)G.nphys();
  if constexpr (std::is_same<T, dfl>::value) {
    // one slot at a time from the thread's own slots of the transform buffer
    // (free again after the transform; no other thread touches them): one
    // copy of the double-float reciprocal code instead of sixteen.
    // N = Nx Ny is a power of two: the scaling by 1/N is exact.
    store_slots(v, sm, L.t, T_, 0);
    const float fN = (float)invN;
#pragma unroll 1
    for (int s = 0; s < 8; ++s) {
      const int x = L.t + s * T_;
      const cpx<T> z = sm[sidx<T>(x, 0)];
      coef_point_df(scale_pow2(z.x, fN), fN, h, cr, cc, (size_t)L.y0 * N + x, flags, cp);
      coef_point_df(scale_pow2(z.y, fN), fN, h, cr, cc, (size_t)L.y1 * N + x, flags, cp);
    }
  } else {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int x = L.t + s * T_;
      coef_point<T>((double)v[s].x * invN, invN, h, cr, cc, (size_t)L.y0 * N + x, flags, cp);
      coef_point<T>((double)v[s].y * invN, invN, h, cr, cc, (size_t)L.y1 * N + x, flags, cp);
    }
  }
}

template <typename T>
__global__ void k_coef_phys(Geom G, const double* __restrict__ hp, T* h, T* cr, T* cc, int* flags, CoefCopy cp) {
  const double invN = 1.0 / (double)G.nphys();
  const size_t n = G.nphys();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<T, dfl>::value)
      coef_point_df(dfl_from_f64(hp[i]), (float)invN, h, cr, cc, i, flags, cp);
    else
      coef_point<T>(hp[i], invN, h, cr, cc, i, flags, cp);
  }
}

// ---------------------------------------------------------- fused matvec x

// Resident 256-thread blocks per SM the x-passes ask the compiler for: the
// FP32 passes are latency bound and need the warps; the FP64 ones are
// FP64-issue bound and keep their registers.
// At 4096 points (LN = 12) a row pair takes 512 threads: one block per SM.
template <int LN>
constexpr int xpass_threads() { return LN == 12 ? 512 : 256; }
template <typename T, int LN>
constexpr int mv_min_blocks() { return LN == 12 ? 1 : ((sizeof(T) == 4 || std::is_same<T, dfl>::value) ? 3 : 2); }
template <typename T, int LN>
constexpr int rhs_min_blocks() { return LN == 12 ? 1 : ((sizeof(T) == 4 || std::is_same<T, dfl>::value) ? 2 : 1); }
// shared-memory elements per row pair of the fused RHS x-pass beyond its
// transform buffer: the double-float pass keeps its accumulators QX, QY there
// (8 slots per thread each)
template <typename T>
__host__ __device__ constexpr int rhs_acc_elems(int N) { return std::is_same<T, dfl>::value ? 2 * N : 0; }

// S = y-inverse of sigma_hat, Sy = y-inverse of i ky sigma_hat. Writes
// Cout = (a - i kx bx)^x and Byout = by^x (x-spectral, y-physical). A block
// reads only its own row pair before writing it: Cout/Byout may alias S/Sy.
// Three phases, each an inverse transform, a pointwise product and a forward
// transform, so that one 8-slot signal is live at a time (plus the a^x half
// spectra of phase 1 until phase 2 combines them): a = 3 sigma/h^3, then
// bx = sigma_x/h, then by = sigma_y/h.
// Shared-memory elements per row pair of the matvec x-pass beyond its
// transform buffer: phase 1's half spectra a0, a1 (5 slots each per thread)
// wait there while phase 2 transforms, instead of in 20 live registers.
__host__ __device__ constexpr int mv_stash_elems(int N) { return 10 * (N >> 3); }

template <typename T, int LN = 0, int PLAN = 0>
__global__ void __launch_bounds__(xpass_threads<LN>(), mv_min_blocks<T, LN>()) k_mv_x(Geom G, const cpx<T>* __restrict__ tw, const T* __restrict__ kx,
                                               const cpx<T>* S, const cpx<T>* Sy, const T* __restrict__ cr,
                                               const T* __restrict__ cc, cpx<T>* Cout, cpx<T>* Byout) {
  const XLayout L = x_layout<LN>(G);
  cpx<T>* sm = x_smem<T>(G, L.grp);
  const int lN = LN > 0 ? LN : G.lNx;
  const int N = 1 << lN, T_ = N >> 3;
  const size_t o0 = (size_t)L.y0 * G.ldS, o1 = (size_t)L.y1 * G.ldS;
  const size_t p0 = (size_t)L.y0 * N, p1 = (size_t)L.y1 * N;
  // this row pair's stash, after the P transform buffers of the block; each
  // thread writes and reads back only its own slots (no barrier needed)
  extern __shared__ __align__(16) unsigned char smraw[];
  const int P = blockDim.x >> (lN - 3);
  cpx<T>* stash =
      reinterpret_cast<cpx<T>*>(smraw) + (size_t)P * smem_elems_of<T>(N) + (size_t)L.grp * mv_stash_elems(N);
  cpx<T> Z[8];
  cpx<T> b0[5], b1[5];
  // phase 0: a = 3 sigma / h^3 (kept in the stash); phase 1: bx = sigma_x / h,
  // combined with a into Cout; phase 2: by = sigma_y / h into Byout
  auto phase = [&](int ph) {
    const cpx<T>* in = ph == 2 ? Sy : S;
    const T* __restrict__ cf = ph == 0 ? cc : cr;
    load_packed(Z, in + o0, in + o1, ph == 1, kx, L.t, lN);
    fft_regs<true>(Z, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int x = L.t + s * T_;
      Z[s] = mk(cf[p0 + x] * Z[s].x, cf[p1 + x] * Z[s].y);
    }
    fft_regs<false>(Z, sm, tw, L.t, lN, 0, PLAN);
    split_pair(Z, sm, L.t, lN, b0, b1);
    if (ph == 0) {
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        stash[(2 * s) * T_ + L.t] = b0[s];
        stash[(2 * s + 1) * T_ + L.t] = b1[s];
      }
    } else {
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        if (!split_owns(s, L.t) || !L.valid) continue;
        const int k = L.t + s * T_;
        if (ph == 1) {
          const T kv = ldr(kx + k);
          Cout[o0 + k] = stash[(2 * s) * T_ + L.t] - mul_ik(b0[s], kv);
          Cout[o1 + k] = stash[(2 * s + 1) * T_ + L.t] - mul_ik(b1[s], kv);
        } else {
          Byout[o0 + k] = b0[s];
          Byout[o1 + k] = b1[s];
        }
      }
    }
  };
  if constexpr (std::is_same<T, dfl>::value) {
    // one copy of the phase for all three: six inlined double-float
    // transforms do not fit the instruction cache (ncu: "no instruction" was
    // the largest stall of this pass with them unrolled)
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) {
      phase(ph);
      __syncthreads();
    }
  } else {
    phase(0);
    __syncthreads();
    phase(1);
    __syncthreads();
    phase(2);
  }
}

// ------------------------------------------------------------- fused RHS x

// Inputs (y-inverse outputs): Vx, Vy, S = sigma, Sy = i ky sigma, and the
// depth anomaly hh = h - 1. Writes Cq = -i kx (h u_x)^x, Qy = (h u_y)^x and
// Fh = F^x with F = |v|^2/2 - |grad sigma|^2/(2h^2) + g (h - 1) - 9 sigma^2/(2h^4).
//
// In FP32 (rhs_lin_split) the pass leaves out the terms linear in the state:
// h u = v + (h - 1) v - grad sigma keeps only (h - 1) v, and F drops g (h - 1).
// k_rk_update adds them back in the state's arithmetic from its spectra
// (-i k.v_hat - |k|^2 sigma_hat and -i k g h_hat), so the FP32 rounding of
// the right-hand side scales with its nonlinear part, not with the whole.
template <typename T>
constexpr bool rhs_lin_split() { return std::is_same<T, float>::value; }

template <typename T, int LN = 0, int PLAN = 0>
__global__ void __launch_bounds__(xpass_threads<LN>(), rhs_min_blocks<T, LN>()) k_rhs_x(Geom G, const cpx<T>* __restrict__ tw, const T* __restrict__ kx,
                                                const cpx<T>* Vx, const cpx<T>* Vy, const cpx<T>* S,
                                                const cpx<T>* Sy, const T* __restrict__ hh,
                                                const T* __restrict__ cr, T g, cpx<T>* Cq, cpx<T>* Qy,
                                                cpx<T>* Fh) {
  const XLayout L = x_layout<LN>(G);
  cpx<T>* sm = x_smem<T>(G, L.grp);
  const int lN = LN > 0 ? LN : G.lNx;
  const int N = 1 << lN, T_ = N >> 3;
  const size_t o0 = (size_t)L.y0 * G.ldS, o1 = (size_t)L.y1 * G.ldS;
  const size_t p0 = (size_t)L.y0 * N, p1 = (size_t)L.y1 * N;
  const T n = (T)(1.0 / (double)G.nphys());
  const T twoN = (T)(2.0 * (double)G.nphys());
  if constexpr (std::is_same<T, dfl>::value) {
    // Double-float (precision 3): the same sums with one copy of the inverse
    // and one of the forward transform code (rolled loops over the five inputs
    // and the three outputs; eight inlined double-float transforms overflow
    // the instruction cache) and the accumulators QX, QY in the thread's own
    // slots of shared memory, so that F and one signal are the registers that
    // live across a transform (two blocks per SM instead of one that spilled)
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = blockDim.x >> (lN - 3);
    cpx<T>* acc = reinterpret_cast<cpx<T>*>(smraw) + (size_t)P * smem_elems_of<T>(N) +
                  (size_t)L.grp * rhs_acc_elems<T>(N);
    cpx<T> F[8], Z[8];
    // inputs: 0 i kx sigma_hat, 1 Sy = i ky sigma_hat, 2 sigma_hat, 3 vx, 4 vy
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
      const cpx<T>* in = i == 1 ? Sy : (i == 3 ? Vx : (i == 4 ? Vy : S));
      load_packed(Z, in + o0, in + o1, i == 0, kx, L.t, lN);
      fft_regs<true>(Z, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int x = L.t + s * T_;
        cpx<T>* qx = acc + (size_t)s * T_ + L.t;
        cpx<T>* qy = acc + (size_t)(8 + s) * T_ + L.t;
        const T z0 = Z[s].x * n, z1 = Z[s].y * n;
        if (i == 0) {
          *qx = mk(-z0, -z1);  // -sigma_x
        } else if (i == 1) {
          // sigma_y; -|grad sigma|^2 / (2 h^2) with sigma_x from the slot
          const T r0 = cr[p0 + x] * twoN, r1 = cr[p1 + x] * twoN;
          const cpx<T> q = *qx;
          *qy = mk(-z0, -z1);
          F[s] = mk((T)-0.5 * r0 * r0 * (q.x * q.x + z0 * z0), (T)-0.5 * r1 * r1 * (q.y * q.y + z1 * z1));
        } else if (i == 2) {
          // sigma: -9 sigma^2 / (2 h^4)
          const T r0 = cr[p0 + x] * twoN, r1 = cr[p1 + x] * twoN;
          const T q0 = z0 * r0 * r0, q1 = z1 * r1 * r1;
          F[s].x -= (T)4.5 * q0 * q0;
          F[s].y -= (T)4.5 * q1 * q1;
        } else {
          // vx, vy: h v and |v|^2/2; with vy also g (h - 1) (see below)
          const T a0 = hh[p0 + x], a1 = hh[p1 + x];  // h - 1
          cpx<T>* q = i == 3 ? qx : qy;
          cpx<T> w = *q;
          w.x += z0 + a0 * z0;
          w.y += z1 + a1 * z1;
          const T gh0 = i == 4 ? g * a0 : (T)0, gh1 = i == 4 ? g * a1 : (T)0;
          F[s].x += (T)0.5 * z0 * z0 + gh0;
          F[s].y += (T)0.5 * z1 * z1 + gh1;
          // the split returns twice the half spectra: pre-scale by 1/2
          *q = scl(w, (T)0.5);
          if (i == 4) F[s] = scl(F[s], (T)0.5);
        }
      }
    }
    cpx<T> f0[5], f1[5];
    // F first, so that its registers are free for the loop over QX, QY
    fft_regs<false>(F, sm, tw, L.t, lN, 0, PLAN);
    split_pair(F, sm, L.t, lN, f0, f1);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      if (!split_owns(s, L.t) || !L.valid) continue;
      const int k = L.t + s * T_;
      Fh[o0 + k] = f0[s];
      Fh[o1 + k] = f1[s];
    }
    __syncthreads();
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int s = 0; s < 8; ++s) Z[s] = acc[(size_t)(8 * j + s) * T_ + L.t];
      fft_regs<false>(Z, sm, tw, L.t, lN, 0, PLAN);
      split_pair(Z, sm, L.t, lN, f0, f1);
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        if (!split_owns(s, L.t) || !L.valid) continue;
        const int k = L.t + s * T_;
        if (j == 0) {
          const T kv = ldr(kx + k);
          Cq[o0 + k] = mul_ik(f0[s], -kv);
          Cq[o1 + k] = mul_ik(f1[s], -kv);
        } else {
          Qy[o0 + k] = f0[s];
          Qy[o1 + k] = f1[s];
        }
      }
      __syncthreads();
    }
    return;
  }
  cpx<T> QX[8], QY[8], F[8], Z[8];
  // grad sigma
  load_packed(QX, S + o0, S + o1, true, kx, L.t, lN);
  fft_regs<true>(QX, sm, tw, L.t, lN, 0, PLAN);
  load_packed(QY, Sy + o0, Sy + o1, false, kx, L.t, lN);
  fft_regs<true>(QY, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    const T r0 = cr[p0 + x] * twoN, r1 = cr[p1 + x] * twoN;
    const T sx0 = QX[s].x * n, sx1 = QX[s].y * n, sy0 = QY[s].x * n, sy1 = QY[s].y * n;
    QX[s] = rhs_lin_split<T>() ? mk((T)0, (T)0) : mk(-sx0, -sx1);
    QY[s] = rhs_lin_split<T>() ? mk((T)0, (T)0) : mk(-sy0, -sy1);
    F[s] = mk((T)-0.5 * r0 * r0 * (sx0 * sx0 + sy0 * sy0), (T)-0.5 * r1 * r1 * (sx1 * sx1 + sy1 * sy1));
  }
  // sigma: -9 sigma^2 / (2 h^4)
  load_packed(Z, S + o0, S + o1, false, kx, L.t, lN);
  fft_regs<true>(Z, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    const T r0 = cr[p0 + x] * twoN, r1 = cr[p1 + x] * twoN;
    const T s0 = Z[s].x * n, s1 = Z[s].y * n;
    const T q0 = s0 * r0 * r0, q1 = s1 * r1 * r1;
    F[s].x -= (T)4.5 * q0 * q0;
    F[s].y -= (T)4.5 * q1 * q1;
  }
  // vx: h vx and |vx|^2/2
  load_packed(Z, Vx + o0, Vx + o1, false, kx, L.t, lN);
  fft_regs<true>(Z, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    const T a0 = hh[p0 + x], a1 = hh[p1 + x];  // h - 1
    const T v0 = Z[s].x * n, v1 = Z[s].y * n;
    QX[s].x += rhs_lin_split<T>() ? a0 * v0 : v0 + a0 * v0;
    QX[s].y += rhs_lin_split<T>() ? a1 * v1 : v1 + a1 * v1;
    F[s].x += (T)0.5 * v0 * v0;
    F[s].y += (T)0.5 * v1 * v1;
  }
  // vy: h vy, |vy|^2/2 and g h
  load_packed(Z, Vy + o0, Vy + o1, false, kx, L.t, lN);
  fft_regs<true>(Z, sm, tw, L.t, lN, 0, PLAN);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = L.t + s * T_;
    const T a0 = hh[p0 + x], a1 = hh[p1 + x];  // h - 1
    const T v0 = Z[s].x * n, v1 = Z[s].y * n;
    QY[s].x += rhs_lin_split<T>() ? a0 * v0 : v0 + a0 * v0;
    QY[s].y += rhs_lin_split<T>() ? a1 * v1 : v1 + a1 * v1;
    // g (h - h_inf): the constant g h_inf of the Bernoulli equation (2) has no
    // gradient; leaving it out keeps F's rounding relative to its variation
    const T gh0 = rhs_lin_split<T>() ? (T)0 : g * a0, gh1 = rhs_lin_split<T>() ? (T)0 : g * a1;
    F[s].x += (T)0.5 * v0 * v0 + gh0;
    F[s].y += (T)0.5 * v1 * v1 + gh1;
    // the split returns twice the half spectra: pre-scale by 1/2
    QX[s] = scl(QX[s], (T)0.5);
    QY[s] = scl(QY[s], (T)0.5);
    F[s] = scl(F[s], (T)0.5);
  }
  cpx<T> f0[5], f1[5];
  fft_regs<false>(QX, sm, tw, L.t, lN, 0, PLAN);
  split_pair(QX, sm, L.t, lN, f0, f1);
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (!split_owns(s, L.t) || !L.valid) continue;
    const int k = L.t + s * T_;
    const T kv = ldr(kx + k);
    Cq[o0 + k] = mul_ik(f0[s], -kv);
    Cq[o1 + k] = mul_ik(f1[s], -kv);
  }
  __syncthreads();
  fft_regs<false>(QY, sm, tw, L.t, lN, 0, PLAN);
  split_pair(QY, sm, L.t, lN, f0, f1);
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (!split_owns(s, L.t) || !L.valid) continue;
    const int k = L.t + s * T_;
    Qy[o0 + k] = f0[s];
    Qy[o1 + k] = f1[s];
  }
  __syncthreads();
  fft_regs<false>(F, sm, tw, L.t, lN, 0, PLAN);
  split_pair(F, sm, L.t, lN, f0, f1);
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (!split_owns(s, L.t) || !L.valid) continue;
    const int k = L.t + s * T_;
    Fh[o0 + k] = f0[s];
    Fh[o1 + k] = f1[s];
  }
}

// ------------------------------------------------------------------ y-pass

template <typename T, int NIN, typename S = T>
struct YIn {
  const cpx<S>* src[NIN];  // storage type S, converted to the compute type T on load
  int deriv[NIN];          // pre-multiply by i ky (inverse passes)
  const int* sel;          // may be null: every src is offset by (*sel) * sel_stride
  size_t sel_stride;
};

template <typename T, typename S>
__device__ __forceinline__ cpx<T> ld_as(const cpx<S>* p) {
  const cpx<S> v = *p;
  // double-float from FP64 without FP64 instructions; FP32 from FP64 with the
  // native conversion (measured: the bit-level one costs more issue slots in
  // the issue-bound RHS y-inverse than the FP64-pipe conversion saves)
  if constexpr (std::is_same<T, dfl>::value && std::is_same<S, double>::value)
    return mk(dfl_from_f64(v.x), dfl_from_f64(v.y));
  else
    return mk((T)v.x, (T)v.y);
}

// Column tile: C = blockDim / (Ny/8) neighbouring kx columns, thread index
// c + C*t. Each input column is transformed in registers; the epilogue gets
// all NIN results of the thread's 8 rows.
// Threads of a y-pass block. FP32: 512 (two columns per block at Ny = 2048,
// twice the bytes per row segment). FP64: 256, the registers of one column per
// block (measured at 2048^2: inverse 321 against 371 us and forward 327
// against 386 us with 512). Double-float: 256, one column per block, three
// blocks per SM for the passes that hold one signal at a time (see
// ypass_body).
// At 4096 points (LN = 12) one column takes 512 threads in every type.
// FP32 passes with at most two inputs (NIN <= 2): 1024 threads, four columns
// per block at Ny = 2048, so that a warp's access covers 8 rows x 32 bytes (8
// cache lines) instead of 16 rows x 16 bytes (16 lines): the strided column
// accesses cost L1 wavefronts per line touched.
template <typename T, bool INV, int LN = 0, int NIN = 0>
constexpr int ypass_threads() {
  if (sizeof(T) == 4 && NIN >= 1 && NIN <= 2) return 1024;
  return (sizeof(T) == 4 || LN == 12) ? 512 : 256;
}

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
// LN > 0: compile-time column length 2^LN, and the built-in shape's column
// interleave 2^LC (folds the index arithmetic of the stages; a tuned shape
// other than the built-in one runs the runtime-length kernel, LN = 0)
template <typename T, bool INV, int LN, int NIN>
constexpr int ypass_lc() {
  return LN == 0 ? -1 : clampi(ilog2c(ypass_threads<T, INV, LN, NIN>()) - (LN - 3), 0, 6);
}

// Input staging of a y-pass (compile-time mask FL). The inputs are column
// segments read at a stride of one row, so a thread's loads wait out the full
// memory latency and, with one transform per input, the next input's loads
// only start after the previous transform:
//   yf_pf(i), i >= 1: input i is copied to shared memory by cp.async when the
//     block starts, so its loads overlap the loads and transforms of the
//     inputs before it;
//   yf_dup(i), i >= 1: input i is i ky times input i-1 (same source, deriv 0
//     there): the raw values of input i-1 are kept in shared memory and input
//     i is formed from them instead of being read again.
// Each thread stages only the elements it reads back itself (slot s of thread
// tid at s * blockDim + tid), so no barrier orders the copies.
__host__ __device__ constexpr int yf_pf(int i) { return 1 << i; }
__host__ __device__ constexpr int yf_dup(int i) { return 1 << (8 + i); }

// staging bytes per thread of the inputs before input `upto`
template <typename T, typename S, int FL>
__host__ __device__ constexpr int ystage_bytes(int upto) {
  int b = 0;
  for (int j = 1; j < upto; ++j) {
    if (FL & yf_pf(j)) b += 8 * (int)sizeof(cpx<S>);
    else if (FL & yf_dup(j)) b += 8 * (int)sizeof(cpx<T>);
  }
  return b;
}

// byte offset of the staging area: the transform buffers, rounded up to 16
template <typename T>
__host__ __device__ constexpr size_t ystage_offset(int lN, int lC) {
  return ((((size_t)smem_elems_of<T>(1 << lN) << lC) * sizeof(cpx<T>)) + 15) & ~(size_t)15;
}

// staging masks of the fused passes (see ypass_body): the matvec y-inverse
// prefetches its second input (sigma_hat again, for i ky sigma_hat: keeping the
// first input's raw values in shared memory instead spilled 244 bytes at the
// 64 registers of the FP32 pass); the y-forward passes stage every input after
// the first; the RHS y-inverse forms i ky sigma_hat from a staged copy of
// sigma_hat and, in FP64 below 4096 points, also stages v_y and sigma_hat (the
// FP32 one measured 117 against 107 us with them staged: 196 KB of shared
// memory leave little L1; FP64 at 4096 has no room for them; the double-float
// one transforms one input at a time at three blocks per SM instead)
constexpr int FL_MV_INV = yf_pf(1);
constexpr int FL_MV_FWD = yf_pf(1);
constexpr int FL_RHS_FWD = yf_pf(1) | yf_pf(2);
// the double-float forward passes stage nothing: they transform one input at
// a time and keep each finished transform in the thread's own shared-memory
// slots for the epilogue instead (ystash_bytes, see ypass_body). (The FP32 RHS
// y-forward the same way, at two blocks of 512 per SM without its prefetch,
// ran 68 us against 53.5: that pass is latency bound.)
template <typename T, bool INV, int NIN>
__host__ __device__ constexpr bool y_stashed() {
  return !INV && std::is_same<T, dfl>::value && NIN >= 2;
}
template <typename T>
constexpr int fl_mv_fwd() { return y_stashed<T, false, 2>() ? 0 : FL_MV_FWD; }
template <typename T>
constexpr int fl_rhs_fwd() { return y_stashed<T, false, 3>() ? 0 : FL_RHS_FWD; }
template <typename T, bool INV, int NIN>
__host__ __device__ constexpr int ystash_bytes() {
  return y_stashed<T, INV, NIN>() ? (NIN - 1) * 8 * (int)sizeof(cpx<T>) : 0;
}
template <typename T, int LN>
constexpr int fl_rhs_inv() {
  return (sizeof(T) == 4 || LN == 12 || std::is_same<T, dfl>::value) ? yf_dup(3)
                                                                      : (yf_pf(1) | yf_pf(2) | yf_dup(3));
}

template <typename E>
__device__ __forceinline__ void cp_async_elem(E* dst, const E* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(E) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
// shared-memory read that stays where it is written (FP32 pairs by an asm
// load, so that the compiler does not schedule it early and hold the value
// across the transform before it)
template <typename T>
__device__ __forceinline__ cpx<T> lds_fenced(const cpx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    float a, b;
    const unsigned d = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(a), "=f"(b) : "r"(d) : "memory");
    return mk((T)a, (T)b);
  } else {
    return *p;
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Tensor copies (TMA) of column tiles. yf_tma(i): input i arrives as one tile
// of [Ny rows][C columns] copied by the tensor engine (boxes of up to 256 rows,
// issued by one thread); its mbarrier completes on the tile's bytes. The FP32
// matvec passes take their inputs this way: one thread's few bulk copies
// replace 8 strided loads per thread and input, whose queue (LSU throttle) was
// the first stall of those passes.
__host__ __device__ constexpr int yf_tma(int i) { return 1 << (16 + i); }
constexpr int kTmaMaxMaps = 2;
struct YTma {
  CUtensorMap map[kTmaMaxMaps];
  int z[kTmaMaxMaps];  // coordinate along the vector dimension of each map
  const int* zsel;     // may be null: map 0's z read from the device instead
  int* flags;          // FLAG_WAIT when a wait runs out
};
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait on phase 0 of bar: about a second at most (try_wait suspends
// between polls). The block-wide vote keeps every thread on the same path.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar) {
  bool ok = false;
  for (int it = 0; it < (1 << 20) && !ok; ++it) ok = mbar_try_wait(bar, 0);
  return __syncthreads_and(ok ? 1 : 0) != 0;
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T, int NIN>
struct EpiStore;
template <class E>
struct is_epi_store : std::false_type {};
template <typename T, int NIN>
struct is_epi_store<EpiStore<T, NIN>> : std::true_type {};

template <typename T, bool INV, int NIN, class Epi, typename S, int LN, int FL, int PLAN>
__device__ __forceinline__ void ypass_body(const Geom& G, const cpx<T>* __restrict__ tw, const T* __restrict__ ky,
                                           const YIn<T, NIN, S>& in, const Epi& epi,
                                           const YTma* tm = nullptr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* smb = reinterpret_cast<cpx<T>*>(smraw);
  const int lN = LN > 0 ? LN : G.lNy;
  const int T_ = 1 << (lN - 3);
  constexpr int LCc = ypass_lc<T, INV, LN, NIN>();
  const int lC = LCc >= 0 ? LCc : __ffs(blockDim.x >> (lN - 3)) - 1;
  const int c = threadIdx.x & ((1 << lC) - 1);
  const int t = threadIdx.x >> lC;
  int col = (blockIdx.x << lC) + c;
  const bool valid = col < G.Nxh;
  if (!valid) col = G.Nxh - 1;
  cpx<T> r[NIN][8];
  const size_t soff = in.sel ? (size_t)(*in.sel) * in.sel_stride : 0;
  // staging area: after the C transform buffers of the exchanges
  unsigned char* stage = smraw + ystage_offset<T>(lN, lC);
  const int nthr = blockDim.x, tid = threadIdx.x;
  // tensor-copied tiles: [Ny][C] per map, 128-byte aligned in the shared window
  constexpr int NMAP = ((FL & yf_tma(0)) ? 1 : 0) + ((NIN > 1 && (FL & yf_tma(1))) ? 1 : 0);
  cpx<T>* tstage = nullptr;
  __shared__ uint64_t tbar[NMAP > 0 ? NMAP : 1];
  if constexpr (NMAP > 0) {
    const unsigned sb = smem_u32(stage);
    tstage = reinterpret_cast<cpx<T>*>(stage + (((sb + 127u) & ~127u) - sb));
    if (tid == 0) {
#pragma unroll
      for (int m = 0; m < NMAP; ++m) mbar_init(&tbar[m], 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      const int Ny = 1 << lN, C = 1 << lC, BR = Ny < 256 ? Ny : 256;
#pragma unroll
      for (int m = 0; m < NMAP; ++m) {
        const int z = (m == 0 && tm->zsel) ? *tm->zsel : tm->z[m];
        mbar_expect_tx(&tbar[m], (unsigned)(Ny * C * (int)sizeof(cpx<T>)));
        for (int b = 0; b < Ny; b += BR)
          tma_load_3d(tstage + ((size_t)m * Ny + b) * C, &tm->map[m], 2 * (int)(blockIdx.x << lC), b, z, &tbar[m]);
      }
    }
  }
  if constexpr (FL != 0) {
#pragma unroll
    for (int i = 1; i < NIN; ++i) {
      if (FL & yf_pf(i)) {
        cpx<S>* st = reinterpret_cast<cpx<S>*>(stage + (size_t)nthr * ystage_bytes<T, S, FL>(i));
        const cpx<S>* src = in.src[i] + soff;
#pragma unroll
        for (int s = 0; s < 8; ++s) cp_async_elem(st + s * nthr + tid, src + (size_t)(t + s * T_) * G.ldS + col);
      }
    }
    cp_async_commit();
  }
  if constexpr (y_stashed<T, INV, NIN>() && NMAP == 0 && FL == 0) {
    // double-float y-forward passes (the refinement matvec's, precision 3's
    // right-hand side): one copy of the transform code for every input (a
    // rolled loop), each finished transform but the last kept in the thread's
    // own slots of shared memory until the epilogue, which needs them all, so
    // that one signal is live during a transform
    cpx<T>* stash = reinterpret_cast<cpx<T>*>(stage);
    const cpx<S>* srcs[NIN];
    int ders[NIN];
#pragma unroll
    for (int j = 0; j < NIN; ++j) {
      srcs[j] = in.src[j] + soff;
      ders[j] = in.deriv[j];
    }
    cpx<T> z[8];
#pragma unroll 1
    for (int i = 0; i < NIN; ++i) {
      const cpx<S>* src = srcs[0];
      bool der = ders[0] != 0;
#pragma unroll
      for (int j = 1; j < NIN; ++j)
        if (i == j) {
          src = srcs[j];
          der = ders[j] != 0;
        }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int row = t + s * T_;
        z[s] = ld_as<T, S>(src + (size_t)row * G.ldS + col);
        if (der) z[s] = mul_ik(z[s], ldr(ky + row));
      }
      fft_regs<INV>(z, smb + c, tw, t, lN, lC, PLAN);
      if (i + 1 < NIN) {
#pragma unroll
        for (int s = 0; s < 8; ++s) stash[(size_t)(i * 8 + s) * nthr + tid] = z[s];
      }
    }
    // the epilogue one slot at a time (a rolled loop: the reloads of the
    // stashed transforms are not hoisted into registers); the last transform
    // goes to the thread's own slots of its exchange buffer, free after the
    // transform, so that the loop indexes no register array
    if (!valid) return;
    store_slots(z, smb + c, t, T_, lC);
    const T kxv = ldr(epi.kx + col);
#pragma unroll 1
    for (int s = 0; s < 8; ++s) {
      cpx<T> v[NIN];
#pragma unroll
      for (int i = 0; i + 1 < NIN; ++i) v[i] = stash[(size_t)(i * 8 + s) * nthr + tid];
      v[NIN - 1] = smb[c + sidx<T>(t + s * T_, lC)];
      epi.at(v, t + s * T_, col, kxv, G, ky);
    }
    return;
  }
  if constexpr ((std::is_same<T, dfl>::value || (sizeof(T) == 4 && NIN >= 3)) && INV && is_epi_store<Epi>::value &&
                NMAP == 0) {
    // double-float y-inverse passes whose epilogue only stores (the
    // refinement matvec's, precision 3's right-hand side) and the FP32 RHS
    // y-inverse: one copy of the transform code for every input (a rolled
    // loop; inlined double-float transforms overflow the instruction cache),
    // each output stored right after its transform, so that one signal is
    // live at a time (FP32: 64 registers, two blocks of 512 per SM instead of
    // one at 128, 92.5 -> 73.8 us at 2048^2)
    const cpx<S>* srcs[NIN];
    int ders[NIN];
#pragma unroll
    for (int j = 0; j < NIN; ++j) {
      srcs[j] = in.src[j] + soff;
      ders[j] = in.deriv[j];
    }
#pragma unroll 1
    for (int i = 0; i < NIN; ++i) {
      const cpx<S>* src = srcs[0];
      bool der = ders[0] != 0;
#pragma unroll
      for (int j = 1; j < NIN; ++j)
        if (i == j) {
          src = srcs[j];
          der = ders[j] != 0;
        }
      const int fpf = (FL >> i) & 1, fdup = (FL >> (8 + i)) & 1, fdup_next = (FL >> (9 + i)) & 1;
      unsigned char* st_i = stage + (size_t)nthr * ystage_bytes<T, S, FL>(i);
      cpx<T> z[8];
      if (i > 0 && fpf) {
        cp_async_wait_all();
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          z[s] = ld_as<T, S>(reinterpret_cast<const cpx<S>*>(st_i) + s * nthr + tid);
          if (der) z[s] = mul_ik(z[s], ldr(ky + t + s * T_));
        }
      } else if (i > 0 && fdup) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
          z[s] = mul_ik(reinterpret_cast<const cpx<T>*>(st_i)[s * nthr + tid], ldr(ky + t + s * T_));
      } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int row = t + s * T_;
          z[s] = ld_as<T, S>(src + (size_t)row * G.ldS + col);
          if (der) z[s] = mul_ik(z[s], ldr(ky + row));
        }
      }
      if (fdup_next && i + 1 < NIN) {
        // input i + 1 is i ky times this one: keep the raw values
        cpx<T>* st = reinterpret_cast<cpx<T>*>(stage + (size_t)nthr * ystage_bytes<T, S, FL>(i + 1));
#pragma unroll
        for (int s = 0; s < 8; ++s) st[s * nthr + tid] = z[s];
      }
      fft_regs<INV>(z, smb + c, tw, t, lN, lC, PLAN);
      if (valid) {
        cpx<T>* dst = epi.dst[0];
#pragma unroll
        for (int j = 1; j < NIN; ++j)
          if (i == j) dst = epi.dst[j];
#pragma unroll
        for (int s = 0; s < 8; ++s) dst[(size_t)(t + s * T_) * G.ldS + col] = z[s];
      }
    }
    return;
  }
  bool waited = false;
#pragma unroll
  for (int i = 0; i < NIN; ++i) {
    if constexpr (NMAP > 0) {
      if ((FL & yf_tma(i)) || (i > 0 && (FL & yf_dup(i)) && (FL & yf_tma(i - 1)))) {
        const int m = (i > 0 && (FL & yf_tma(0)) && (FL & yf_tma(i))) ? 1 : 0;
        const bool dup = !(FL & yf_tma(i));
        if (!dup) {
          if (!mbar_wait_bounded(&tbar[m])) {
            // before the block's shared memory goes: one more bounded wait
            // for every tensor copy of this block still in flight
            if (tid == 0) {
              atomicOr(tm->flags, FLAG_WAIT);
#pragma unroll 1
              for (int q = 0; q < NMAP; ++q)
                for (int it = 0; it < (1 << 20) && !mbar_try_wait(&tbar[q], 0); ++it) {
                }
            }
            return;
          }
        }
        const cpx<T>* st = tstage + (size_t)m * (1 << lN) * (1 << lC);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int row = t + s * T_;
          cpx<T> z = st[(row << lC) + c];
          if (in.deriv[i]) z = mul_ik(z, ldr(ky + row));
          r[i][s] = z;
        }
        fft_regs<INV>(r[i], smb + c, tw, t, lN, lC, PLAN);
        continue;
      }
    }
    if (i > 0 && (FL & yf_pf(i))) {
      if (!waited) cp_async_wait_all();
      waited = true;
      const cpx<S>* st = reinterpret_cast<const cpx<S>*>(stage + (size_t)nthr * ystage_bytes<T, S, FL>(i));
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        cpx<T> z = ld_as<T, S>(st + s * nthr + tid);
        if (in.deriv[i]) z = mul_ik(z, ldr(ky + t + s * T_));
        r[i][s] = z;
      }
    } else if (i > 0 && (FL & yf_dup(i))) {
      const cpx<T>* st = reinterpret_cast<const cpx<T>*>(stage + (size_t)nthr * ystage_bytes<T, S, FL>(i));
#pragma unroll
      for (int s = 0; s < 8; ++s) r[i][s] = mul_ik(lds_fenced(st + s * nthr + tid), ldr(ky + t + s * T_));
    } else {
      const cpx<S>* src = in.src[i] + soff;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int row = t + s * T_;
        cpx<T> z = ld_as<T, S>(src + (size_t)row * G.ldS + col);
        if (in.deriv[i]) z = mul_ik(z, ldr(ky + row));
        r[i][s] = z;
      }
    }
    if (i + 1 < NIN && (FL & yf_dup(i + 1))) {
      cpx<T>* st = reinterpret_cast<cpx<T>*>(stage + (size_t)nthr * ystage_bytes<T, S, FL>(i + 1));
#pragma unroll
      for (int s = 0; s < 8; ++s) st[s * nthr + tid] = r[i][s];
      // the copy is read back after the transform: keep the compiler from
      // carrying the raw values in registers across it instead
      asm volatile("" ::: "memory");
    }
    fft_regs<INV>(r[i], smb + c, tw, t, lN, lC, PLAN);
  }
  epi(r, col, t, T_, valid, G, ky);
}

template <typename T, bool INV, int NIN, class Epi, typename S = T, int LN = 0, int FL = 0, int PLAN = 0>
__global__ void __launch_bounds__(ypass_threads<T, INV, LN, NIN>()) k_ypass(Geom G, const cpx<T>* __restrict__ tw,
                                                                   const T* __restrict__ ky, YIn<T, NIN, S> in,
                                                                   Epi epi) {
  ypass_body<T, INV, NIN, Epi, S, LN, FL, PLAN>(G, tw, ky, in, epi);
}
// FP32 passes with at most two transforms per thread: 64 registers, 32 warps
// per SM (measured with two 512-thread blocks: matvec y-forward 34 against
// 39 us at 2048^2 with the compiler's choice). The other passes keep the
// compiler's register choice.
template <typename T, bool INV, int NIN>
constexpr int ypass_o2_blocks() { return ypass_threads<T, INV, 0, NIN>() >= 1024 ? 1 : 2; }
template <typename T, bool INV, int NIN, class Epi, typename S = T, int LN = 0, int FL = 0, int PLAN = 0>
__global__ void __launch_bounds__(ypass_threads<T, INV, LN, NIN>(), ypass_o2_blocks<T, INV, NIN>()) k_ypass_o2(Geom G, const cpx<T>* __restrict__ tw,
                                                                        const T* __restrict__ ky,
                                                                        YIn<T, NIN, S> in, Epi epi) {
  ypass_body<T, INV, NIN, Epi, S, LN, FL, PLAN>(G, tw, ky, in, epi);
}
// FP32 passes whose inputs arrive by tensor copies (see yf_tma)
template <typename T, bool INV, int NIN, class Epi, int LN, int FL, int PLAN = 0>
__global__ void __launch_bounds__(ypass_threads<T, INV, LN, NIN>(), ypass_o2_blocks<T, INV, NIN>())
    k_ypass_tma(Geom G, const cpx<T>* __restrict__ tw, const T* __restrict__ ky, YIn<T, NIN, T> in,
                const __grid_constant__ YTma tm, Epi epi) {
  ypass_body<T, INV, NIN, Epi, T, LN, FL, PLAN>(G, tw, ky, in, epi, &tm);
}
constexpr int FL_MV_INV_TMA = yf_tma(0) | yf_dup(1);
constexpr int FL_MV_FWD_TMA = yf_tma(0) | yf_tma(1);

// Double-float passes of two or more inputs with one signal live at a time
// (see ypass_body): the y-inverses that only store and the y-forward passes,
// 256 threads, MINB blocks per SM: three, two for the three-input y-forward
// (its stash of two transforms leaves room for two). One input keeps k_ypass:
// 107 registers there, against 80 with 36 bytes spilled.
template <int MINB, typename T, bool INV, int NIN, class Epi, typename S = T, int LN = 0, int FL = 0, int PLAN = 0>
__global__ void __launch_bounds__(256, MINB) k_ypass_df(Geom G, const cpx<T>* __restrict__ tw,
                                                        const T* __restrict__ ky, YIn<T, NIN, S> in, Epi epi) {
  ypass_body<T, INV, NIN, Epi, S, LN, FL, PLAN>(G, tw, ky, in, epi);
}
// FP32 y-inverses of three or more inputs that only store (the RHS's), one
// signal live at a time (see ypass_body): two blocks of 512 per SM
template <typename T, bool INV, int NIN, class Epi, typename S = T, int LN = 0, int FL = 0, int PLAN = 0>
__global__ void __launch_bounds__(512, 2) k_ypass_f2(Geom G, const cpx<T>* __restrict__ tw,
                                                     const T* __restrict__ ky, YIn<T, NIN, S> in, Epi epi) {
  ypass_body<T, INV, NIN, Epi, S, LN, FL, PLAN>(G, tw, ky, in, epi);
}
template <typename T, bool INV, int NIN, class Epi, typename S = T, int LN = 0, int FL = 0, int PLAN = 0>
constexpr auto ypass_fn() {
  if constexpr (sizeof(T) == 4 && NIN <= 2)
    return &k_ypass_o2<T, INV, NIN, Epi, S, LN, FL, PLAN>;
  else if constexpr (sizeof(T) == 4 && INV && is_epi_store<Epi>::value && LN != 12)
    return &k_ypass_f2<T, INV, NIN, Epi, S, LN, FL, PLAN>;
  else if constexpr (std::is_same<T, dfl>::value && (!INV || is_epi_store<Epi>::value) && NIN >= 2 && LN != 12)
    return &k_ypass_df<(!INV && NIN >= 3) ? 2 : 3, T, INV, NIN, Epi, S, LN, FL, PLAN>;
  else
    return &k_ypass<T, INV, NIN, Epi, S, LN, FL, PLAN>;
}

// Calls f with std::integral_constant<int, 0> or <int, 1>: the radix plan of a
// tuned pass as a template argument (each plan is compiled on its own, so the
// built-in plan's kernels carry no code of the other)
// (a compile-time length 2^L with 3 | L has one plan: plan 0 serves both)
template <int L, class F>
static inline void dispatch_plan(int plan, F f) {
  if constexpr (L > 0 && L % 3 == 0) {
    f(std::integral_constant<int, 0>{});
  } else {
    if (plan)
      f(std::integral_constant<int, 1>{});
    else
      f(std::integral_constant<int, 0>{});
  }
}

template <typename T, int NIN>
struct EpiStore {
  cpx<T>* dst[NIN];
  __device__ __forceinline__ void operator()(cpx<T> (&r)[NIN][8], int col, int t, int T_, bool valid,
                                             const Geom& G, const T* ky) const {
    if (!valid) return;
#pragma unroll
    for (int i = 0; i < NIN; ++i)
#pragma unroll
      for (int s = 0; s < 8; ++s) dst[i][(size_t)(t + s * T_) * G.ldS + col] = r[i][s];
  }
};

// one transform stored as FP64 (the double-float conversion passes of the
// state of precision 2)
template <typename T>
struct EpiStoreF64 {
  cpx<double>* dst;
  __device__ __forceinline__ void operator()(cpx<T> (&r)[1][8], int col, int t, int T_, bool valid, const Geom& G,
                                             const T* ky) const {
    if (!valid) return;
#pragma unroll
    for (int s = 0; s < 8; ++s) dst[(size_t)(t + s * T_) * G.ldS + col] = mk(to_f64<T>(r[0][s].x), to_f64<T>(r[0][s].y));
  }
};

// w = [M^-1] (C - i ky By), M = 3 + kx^2 + ky^2 (Section 3 preconditioner)
// minv (may be null): the FP64 and double-float passes read M^-1 from a table,
// because a division costs about 25 FP64 instructions here; FP32 divides
// (cheap) on the fly. SO: the storage type of w (the double-float refinement
// matvec hands its result to the FP64 residual).
template <typename T, typename SO = T>
struct EpiMatvec {
  cpx<SO>* w;
  const T* kx;
  int precond;
  const T* minv;
  // the output at (row, col) from the two transforms' values v there
  __device__ __forceinline__ void at(const cpx<T> (&v)[2], int row, int col, T kxv, const Geom& G,
                                     const T* ky) const {
    const T kyv = ldr(ky + row);
    const size_t e = (size_t)row * G.ldS + col;
    cpx<T> z = v[0] - mul_ik(v[1], kyv);
    if (precond) z = scl(z, minv ? ldr(minv + e) : (T)1 / ((T)3 + kxv * kxv + kyv * kyv));
    if constexpr (std::is_same<T, dfl>::value && std::is_same<SO, double>::value)
      w[e] = mk(dfl_to_f64(z.x), dfl_to_f64(z.y));
    else
      w[e] = mk((SO)z.x, (SO)z.y);
  }
  __device__ __forceinline__ void operator()(cpx<T> (&r)[2][8], int col, int t, int T_, bool valid,
                                             const Geom& G, const T* ky) const {
    if (!valid) return;
    const T kxv = ldr(kx + col);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const cpx<T> v[2] = {r[0][s], r[1][s]};
      at(v, t + s * T_, col, kxv, G, ky);
    }
  }
};

// K = (h_t, vx_t, vy_t) from r0 = Cq^y, r1 = Qy^y, r2 = F^y:
// h_t = -i kx (h u_x)^ - i ky (h u_y)^, v_t = -i k F^ (2/3-masked if asked).
// Stored in the pass's type; the RK4 stage update is a separate flat kernel
// (k_rk_update) so that the FP64 state is read and written with coalesced rows
// rather than in the column layout of this pass.
template <typename T>
struct EpiK {
  cpx<T>* K[3];
  const T* kx;
  int dealias;
  // the outputs at (row, col) from the three transforms' values v there
  __device__ __forceinline__ void at(const cpx<T> (&v)[3], int row, int col, T kxv, const Geom& G,
                                     const T* ky) const {
    const T kyv = ldr(ky + row);
    const size_t e = (size_t)row * G.ldS + col;
    cpx<T> k0 = v[0] - mul_ik(v[1], kyv);
    cpx<T> k1 = mul_ik(v[2], -kxv);
    cpx<T> k2 = mul_ik(v[2], -kyv);
    if (dealias) {
      const int my = row <= (G.Ny >> 1) ? row : G.Ny - row;
      if (3 * col > G.Nx || 3 * my > G.Ny) {
        k0 = mk((T)0, (T)0);
        k1 = k0;
        k2 = k0;
      }
    }
    K[0][e] = k0;
    K[1][e] = k1;
    K[2][e] = k2;
  }
  __device__ __forceinline__ void operator()(cpx<T> (&r)[3][8], int col, int t, int T_, bool valid,
                                             const Geom& G, const T* ky) const {
    if (!valid) return;
    const T kxv = ldr(kx + col);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const cpx<T> v[3] = {r[0][s], r[1][s], r[2][s]};
      at(v, t + s * T_, col, kxv, G, ky);
    }
  }
};

// RK4 stage update (Section 3) on the state type S from K in type T, then
// b_hat = -(i kx vx + i ky vy) of the next stage state:
//   stage 1: acc = K,    U_s = U_n + dt/2 K;   stage 2: acc += 2K, U_s = U_n + dt/2 K
//   stage 3: acc += 2K,  U_s = U_n + dt K;     final:   U_n += dt/6 (acc + K), Krasny
//   RK_STORE_K: acc = K (one RHS evaluation)
// With an FP32 right-hand side (rhs_lin_split), K holds only its nonlinear
// part; the linear part comes from the stage state Y and sigma_hat here:
//   h_t += -i kx vx - i ky vy - (kx^2 + ky^2) sigma,  v_t += -i k g h,
// with the zeroed-Nyquist wavenumbers and the 2/3 mask of the FP32 pass.
// c6 = dt/6, cdt = the stage's dt (dt/2 or dt) and thr2 = the squared Krasny
// threshold times (Nx Ny)^2 come from the host (in every thread they would
// cost an FP64 division and products on the slow FP64 pipe).
template <typename T, typename S>
__global__ void k_rk_update(Geom G, RkK<T, S> a, double c6d, double cdtd, double thr2) {
  const RkArgs rk = a.rk;
  const S c6 = (S)c6d;
  const S cdt = (S)cdtd;
  const S g = (S)rk.g;
  for (Walk it(G); it.ok(); it.next()) {
    const size_t e = it.e;
    cpx<S> kk[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) kk[f] = mk(cvt<S>(a.K[f][e].x), cvt<S>(a.K[f][e].y));
    if (rhs_lin_split<T>()) {
      const int my = it.row <= (G.Ny >> 1) ? it.row : G.Ny - it.row;
      const bool keep = it.col < G.Nxh && (!rk.dealias || (3 * it.col <= G.Nx && 3 * my <= G.Ny));
      if (keep) {
        const S kxv = __ldg(a.kxs + it.col);
        const S kyv = __ldg(a.kys + it.row);
        const cpx<S> yh = a.Y[0][e], yx = a.Y[1][e], yy = a.Y[2][e], sg = a.sig[e];
        kk[0] = kk[0] - mul_ik(yx, kxv) - mul_ik(yy, kyv) - scl(sg, kxv * kxv + kyv * kyv);
        kk[1] = kk[1] - mul_ik(yh, g * kxv);
        kk[2] = kk[2] - mul_ik(yh, g * kyv);
      }
    }
    if (rk.mode == RK_STORE_K) {
#pragma unroll
      for (int f = 0; f < 3; ++f) a.acc[f][e] = kk[f];
      continue;
    }
    cpx<S> u[3];
    if (rk.mode == RK_FINAL) {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        cpx<S> z = a.Un[f][e] + scl(a.acc[f][e] + kk[f], c6);
        if (rk.krasny && (double)z.x * z.x + (double)z.y * z.y < thr2) z = mk((S)0, (S)0);
        a.Un[f][e] = z;
        u[f] = z;
      }
    } else {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        a.acc[f][e] = (rk.mode == RK_STAGE1) ? kk[f] : a.acc[f][e] + scl(kk[f], (S)2);
        u[f] = a.Un[f][e] + scl(kk[f], cdt);
        a.Unext[f][e] = u[f];
      }
    }
    if (a.b) {
      const S kxv = it.col < G.Nxh ? __ldg(a.kxs + it.col) : (S)0;
      a.b[e] = mul_ik(u[1], -kxv) - mul_ik(u[2], __ldg(a.kys + it.row));
    }
  }
}

// The kx = 0 and kx = Nx/2 columns of the half spectrum of a real field are
// Hermitian in ky: x(-ky) = conj(x(ky)), real at ky = 0 and ky = Ny/2. The
// inverse transforms read only that part, so an anti-Hermitian remainder (FP32
// rounding of RK4 increments leaves one in the state) lies in the null space
// of the discrete operator; left in b_hat it would stall GMRES at its size.
// This projects both columns onto their Hermitian part, in place.
template <typename T>
__global__ void k_hermitian_fix(Geom G, cpx<T>* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // 0 .. Ny/2 for each of the 2 columns
  const int half = G.Ny >> 1;
  if (i > 2 * half + 1) return;
  const int col = (i <= half) ? 0 : (G.Nx >> 1);
  const int ky = (i <= half) ? i : i - half - 1;
  const int kn = (G.Ny - ky) & (G.Ny - 1);
  cpx<T>* a = x + (size_t)ky * G.ldS + col;
  cpx<T>* b = x + (size_t)kn * G.ldS + col;
  if (ky == kn) {
    a->y = (T)0;
  } else {
    const cpx<T> va = *a, vb = *b;
    const cpx<T> h = mk((T)0.5 * (va.x + vb.x), (T)0.5 * (va.y - vb.y));
    *a = h;
    *b = conjg(h);
  }
}

template <typename T>
cudaError_t launch_hermitian_fix(const Geom& G, cpx<T>* x, const Exec& ex) {
  const int n = 2 * ((G.Ny >> 1) + 1);
  ex.begin(PK_KRYLOV);
  k_hermitian_fix<T><<<(n + 127) / 128, 128, 0, ex.s>>>(G, x);
  ex.end();
  return cudaGetLastError();
}

// ------------------------------------------------------------ launchers

// Calls f(std::integral_constant<int, LN>) with LN = lN for the sizes that have
// compile-time kernels (FP32: 256..4096 points; every type: 4096, whose
// transforms take 512 threads), LN = 0 (runtime size) otherwise.
template <typename T, class F>
static inline void dispatch_ln(int lN, F&& f) {
  if (lN == 12) {
    f(std::integral_constant<int, 12>());
    return;
  }
  if constexpr (sizeof(T) == 4) {
    switch (lN) {
      case 8: f(std::integral_constant<int, 8>()); return;
      case 9: f(std::integral_constant<int, 9>()); return;
      case 10: f(std::integral_constant<int, 10>()); return;
      case 11: f(std::integral_constant<int, 11>()); return;
      default: break;
    }
  }
  f(std::integral_constant<int, 0>());
}

// LN = 12 at 4096 points, else LN = 0: the passes that have no other
// compile-time sizes.
template <class F>
static inline void dispatch_l12(int lN, F&& f) {
  if (lN == 12)
    f(std::integral_constant<int, 12>());
  else
    f(std::integral_constant<int, 0>());
}

template <typename T>
static inline int x_pairs_per_block(const Geom& G) {
  int Tn = G.Nx >> 3;
  int P = Tn >= 256 ? 1 : 256 / Tn;
  int half = G.Ny >> 1;
  if (P > half) P = half;
  return P;
}
template <typename T>
static inline void x_config(const Geom& G, dim3& grid, dim3& block, size_t& smem, int nf, int tpb = 0,
                            int extra_elems_per_group = 0) {
  int P = x_pairs_per_block<T>(G);
  // tuned shape: whole row pairs, a power of two, within the launch bound
  const int Tn = G.Nx >> 3;
  if (tpb > 0 && tpb % Tn == 0) {
    const int q = tpb / Tn;
    if ((q & (q - 1)) == 0 && tpb <= (G.lNx == 12 ? 512 : 256) && q <= (G.Ny >> 1)) P = q;
  }
  block = dim3((G.Nx >> 3) * P);
  grid = dim3((G.Ny / 2 + P - 1) / P, nf);
  smem = (size_t)P * (smem_elems_of<T>(G.Nx) + extra_elems_per_group) * sizeof(cpx<T>);
}
template <typename T, bool INV, int NIN>
static inline void y_config(const Geom& G, dim3& grid, dim3& block, size_t& smem, int stage_per_thread = 0,
                            int tpb_tuned = 0, bool* builtin = nullptr) {
  const int Tn = G.Ny >> 3;
  const int bound = G.lNy == 12 ? ypass_threads<T, INV, 12, NIN>() : ypass_threads<T, INV, 0, NIN>();
  int C = bound / Tn;
  if (C < 1) C = 1;
  if (C > 64) C = 64;
  const int C0 = C;
  // tuned shape: whole columns, a power of two, within the launch bound
  if (tpb_tuned > 0 && tpb_tuned % Tn == 0) {
    const int q = tpb_tuned / Tn;
    if ((q & (q - 1)) == 0 && q <= 64 && tpb_tuned <= bound && tpb_tuned >= 32) C = q;
  }
  if (builtin) *builtin = C == C0;
  block = dim3(Tn * C);
  grid = dim3((G.Nxh + C - 1) / C);
  int lC = 0;
  while ((1 << lC) < C) ++lC;
  smem = ystage_offset<T>(G.lNy, lC) + (size_t)block.x * stage_per_thread;
}

static constexpr int kMaxDynSmem = 227 * 1024;

// Dynamic shared memory limit of a kernel: the device's opt-in maximum less
// the kernel's static shared memory (the mbarriers of the tensor-copy passes),
// capped at 227 KB.
template <typename T>
static void set_smem(const void* fn) {
  int dev = 0, optin = kMaxDynSmem;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, fn);
  int lim = optin - (int)fa.sharedSizeBytes;
  if (lim > kMaxDynSmem) lim = kMaxDynSmem;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// the kernels sgn_autotune can give either radix plan, at compile-time length L
template <typename T, int L, int P>
static void set_attrs_ln_plan() {
  set_smem<T>((const void*)k_mv_x<T, L, P>);
  set_smem<T>((const void*)k_rhs_x<T, L, P>);
  set_smem<T>((const void*)ypass_fn<T, true, 2, EpiStore<T, 2>, T, L, FL_MV_INV, P>());
  set_smem<T>((const void*)ypass_fn<T, false, 2, EpiMatvec<T>, T, L, fl_mv_fwd<T>(), P>());
  if constexpr (sizeof(T) == 4) {
    set_smem<T>((const void*)k_ypass_tma<T, true, 2, EpiStore<T, 2>, L, FL_MV_INV_TMA, P>);
    set_smem<T>((const void*)k_ypass_tma<T, false, 2, EpiMatvec<T, T>, L, FL_MV_FWD_TMA, P>);
  }
  set_smem<T>((const void*)ypass_fn<T, true, 4, EpiStore<T, 4>, double, L, fl_rhs_inv<T, L>(), P>());
  set_smem<T>((const void*)ypass_fn<T, false, 3, EpiK<T>, T, L, fl_rhs_fwd<T>(), P>());
}

template <typename T, int L>
static void set_attrs_ln() {
  set_attrs_ln_plan<T, L, 0>();
  if constexpr (L % 3 != 0) set_attrs_ln_plan<T, L, 1>();
  if constexpr (L == 12) {
    set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>, T, L>());
    set_smem<T>((const void*)ypass_fn<T, false, 1, EpiStore<T, 1>, T, L>());
    set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>, double, L>());
  }
}

// the same at runtime length (LN = 0)
template <typename T, int P>
static void set_attrs_plan() {
  set_smem<T>((const void*)k_mv_x<T, 0, P>);
  set_smem<T>((const void*)k_rhs_x<T, 0, P>);
  set_smem<T>((const void*)ypass_fn<T, true, 2, EpiStore<T, 2>, T, 0, FL_MV_INV, P>());
  if constexpr (sizeof(T) == 4) {
    set_smem<T>((const void*)k_ypass_tma<T, true, 2, EpiStore<T, 2>, 0, FL_MV_INV_TMA, P>);
    set_smem<T>((const void*)k_ypass_tma<T, false, 2, EpiMatvec<T, T>, 0, FL_MV_FWD_TMA, P>);
  }
  set_smem<T>((const void*)ypass_fn<T, true, 4, EpiStore<T, 4>, T, 0, fl_rhs_inv<T, 0>(), P>());
  set_smem<T>((const void*)ypass_fn<T, false, 2, EpiMatvec<T>, T, 0, fl_mv_fwd<T>(), P>());
  set_smem<T>((const void*)ypass_fn<T, false, 3, EpiK<T>, T, 0, fl_rhs_fwd<T>(), P>());
  set_smem<T>((const void*)ypass_fn<T, true, 4, EpiStore<T, 4>, double, 0, fl_rhs_inv<T, 0>(), P>());
}

template <typename T>
void init_kernel_attributes() {
  if constexpr (sizeof(T) == 4) {
    set_attrs_ln<T, 8>();
    set_attrs_ln<T, 9>();
    set_attrs_ln<T, 10>();
    set_attrs_ln<T, 11>();
  }
  set_attrs_ln<T, 12>();
  set_attrs_plan<T, 0>();
  set_attrs_plan<T, 1>();
  set_smem<T>((const void*)k_x_r2c<T>);
  set_smem<T>((const void*)k_x_c2r<T>);
  set_smem<T>((const void*)k_coef_x<T>);
  set_smem<T>((const void*)ypass_fn<T, false, 1, EpiStore<T, 1>>());
  set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>>());
  set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>, double>());
  cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_r2c(const Geom& G, const Tables<T>& tb, const double* const* f, int nf,
                         cpx<T>* const* out, const Exec& ex) {
  XR2CArgs<T> a{};
  for (int i = 0; i < nf; ++i) {
    a.f[i] = f[i];
    a.out[i] = out[i];
  }
  dim3 grid, block;
  size_t smem;
  x_config<T>(G, grid, block, smem, nf);
  ex.begin(PK_IO);
  k_x_r2c<T><<<grid, block, smem, ex.s>>>(G, tb.twx, a);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_c2r(const Geom& G, const Tables<T>& tb, const cpx<T>* const* in, const int* deriv,
                         int nf, double* const* out, double scale, const Exec& ex) {
  XC2RArgs<T> a{};
  for (int i = 0; i < nf; ++i) {
    a.in[i] = in[i];
    a.out[i] = out[i];
    a.deriv[i] = deriv ? deriv[i] : 0;
  }
  dim3 grid, block;
  size_t smem;
  x_config<T>(G, grid, block, smem, nf);
  ex.begin(PK_IO);
  k_x_c2r<T><<<grid, block, smem, ex.s>>>(G, tb.twx, tb.kx, a, scale);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_y_fft(const Geom& G, const Tables<T>& tb, bool inverse, const cpx<T>* const* in,
                         const int* deriv, int nf, cpx<T>* const* out, const Exec& ex) {
  dim3 grid, block;
  size_t smem;
  if (inverse)
    y_config<T, true, 1>(G, grid, block, smem);
  else
    y_config<T, false, 1>(G, grid, block, smem);
  for (int i = 0; i < nf; ++i) {
    YIn<T, 1> yi{};
    yi.src[0] = in[i];
    yi.deriv[0] = deriv ? deriv[i] : 0;
    EpiStore<T, 1> ep{};
    ep.dst[0] = out[i];
    dispatch_l12(G.lNy, [&](auto ln) {
      constexpr int L = decltype(ln)::value;
      ex.begin(PK_IO);
      if (inverse)
        ypass_fn<T, true, 1, EpiStore<T, 1>, T, L>()<<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, ep);
      else
        ypass_fn<T, false, 1, EpiStore<T, 1>, T, L>()<<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, ep);
      ex.end();
    });
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coef_x(const Geom& G, const Tables<T>& tb, const cpx<T>* Hy, T* h, T* cr, T* cc, int* flags,
                          const CoefCopy& cp, const Exec& ex) {
  dim3 grid, block;
  size_t smem;
  x_config<T>(G, grid, block, smem, 1);
  ex.begin(PK_COEF);
  k_coef_x<T><<<grid, block, smem, ex.s>>>(G, tb.twx, tb.kx, Hy, h, cr, cc, flags, cp);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coef_phys(const Geom& G, const double* hphys, T* h, T* cr, T* cc, int* flags,
                             const CoefCopy& cp, const Exec& ex) {
  ex.begin(PK_COEF);
  k_coef_phys<T><<<NBLK, 256, 0, ex.s>>>(G, hphys, h, cr, cc, flags, cp);
  ex.end();
  return cudaGetLastError();
}

// S: storage type of sigma_hat and w; T: arithmetic of the passes
// Columns per block of the FP32 two-input y-passes (tpb: tuned threads or 0).
static inline int mv_y_columns(const Geom& G, int tpb) {
  dim3 grid, block;
  size_t smem;
  y_config<float, false, 2>(G, grid, block, smem, 0, tpb);
  return (int)block.x / (G.Ny >> 3);
}

// Launch bound of a y-pass in threads, per arithmetic and pass (mirrors
// ypass_threads), and of an x-pass.
static int y_bound(const Geom& G, int type, int pass) {
  const bool inv = pass == TP_MV_YINV || pass == TP_RHS_YINV;
  const int nin = (pass == TP_MV_YINV || pass == TP_MV_YFWD) ? 2 : (pass == TP_RHS_YINV ? 4 : 3);
  const bool l12 = G.lNy == 12;
  if (type == TT_F32) return nin <= 2 ? 1024 : 512;
  if (type == TT_F64) return l12 ? 512 : 256;
  if (nin >= 3) return l12 ? 512 : 256;
  return (l12 || !inv) ? 512 : 256;
}
static bool is_y_pass(int pass) { return pass <= TP_RHS_YFWD; }

#ifdef SGN_SPECTRAL_COMMON
int pass_default_threads(const Geom& G, int type, int pass) {
  if (is_y_pass(pass)) {
    const int Tn = G.Ny >> 3;
    int C = y_bound(G, type, pass) / Tn;
    if (C < 1) C = 1;
    if (C > 64) C = 64;
    return Tn * C;
  }
  const int Tn = G.Nx >> 3;
  int P = Tn >= 256 ? 1 : 256 / Tn;
  if (P > (G.Ny >> 1)) P = G.Ny >> 1;
  return Tn * P;
}
#endif  // SGN_SPECTRAL_COMMON

#ifdef SGN_SPECTRAL_COMMON
int pass_candidates(const Geom& G, int type, int pass, int* out, int max_out) {
  int n = 0;
  if (is_y_pass(pass)) {
    const int Tn = G.Ny >> 3, bound = y_bound(G, type, pass);
    for (int C = 1; C <= 64 && n < max_out; C *= 2) {
      const int t = Tn * C;
      if (t > bound) break;
      if (t >= 32) out[n++] = t;
    }
  } else {
    const int Tn = G.Nx >> 3, bound = G.lNx == 12 ? 512 : 256;
    for (int P = 1; P <= (G.Ny >> 1) && n < max_out; P *= 2) {
      const int t = Tn * P;
      if (t > bound) break;
      if (t >= 32 || P == (G.Ny >> 1) || t * 2 > bound) out[n++] = t;
    }
  }
  if (n == 0 && max_out > 0) out[n++] = pass_default_threads(G, type, pass);
  return n;
}
#endif  // SGN_SPECTRAL_COMMON

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// [nvec][Ny][2 ldS] FP32 tensor at base, box [1][min(Ny, 256)][2 C]
static bool encode_spectra(EncodeTiledFn enc, const Geom& G, const void* base, int nvec, int C, CUtensorMap* m) {
  const cuuint64_t dims[3] = {(cuuint64_t)2 * G.ldS, (cuuint64_t)G.Ny, (cuuint64_t)nvec};
  const cuuint64_t strides[2] = {(cuuint64_t)G.ldS * 8, (cuuint64_t)G.ldS * 8 * G.Ny};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * C), (cuuint32_t)(G.Ny < 256 ? G.Ny : 256), 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

#ifdef SGN_SPECTRAL_COMMON
bool make_mv_tma(const Geom& G, const void* V, int nvec, const void* t0, const void* t1, int* flags,
                 const Tune* tune, MvTma* out) {
  *out = MvTma{};
  // row strides must be multiples of 16 bytes, and a box at most 256 wide
  const int Ci = mv_y_columns(G, tune ? tune->tpb[TT_F32][TP_MV_YINV] : 0);
  const int Cf = mv_y_columns(G, tune ? tune->tpb[TT_F32][TP_MV_YFWD] : 0);
  if ((G.ldS * 8) % 16 != 0 || 2 * Ci > 256 || 2 * Cf > 256) return false;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(fn);
  if (!encode_spectra(enc, G, V, nvec, Ci, &out->v) || !encode_spectra(enc, G, t0, 1, Cf, &out->t0) ||
      !encode_spectra(enc, G, t1, 1, Cf, &out->t1))
    return false;
  out->cinv = Ci;
  out->cfwd = Cf;
  out->vbase = V;
  out->t0base = t0;
  out->t1base = t1;
  out->vs = G.nspec();
  out->nvec = nvec;
  out->flags = flags;
  out->ok = 1;
  return true;
}
#endif  // SGN_SPECTRAL_COMMON

// The FP32 matvec with tensor-copied y-pass inputs; false if it does not apply.
template <typename T>
static bool matvec_tma(const Geom& G, const Tables<T>& tb, const cpx<T>* sig, const T* cr, const T* cc, cpx<T>* w,
                       cpx<T>* const* tmp, bool precond, const Exec& ex, const int* jsel, const MvTma* tma) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    if (!tma || !tma->ok || tmp[0] != tma->t0base || tmp[1] != tma->t1base) return false;
    long long zj = 0;
    if (!jsel) {
      const long long off = (const char*)sig - (const char*)tma->vbase;
      const long long vb = (long long)(tma->vs * sizeof(cpx<T>));
      if (off < 0 || off % vb != 0 || off / vb >= tma->nvec) return false;
      zj = off / vb;
    } else if (sig != tma->vbase) {
      return false;
    }
    dim3 grid, block;
    size_t smem;
    // the boxes of the maps fix the columns per block
    bool bi = true, bf = true;
    y_config<T, true, 2>(G, grid, block, smem, 0, ex.tpb(TT_F32, TP_MV_YINV), &bi);
    const int C = (int)block.x / (G.Ny >> 3);
    {
      dim3 g2, b2;
      size_t s2;
      y_config<T, false, 2>(G, g2, b2, s2, 0, ex.tpb(TT_F32, TP_MV_YFWD), &bf);
      if (C != tma->cinv || (int)b2.x / (G.Ny >> 3) != tma->cfwd) return false;
    }
    int lC = 0;
    while ((1 << lC) < C) ++lC;
    const size_t tile = (size_t)G.Ny * C * sizeof(cpx<T>);
    YTma ti{};
    ti.map[0] = tma->v;
    ti.z[0] = (int)zj;
    ti.zsel = jsel;
    ti.flags = tma->flags;
    smem = ystage_offset<T>(G.lNy, lC) + 128 + tile;
    dispatch_ln<T>(bi ? G.lNy : 0, [&](auto ln) {
      constexpr int L = decltype(ln)::value;
      YIn<T, 2> yi{};
      yi.src[0] = sig;
      yi.src[1] = sig;
      yi.deriv[1] = 1;
      EpiStore<T, 2> ep{};
      ep.dst[0] = tmp[0];
      ep.dst[1] = tmp[1];
      ex.begin(PK_MV_YINV);
      dispatch_plan<L>(ex.plan(TT_F32, TP_MV_YINV), [&](auto pl) {
        k_ypass_tma<T, true, 2, EpiStore<T, 2>, L, FL_MV_INV_TMA, decltype(pl)::value>
            <<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, ti, ep);
      });
      ex.end();
    });
    x_config<T>(G, grid, block, smem, 1, ex.tpb(TT_F32, TP_MV_X), mv_stash_elems(G.Nx));
    dispatch_ln<T>(G.lNx, [&](auto ln) {
      constexpr int L = decltype(ln)::value;
      ex.begin(PK_MV_X);
      dispatch_plan<L>(ex.plan(TT_F32, TP_MV_X), [&](auto pl) {
        k_mv_x<T, L, decltype(pl)::value>
            <<<grid, block, smem, ex.s>>>(G, tb.twx, tb.kx, tmp[0], tmp[1], cr, cc, tmp[0], tmp[1]);
      });
      ex.end();
    });
    y_config<T, false, 2>(G, grid, block, smem, 0, ex.tpb(TT_F32, TP_MV_YFWD));
    const int Cf = (int)block.x / (G.Ny >> 3);
    int lCf = 0;
    while ((1 << lCf) < Cf) ++lCf;
    const size_t tilef = (size_t)G.Ny * Cf * sizeof(cpx<T>);
    YTma tf{};
    tf.map[0] = tma->t0;
    tf.map[1] = tma->t1;
    tf.flags = tma->flags;
    smem = ystage_offset<T>(G.lNy, lCf) + 128 + 2 * tilef;
    dispatch_ln<T>(bf ? G.lNy : 0, [&](auto ln) {
      constexpr int L = decltype(ln)::value;
      YIn<T, 2> yi{};
      yi.src[0] = tmp[0];
      yi.src[1] = tmp[1];
      EpiMatvec<T, T> ep{w, tb.kx, precond ? 1 : 0, tb.minv};
      ex.begin(PK_MV_YFWD);
      dispatch_plan<L>(ex.plan(TT_F32, TP_MV_YFWD), [&](auto pl) {
        k_ypass_tma<T, false, 2, EpiMatvec<T, T>, L, FL_MV_FWD_TMA, decltype(pl)::value>
            <<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, tf, ep);
      });
      ex.end();
    });
    return true;
  }
}

template <typename T, typename S>
cudaError_t launch_matvec_io(const Geom& G, const Tables<T>& tb, const cpx<S>* sig, const T* cr, const T* cc,
                             cpx<S>* w, cpx<T>* const* tmp, bool precond, const Exec& ex, const int* jsel,
                             size_t jstride) {
  dim3 grid, block;
  size_t smem;
  // y-inverse of sigma_hat and i ky sigma_hat (read once, the second formed
  // from the staged copy)
  bool bi = true;
  y_config<T, true, 2>(G, grid, block, smem, ystage_bytes<T, S, FL_MV_INV>(2), ex.tpb(tune_type<T>(), TP_MV_YINV),
                       &bi);
  dispatch_ln<T>(bi ? G.lNy : 0, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    YIn<T, 2, S> yi{};
    yi.src[0] = sig;
    yi.src[1] = sig;
    yi.deriv[0] = 0;
    yi.deriv[1] = 1;
    yi.sel = jsel;
    yi.sel_stride = jstride;
    EpiStore<T, 2> ep{};
    ep.dst[0] = tmp[0];
    ep.dst[1] = tmp[1];
    ex.begin(PK_MV_YINV);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_MV_YINV), [&](auto pl) {
      ypass_fn<T, true, 2, EpiStore<T, 2>, S, L, FL_MV_INV, decltype(pl)::value>()<<<grid, block, smem, ex.s>>>(
          G, tb.twy, tb.ky, yi, ep);
    });
    ex.end();
  });
  x_config<T>(G, grid, block, smem, 1, ex.tpb(tune_type<T>(), TP_MV_X), mv_stash_elems(G.Nx));
  dispatch_ln<T>(G.lNx, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    ex.begin(PK_MV_X);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_MV_X), [&](auto pl) {
      k_mv_x<T, L, decltype(pl)::value>
          <<<grid, block, smem, ex.s>>>(G, tb.twx, tb.kx, tmp[0], tmp[1], cr, cc, tmp[0], tmp[1]);
    });
    ex.end();
  });
  bool bf = true;
  y_config<T, false, 2>(G, grid, block, smem, ystage_bytes<T, T, fl_mv_fwd<T>()>(2) + ystash_bytes<T, false, 2>(),
                        ex.tpb(tune_type<T>(), TP_MV_YFWD),
                        &bf);
  dispatch_ln<T>(bf ? G.lNy : 0, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    YIn<T, 2> yi{};
    yi.src[0] = tmp[0];
    yi.src[1] = tmp[1];
    EpiMatvec<T, S> ep{w, tb.kx, precond ? 1 : 0, tb.minv};
    ex.begin(PK_MV_YFWD);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_MV_YFWD), [&](auto pl) {
      ypass_fn<T, false, 2, EpiMatvec<T, S>, T, L, fl_mv_fwd<T>(), decltype(pl)::value>()<<<grid, block, smem, ex.s>>>(
          G, tb.twy, tb.ky, yi, ep);
    });
    ex.end();
  });
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_matvec(const Geom& G, const Tables<T>& tb, const cpx<T>* sig, const T* cr, const T* cc,
                          cpx<T>* w, cpx<T>* const* tmp, bool precond, const Exec& ex, const int* jsel,
                          size_t jstride, const MvTma* tma) {
  if (matvec_tma<T>(G, tb, sig, cr, cc, w, tmp, precond, ex, jsel, tma)) return cudaGetLastError();
  return launch_matvec_io<T, T>(G, tb, sig, cr, cc, w, tmp, precond, ex, jsel, jstride);
}

// y-inverse of one FP64 half spectrum into the pass type T (the coefficient
// pass of the double-float path)
template <typename T>
cudaError_t launch_y_inv64(const Geom& G, const Tables<T>& tb, const cpx<double>* in, cpx<T>* out, const Exec& ex) {
  dim3 grid, block;
  size_t smem;
  y_config<T, true, 1>(G, grid, block, smem);
  YIn<T, 1, double> yi{};
  yi.src[0] = in;
  EpiStore<T, 1> ep{};
  ep.dst[0] = out;
  dispatch_l12(G.lNy, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    ex.begin(PK_IO);
    ypass_fn<T, true, 1, EpiStore<T, 1>, double, L>()<<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, ep);
    ex.end();
  });
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_y_fwd64(const Geom& G, const Tables<T>& tb, const cpx<T>* in, cpx<double>* out, const Exec& ex) {
  dim3 grid, block;
  size_t smem;
  y_config<T, false, 1>(G, grid, block, smem);
  YIn<T, 1> yi{};
  yi.src[0] = in;
  EpiStoreF64<T> ep{out};
  dispatch_l12(G.lNy, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    ex.begin(PK_IO);
    ypass_fn<T, false, 1, EpiStoreF64<T>, T, L>()<<<grid, block, smem, ex.s>>>(G, tb.twy, tb.ky, yi, ep);
    ex.end();
  });
  return cudaGetLastError();
}

// dynamic shared memory limits of the double-float kernels
template <int P>
static void set_attrs_df_plan() {
  typedef dfl T;
  set_smem<T>((const void*)k_mv_x<T, 0, P>);
  set_smem<T>((const void*)ypass_fn<T, true, 2, EpiStore<T, 2>, double, 0, FL_MV_INV, P>());
  set_smem<T>((const void*)ypass_fn<T, false, 2, EpiMatvec<T, double>, T, 0, fl_mv_fwd<T>(), P>());
  if constexpr (P == 0) {  // 4096 points: one plan
    set_smem<T>((const void*)k_mv_x<T, 12, P>);
    set_smem<T>((const void*)ypass_fn<T, true, 2, EpiStore<T, 2>, double, 12, FL_MV_INV, P>());
    set_smem<T>((const void*)ypass_fn<T, false, 2, EpiMatvec<T, double>, T, 12, fl_mv_fwd<T>(), P>());
  }
}

// precision 3: the double-float right-hand side
template <int P>
static void set_attrs_df_rhs_plan() {
  typedef dfl T;
  set_smem<T>((const void*)k_rhs_x<T, 0, P>);
  set_smem<T>((const void*)ypass_fn<T, true, 4, EpiStore<T, 4>, double, 0, fl_rhs_inv<T, 0>(), P>());
  set_smem<T>((const void*)ypass_fn<T, false, 3, EpiK<T>, T, 0, fl_rhs_fwd<T>(), P>());
  if constexpr (P == 0) {  // 4096 points: one plan
    set_smem<T>((const void*)k_rhs_x<T, 12, P>);
    set_smem<T>((const void*)ypass_fn<T, true, 4, EpiStore<T, 4>, double, 12, fl_rhs_inv<T, 12>(), P>());
    set_smem<T>((const void*)ypass_fn<T, false, 3, EpiK<T>, T, 12, fl_rhs_fwd<T>(), P>());
  }
}

#ifdef SGN_SPECTRAL_DF_RHS
void init_kernel_attributes_df_rhs() {
  set_attrs_df_rhs_plan<0>();
  set_attrs_df_rhs_plan<1>();
  cudaGetLastError();
}
#endif  // SGN_SPECTRAL_DF_RHS

#ifdef SGN_SPECTRAL_DF
void init_kernel_attributes_df() {
  typedef dfl T;
  set_attrs_df_plan<0>();
  set_attrs_df_plan<1>();
  init_kernel_attributes_df_rhs();
  set_smem<T>((const void*)k_coef_x<T>);
  set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>, double>());
  set_smem<T>((const void*)ypass_fn<T, true, 1, EpiStore<T, 1>, double, 12>());
  set_smem<T>((const void*)k_x_r2c<T>);
  set_smem<T>((const void*)k_x_c2r<T>);
  set_smem<T>((const void*)ypass_fn<T, false, 1, EpiStoreF64<T>, T, 0>());
  set_smem<T>((const void*)ypass_fn<T, false, 1, EpiStoreF64<T>, T, 12>());
  cudaGetLastError();
}
#endif  // SGN_SPECTRAL_DF

template <typename T, typename S>
cudaError_t launch_rhs(const Geom& G, const Tables<T>& tb, const Tables<S>& tbs, cpx<S>* const* U,
                       const cpx<S>* sig, const T* h, const T* cr, cpx<T>* const* tmp, cpx<S>* const* Un,
                       cpx<S>* const* Unext, cpx<S>* const* acc, cpx<S>* bhat, const RkArgs& rk, const Exec& ex) {
  dim3 grid, block;
  size_t smem;
  bool bi = true;
  y_config<T, true, 4>(G, grid, block, smem, 0, ex.tpb(tune_type<T>(), TP_RHS_YINV), &bi);
  dispatch_ln<T>(bi ? G.lNy : 0, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    constexpr int FL = fl_rhs_inv<T, L>();
    y_config<T, true, 4>(G, grid, block, smem, ystage_bytes<T, S, FL>(4), ex.tpb(tune_type<T>(), TP_RHS_YINV));
    YIn<T, 4, S> yi{};
    yi.src[0] = U[1];
    yi.src[1] = U[2];
    yi.src[2] = sig;
    yi.src[3] = sig;
    yi.deriv[3] = 1;
    EpiStore<T, 4> ep{};
    for (int i = 0; i < 4; ++i) ep.dst[i] = tmp[i];
    ex.begin(PK_RHS_YINV);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_RHS_YINV), [&](auto pl) {
      ypass_fn<T, true, 4, EpiStore<T, 4>, S, L, FL, decltype(pl)::value>()<<<grid, block, smem, ex.s>>>(
          G, tb.twy, tb.ky, yi, ep);
    });
    ex.end();
  });
  // each block reads only its own row pair before writing it, so the outputs
  // may overwrite the inputs
  x_config<T>(G, grid, block, smem, 1, ex.tpb(tune_type<T>(), TP_RHS_X), rhs_acc_elems<T>(G.Nx));
  dispatch_ln<T>(G.lNx, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    ex.begin(PK_RHS_X);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_RHS_X), [&](auto pl) {
      k_rhs_x<T, L, decltype(pl)::value><<<grid, block, smem, ex.s>>>(G, tb.twx, tb.kx, tmp[0], tmp[1], tmp[2],
                                                                      tmp[3], h, cr, (T)rk.g, tmp[0], tmp[1],
                                                                      tmp[2]);
    });
    ex.end();
  });
  bool bf = true;
  y_config<T, false, 3>(G, grid, block, smem, ystage_bytes<T, T, fl_rhs_fwd<T>()>(3) + ystash_bytes<T, false, 3>(),
                        ex.tpb(tune_type<T>(), TP_RHS_YFWD),
                        &bf);
  dispatch_ln<T>(bf ? G.lNy : 0, [&](auto ln) {
    constexpr int L = decltype(ln)::value;
    YIn<T, 3> yi{};
    yi.src[0] = tmp[0];
    yi.src[1] = tmp[1];
    yi.src[2] = tmp[2];
    // K overwrites the three inputs column by column (each block reads its
    // columns completely before writing them)
    EpiK<T> ep{};
    for (int f = 0; f < 3; ++f) ep.K[f] = tmp[f];
    ep.kx = tb.kx;
    ep.dealias = rk.dealias;
    ex.begin(PK_RHS_YFWD);
    dispatch_plan<L>(ex.plan(tune_type<T>(), TP_RHS_YFWD), [&](auto pl) {
      ypass_fn<T, false, 3, EpiK<T>, T, L, fl_rhs_fwd<T>(), decltype(pl)::value>()<<<grid, block, smem, ex.s>>>(
          G, tb.twy, tb.ky, yi, ep);
    });
    ex.end();
  });
  {
    RkK<T, S> a{};
    for (int f = 0; f < 3; ++f) {
      a.K[f] = tmp[f];
      a.Un[f] = Un[f];
      a.Unext[f] = Unext ? Unext[f] : nullptr;
      a.acc[f] = acc[f];
    }
    a.b = bhat;
    a.kxs = tbs.kx;
    a.kys = tbs.ky;
    for (int f = 0; f < 3; ++f) a.Y[f] = U[f];
    a.sig = sig;
    a.rk = rk;
    ex.begin(PK_RK);
    k_rk_update<T, S><<<NBLK, 256, 0, ex.s>>>(G, a, rk.dt / 6.0, rk.mode == RK_STAGE3 ? rk.dt : 0.5 * rk.dt,
                                               rk.krasny_thr * rk.krasny_thr * (double)G.nphys() *
                                                   (double)G.nphys());
    ex.end();
  }
  return cudaGetLastError();
}

// ------------------------------------------------ spectral pointwise kernels

template <typename T>
__global__ void k_spec_div(Geom G, const T* __restrict__ kx, const T* __restrict__ ky, const cpx<T>* vx,
                           const cpx<T>* vy, cpx<T>* b) {
  for (Walk it(G); it.ok(); it.next()) {
    const T kxv = it.col < G.Nxh ? __ldg(kx + it.col) : (T)0;
    b[it.e] = mul_ik(vx[it.e], -kxv) - mul_ik(vy[it.e], __ldg(ky + it.row));
  }
}

template <typename T>
cudaError_t launch_spec_div(const Geom& G, const Tables<T>& tb, const cpx<T>* vx, const cpx<T>* vy, cpx<T>* b,
                            const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_spec_div<T><<<NBLK, 256, 0, ex.s>>>(G, tb.kx, tb.ky, vx, vy, b);
  ex.end();
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_precond(Geom G, const T* __restrict__ kx, const T* __restrict__ ky,
                                                 const T* __restrict__ minv, const cpx<T>* in, cpx<T>* out,
                                                 double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (Walk it(G); it.ok(); it.next()) {
    const T kxv = it.col < G.Nxh ? __ldg(kx + it.col) : (T)0;
    const T kyv = __ldg(ky + it.row);
    const T m = minv ? __ldg(minv + it.e) : (T)1 / ((T)3 + kxv * kxv + kyv * kyv);
    const cpx<T> z = scl(in[it.e], m);
    out[it.e] = z;
    acc += col_weight_k(G, it.col) * ((double)z.x * z.x + (double)z.y * z.y);
  }
  const double tot = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename T>
cudaError_t launch_precond(const Geom& G, const Tables<T>& tb, const cpx<T>* in, cpx<T>* out, double* partials,
                           const Exec& ex) {
  ex.begin(PK_KRYLOV);
  k_precond<T><<<NBLK, 256, 0, ex.s>>>(G, tb.kx, tb.ky, tb.minv, in, out, partials);
  ex.end();
  return cudaGetLastError();
}

// ------------------------------------------------------- instantiations
// the launchers of one arithmetic (used by the per-type units)
#define SGN_INST(T)                                                                                          \
  template void init_kernel_attributes<T>();                                                                 \
  template cudaError_t launch_x_r2c<T>(const Geom&, const Tables<T>&, const double* const*, int,             \
                                       cpx<T>* const*, const Exec&);                                        \
  template cudaError_t launch_x_c2r<T>(const Geom&, const Tables<T>&, const cpx<T>* const*, const int*, int, \
                                       double* const*, double, const Exec&);                                \
  template cudaError_t launch_y_fft<T>(const Geom&, const Tables<T>&, bool, const cpx<T>* const*,            \
                                       const int*, int, cpx<T>* const*, const Exec&);                       \
  template cudaError_t launch_coef_x<T>(const Geom&, const Tables<T>&, const cpx<T>*, T*, T*, T*, int*,      \
                                        const CoefCopy&, const Exec&);                                      \
  template cudaError_t launch_coef_phys<T>(const Geom&, const double*, T*, T*, T*, int*, const CoefCopy&,   \
                                           const Exec&);                                                    \
  template cudaError_t launch_matvec<T>(const Geom&, const Tables<T>&, const cpx<T>*, const T*, const T*,    \
                                        cpx<T>*, cpx<T>* const*, bool, const Exec&, const int*, size_t,     \
                                        const MvTma*);                                                      \
  template cudaError_t launch_spec_div<T>(const Geom&, const Tables<T>&, const cpx<T>*, const cpx<T>*,      \
                                          cpx<T>*, const Exec&);                                            \
  template cudaError_t launch_precond<T>(const Geom&, const Tables<T>&, const cpx<T>*, cpx<T>*, double*,    \
                                         const Exec&);                                                      \
  template cudaError_t launch_hermitian_fix<T>(const Geom&, cpx<T>*, const Exec&);

}  // namespace sgn
