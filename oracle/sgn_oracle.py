"""Plain FP64 CPU oracle of the 2D SGN hot path (test infrastructure only).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. The GPU library never
calls it, and it shares no code with the CUDA path.

It restates, step by step and without fusion or reordering, what Gavrilyuk &
Klein, "Numerical study of the Serre-Green-Naghdi equations in 2D" define:

* potential form of SGN in (h, v = grad phi), Section 2.2, Eqs. (1)-(3), and the
  v-form of the Bernoulli equation, Section 3 (the equation before (sigmav));
* the elliptic equation L[sigma] = 3 sigma/h^3 - div(grad sigma / h) = -div v,
  Section 3, Eq. (sigmav);
* Fourier collocation on the torus with derivatives as i k multipliers,
  Section 3 (Fourier convention and g_x ~ i k_x g);
* left-preconditioned restarted GMRES (Saad-Schultz) with M = 3 + kx^2 + ky^2,
  Section 3 (preconditioner paragraph);
* classic explicit RK4 on (h, v), GMRES warm-started with the last sigma,
  Section 3 (time integration paragraph);
* the Krasny filter, Section 3;
* mass, momentum and energy integrals, Section 2.3, Eqs. (total_mass),
  (total_momentum), (total_energy);
* the monitoring quantities of the transverse-stability runs, Sections 3,
  4.1 and 4.2 (L-infinity norm and crest of h, the fitted solitary wave, the
  decay of the DFT coefficients).

Readings where the paper is silent or garbled:
* grid x_j = -Lx/2 + j Lx/Nx with the FULL period Lx (the paper's period is
  2 pi L_x; its collocation formula lost the "/N_x");
* the Nyquist wavenumber is set to zero in i k, and the same zeroed k enter
  M = 3 + kx^2 + ky^2, so that M equals L exactly at h = 1;
* GMRES: restart m, stop when the estimate of ||M^-1 (b - L sigma)||_2 is at
  most tol * ||M^-1 b||_2 (Euclidean norm over grid values); an iteration cap
  ``maxit`` counts matvecs over all cycles; Arnoldi by modified Gram-Schmidt;
* Krasny: zero a DFT coefficient when |DFT| / (Nx Ny) < thr, on h, vx, vy
  after each full RK4 step;
* optional 2/3 dealiasing (not in the paper): the RHS spectra keep only modes
  with 3|m_x| <= Nx and 3|m_y| <= Ny (m the integer wavenumber);
* h_inf = 1.

numpy.fft serves as the DFT primitive (unnormalised forward transform,
1/N on the inverse), full complex transforms, real part taken after inversion.
"""
from __future__ import annotations

import math

import numpy as np

H_INF = 1.0


class Grid:
    """Periodic collocation grid and wavenumbers (Section 3, collocation points)."""

    def __init__(self, Nx: int, Ny: int, Lx: float, Ly: float):
        assert Nx % 2 == 0 and Ny % 2 == 0
        self.Nx, self.Ny, self.Lx, self.Ly = Nx, Ny, float(Lx), float(Ly)
        self.x = -0.5 * Lx + Lx * np.arange(Nx) / Nx
        self.y = -0.5 * Ly + Ly * np.arange(Ny) / Ny
        mx = np.fft.fftfreq(Nx, d=1.0 / Nx)  # 0..Nx/2-1, -Nx/2..-1
        my = np.fft.fftfreq(Ny, d=1.0 / Ny)
        self.mx, self.my = mx, my
        kx = 2.0 * math.pi * mx / Lx
        ky = 2.0 * math.pi * my / Ly
        kx[Nx // 2] = 0.0  # Nyquist set to zero (reading)
        ky[Ny // 2] = 0.0
        # broadcastable (Ny, Nx) shapes: rows are y, columns are x
        self.KX = kx[None, :]
        self.KY = ky[:, None]
        self.M = 3.0 + self.KX ** 2 + self.KY ** 2
        self.dxdy = self.Lx * self.Ly / (Nx * Ny)


def fft2(f):
    return np.fft.fft2(f)


def ifft2_real(F):
    return np.fft.ifft2(F).real


def dx(G: Grid, f):
    """Spectral x-derivative: DFT, multiply by i kx, inverse DFT (Section 3)."""
    return ifft2_real(1j * G.KX * fft2(f))


def dy(G: Grid, f):
    """Spectral y-derivative: DFT, multiply by i ky, inverse DFT (Section 3)."""
    return ifft2_real(1j * G.KY * fft2(f))


def elliptic_apply(G: Grid, h, sigma):
    """L[sigma] = 3 sigma / h^3 - d/dx(sigma_x / h) - d/dy(sigma_y / h), Eq. (sigmav)."""
    return 3.0 * sigma / h ** 3 - dx(G, dx(G, sigma) / h) - dy(G, dy(G, sigma) / h)


def precond_solve(G: Grid, f):
    """M^{-1} f with M = 3 + kx^2 + ky^2 (L at h = 1), Section 3."""
    return ifft2_real(fft2(f) / G.M)


def divergence_rhs(G: Grid, vx, vy):
    """b = -div v, the right-hand side of Eq. (sigmav)."""
    return -(dx(G, vx) + dy(G, vy))


def gmres(G: Grid, h, b, sigma0, tol=1e-10, restart=20, maxit=1000):
    """Left-preconditioned restarted GMRES for L sigma = b (Saad-Schultz).

    Solves A x = c with A = M^{-1} L and c = M^{-1} b. Arnoldi by modified
    Gram-Schmidt, Givens rotations on the Hessenberg matrix, stop when the
    residual estimate |g_{j+1}| <= tol ||c||. Returns (sigma, iters, relres, converged).
    """
    def A(x):
        return precond_solve(G, elliptic_apply(G, h, x))

    def norm(x):
        return math.sqrt(float(np.sum(x * x)))

    c = precond_solve(G, b)
    cnorm = norm(c)
    if cnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    x = np.array(sigma0, dtype=np.float64, copy=True)
    its = 0
    m = restart
    while True:
        r = c - A(x)
        beta = norm(r)
        if beta <= tol * cnorm:
            return x, its, beta / cnorm, True
        if its >= maxit:
            return x, its, beta / cnorm, False
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        k = 0
        res = beta
        for j in range(m):
            w = A(V[j])
            its += 1
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = float(np.sum(V[i] * w))
                w = w - H[i, j] * V[i]
            hnext = norm(w)
            H[j + 1, j] = hnext
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d
            sn[j] = H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            res = abs(gvec[j + 1])
            k = j + 1
            if res <= tol * cnorm or its >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        # back substitution on the k x k upper triangle
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (gvec[i] - float(np.dot(H[i, i + 1:k], y[i + 1:k]))) / H[i, i]
        for i in range(k):
            x = x + y[i] * V[i]
        if res <= tol * cnorm:
            return x, its, res / cnorm, True


def dealias_mask(G: Grid):
    """2/3 rule: keep modes with 3|m_x| <= Nx and 3|m_y| <= Ny."""
    keep_x = 3.0 * np.abs(G.mx) <= G.Nx
    keep_y = 3.0 * np.abs(G.my) <= G.Ny
    return (keep_y[:, None] & keep_x[None, :]).astype(np.float64)


def rhs(G: Grid, h, vx, vy, sigma0, g=1.0, tol=1e-10, restart=20, maxit=1000,
        dealias=False):
    """Time derivatives of (h, vx, vy); Section 2.2 Eq. (1) and the v-form of Eq. (2).

    sigma solves Eq. (sigmav) by GMRES from the warm start sigma0. Then
    u = v - grad sigma / h, h_t = -div(h u), and v_t = -grad F with
    F = |v|^2/2 - |grad sigma|^2/(2h^2) + g h - 9 sigma^2/(2h^4).
    Returns (ht, vxt, vyt, sigma, gmres_info).
    """
    b = divergence_rhs(G, vx, vy)
    sigma, its, relres, conv = gmres(G, h, b, sigma0, tol=tol, restart=restart, maxit=maxit)
    sx = dx(G, sigma)
    sy = dy(G, sigma)
    ux = vx - sx / h
    uy = vy - sy / h
    ht = -(dx(G, h * ux) + dy(G, h * uy))
    F = 0.5 * (vx ** 2 + vy ** 2) - (sx ** 2 + sy ** 2) / (2.0 * h ** 2) + g * h \
        - 4.5 * sigma ** 2 / h ** 4
    vxt = -dx(G, F)
    vyt = -dy(G, F)
    if dealias:
        mask = dealias_mask(G)
        ht = ifft2_real(mask * fft2(ht))
        vxt = ifft2_real(mask * fft2(vxt))
        vyt = ifft2_real(mask * fft2(vyt))
    return ht, vxt, vyt, sigma, dict(iters=its, relres=relres, converged=conv)


def krasny(G: Grid, f, thr=1e-12):
    """Krasny filter: zero DFT coefficients with |DFT|/(Nx Ny) < thr (Section 3)."""
    F = fft2(f)
    F[np.abs(F) / (G.Nx * G.Ny) < thr] = 0.0
    return ifft2_real(F)


def rk4_step(G: Grid, h, vx, vy, sigma, dt, nsteps=1, g=1.0, tol=1e-10, restart=20,
             maxit=1000, krasny_on=False, krasny_thr=1e-12, dealias=False, log=None):
    """Classic explicit RK4 on (h, vx, vy), Section 3.

    Each stage's GMRES starts from the sigma of the previous stage (the last
    computed sigma, also across steps). Returns (h, vx, vy, sigma).
    """
    kw = dict(g=g, tol=tol, restart=restart, maxit=maxit, dealias=dealias)
    for _ in range(nsteps):
        k1h, k1x, k1y, sigma, i1 = rhs(G, h, vx, vy, sigma, **kw)
        k2h, k2x, k2y, sigma, i2 = rhs(G, h + 0.5 * dt * k1h, vx + 0.5 * dt * k1x,
                                       vy + 0.5 * dt * k1y, sigma, **kw)
        k3h, k3x, k3y, sigma, i3 = rhs(G, h + 0.5 * dt * k2h, vx + 0.5 * dt * k2x,
                                       vy + 0.5 * dt * k2y, sigma, **kw)
        k4h, k4x, k4y, sigma, i4 = rhs(G, h + dt * k3h, vx + dt * k3x, vy + dt * k3y,
                                       sigma, **kw)
        h = h + dt / 6.0 * (k1h + 2.0 * k2h + 2.0 * k3h + k4h)
        vx = vx + dt / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x)
        vy = vy + dt / 6.0 * (k1y + 2.0 * k2y + 2.0 * k3y + k4y)
        if krasny_on:
            h = krasny(G, h, krasny_thr)
            vx = krasny(G, vx, krasny_thr)
            vy = krasny(G, vy, krasny_thr)
        if log is not None:
            log.append([i1, i2, i3, i4])
    return h, vx, vy, sigma


def invariants(G: Grid, h, vx, vy, sigma, g=1.0):
    """Mass, momentum (x, y) and energy by the rectangle rule on the torus.

    Eqs. (total_mass), (total_momentum), (total_energy) with u = v - grad sigma / h.
    """
    sx = dx(G, sigma)
    sy = dy(G, sigma)
    ux = vx - sx / h
    uy = vy - sy / h
    mass = G.dxdy * float(np.sum(h - H_INF))
    px = G.dxdy * float(np.sum(h * ux))
    py = G.dxdy * float(np.sum(h * uy))
    energy = G.dxdy * float(np.sum(0.5 * h * (ux ** 2 + uy ** 2)
                                   + 1.5 * sigma ** 2 / h ** 3
                                   + 0.5 * g * (h - H_INF) ** 2))
    return np.array([mass, px, py, energy])


def line_soliton_profile(xi, a, g=1.0):
    """h and v of the line solitary wave of Eq. (sol) with crest h_inf + a at xi = 0.

    h = h_inf + a sech^2(kappa xi), kappa^2 = 3a / (4 h_inf^2 (h_inf + a)),
    c^2 = g (h_inf + a), v = c - (c h_inf / h) (1 + (h^2)_xixi / 6).
    """
    c = np.sqrt(g * (H_INF + a))
    kappa = np.sqrt(3.0 * a / (4.0 * H_INF ** 2 * (H_INF + a)))
    sech2 = 1.0 / np.cosh(kappa * xi) ** 2
    h = H_INF + a * sech2
    # (h^2)'' = 2 (h'^2 + h h''), h' = a (sech^2)', (sech^2)'' = kappa^2 (4 sech^2 - 6 sech^4)
    d1 = -2.0 * kappa * sech2 * np.tanh(kappa * xi)
    d2 = kappa ** 2 * (4.0 * sech2 - 6.0 * sech2 ** 2)
    h2xx = 2.0 * ((a * d1) ** 2 + h * a * d2)
    v = c - (c * H_INF / h) * (1.0 + h2xx / 6.0)
    return h, v


def diagnostics(G: Grid, h, vx, vy, g=1.0):
    """The monitoring quantities of Sections 3 and 4.

    * the L-infinity norm of h and the grid point of the maximum (the crest
      location x_s of Section 4.1; the first maximum in row-major order);
    * the speed of the line solitary wave of Eq. (sol) whose maximum equals it,
      c = sqrt(g h_max) (Section 4.2 fits c this way, h_inf = 1);
    * the largest differences of h and vx from that solitary wave centred at
      x_s (Sections 4.1, 4.2), the nearest periodic image in x, and max |vy|;
    * the size of the DFT coefficients of h, vx, vy on the outermost modes,
      16 |m_x| >= 7 Nx or 16 |m_y| >= 7 Ny, divided by Nx Ny (Section 3 reads
      resolution from their decay).
    """
    i_max = int(np.argmax(h))
    h_max = float(h.flat[i_max])
    jy, jx = divmod(i_max, G.Nx)
    x_s = float(G.x[jx])
    y_s = float(G.y[jy])
    c_fit = float(np.sqrt(g * h_max))
    a = h_max - H_INF
    if a > 0.0:
        xi = G.x - x_s
        xi = np.where(xi >= 0.5 * G.Lx, xi - G.Lx, xi)
        xi = np.where(xi < -0.5 * G.Lx, xi + G.Lx, xi)
        hc, vc = line_soliton_profile(xi, a, g)
        dev_h = float(np.max(np.abs(h - hc[None, :])))
        dev_vx = float(np.max(np.abs(vx - vc[None, :])))
    else:
        dev_h = dev_vx = float("nan")
    mx = np.abs(np.fft.fftfreq(G.Nx, 1.0 / G.Nx))
    my = np.abs(np.fft.fftfreq(G.Ny, 1.0 / G.Ny))
    band = (16 * mx[None, :] >= 7 * G.Nx) | (16 * my[:, None] >= 7 * G.Ny)
    tail = [float(np.max(np.abs(fft2(f))[band]) / (G.Nx * G.Ny)) for f in (h, vx, vy)]
    return dict(h_max=h_max, i_max=i_max, x_s=x_s, y_s=y_s, c_fit=c_fit, dev_h=dev_h, dev_vx=dev_vx,
                max_vy=float(np.max(np.abs(vy))), tail=tail)


def _band(N, n):
    m = np.fft.fftfreq(N, 1.0 / N)
    return np.abs(m) < n / 2


def coarse_sample(G: Grid, f, n):
    """The Fourier modes |m_x|, |m_y| < n/2 of f, evaluated at the grid points
    (j Nx/n, i Ny/n): the coarse inputs of the learned GMRES start."""
    F = fft2(f) * (_band(G.Ny, n)[:, None] & _band(G.Nx, n)[None, :])
    return ifft2_real(F)[::G.Ny // n, ::G.Nx // n]


def coarse_embed(G: Grid, fc, n, scale=1.0):
    """The field on the fine grid with Fourier modes |m| < n/2 only whose
    samples at the points of coarse_sample are scale * fc (modes of fc with
    |m| >= n/2 dropped)."""
    D = np.fft.fft2(scale * np.asarray(fc, dtype=np.float64)) * (_band(n, n)[:, None] & _band(n, n)[None, :])
    F = np.zeros((G.Ny, G.Nx), dtype=complex)
    m = np.fft.fftfreq(n, 1.0 / n).astype(int)
    F[np.ix_(m % G.Ny, m % G.Nx)] = D * (G.Nx * G.Ny / (n * n))
    return ifft2_real(F)


def dense_elliptic_matrix(G: Grid, h):
    """Columns L e_j of the discrete operator, for tiny grids (N <= a few hundred)."""
    N = G.Nx * G.Ny
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = elliptic_apply(G, h, e.reshape(G.Ny, G.Nx)).ravel()
    return A
