"""Plain FP64 CPU oracle for contour-deformation G0W0 (arXiv 2107.10423).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA library; both take their inputs from ``paper_2107_10423_gb300.synth``.

Everything is numpy float64, written for a reader to check against the paper
by eye: no blocking, fusion or reordering beyond what the equations state.
Library primitives used as single steps: matrix products, ``numpy.linalg.solve``
(LAPACK LU), ``numpy.linalg.eigh`` and ``numpy.polynomial.legendre.leggauss``.

Notation (Sec. 3.1-3.3): closed shell, orthonormal Coulomb-metric auxiliary
basis, B[P, ia] = (P|ia) with pair index ia = i*n_virt + a, D_ia = e_a - e_i,
b_nm = B[:, nm] for a target state n and any state m.

Readings where the paper is silent or garbled:
  * Pi on the imaginary axis uses eta = 0; on the real axis Pi(x) keeps the
    paper's +i*eta inside both pole terms and the residue frequency is the
    real x = e_m - omega (no second i*eta);
  * W in the CD formulas is the correlation part (1-Pi)^-1 - 1; the bare
    part is Sigma_x;
  * the I term is written over xi >= 0 by evenness of W(i xi), with a static
    subtraction W(0) * sgn(a)/2 that is an exact rewrite of the integral;
  * theta(0) = 1/2;
  * modified Gauss-Legendre grid xi = x0 (1+t)/(1-t), w = 2 x0 w_GL/(1-t)^2;
  * V_xc defaults to Sigma_x (so e_QP = e + Re Sigma_c(e_QP));
  * step-tree QP solver constants 0.3 / 0.1 / 0.7 / cap 0.1 Ha and the
    bracket rules as described in ``qp_steptree``.
"""
from __future__ import annotations

import math

import numpy as np

GOLD = (3.0 - math.sqrt(5.0)) / 2.0     # 1 - 1/phi, the golden-section fraction


# --------------------------------------------------------------------------
# Frequency grid (Sec. 3.3, text after eq. "inn": modified Gauss-Legendre grid)
# --------------------------------------------------------------------------
def mgl_grid(n: int, x0: float = 0.5):
    """Modified Gauss-Legendre grid on [0, inf): Gauss-Legendre nodes t_k on
    [-1, 1] mapped by xi = x0 (1+t)/(1-t); weights carry the Jacobian
    2 x0/(1-t)^2.  Returns (xi, w) ascending."""
    t, wgl = np.polynomial.legendre.leggauss(n)
    xi = x0 * (1.0 + t) / (1.0 - t)
    w = 2.0 * x0 * wgl / (1.0 - t) ** 2
    return xi, w


# --------------------------------------------------------------------------
# Polarizability in the auxiliary basis (Sec. 3.3, equation after "wauxbas")
# --------------------------------------------------------------------------
def pair_energies(eps, n_occ):
    """D_ia = e_a - e_i for i occupied, a virtual, flattened as i*n_virt + a."""
    eps = np.asarray(eps, dtype=np.float64)
    return (eps[None, n_occ:] - eps[:n_occ, None]).reshape(-1)


def pi_imag(eps, n_occ, B_ia, xi):
    """Pi_PQ(i xi) = sum_sigma sum_ia B_P,ia [1/(i xi - D) + 1/(-i xi - D)] B_Q,ia
                  = -4 sum_ia B_P,ia B_Q,ia D_ia / (D_ia^2 + xi^2)   (closed shell, eta = 0)."""
    D = pair_energies(eps, n_occ)
    return (B_ia * (-4.0 * D / (D * D + xi * xi))) @ B_ia.T


def pi_complex(eps, n_occ, B_ia, z, eta):
    """Pi_PQ(z) for a complex frequency z with the paper's +i*eta in both pole terms:
    2 sum_ia B_P,ia [1/(z - D + i eta) + 1/(-z - D + i eta)] B_Q,ia."""
    D = pair_energies(eps, n_occ)
    c = 2.0 * (1.0 / (z - D + 1j * eta) + 1.0 / (-z - D + 1j * eta))
    return (B_ia * c) @ B_ia.T


def dpi_complex(eps, n_occ, B_ia, z, eta):
    """d Pi(z)/dz = 2 sum_ia B B [-1/(z - D + i eta)^2 + 1/(-z - D + i eta)^2]."""
    D = pair_energies(eps, n_occ)
    c = 2.0 * (-1.0 / (z - D + 1j * eta) ** 2 + 1.0 / (-z - D + 1j * eta) ** 2)
    return (B_ia * c) @ B_ia.T


def w_corr(Pi, b):
    """Correlation part of W (Sec. 3.3, eq. "wauxbas" minus the bare term):
    b^T [(1 - Pi)^-1 - 1] b, dense LU solve.  ``b`` is [n_aux] or [n_aux, k]
    (one value per column).  Works for real or complex (symmetric) Pi."""
    A = np.eye(Pi.shape[0], dtype=Pi.dtype) - Pi
    y = np.linalg.solve(A, b)
    if b.ndim == 1:
        return b @ y - b @ b
    return np.einsum("pk,pk->k", b, y) - np.einsum("pk,pk->k", b, b)


def w_corr_and_deriv(Pi, dPi, b):
    """W(x) = b^T[(1-Pi)^-1 - 1]b and dW/dx = y^T Pi'(x) y with y = (1-Pi)^-1 b
    (complex symmetric: plain transpose, no conjugation)."""
    A = np.eye(Pi.shape[0], dtype=Pi.dtype) - Pi
    y = np.linalg.solve(A, b)
    return b @ y - b @ b, y @ (dPi @ y)


# --------------------------------------------------------------------------
# Exchange self-energy (Algorithm 1, Init: Sigma_x_nn = -sum_i sum_P (P|ni)^2)
# --------------------------------------------------------------------------
def sigma_x(B_nm_t, n_occ):
    """Sigma^x_nn = -sum_{i occ} sum_P B_P,ni^2, for one target's rows B_nm_t [n_bas, n_aux]."""
    return -np.sum(B_nm_t[:n_occ, :] ** 2)


# --------------------------------------------------------------------------
# Spectral decomposition (Sec. 2.2 and 3.2)
# --------------------------------------------------------------------------
def casida(eps, n_occ, B_ia):
    """Hermitian Casida form (Sec. 3.2): (A-B)^1/2 (A+B) (A-B)^1/2 T = Omega^2 T with
    A-B = diag(D) and A+B = diag(D) + 4 B^T B.  Returns Omega [N_ov] ascending and
    V = 2 B D^1/2 T [n_aux, N_ov] so that the correlation part of W is
    W^c_nm(z) = sum_s (b_nm . V_s)^2 / (2 Omega_s) [1/(z - Omega_s) - 1/(z + Omega_s)]."""
    D = pair_energies(eps, n_occ)
    K = B_ia.T @ B_ia
    sD = np.sqrt(D)
    M = sD[:, None] * (np.diag(D) + 4.0 * K) * sD[None, :]
    Om2, T = np.linalg.eigh(M)
    Omega = np.sqrt(Om2)
    V = (2.0 * B_ia * sD[None, :]) @ T
    return Omega, V


def casida_full_omegas(eps, n_occ, B_ia):
    """Positive eigenvalues of the non-Hermitian Casida problem [[A, B],[-B, -A]] (eq. "rpa")
    with A = diag(D) + 2K, B = 2K, K_ia,jb = (ia|jb) = sum_P B_P,ia B_P,jb."""
    D = pair_energies(eps, n_occ)
    K = B_ia.T @ B_ia
    A = np.diag(D) + 2.0 * K
    Bm = 2.0 * K
    H = np.block([[A, Bm], [-Bm, -A]])
    ev = np.linalg.eigvals(H)
    ev = np.sort(ev.real)
    return ev[ev > 0]


def w_corr_sd(Omega, V, b, z):
    """W^c(z) from the spectral sum (eq. "analytic_w" minus the bare term)."""
    w2 = (V.T @ b) ** 2 / (2.0 * Omega)
    return np.sum(w2 * (1.0 / (z - Omega) - 1.0 / (z + Omega)))


def sigma_c_sd(eps, n_occ, B_nm_t, Omega, V, omega, eta=0.0):
    """Sigma^c_nn(omega) by spectral decomposition (Sec. 3.2, last equation):
    sum_i sum_s (w^s_ni)^2/(omega - e_i + Omega_s - i eta) + sum_a sum_s (w^s_na)^2/(omega - e_a - Omega_s + i eta)
    with w^s_nm = b_nm . V_s / sqrt(2 Omega_s).  Returns (Re Sigma, Re dSigma/domega)."""
    eps = np.asarray(eps)
    w2 = (B_nm_t @ V) ** 2 / (2.0 * Omega[None, :])        # [n_bas, n_s]
    den = np.empty_like(w2, dtype=np.complex128)
    den[:n_occ] = omega - eps[:n_occ, None] + Omega[None, :] - 1j * eta
    den[n_occ:] = omega - eps[n_occ:, None] - Omega[None, :] + 1j * eta
    s = np.sum(w2 / den)
    ds = -np.sum(w2 / den ** 2)
    return s.real, ds.real


# --------------------------------------------------------------------------
# Contour deformation (Sec. 2.3 and 3.3, eqs. "R", "I", "inn", "rnn"; Algorithm 1)
# --------------------------------------------------------------------------
def theta(x):
    """Heaviside step with the half-maximum convention theta(0) = 1/2."""
    return 1.0 if x > 0 else (0.5 if x == 0 else 0.0)


def residue_set(eps, n_occ, omega):
    """Residues of eq. "rnn" at frequency omega: list of (m, sign, theta) with sign -1 for
    occupied m (theta(e_m - omega)) and +1 for virtual m (theta(omega - e_m)), theta != 0."""
    out = []
    for m, e in enumerate(eps):
        th = theta(e - omega) if m < n_occ else theta(omega - e)
        if th != 0.0:
            out.append((m, -1.0 if m < n_occ else 1.0, th))
    return out


class CDSelfEnergy:
    """Correlation self-energy Sigma^c_nn(omega) = R_nn(omega) - I_nn(omega) by contour deformation.

    Imaginary-axis table (Algorithm 1, loop over the imaginary grid): W^c_nm(i xi_g) for every
    grid point, plus the static W^c_nm(0), each from a dense LU solve with 1 - Pi(i xi).
    Residues (eq. "rnn"): W^c_nm(e_m - omega) from a dense complex LU solve with 1 - Pi(x).

    ``eps`` are the energies in Pi (the pair energies D_ia of W); ``eps_g`` (default ``eps``) are the poles of
    G, the e_m of the I and R terms.  They differ inside the eigenvalue self-consistency loop of Algorithm 1
    (``evgw``)."""

    def __init__(self, eps, n_occ, B_ia, B_nm, targets, xi, wt, eta=1e-3, eps_g=None):
        self.eps = np.asarray(eps, dtype=np.float64)
        self.eps_g = self.eps if eps_g is None else np.asarray(eps_g, dtype=np.float64)
        self.n_occ = int(n_occ)
        self.B_ia = B_ia
        self.B_nm = B_nm                       # [n_t, n_bas, n_aux]
        self.targets = list(targets)
        self.xi = np.asarray(xi, dtype=np.float64)
        self.wt = np.asarray(wt, dtype=np.float64)
        self.eta = float(eta)
        n_t, n_bas, _ = B_nm.shape
        self.W = np.empty((n_t, n_bas, len(self.xi)))   # W^c_nm(i xi_g)
        self.W0 = np.empty((n_t, n_bas))                  # W^c_nm(0)
        for g, x in enumerate(self.xi):
            Pi = pi_imag(self.eps, self.n_occ, B_ia, x)
            for t in range(n_t):
                self.W[t, :, g] = w_corr(Pi, B_nm[t].T)
        Pi0 = pi_imag(self.eps, self.n_occ, B_ia, 0.0)
        for t in range(n_t):
            self.W0[t] = w_corr(Pi0, B_nm[t].T)
        self.n_residue_solves = 0

    def sigma_x(self, t):
        return sigma_x(self.B_nm[t], self.n_occ)

    def i_term(self, t, omega, static_subtraction=True):
        """I_nn(omega) of eq. "inn" over xi >= 0 and its omega-derivative.
        Literal form (Algorithm 1): (1/pi) sum_m sum_g w_g W_nm(i xi_g) a/(a^2 + xi_g^2), a = omega - e_m.
        Static-subtracted form: W_nm(i xi_g) -> W_nm(i xi_g) - W_nm(0) plus the exact
        W_nm(0) sgn(a)/2 (whose delta-function derivative cancels the theta jump of R)."""
        a = omega - self.eps_g                                # [n_bas]
        xi2 = self.xi[None, :] ** 2
        a2 = a[:, None] ** 2
        if static_subtraction:
            Wg = self.W[t] - self.W0[t][:, None]
        else:
            Wg = self.W[t]
        lor = a[:, None] / (a2 + xi2)
        dlor = (xi2 - a2) / (a2 + xi2) ** 2
        I = np.sum(self.wt[None, :] * Wg * lor) / math.pi
        dI = np.sum(self.wt[None, :] * Wg * dlor) / math.pi
        if static_subtraction:
            I += np.sum(self.W0[t] * np.sign(a)) / 2.0
        return I, dI

    def residue_w(self, t, m, x):
        """W^c_nm(x) and dW^c_nm/dx on the real axis, dense complex LU."""
        Pi = pi_complex(self.eps, self.n_occ, self.B_ia, x, self.eta)
        dPi = dpi_complex(self.eps, self.n_occ, self.B_ia, x, self.eta)
        self.n_residue_solves += 1
        return w_corr_and_deriv(Pi, dPi, self.B_nm[t, m])

    def r_term(self, t, omega, residue_fn=None):
        """R_nn(omega) of eq. "rnn" (real part) and its omega-derivative."""
        R = 0.0
        dR = 0.0
        for m, sgn, th in residue_set(self.eps_g, self.n_occ, omega):
            x = self.eps_g[m] - omega
            w, dw = (residue_fn or self.residue_w)(t, m, x)
            R += sgn * th * w.real
            dR -= sgn * th * dw.real          # d/domega W(e_m - omega) = -W'(x)
        return R, dR

    def sigma_c(self, t, omega, static_subtraction=True, residue_fn=None):
        """Re Sigma^c_nn(omega) = R - I and its omega-derivative."""
        R, dR = self.r_term(t, omega, residue_fn)
        I, dI = self.i_term(t, omega, static_subtraction)
        return R - I, dR - dI


# --------------------------------------------------------------------------
# MINRES (Paige & Saunders 1975; Sec. 3.3 residue solves)
# --------------------------------------------------------------------------
def minres(matvec, b, tol=1e-10, maxit=1000):
    """Unpreconditioned MINRES for a real symmetric (possibly indefinite) operator.

    Lanczos: beta_1 v_1 = b; beta_{k+1} v_{k+1} = A v_k - alpha_k v_k - beta_k v_{k-1}.
    The (k+1) x k tridiagonal least-squares problem min ||beta_1 e_1 - T_k y|| is reduced
    by Givens rotations; x_k is updated through direction vectors d_k.  Stops when the
    recurrence residual norm |phibar_k| <= tol * ||b||.
    Returns (x, iterations, relative residual estimate)."""
    n = b.shape[0]
    x = np.zeros(n)
    beta1 = np.linalg.norm(b)
    if beta1 == 0.0:
        return x, 0, 0.0
    v_prev = np.zeros(n)
    v = b / beta1
    beta = 0.0                      # coupling between v_{k-1} and v_k (none for k = 1)
    c_m2, s_m2 = 1.0, 0.0           # rotation G_{k-2}
    c_m1, s_m1 = 1.0, 0.0           # rotation G_{k-1}
    d_m2 = np.zeros(n)
    d_m1 = np.zeros(n)
    phibar = beta1
    k = 0
    for k in range(1, maxit + 1):
        p = matvec(v) - beta * v_prev
        alpha = v @ p
        p = p - alpha * v
        beta_next = np.linalg.norm(p)
        # column k of T: (beta at row k-1, alpha at row k, beta_next at row k+1)
        eps_k = s_m2 * beta                        # after G_{k-2}: row k-2
        dbar = c_m2 * beta                         # row k-1 before G_{k-1}
        delta_k = c_m1 * dbar + s_m1 * alpha       # row k-1 after G_{k-1}
        gbar = -s_m1 * dbar + c_m1 * alpha         # row k after G_{k-1}
        gamma = math.hypot(gbar, beta_next)
        c_k, s_k = gbar / gamma, beta_next / gamma
        tau = c_k * phibar
        phibar = -s_k * phibar
        d = (v - delta_k * d_m1 - eps_k * d_m2) / gamma
        x = x + tau * d
        d_m2, d_m1 = d_m1, d
        c_m2, s_m2, c_m1, s_m1 = c_m1, s_m1, c_k, s_k
        if abs(phibar) <= tol * beta1 or beta_next == 0.0:
            break
        v_prev, v = v, p / beta_next
        beta = beta_next
    return x, k, abs(phibar) / beta1


def complex_symmetric_embed_matvec(A):
    """Real symmetric 2n operator [[A_r, A_i], [A_i, -A_r]] for a complex symmetric A = A_r + i A_i.
    Solving it for [y_r; -y_i] with right-hand side [c; 0] gives A y = c."""
    Ar, Ai = A.real, A.imag
    n = A.shape[0]

    def mv(u):
        return np.concatenate([Ar @ u[:n] + Ai @ u[n:], Ai @ u[:n] - Ar @ u[n:]])
    return mv


def residue_w_minres(eps, n_occ, B_ia, b, x, eta, tol=1e-10, maxit=1000):
    """W^c(x) = b^T delta with (1 - Pi(x)) delta = Pi(x) b, solved by MINRES on the real 2n
    embedding of the complex symmetric system; dW/dx = y^T Pi'(x) y with y = b + delta.
    Returns (W, dW, iterations, relative residual)."""
    Pi = pi_complex(eps, n_occ, B_ia, x, eta)
    dPi = dpi_complex(eps, n_occ, B_ia, x, eta)
    A = np.eye(Pi.shape[0]) - Pi
    rhs = Pi @ b
    n = b.shape[0]
    rr = np.concatenate([rhs.real, rhs.imag])
    # complex rhs c = c_r + i c_i: embedding rows give A_r y_r - A_i y_i = c_r and A_i y_r + A_r y_i = c_i,
    # i.e. [[A_r, A_i],[A_i, -A_r]] [y_r; -y_i] = [c_r; c_i]
    u, it, rel = minres(complex_symmetric_embed_matvec(A), rr, tol=tol, maxit=maxit)
    delta = u[:n] - 1j * u[n:]
    y = b + delta
    return b @ delta, y @ (dPi @ y), it, rel


# --------------------------------------------------------------------------
# Quasiparticle equation (Sec. 3.4, eq. "qpeqn", Fig. "steptree")
# --------------------------------------------------------------------------
def qp_linearised(e_n, shift, sigma_fn):
    """One Newton step of e_QP = e + shift + Re Sigma_c(e_QP) from omega = e:
    e_QP = e + Z (shift + Sigma_c(e)), Z = 1/(1 - dSigma_c/domega); shift = Sigma_x - V_xc."""
    s, ds = sigma_fn(e_n)
    Z = 1.0 / (1.0 - ds)
    return e_n + Z * (shift + s), Z


def _sign(v):
    return 1.0 if v > 0 else (-1.0 if v < 0 else 0.0)


def qp_steptree(e_n, shift, sigma_fn, tol=1e-8, maxit=50, cap=0.1):
    """Iterative QP solver with the step-selection tree of Fig. "steptree" (Sec. 3.4).

    f(w) = e_n + shift + Re Sigma_c(w) - w,  Z = -(df/dw)^-1 = 1/(1 - dSigma_c/dw).
    iter 0: scaled residual.  Later: Z >= 0.3 -> Newton (w += Z f); else bracketed -> golden
    section; else Z >= 0.1 -> scaled Newton (w += 0.7 Z f); else scaled residual.
    Scaled residual: w += c f with c = min(1, cap/|f|) (step at most ``cap`` Ha).
    Bracket: opened by a sign change of f between consecutive iterates ("sign" bracket), or by
    the same sign with growing |f| ("same" bracket, a skipped root).  A sign bracket [a, b] is
    narrowed by golden-section points taken from the end with the smaller |f|; a same-sign
    bracket runs a golden-section minimisation of |f| around its best point x, and turns into a
    sign bracket as soon as a sign change appears.  Converged when |f| < tol.
    Returns (omega, Z, status, n_evaluations, trace) with status 0 converged, 1 not converged."""
    omega = float(e_n)
    prev = None
    br = None
    trace = []
    Z = 1.0
    for k in range(maxit):
        s, ds = sigma_fn(omega)
        f = e_n + shift + s - omega
        Z = 1.0 / (1.0 - ds)
        trace.append((omega, f, Z))
        if abs(f) < tol:
            return omega, Z, 0, k + 1, trace
        br = _update_bracket(br, prev, (omega, f))
        if k == 0:
            kind = "residual"
        elif Z >= 0.3:
            kind = "newton"
        elif br is not None:
            kind = "golden"
        elif Z >= 0.1:
            kind = "scaled_newton"
        else:
            kind = "residual"
        if kind == "residual":
            step = min(1.0, cap / abs(f)) * f
            new = omega + step
        elif kind == "newton":
            new = omega + Z * f
        elif kind == "scaled_newton":
            new = omega + 0.7 * Z * f
        else:
            new = _golden_point(br)
        prev = (omega, f)
        omega = new
    return trace[-1][0], trace[-1][2], 1, maxit, trace


def _update_bracket(br, prev, cur):
    """Bracket bookkeeping for ``qp_steptree``; br = [kind, a, fa, b, fb, x, fx]."""
    w1, f1 = cur
    if br is not None and br[1] < w1 < br[3]:
        kind, a, fa, b, fb, x, fx = br
        if kind == "sign":
            if _sign(f1) == _sign(fa):
                a, fa = w1, f1
            else:
                b, fb = w1, f1
            return ["sign", a, fa, b, fb, None, None]
        # same-sign bracket: golden-section minimisation of |f| around x
        if _sign(f1) != _sign(fx):
            lo, hi = sorted([(w1, f1), (x, fx)])
            return ["sign", lo[0], lo[1], hi[0], hi[1], None, None]
        if abs(f1) < abs(fx):
            if w1 > x:
                a, fa = x, fx
            else:
                b, fb = x, fx
            x, fx = w1, f1
        else:
            if w1 > x:
                b, fb = w1, f1
            else:
                a, fa = w1, f1
        return ["same", a, fa, b, fb, x, fx]
    if prev is None:
        return br
    w0, f0 = prev
    if _sign(f1) != _sign(f0):
        lo, hi = sorted([(w0, f0), (w1, f1)])
        return ["sign", lo[0], lo[1], hi[0], hi[1], None, None]
    if br is None and abs(f1) > abs(f0):
        lo, hi = sorted([(w0, f0), (w1, f1)])
        return ["same", lo[0], lo[1], hi[0], hi[1], w0, f0]
    return br


def _golden_point(br):
    kind, a, fa, b, fb, x, fx = br
    if kind == "sign":
        return a + GOLD * (b - a) if abs(fa) <= abs(fb) else b - GOLD * (b - a)
    return x + GOLD * (b - x) if (b - x) >= (x - a) else x - GOLD * (x - a)


# --------------------------------------------------------------------------
# Driver: G0W0 QP energies of the targets (Algorithm 1 with maxeviter = 0)
# --------------------------------------------------------------------------
def g0w0_cd(eps, n_occ, B_ia, B_nm, targets, n_freq=128, x0=0.5, eta=1e-3, mode="steptree",
            vxc=None, qp_tol=1e-8, qp_maxit=50, static_subtraction=True, cluster_gap=0.0, window=0.5,
            n_window=64):
    """CD-G0W0 QP energies.  ``mode``: "linearised", "steptree" or "graphical" (window of +-``window`` Ha around
    the starting point, ``n_window`` points).  ``cluster_gap`` > 0 turns on the cluster layer of Sec. 3.4: targets
    within cluster_gap of each other in KS energy form a cluster; its first member is solved from its KS energy,
    the others start from their KS energy shifted by the first member's QP correction (if it converged).
    Returns dict with e_qp, Z, status, sigma_x, n_residue_solves, n_sigma (Sigma evaluations per target)."""
    xi, wt = mgl_grid(n_freq, x0)
    cd = CDSelfEnergy(eps, n_occ, B_ia, B_nm, targets, xi, wt, eta)
    nt = len(targets)
    e_qp, Zs, st, sx, nsig = [0.0] * nt, [1.0] * nt, [0] * nt, [0.0] * nt, [0] * nt
    groups = clusters([eps[n] for n in targets], cluster_gap) if cluster_gap > 0 else [[t] for t in range(nt)]
    for grp in groups:
        for k, t in enumerate(grp):
            n = targets[t]
            sxn = cd.sigma_x(t)
            shift = 0.0 if vxc is None else sxn - vxc[t]
            fn = lambda w, t=t: cd.sigma_c(t, w, static_subtraction)
            rep = grp[0]
            start = eps[n] + (e_qp[rep] - eps[targets[rep]]) if k > 0 and st[rep] == 0 else eps[n]
            if mode == "linearised":
                e, Z = qp_linearised(eps[n], shift, fn)
                s, ne = 0, 1
            elif mode == "graphical":
                e, Z, s, ne = qp_graphical(eps[n], shift, fn, start, window, n_window, tol=qp_tol, maxit=qp_maxit)
            else:
                e, Z, s, ne, _ = qp_steptree(start, eps[n] + shift - start, fn, tol=qp_tol, maxit=qp_maxit)
            e_qp[t], Zs[t], st[t], sx[t], nsig[t] = e, Z, s, sxn, ne
    return {"e_qp": np.array(e_qp), "Z": np.array(Zs), "status": np.array(st), "sigma_x": np.array(sx),
            "n_residue_solves": cd.n_residue_solves, "n_sigma": np.array(nsig), "cd": cd}


# --------------------------------------------------------------------------
# Open shell (spin-unrestricted, Sec. 2.2/3.3: the sum over sigma in Pi and spin-resolved Sigma)
# --------------------------------------------------------------------------
def pi_imag_uks(channels, xi):
    """Pi_PQ(i xi) = sum_sigma sum_{ia in sigma} B^s_P,ia [1/(i xi - D) + 1/(-i xi - D)] B^s_Q,ia
                  = -2 sum_sigma sum_ia B B D/(D^2 + xi^2).  channels = [(eps_sigma, n_occ_sigma, B_ia_sigma), ...]."""
    out = 0.0
    for eps, n_occ, B in channels:
        D = pair_energies(eps, n_occ)
        out = out + (B * (-2.0 * D / (D * D + xi * xi))) @ B.T
    return out


def pi_complex_uks(channels, z, eta):
    """Pi_PQ(z) = sum_sigma sum_ia B B [1/(z - D + i eta) + 1/(-z - D + i eta)] (one spin channel per term)."""
    out = 0.0
    for eps, n_occ, B in channels:
        D = pair_energies(eps, n_occ)
        c = 1.0 / (z - D + 1j * eta) + 1.0 / (-z - D + 1j * eta)
        out = out + (B * c) @ B.T
    return out


def dpi_complex_uks(channels, z, eta):
    out = 0.0
    for eps, n_occ, B in channels:
        D = pair_energies(eps, n_occ)
        c = -1.0 / (z - D + 1j * eta) ** 2 + 1.0 / (-z - D + 1j * eta) ** 2
        out = out + (B * c) @ B.T
    return out


class CDSelfEnergyUKS:
    """Sigma^c_nn,sigma(omega) by contour deformation for an open-shell system: W from the spin-summed Pi, G of the
    target's own spin (its energies and occupations), b_nm the target's rows.  ``targets`` = [(spin, n), ...],
    ``B_nm`` [n_t][n_bas][n_aux] rows of each target's spin."""

    def __init__(self, channels, B_nm, targets, xi, wt, eta=1e-3):
        self.ch = [(np.asarray(e, dtype=np.float64), int(o), B) for e, o, B in channels]
        self.B_nm = B_nm
        self.targets = list(targets)
        self.xi = np.asarray(xi, dtype=np.float64)
        self.wt = np.asarray(wt, dtype=np.float64)
        self.eta = float(eta)
        n_t, n_bas, _ = B_nm.shape
        self.W = np.empty((n_t, n_bas, len(self.xi)))
        self.W0 = np.empty((n_t, n_bas))
        for g, x in enumerate(self.xi):
            Pi = pi_imag_uks(self.ch, x)
            for t in range(n_t):
                self.W[t, :, g] = w_corr(Pi, B_nm[t].T)
        Pi0 = pi_imag_uks(self.ch, 0.0)
        for t in range(n_t):
            self.W0[t] = w_corr(Pi0, B_nm[t].T)

    def sigma_x(self, t):
        sp, _ = self.targets[t]
        return sigma_x(self.B_nm[t], self.ch[sp][1])

    def sigma_c(self, t, omega, static_subtraction=True):
        sp, _ = self.targets[t]
        eps, n_occ, _ = self.ch[sp]
        a = omega - eps
        xi2 = self.xi[None, :] ** 2
        a2 = a[:, None] ** 2
        Wg = self.W[t] - self.W0[t][:, None] if static_subtraction else self.W[t]
        I = np.sum(self.wt[None, :] * Wg * a[:, None] / (a2 + xi2)) / math.pi
        dI = np.sum(self.wt[None, :] * Wg * (xi2 - a2) / (a2 + xi2) ** 2) / math.pi
        if static_subtraction:
            I += np.sum(self.W0[t] * np.sign(a)) / 2.0
        R = dR = 0.0
        for m, sgn, th in residue_set(eps, n_occ, omega):
            x = eps[m] - omega
            w, dw = w_corr_and_deriv(pi_complex_uks(self.ch, x, self.eta), dpi_complex_uks(self.ch, x, self.eta),
                                     self.B_nm[t, m])
            R += sgn * th * w.real
            dR -= sgn * th * dw.real
        return R - I, dR - dI


def casida_uks(channels):
    """Casida form with two spin blocks: M = D^1/2 (D + 2K) D^1/2 over the pairs of both spins, K = B^T B with the
    spin blocks' B side by side (each spin channel carries its own factor 1 where the closed shell has 2).
    Returns Omega and V = sqrt(2) B D^1/2 T (W^c as in ``casida``)."""
    D = np.concatenate([pair_energies(e, o) for e, o, _ in channels])
    B = np.concatenate([b for _, _, b in channels], axis=1)
    K = B.T @ B
    sD = np.sqrt(D)
    M = sD[:, None] * (np.diag(D) + 2.0 * K) * sD[None, :]
    Om2, T = np.linalg.eigh(M)
    return np.sqrt(Om2), (math.sqrt(2.0) * B * sD[None, :]) @ T


# --------------------------------------------------------------------------
# Graphical solution and cluster guesses (Sec. 3.4)
# --------------------------------------------------------------------------
def qp_graphical(e_n, shift, sigma_fn, center, half_width=0.5, n_pts=64, tol=1e-8, maxit=50):
    """Graphical solution of e_QP = e_n + shift + Re Sigma_c(e_QP) (Sec. 3.4): f(w) = e_n + shift + Sigma_c(w) - w
    on n_pts evenly spaced points of [center - half_width, center + half_width]; every sign change of f between
    neighbouring points with f decreasing across it (a root of the QP equation, not a pole of Sigma, where f jumps
    upwards) is a candidate, located by linear interpolation; the candidate closest to ``center`` is refined by the
    step tree started there.  Returns (omega, Z, status, n_grid_evaluations) with status 0 converged, 1 step tree
    not converged, 3 no root in the window."""
    ws = center + half_width * np.linspace(-1.0, 1.0, n_pts)
    fs = np.array([e_n + shift + sigma_fn(w)[0] - w for w in ws])
    best = None
    for k in range(n_pts - 1):
        f0, f1 = fs[k], fs[k + 1]
        if f0 > 0.0 >= f1 or (f0 == 0.0 and f1 < 0.0):
            r = ws[k] + (ws[k + 1] - ws[k]) * f0 / (f0 - f1)
            if best is None or abs(r - center) < abs(best - center):
                best = r
    if best is None:
        return center, float("nan"), 3, n_pts
    w, Z, st, n, _ = qp_steptree(best, e_n + shift - best, sigma_fn, tol=tol, maxit=maxit)
    return w, Z, st, n_pts + n


def clusters(eps_t, gap):
    """Targets grouped by KS energy (Sec. 3.4, cluster layer): sorted energies split wherever two neighbours are
    more than ``gap`` apart.  Returns lists of positions into eps_t; each cluster's representative is its first
    member in energy order."""
    order = sorted(range(len(eps_t)), key=lambda t: eps_t[t])
    out = []
    for t in order:
        if out and eps_t[t] - eps_t[out[-1][-1]] <= gap:
            out[-1].append(t)
        else:
            out.append([t])
    return out


# --------------------------------------------------------------------------
# Eigenvalue self-consistency (Algorithm 1, outer loop over iter; Sec. 1 evGW0 / evGW)
# --------------------------------------------------------------------------
def scissor_energies(eps_ks, n_occ, targets, e_qp):
    """Energies for the next cycle: the targets take their QP energies; every other occupied state moves by the
    QP correction of the highest occupied target, every other virtual state by that of the lowest virtual
    target (no shift where a class has no target)."""
    eps_ks = np.asarray(eps_ks, dtype=np.float64)
    out = eps_ks.copy()
    occ = [(eps_ks[n], e - eps_ks[n]) for n, e in zip(targets, e_qp) if n < n_occ]
    vir = [(eps_ks[n], e - eps_ks[n]) for n, e in zip(targets, e_qp) if n >= n_occ]
    d_occ = max(occ)[1] if occ else 0.0
    d_vir = min(vir)[1] if vir else 0.0
    out[:n_occ] += d_occ
    out[n_occ:] += d_vir
    for n, e in zip(targets, e_qp):
        out[n] = e
    return out


def evgw(eps, n_occ, B_ia, B_nm, targets, update_w=False, mode="steptree", max_iter=30, tol=1e-6, n_freq=128,
         x0=0.5, eta=1e-3, qp_tol=1e-8, qp_maxit=50, static_subtraction=True):
    """Eigenvalue self-consistent GW: each cycle of Algorithm 1's outer loop solves the QP equations
    e_QP = e_KS + Re Sigma_c[G, W](e_QP) (V_xc := Sigma_x) with G built from the current energies (evGW0) and, if
    ``update_w``, W built from them too (evGW); the energies are then updated (``scissor_energies``).  Cycle 0 is
    G0W0.  The QP search of each cycle starts from the previous cycle's energy: one Newton step (linearised) or the
    step tree.  Stops when no target moves by more than ``tol``.  Returns dict e_qp, Z, status, iterations."""
    eps_ks = np.asarray(eps, dtype=np.float64)
    xi, wt = mgl_grid(n_freq, x0)
    cur = eps_ks.copy()
    e_prev = np.array([eps_ks[n] for n in targets])
    e_qp, Zs, st = e_prev.copy(), np.ones(len(targets)), np.zeros(len(targets), dtype=int)
    it = 0
    for it in range(1, max_iter + 1):
        cd = CDSelfEnergy(cur if update_w else eps_ks, n_occ, B_ia, B_nm, targets, xi, wt, eta, eps_g=cur)
        e_new, Zs, st = [], [], []
        for t, n in enumerate(targets):
            fn = lambda w, t=t: cd.sigma_c(t, w, static_subtraction)
            if mode == "linearised":
                w0 = e_prev[t]
                sg, dsg = fn(w0)
                Z = 1.0 / (1.0 - dsg)
                e, s = w0 + Z * (eps_ks[n] + sg - w0), 0
            else:
                e, Z, s = _qp_steptree_from(eps_ks[n], e_prev[t], fn, qp_tol, qp_maxit)
            e_new.append(e)
            Zs.append(Z)
            st.append(s)
        e_new = np.array(e_new)
        delta = np.max(np.abs(e_new - e_prev))
        e_qp, e_prev = e_new, e_new
        cur = scissor_energies(eps_ks, n_occ, targets, e_qp)
        if delta < tol:
            break
    return {"e_qp": e_qp, "Z": np.array(Zs), "status": np.array(st), "iterations": it,
            "converged": bool(delta < tol), "eps_final": cur}


def _qp_steptree_from(e_ks, w0, sigma_fn, tol, maxit):
    """The step tree of ``qp_steptree`` for f(w) = e_ks + Sigma_c(w) - w, started at w0 instead of e_ks."""
    shifted = lambda w: sigma_fn(w)
    # qp_steptree starts at its first argument and solves e + shift + Sigma(w) - w = 0: start at w0 with
    # shift = e_ks - w0 so that the equation is unchanged
    w, Z, st, n, trace = qp_steptree(w0, e_ks - w0, shifted, tol=tol, maxit=maxit)
    return w, Z, st


def g0w0_sd(eps, n_occ, B_ia, B_nm, targets, eta=0.0, mode="steptree", vxc=None, qp_tol=1e-8, qp_maxit=50):
    """SD-G0W0 QP energies from the Casida spectral sum (same QP solvers as the CD route)."""
    Omega, V = casida(eps, n_occ, B_ia)
    e_qp, Zs, st = [], [], []
    for t, n in enumerate(targets):
        sxn = sigma_x(B_nm[t], n_occ)
        shift = 0.0 if vxc is None else sxn - vxc[t]
        fn = lambda w, t=t: sigma_c_sd(eps, n_occ, B_nm[t], Omega, V, w, eta)
        if mode == "linearised":
            e, Z = qp_linearised(eps[n], shift, fn)
            s = 0
        else:
            e, Z, s, _, _ = qp_steptree(eps[n], shift, fn, tol=qp_tol, maxit=qp_maxit)
        e_qp.append(e)
        Zs.append(Z)
        st.append(s)
    return {"e_qp": np.array(e_qp), "Z": np.array(Zs), "status": np.array(st), "Omega": Omega}
