"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, a second independent route, invariants, library routines)."""
import math

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth


# ---------------------------------------------------------------- generator
def test_philox_known_answers():
    # Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11, Random123 distribution).
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert synth.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == [0x408f276d, 0x41c83b0e, 0xa20bc7c6,
                                                                        0x6d5451fd]
    assert synth.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_synth_slices_agree_and_statistics():
    s = synth.water_cluster(2, 7, targets=[0, 3, 9, 10, 20])
    B = s.b_ia()
    Bn = s.b_nm()
    nv = s.n_virt
    for t, n in enumerate(s.targets):
        if n < s.n_occ:
            np.testing.assert_array_equal(Bn[t, s.n_occ:, :].T, B[:, n * nv:(n + 1) * nv])
    # B_{P,pq} = B_{P,qp}: target 3 row m=9 equals target 9 row m=3
    np.testing.assert_array_equal(Bn[1, 9], Bn[2, 3])
    big = synth.water_cluster(4, 3).b_ia()
    assert abs(big.mean()) < 3e-3 * s.sigma_b * 10
    assert abs(big.std() / (0.6 / math.sqrt(504)) - 1) < 0.01


# ---------------------------------------------------------------- grid
def test_grid_nodes_are_mapped_gauss_legendre():
    xi, w = O.mgl_grid(64, 0.7)
    t, wgl = np.polynomial.legendre.leggauss(64)
    # inverse map t = (xi - x0)/(xi + x0) recovers the Legendre nodes
    np.testing.assert_allclose((xi - 0.7) / (xi + 0.7), t, atol=1e-14)
    assert np.all(np.diff(xi) > 0) and np.all(w > 0)


@pytest.mark.parametrize("n", [32, 128, 200])
def test_grid_lorentzian_identity(n):
    # int_0^inf x0/(x0^2 + xi^2) dxi = pi/2 exactly (the map sends it to int_-1^1 dt/(1+t^2))
    xi, w = O.mgl_grid(n, 0.5)
    assert abs(np.sum(w * 0.5 / (0.25 + xi ** 2)) - math.pi / 2) < 1e-14


def test_grid_other_integrals():
    xi, w = O.mgl_grid(128, 0.5)
    assert abs(np.sum(w * np.exp(-xi)) - 1.0) < 1e-10
    assert abs(np.sum(w / (1 + xi ** 2) ** 2) - math.pi / 4) < 1e-12
    for a in [0.05, 0.3, 2.0, 20.0]:
        assert abs(np.sum(w * a / (a * a + xi ** 2)) - math.pi / 2) < 1e-7


# ---------------------------------------------------------------- pole model (closed form)
def _pole_model(e_i=-0.6, e_a=0.4, b=0.35, b_ii=0.8, b_aa=0.55):
    eps = np.array([e_i, e_a])
    B_ia = np.array([[b]])
    B_nm = np.array([[[b_ii], [b]], [[b], [b_aa]]])          # targets 0 (HOMO), 1 (LUMO)
    D = e_a - e_i
    Om = math.sqrt(D * (D + 4 * b * b))
    return eps, B_ia, B_nm, D, Om, (b, b_ii, b_aa)


def _pole_sigma(omega, t, eps, D, Om, bs):
    b, b_ii, b_aa = bs
    pref = 2 * b * b * D / Om
    ni, na = (b_ii, b) if t == 0 else (b, b_aa)
    s = pref * (ni ** 2 / (omega - eps[0] + Om) + na ** 2 / (omega - eps[1] - Om))
    ds = -pref * (ni ** 2 / (omega - eps[0] + Om) ** 2 + na ** 2 / (omega - eps[1] - Om) ** 2)
    return s, ds


def test_pole_model_pi_and_w():
    eps, B_ia, B_nm, D, Om, (b, b_ii, b_aa) = _pole_model()
    for xi in [0.0, 0.1, 1.0, 7.0]:
        Pi = O.pi_imag(eps, 1, B_ia, xi)
        assert abs(Pi[0, 0] + 4 * b * b * D / (D * D + xi * xi)) < 1e-15
        for bn in [b_ii, b, b_aa]:
            w = O.w_corr(Pi, np.array([bn]))
            assert abs(w - bn * bn * 4 * b * b * D / (-xi * xi - Om * Om)) < 1e-14
    # real axis, eta = 0, away from the pole: W = B^2 4 b^2 D/(x^2 - Om^2)
    for x in [0.2, -0.5, 1.9, 3.0]:
        Pi = O.pi_complex(eps, 1, B_ia, x, 0.0)
        w = O.w_corr(Pi, np.array([b_ii]))
        assert abs(w - b_ii ** 2 * 4 * b * b * D / (x * x - Om * Om)) < 1e-13


def test_pole_model_sigma_cd_and_sd():
    eps, B_ia, B_nm, D, Om, bs = _pole_model()
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(eps, 1, B_ia, B_nm, [0, 1], xi, wt, eta=0.0)
    Omega, V = O.casida(eps, 1, B_ia)
    assert abs(Omega[0] - Om) < 1e-14
    for t in (0, 1):
        assert abs(cd.sigma_x(t) - (-(bs[1] ** 2) if t == 0 else -(bs[0] ** 2))) < 1e-15
        for w in [-1.7, -0.9, -0.6, -0.3, 0.0, 0.4, 0.9, 2.5]:
            s_ref, ds_ref = _pole_sigma(w, t, eps, D, Om, bs)
            s_sd, ds_sd = O.sigma_c_sd(eps, 1, B_nm[t], Omega, V, w, 0.0)
            s_cd, ds_cd = cd.sigma_c(t, w)
            assert abs(s_sd - s_ref) < 1e-13 and abs(ds_sd - ds_ref) < 1e-12
            assert abs(s_cd - s_ref) < 1e-9, (t, w, s_cd, s_ref)
            assert abs(ds_cd - ds_ref) < 1e-7, (t, w, ds_cd, ds_ref)


def test_static_subtraction_matters_only_near_poles():
    eps, B_ia, B_nm, D, Om, bs = _pole_model()
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(eps, 1, B_ia, B_nm, [0, 1], xi, wt, eta=0.0)
    s_ref, _ = _pole_sigma(-0.6 - 1e-6, 0, eps, D, Om, bs)
    s_sub, _ = cd.sigma_c(0, -0.6 - 1e-6, static_subtraction=True)
    s_lit, _ = cd.sigma_c(0, -0.6 - 1e-6, static_subtraction=False)
    assert abs(s_sub - s_ref) < 1e-8
    assert abs(s_lit - s_ref) > 1e-3          # the literal quadrature misses the Lorentzian jump


# ---------------------------------------------------------------- SD <-> CD (two routes to one Sigma)
def test_sd_vs_cd_single_water():
    s = synth.workload(0)
    B, Bn = s.b_ia(), s.b_nm()
    cd = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=0.0, mode="linearised")
    sd = O.g0w0_sd(s.eps, s.n_occ, B, Bn, s.targets, eta=0.0, mode="linearised")
    np.testing.assert_allclose(cd["e_qp"], sd["e_qp"], atol=1e-8, rtol=0)
    cdt = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=0.0)
    sdt = O.g0w0_sd(s.eps, s.n_occ, B, Bn, s.targets, eta=0.0)
    np.testing.assert_allclose(cdt["e_qp"], sdt["e_qp"], atol=1e-8, rtol=0)
    assert np.all(cdt["status"] == 0)
    Omega, V = O.casida(s.eps, s.n_occ, B)
    c = cd["cd"]
    for w in np.linspace(-1.6, 0.6, 23):
        a = c.sigma_c(0, w)
        b = O.sigma_c_sd(s.eps, s.n_occ, Bn[0], Omega, V, w, 0.0)
        assert abs(a[0] - b[0]) < 1e-8 and abs(a[1] - b[1]) < 1e-6


@pytest.mark.parametrize("seed", range(6))
def test_sd_vs_cd_tiny_random(seed):
    rng = np.random.default_rng(100 + seed)
    n_occ, n_virt, n_aux = rng.integers(1, 4), rng.integers(2, 5), rng.integers(3, 7)
    occ = np.sort(rng.uniform(-2.0, -0.3, n_occ))
    vir = np.sort(rng.uniform(0.1, 3.0, n_virt))
    eps = np.concatenate([occ, vir])
    n_bas = len(eps)
    Bfull = rng.normal(0, 0.3, (n_aux, n_bas, n_bas))
    Bfull = 0.5 * (Bfull + Bfull.transpose(0, 2, 1))
    B_ia = Bfull[:, :n_occ, n_occ:].reshape(n_aux, -1)
    targets = list(range(n_bas))
    B_nm = np.stack([Bfull[:, n, :].T for n in targets])
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(eps, n_occ, B_ia, B_nm, targets, xi, wt, eta=0.0)
    Omega, V = O.casida(eps, n_occ, B_ia)
    for t in targets:
        for w in [eps[t], eps[t] - 0.07, eps[t] + 0.11]:
            a = cd.sigma_c(t, w)
            b = O.sigma_c_sd(eps, n_occ, B_nm[t], Omega, V, w, 0.0)
            assert abs(a[0] - b[0]) < 1e-8, (t, w, a, b)


def test_casida_hermitian_vs_full():
    s = synth.workload(0)
    B = s.b_ia()
    Omega, _ = O.casida(s.eps, s.n_occ, B)
    full = O.casida_full_omegas(s.eps, s.n_occ, B)
    np.testing.assert_allclose(np.sort(full), Omega, rtol=1e-10)
    D = O.pair_energies(s.eps, s.n_occ)
    assert Omega.min() >= D.min() - 1e-12          # RPA: Omega_s >= min D


# ---------------------------------------------------------------- invariants
def test_pi_invariants_and_w_sign():
    s = synth.water_cluster(1, 11)
    B, Bn = s.b_ia(), s.b_nm()
    prev = None
    for xi in [0.0, 0.05, 0.3, 1.0, 5.0, 40.0]:
        Pi = O.pi_imag(s.eps, s.n_occ, B, xi)
        assert np.abs(Pi - Pi.T).max() <= 1e-15 * np.abs(Pi).max()
        ev = np.linalg.eigvalsh(Pi)
        assert ev.max() <= 1e-12 * np.abs(ev).max()
        assert np.linalg.eigvalsh(np.eye(len(Pi)) - Pi).min() >= 1.0 - 1e-12
        np.testing.assert_allclose(O.pi_complex(s.eps, s.n_occ, B, 1j * xi, 0.0).real, Pi, atol=1e-13)
        W = O.w_corr(Pi, Bn[0].T)
        assert np.all(W <= 1e-15)
        if prev is not None:
            assert np.all(W >= prev - 1e-15)          # W^c(i xi) rises towards 0
        prev = W


def test_w_imag_matches_spectral_route():
    s = synth.workload(0)
    B, Bn = s.b_ia(), s.b_nm()
    Omega, V = O.casida(s.eps, s.n_occ, B)
    for xi in [0.0, 0.2, 1.5]:
        Pi = O.pi_imag(s.eps, s.n_occ, B, xi)
        for m in range(0, s.n_bas, 5):
            a = O.w_corr(Pi, Bn[1, m])
            b = O.w_corr_sd(Omega, V, Bn[1, m], 1j * xi)
            assert abs(a - b.real) < 1e-11 * max(1, abs(a))


def test_residue_derivative_matches_finite_difference():
    s = synth.water_cluster(1, 5)
    B, Bn = s.b_ia(), s.b_nm()
    b = Bn[0, 3]
    for x in [0.13, 0.71, 1.37]:
        def cd(h):   # central difference
            Wp = O.w_corr(O.pi_complex(s.eps, s.n_occ, B, x + h, 1e-3), b)
            Wm = O.w_corr(O.pi_complex(s.eps, s.n_occ, B, x - h, 1e-3), b)
            return (Wp - Wm) / (2 * h)
        _, dW = O.w_corr_and_deriv(O.pi_complex(s.eps, s.n_occ, B, x, 1e-3),
                                   O.dpi_complex(s.eps, s.n_occ, B, x, 1e-3), b)
        fd = (4 * cd(5e-6) - cd(1e-5)) / 3      # Richardson extrapolation, O(h^4)
        assert abs(fd - dW) < 1e-6 * max(1, abs(dW))


# ---------------------------------------------------------------- MINRES
def test_minres_matches_dense_and_scipy():
    import scipy.sparse.linalg as sla
    rng = np.random.default_rng(3)
    n = 60
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    for evs in [rng.uniform(0.5, 3, n), np.concatenate([rng.uniform(-3, -0.2, n // 2), rng.uniform(0.2, 3, n // 2)])]:
        A = (Q * evs) @ Q.T
        A = 0.5 * (A + A.T)
        b = rng.normal(size=n)
        x, it, rel = O.minres(lambda v: A @ v, b, tol=1e-12, maxit=500)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-9)
        assert rel <= 1e-12 and np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
        # fixed iteration count: same iterate as scipy's MINRES (same Krylov minimiser)
        x5, _, _ = O.minres(lambda v: A @ v, b, tol=0.0, maxit=5)
        xs, _ = sla.minres(A, b, rtol=1e-30, maxiter=5)
        np.testing.assert_allclose(x5, xs, atol=1e-10)


def test_minres_residue_matches_dense_solve():
    s = synth.water_cluster(1, 5)
    B, Bn = s.b_ia(), s.b_nm()
    b = Bn[1, 2]
    for x in [0.05, 0.6, 1.2]:
        Wd, dWd = O.w_corr_and_deriv(O.pi_complex(s.eps, s.n_occ, B, x, 1e-3),
                                     O.dpi_complex(s.eps, s.n_occ, B, x, 1e-3), b)
        Wm, dWm, it, rel = O.residue_w_minres(s.eps, s.n_occ, B, b, x, 1e-3, tol=1e-12, maxit=2000)
        assert rel <= 1e-12
        assert abs(Wm - Wd) < 1e-10 and abs(dWm - dWd) < 1e-8 * max(1, abs(dWd))


# ---------------------------------------------------------------- QP solvers
def test_linearised_is_exact_for_linear_sigma():
    e, alpha, beta = -0.5, -0.2, -0.4
    eq, Z = O.qp_linearised(e, 0.0, lambda w: (alpha + beta * w, beta))
    assert abs(eq - (e + alpha) / (1 - beta)) < 1e-15 and abs(Z - 1 / (1 - beta)) < 1e-15


def test_steptree_finds_roots_of_pole_model():
    from scipy.optimize import brentq
    eps, B_ia, B_nm, D, Om, bs = _pole_model()
    for t in (0, 1):
        fn = lambda w: _pole_sigma(w, t, eps, D, Om, bs)
        w, Z, st, n, trace = O.qp_steptree(eps[t], 0.0, fn, tol=1e-12)
        assert st == 0
        f = lambda w: eps[t] + fn(w)[0] - w
        assert abs(f(w)) < 1e-12
        assert abs(trace[1][0] - trace[0][0]) <= 0.1 + 1e-15     # first step is a capped scaled residual
        # the root is the one brentq finds in a small bracket around it
        r = brentq(f, w - 1e-3, w + 1e-3, xtol=1e-15)
        assert abs(r - w) < 1e-11


def test_steptree_uses_golden_section_when_z_small():
    # Sigma with a strong pole next to the root: Z < 0.3 near the root, sign-change bracket.
    p, A = -0.52, 0.004
    fn = lambda w: (A / (w - p), -A / (w - p) ** 2)
    e = -0.5
    w, Z, st, n, trace = O.qp_steptree(e, 0.0, fn, tol=1e-10, maxit=200)
    f = lambda w: e + A / (w - p) - w
    assert st == 0 and abs(f(w)) < 1e-10


# ---------------------------------------------------------------- real-axis W at finite eta
def _pair_space_w(eps, n_occ, B, b, x, eta):
    """W^c_eta(x) and dW/dx by a route that never forms Pi: the two pole terms of Pi(x) (Sec. 3.3) combine to
    1/(x - D + i eta) + 1/(-x - D + i eta) = -2 Dt/(Dt^2 - x^2) with the complex pair energy Dt = D - i eta, so
    Pi_eta(x) = -C (Dt^2 - x^2)^-1 C^T with C = 2 B Dt^(1/2).  The Woodbury identity then gives
    W^c = b^T[(1 - Pi)^-1 - 1]b = -u^T (M - x^2)^-1 u with u = C^T b and M = Dt^(1/2)(Dt + 4K)Dt^(1/2), the
    Casida matrix of Sec. 3.2 with K = B^T B, here complex symmetric; dW/dx = -2x v^T v with v = (M - x^2)^-1 u."""
    D = O.pair_energies(eps, n_occ)
    Dt = D - 1j * eta
    sD = np.sqrt(Dt)
    K = B.T @ B
    M = sD[:, None] * (np.diag(Dt) + 4.0 * K) * sD[None, :]
    u = 2.0 * sD * (B.T @ b)
    v = np.linalg.solve(M - x * x * np.eye(len(D)), u)
    return -(u @ v), -2.0 * x * (v @ v)


@pytest.mark.parametrize("seed", [None, 1, 2])
def test_residue_w_at_finite_eta_matches_pair_space_route(seed):
    """Pins pi_complex, dpi_complex and residue_w at eta != 0 (the placement and factor of i eta in both pole
    terms): the N_aux-dimensional dense solve against the N_ov-dimensional Casida form, including frequencies
    within a few eta of a pair energy, where a wrong eta factor or placement changes W at first order."""
    if seed is None:
        s = synth.workload(0)
        B, Bn = s.b_ia(), s.b_nm()
        eps, n_occ, rows = s.eps, s.n_occ, [Bn[1, 3], Bn[0, 10]]
    else:
        rng = np.random.default_rng(seed)
        n_occ, n_virt, n_aux = 2, 4, 5
        eps = np.sort(np.concatenate([rng.uniform(-1.5, -0.3, n_occ), rng.uniform(0.1, 2.0, n_virt)]))
        B = rng.normal(0, 0.3, (n_aux, n_occ * n_virt))
        rows = [rng.normal(0, 0.3, n_aux) for _ in range(2)]
    D = O.pair_energies(eps, n_occ)
    xs = [0.0, 0.31, -0.7, D.min() + 0.002, D.max() - 0.004, -D[len(D) // 2] + 0.001, 1.93]
    for eta in (1e-3, 1e-2, 0.07):
        for x in xs:
            for b in rows:
                cd = O.CDSelfEnergy.__new__(O.CDSelfEnergy)        # residue_w only needs these fields
                cd.eps, cd.n_occ, cd.B_ia, cd.eta, cd.n_residue_solves = eps, n_occ, B, eta, 0
                cd.B_nm = b[None, None, :]
                w, dw = cd.residue_w(0, 0, x)
                wr, dwr = _pair_space_w(eps, n_occ, B, b, x, eta)
                # both routes are FP64 LU solves; near a resonance their condition number grows like 1/eta
                assert abs(w - wr) < 1e-9 * max(1.0, abs(wr)), (eta, x, w, wr)
                assert abs(dw - dwr) < 1e-8 * max(1.0, abs(dwr)), (eta, x, dw, dwr)


def test_pi_complex_properties_at_finite_eta():
    """Consequences of the paper's Pi(x) that hold for any eta: even in x, complex symmetric, -Im Pi positive
    semidefinite, and at an isolated resonance x = D_k, eta Im Pi -> -2 B_k B_k^T as eta -> 0 (the closed-shell
    factor 2 over a unit-residue pole term)."""
    rng = np.random.default_rng(4)
    n_occ, n_virt, n_aux = 2, 3, 4
    eps = np.sort(np.concatenate([[-1.1, -0.6], [0.2, 0.9, 1.7]]))
    B = rng.normal(0, 0.4, (n_aux, n_occ * n_virt))
    eta = 0.05
    for x in (0.0, 0.4, 1.3, 2.6):
        P = O.pi_complex(eps, n_occ, B, x, eta)
        np.testing.assert_allclose(P, O.pi_complex(eps, n_occ, B, -x, eta), atol=1e-14)
        np.testing.assert_allclose(P, P.T, atol=1e-14)
        assert np.linalg.eigvalsh(-P.imag).min() > -1e-13
    # isolated resonance: the lowest pair energy is well separated from the others
    D = O.pair_energies(eps, n_occ)
    k = int(np.argmin(D))
    for e in (1e-4, 1e-6):
        P = O.pi_complex(eps, n_occ, B, D[k], e)
        np.testing.assert_allclose(e * P.imag, -2.0 * np.outer(B[:, k], B[:, k]), atol=50 * e)


# ---------------------------------------------------------------- step tree, worked by hand
# Each case uses a Sigma whose f(w) = e + Sigma(w) - w and Z = 1/(1 - Sigma'(w)) are simple enough to follow
# Fig. "steptree" (Sec. 3.4) by hand; the expected iterates below are those hand computations, written with the
# golden fraction G = (3 - sqrt 5)/2.
G = (3.0 - math.sqrt(5.0)) / 2.0


def _iterates(sigma, e=0.0, maxit=50, tol=1e-8):
    w, Z, st, n, trace = O.qp_steptree(e, 0.0, sigma, tol=tol, maxit=maxit)
    return [t[0] for t in trace], [t[1] for t in trace], st, Z


def test_steptree_capped_residual_then_newton():
    # Sigma = 0.5 - w: f = 0.5 - 2w, Z = 1/2.  Iteration 0: residual step capped at 0.1 (|f| = 0.5);
    # iteration 1: Z >= 0.3, Newton w += Z f = 0.1 + 0.15 lands on the root 0.25.
    ws, fs, st, Z = _iterates(lambda w: (0.5 - w, -1.0))
    assert st == 0 and Z == 0.5
    np.testing.assert_allclose(ws, [0.0, 0.1, 0.25], atol=1e-15)
    np.testing.assert_allclose(fs, [0.5, 0.3, 0.0], atol=1e-15)


def test_steptree_scaled_newton_without_bracket():
    # Sigma = 1 - 4w: f = 1 - 5w, Z = 0.2 (below 0.3, at least 0.1).  Iteration 0: capped step 0.1 (f = 1 -> 0.5,
    # same sign, |f| shrinks: no bracket).  Then w += 0.7 Z f = 0.14 f each time, so f_{k+1} = (1 - 5*0.14) f_k
    # = 0.3 f_k: w = 0.1, 0.17, 0.191, 0.1973, ...
    ws, fs, st, Z = _iterates(lambda w: (1.0 - 4.0 * w, -4.0))
    assert st == 0 and abs(Z - 0.2) < 1e-15
    np.testing.assert_allclose(ws[:5], [0.0, 0.1, 0.17, 0.191, 0.1973], atol=1e-14)
    for k in range(1, len(fs) - 1):
        assert abs(fs[k + 1] - 0.3 * fs[k]) < 1e-14
    assert len(ws) == 17 and abs(fs[-1]) < 1e-8 <= abs(fs[-2])     # f_16 = 0.5 * 0.3^15 < 1e-8 <= f_15


def test_steptree_residual_steps_then_golden_in_sign_bracket():
    # Sigma = 5 - 19w: f = 5 - 20w, Z = 0.05 (below 0.1).  Capped residual steps of 0.1 (f = 5, 3, 1, -1); the sign
    # change between w = 0.2 and 0.3 opens the bracket [0.2, 0.3] with f = 1 and -1.  Bracketed and Z < 0.3:
    # golden points from the end with the smaller |f| (the lower end on a tie):
    #   0.2 + 0.1 G (f = 1 - 2G > 0: replaces the lower end), then
    #   a + G (0.3 - a) with a = 0.2 + 0.1 G (f < 0: replaces the upper end), ...
    ws, fs, st, Z = _iterates(lambda w: (5.0 - 19.0 * w, -19.0), maxit=8)
    w4 = 0.2 + 0.1 * G
    w5 = w4 + G * (0.3 - w4)
    np.testing.assert_allclose(ws[:6], [0.0, 0.1, 0.2, 0.3, w4, w5], atol=1e-14)
    np.testing.assert_allclose(fs[:4], [5.0, 3.0, 1.0, -1.0], atol=1e-13)
    assert fs[4] > 0 > fs[5]
    # at w5 both ends have |f| = 20 |w - 0.25| equal by the golden symmetry: the lower end wins the tie
    w6 = w4 + G * (w5 - w4)
    assert abs(ws[6] - w6) < 1e-14 and st == 1


def test_steptree_same_sign_bracket_turns_into_sign_bracket():
    # f = -0.01 + 4|w - 0.04| (roots 0.0375 and 0.0425): Sigma' = -3 left of 0.04 (Z = 0.25), +5 right of it
    # (Z = -0.25); Z < 0.3 everywhere, so Newton never runs.  Iteration 0: capped step 0.1 from f = 0.15 to 0.23:
    # same sign and growing |f| -> "same" bracket [0, 0.1] around x = 0.  Golden point x + G (b - x) = 0.1 G has
    # f = -0.01 + 4 (0.04 - 0.1 G) < 0: the bracket becomes a sign bracket [0, 0.1 G] with f(0) = 0.15; then
    # golden from the end with the smaller |f| (the upper one): b - G (b - a) = 0.1 G (1 - G).
    def sig(w):
        f = -0.01 + 4.0 * abs(w - 0.04)
        return f + w, (-3.0 if w < 0.04 else 5.0)
    ws, fs, st, Z = _iterates(sig, maxit=6)
    np.testing.assert_allclose(ws[:4], [0.0, 0.1, 0.1 * G, 0.1 * G * (1.0 - G)], atol=1e-15)
    np.testing.assert_allclose(fs[:2], [0.15, 0.23], atol=1e-15)
    assert fs[2] < 0 < fs[3]


# ---------------------------------------------------------------- eigenvalue self-consistency (Algorithm 1 outer loop)
@pytest.mark.parametrize("update_w", [False, True])
def test_evgw_reaches_the_pole_model_fixed_point(update_w):
    """On the one-pair pole model every state is a target, so the converged energies (e_i*, e_a*) must solve the
    closed-form QP equations e* = e_KS + Sigma_c(e*) with G's poles at (e_i*, e_a*) and W's pair energy the KS one
    (evGW0) or D* = e_a* - e_i* with Omega* = sqrt(D* (D* + 4 b^2)) (evGW)."""
    eps, B_ia, B_nm, D, Om, bs = _pole_model()
    r = O.evgw(eps, 1, B_ia, B_nm, [0, 1], update_w=update_w, mode="steptree", tol=1e-12, qp_tol=1e-13,
               max_iter=200, eta=0.0)
    assert r["converged"] and np.all(r["status"] == 0)
    e = r["e_qp"]
    Dw = (e[1] - e[0]) if update_w else D
    Omw = math.sqrt(Dw * (Dw + 4 * bs[0] ** 2))
    for t in (0, 1):
        s, _ = _pole_sigma(e[t], t, e, Dw, Omw, bs)
        assert abs(eps[t] + s - e[t]) < 1e-9, (t, eps[t] + s - e[t])
    # and the loop moved the energies away from the one-shot G0W0 result
    g0 = O.g0w0_cd(eps, 1, B_ia, B_nm, [0, 1], eta=0.0, qp_tol=1e-13)
    assert np.max(np.abs(e - g0["e_qp"])) > 1e-4


def test_scissor_energies():
    eps = np.array([-10.0, -1.0, -0.5, 0.2, 0.9, 3.0])
    out = O.scissor_energies(eps, 3, [1, 2, 3], [-1.2, -0.8, 0.5])
    np.testing.assert_allclose(out, [-10.3, -1.2, -0.8, 0.5, 1.2, 3.3], atol=1e-15)
    out = O.scissor_energies(eps, 3, [4], [1.0])
    np.testing.assert_allclose(out, [-10.0, -1.0, -0.5, 0.3, 1.0, 3.1], atol=1e-15)


# ---------------------------------------------------------------- graphical solver and cluster guesses (Sec. 3.4)
def test_graphical_solver_finds_the_nearest_root_of_the_pole_model():
    """f(w) = e + Sigma_c(w) - w on the one-pair pole model is a rational function: e + A/(w - p1) + B/(w - p2) - w
    with p1 = e_i - Omega, p2 = e_a + Omega.  Its roots are those of a cubic (numpy.roots); the graphical solver
    must return the root with f' < 0 closest to the window centre."""
    eps, B_ia, B_nm, D, Om, bs = _pole_model()
    b, b_ii, b_aa = bs
    pref = 2 * b * b * D / Om
    for t in (0, 1):
        ni, na = (b_ii, b) if t == 0 else (b, b_aa)
        A, Bc = pref * ni ** 2, pref * na ** 2
        p1, p2 = eps[0] - Om, eps[1] + Om
        e = eps[t]
        # (e - w)(w - p1)(w - p2) + A (w - p2) + B (w - p1) = 0
        poly = np.polymul(np.polymul([-1.0, e], [1.0, -p1]), [1.0, -p2])
        poly = np.polyadd(poly, np.polyadd(A * np.array([1.0, -p2]), Bc * np.array([1.0, -p1])))
        fn = lambda w: _pole_sigma(w, t, eps, D, Om, bs)
        f = lambda w: e + fn(w)[0] - w
        df = lambda w: fn(w)[1] - 1.0
        roots = [r.real for r in np.roots(poly) if abs(r.imag) < 1e-12 and df(r.real) < 0]
        for center in (e, e - 0.7, e + 0.9):
            inside = [r for r in roots if abs(r - center) <= 1.5]
            w, Z, st, n = O.qp_graphical(e, 0.0, fn, center, half_width=1.5, n_pts=301, tol=1e-12)
            if not inside:
                assert st == 3
                continue
            ref = min(inside, key=lambda r: abs(r - center))
            assert st == 0 and abs(w - ref) < 1e-10 and abs(f(w)) < 1e-12, (t, center, w, ref)


def test_cluster_guesses_reach_the_same_roots_with_fewer_evaluations():
    s = synth.water_cluster(2, 31, targets=[0, 1])           # the two O1s-like core levels, 0.2 Ha apart
    B, Bn = s.b_ia(), s.b_nm()
    plain = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, qp_tol=1e-7)
    grouped = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, qp_tol=1e-7, cluster_gap=0.5)
    assert O.clusters([s.eps[0], s.eps[1]], 0.5) == [[0, 1]]
    assert np.all(plain["status"] == 0) and np.all(grouped["status"] == 0)
    np.testing.assert_allclose(grouped["e_qp"], plain["e_qp"], rtol=0, atol=1e-6)
    assert grouped["n_sigma"][1] < plain["n_sigma"][1]       # the second state started from the first's shift


def test_clusters_split_on_gaps():
    assert O.clusters([-20.5, -20.4, -1.0, -0.9, -0.2, 3.0], 0.15) == [[0, 1], [2, 3], [4], [5]]
    assert O.clusters([0.3, -0.1, 0.0], 0.2) == [[1, 2], [0]]
    assert O.clusters([0.3, -0.1, 0.0], 0.35) == [[1, 2, 0]]


# ---------------------------------------------------------------- open shell
def _uks_system(seed, n_bas=7, n_occ=(3, 2), n_aux=5):
    rng = np.random.default_rng(seed)
    chans = []
    for o in n_occ:
        eps = np.sort(np.concatenate([rng.uniform(-1.6, -0.3, o), rng.uniform(0.1, 2.2, n_bas - o)]))
        chans.append((eps, o, rng.normal(0, 0.3, (n_aux, o * (n_bas - o)))))
    return chans, rng


def test_uks_with_equal_spins_is_the_closed_shell():
    s = synth.workload(0)
    B, Bn = s.b_ia(), s.b_nm()
    xi, wt = O.mgl_grid(64, 0.5)
    cs = O.CDSelfEnergy(s.eps, s.n_occ, B, Bn, s.targets, xi, wt, eta=1e-3)
    chans = [(s.eps, s.n_occ, B), (s.eps, s.n_occ, B)]
    us = O.CDSelfEnergyUKS(chans, Bn, [(0, n) for n in s.targets], xi, wt, eta=1e-3)
    for x in (0.0, 0.7):
        np.testing.assert_allclose(O.pi_imag_uks(chans, x), O.pi_imag(s.eps, s.n_occ, B, x), atol=1e-14)
    for t, n in enumerate(s.targets):
        for w in (s.eps[n], s.eps[n] - 0.3):
            a, b = us.sigma_c(t, w), cs.sigma_c(t, w)
            assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] - b[1]) < 1e-11
        assert us.sigma_x(t) == cs.sigma_x(t)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uks_cd_matches_spectral_route(seed):
    """Open shell, different occupations per spin: CD (spin-summed Pi, spin-resolved G) against the spectral
    decomposition with two spin blocks, at eta = 0 and omega = e_n (as the closed-shell SD/CD pin)."""
    chans, rng = _uks_system(seed)
    n_bas, n_aux = len(chans[0][0]), chans[0][2].shape[0]
    targets = [(0, 2), (0, 3), (1, 1), (1, 2)]
    Bn = rng.normal(0, 0.3, (len(targets), n_bas, n_aux))
    xi, wt = O.mgl_grid(256, 0.5)
    cd = O.CDSelfEnergyUKS(chans, Bn, targets, xi, wt, eta=0.0)
    Omega, V = O.casida_uks(chans)
    for t, (sp, n) in enumerate(targets):
        eps, n_occ, _ = chans[sp]
        s_sd, ds_sd = O.sigma_c_sd(eps, n_occ, Bn[t], Omega, V, eps[n], 0.0)
        s_cd, ds_cd = cd.sigma_c(t, eps[n])
        assert abs(s_cd - s_sd) < 1e-8, (t, s_cd, s_sd)
        assert abs(ds_cd - ds_sd) < 1e-6 * max(1.0, abs(ds_sd)), (t, ds_cd, ds_sd)
