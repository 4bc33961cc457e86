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
