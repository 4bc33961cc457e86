"""Mixed-precision path (tcgen05 BF16x3 Pi and dense residue matrices, FP32 operators, FP64 recurrences,
quadrature and QP search) vs the FP64 oracle: every QP energy within 5 meV."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu
MEV = 3.6749322175655e-5      # Ha per meV
MIXED = dict()     # production settings: paper MINRES defaults (25 / 5e-5 / dense fallback above 1e-4)


@pytest.fixture(scope="module")
def gw(gwlib):
    from paper_2107_10423_gb300 import gw as m
    return m


@pytest.mark.parametrize("n,targets", [(2, "valence"), (3, "valence")])
def test_mixed_linearised_within_5mev(gw, n, targets):
    s = synth.water_cluster(n, 40 + n, targets=targets)
    B, Bn = s.b_ia(), s.b_nm()
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, mode="linearised")
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, **MIXED) as p:
        e, z, st = p.qp_solve(gw.GW_QP_LINEARISED)
    err = np.abs(e - ref["e_qp"])
    print("mixed linearised |error| meV:", np.round(err / MEV, 4))
    assert np.all(err < 5 * MEV), err / MEV


def test_mixed_core_steptree_within_5mev_of_a_root(gw):
    """O1s core states solved with the step tree: converged, on a root of the exact QP equation (|f Z| from the
    FP64 oracle at the GPU's answer) and on the oracle's own step-tree root, each within 5 meV."""
    s = synth.water_cluster(3, 43, targets=[0, 1, 2])
    B, Bn = s.b_ia(), s.b_nm()
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, qp_tol=1e-6, **MIXED) as p:
        e, z, st = p.qp_solve(gw.GW_QP_STEPTREE)
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, qp_tol=1e-6)
    cd = ref["cd"]
    for t, n in enumerate(s.targets):
        assert st[t] != 1, (t, st)
        sg, dsg = cd.sigma_c(t, e[t])
        assert abs((s.eps[n] + sg - e[t]) / (1.0 - dsg)) < 5 * MEV, (t, e[t])
    print("mixed core step-tree vs oracle root meV:", np.round(np.abs(e - ref["e_qp"]) / MEV, 4))
    assert np.all(np.abs(e - ref["e_qp"]) < 5 * MEV), np.abs(e - ref["e_qp"]) / MEV


def test_mixed_steptree_energies_are_roots(gw):
    """Valence states with the step tree: each mixed-precision energy is converged, within 5 meV of a root of the
    exact equation (|f(e)| |Z(e)| with f, Z from the FP64 oracle at e) and within 5 meV of the oracle's own
    step-tree root."""
    s = synth.water_cluster(2, 42, targets=[8, 9, 10, 11, 12])
    B, Bn = s.b_ia(), s.b_nm()
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, qp_tol=1e-6, **MIXED) as p:
        e, z, st = p.qp_solve(gw.GW_QP_STEPTREE)
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, qp_tol=1e-6)
    cd = ref["cd"]
    for t, n in enumerate(s.targets):
        assert st[t] != 1, (t, st)
        sg, dsg = cd.sigma_c(t, e[t])
        f = s.eps[n] + sg - e[t]
        Z = 1.0 / (1.0 - dsg)
        assert abs(f * Z) < 5 * MEV, (t, f, Z)
    print("mixed valence step-tree vs oracle root meV:", np.round(np.abs(e - ref["e_qp"]) / MEV, 4))
    assert np.all(np.abs(e - ref["e_qp"]) < 5 * MEV), np.abs(e - ref["e_qp"]) / MEV


def test_mixed_sigma_within_tolerance(gw):
    s = synth.water_cluster(2, 7, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(s.eps, s.n_occ, B, Bn, s.targets, xi, wt, eta=1e-3)
    om = s.eps[s.targets] - 0.05
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, **MIXED) as p:
        sc, dsc, _ = p.sigma_cd(om)
    ref = np.array([cd.sigma_c(t, om[t])[0] for t in range(len(s.targets))])
    assert np.all(np.abs(sc - ref) < 1 * MEV), np.abs(sc - ref) / MEV


def test_mixed_pi_accuracy(gw):
    s = synth.water_cluster(2, 7)
    B, Bn = s.b_ia(), s.b_nm()
    xi = np.array([0.0, 0.1, 3.0])
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED) as p:
        Pi = p.polarizability(xi)
    for g, x in enumerate(xi):
        ref = O.pi_imag(s.eps, s.n_occ, B, x)
        assert np.abs(Pi[g] - ref).max() < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("deriv_fp64", [0, 1])
def test_mixed_dsigma_at_the_ks_energy(gw, deriv_fp64):
    """dSigma_c/domega at omega = e_n, the input of the linearised QP equation, against the oracle's exact CD.
    At omega = e_n the I term weighs W(i xi) - W(0) of the diagonal state by w/xi^2 at the first grid nodes, and
    residues sit near the poles of Pi(x); both are where FP32 rounding would show."""
    s = synth.water_cluster(3, 43, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(s.eps, s.n_occ, B, Bn, s.targets, xi, wt, eta=1e-3)
    om = s.eps[s.targets]
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, deriv_fp64=deriv_fp64) as p:
        sc, dsc, _ = p.sigma_cd(om)
    ref = np.array([cd.sigma_c(t, om[t]) for t in range(len(s.targets))])
    print("dSigma_c error:", np.abs(dsc - ref[:, 1]).max(), " Sigma_c error meV:", np.abs(sc - ref[:, 0]).max() / MEV)
    assert np.all(np.abs(sc - ref[:, 0]) < 1 * MEV), np.abs(sc - ref[:, 0]) / MEV
    assert np.all(np.abs(dsc - ref[:, 1]) < 2e-5), np.abs(dsc - ref[:, 1])


def test_double_float_refinement_residual_matches_fp64(gw):
    """The refinement residual of the dense fallback solves in double-float arithmetic (FP32 pairs) against the
    same residual in FP64: the QP energies agree far below the accuracy bar, and both match the oracle."""
    s = synth.water_cluster(3, 43, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, mode="linearised")
    out = {}
    for df in (0, 1):
        with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, refine_df=df) as p:
            out[df] = p.qp_solve(gw.GW_QP_LINEARISED)[0]
            assert p.stats()["n_refine_fp64"] > 0
    assert np.abs(out[1] - out[0]).max() < 0.01 * MEV, np.abs(out[1] - out[0]).max() / MEV
    assert np.abs(out[1] - ref["e_qp"]).max() < 1 * MEV, np.abs(out[1] - ref["e_qp"]).max() / MEV


@pytest.mark.parametrize("n", [1, 3])
def test_mixed_dense_fallback_blocked_lu(gw, n):
    """Residues forced through the mixed dense fallback, whose FP32 LU runs in 64-column panels with the trailing
    updates on the tensor cores (N_aux 126: one update of 62 rows; N_aux 378: five updates and a ragged last
    panel), refined against the FP64 operator: W and dW against the oracle's dense complex solve (Sec. 3.3)."""
    s = synth.water_cluster(n, 9)
    B, Bn = s.b_ia(), s.b_nm()
    ti = np.array([0, 1, 1, 0])
    m = np.array([2, 7, 4, s.n_occ])
    x = np.array([0.3, -0.9, 1.7, 0.62])
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, minres_maxit=2, minres_tol=1e-14,
                 minres_fallback_tol=1e-13) as p:
        r = p.residues(ti, m, x)
    assert np.all(r["used_fallback"] == 1)
    for j in range(len(ti)):
        w, dw = O.w_corr_and_deriv(O.pi_complex(s.eps, s.n_occ, B, x[j], 1e-3),
                                   O.dpi_complex(s.eps, s.n_occ, B, x[j], 1e-3), Bn[ti[j], m[j]])
        print("fallback W error", abs(r["w_re"][j] - w.real), " dW error", abs(r["dw_re"][j] - dw.real))
        assert abs(r["w_re"][j] - w.real) < 2e-6 * max(1, abs(w)), (j, r["w_re"][j], w)
        assert abs(r["w_im"][j] - w.imag) < 2e-6 * max(1, abs(w)), (j, r["w_im"][j], w)
        assert abs(r["dw_re"][j] - dw.real) < 1e-4 * max(1, abs(dw)), (j, r["dw_re"][j], dw)


def test_chunked_workspace_mixed_vs_oracle(gw):
    """The chunked code that full-size mixed jobs run, forced on (H2O)_3 by a 12 MiB workspace cap: two frequency
    matrices per Newton-Schulz chunk (65 chunks), so the difference-form columns of the lowest grid points span many
    chunks after the first and use its stored eps(0)^-1; split-operand sub-batches of the dense fallback; and
    max_rhs_batch = 7 MINRES sub-batches.  Sigma_c, dSigma_c and the linearised QP energies against the oracle at
    the same bars as the unchunked tests."""
    s = synth.water_cluster(3, 43, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    xi, wt = O.mgl_grid(128, 0.5)
    cd = O.CDSelfEnergy(s.eps, s.n_occ, B, Bn, s.targets, xi, wt, eta=1e-3)
    om = s.eps[s.targets]
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, workspace_mb=12,
                 max_rhs_batch=7) as p:
        sc, dsc, _ = p.sigma_cd(om)
        e, z, st = p.qp_solve(gw.GW_QP_LINEARISED)
        stats = p.stats()
    assert stats["launches_kernel"][0] >= 60          # Pi(i xi) in many chunks
    assert stats["n_fallback"] > 7                    # more than one fallback sub-batch
    ref = np.array([cd.sigma_c(t, om[t]) for t in range(len(s.targets))])
    assert np.all(np.abs(sc - ref[:, 0]) < 1 * MEV), np.abs(sc - ref[:, 0]) / MEV
    assert np.all(np.abs(dsc - ref[:, 1]) < 2e-5), np.abs(dsc - ref[:, 1])
    qref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, mode="linearised")
    err = np.abs(e - qref["e_qp"])
    print("chunked mixed linearised |error| meV:", np.round(err / MEV, 4))
    assert np.all(err < 5 * MEV), err / MEV


def test_footprint_bound_holds(gw):
    """The plan's device bytes (counted at every allocation) stay below gw_plan_footprint's bound, and the device's
    own free-memory drop agrees with the count, on a mixed job forced through the dense fallback."""
    import torch
    s = synth.water_cluster(3, 43, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    bound = gw.footprint(s.n_occ, s.n_virt, s.n_aux, len(s.targets), precision=gw.GW_PREC_MIXED, workspace_mb=64)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, workspace_mb=64) as p:
        p.qp_solve(gw.GW_QP_LINEARISED)
        st = p.stats()
        free1, _ = torch.cuda.mem_get_info()
    assert st["n_fallback"] > 0
    assert 0 < st["bytes_device"] <= st["bytes_device_peak"] <= bound, (st["bytes_device_peak"], bound)
    used = free0 - free1
    # allocation granularity: at most 2 MiB per buffer on top of the counted bytes
    assert st["bytes_device"] - (1 << 20) <= used <= st["bytes_device"] + 200 * (2 << 20), (used, st["bytes_device"])


@pytest.mark.parametrize("n,seed,xi,ctas", [
    (1, 3, [0.7], 0),                           # one 128 x 256 tile holding 84 rows, K = 95 (ragged k-block), one entry
    (1, 3, [0.0, 0.2, 1.0, 4.0, 30.0], 1),      # five entries on a single persistent CTA (items in sequence)
    (3, 5, [0.0, 0.05, 2.0, 9.0], 2),           # 378 rows: 4 lower 128 x 256 tiles, ragged in rows and columns, 2 CTAs
    (4, 6, [0.01, 0.3, 1.1], 0)])               # 504 rows, K = 7600 (30 K panels)
def test_fused_pi_tiles_and_entries(gw, n, seed, xi, ctas):
    """Pi(i xi) from the fused-weight tensor-core kernel against the oracle, element by element: ragged row, column
    and k tails, several batch entries and persistent CTAs that each take many (tile, entry) items in sequence.
    Bar: 2e-5 of max |Pi| (BF16x3 with FP32 sums)."""
    s = synth.workload(0) if n == 1 else synth.water_cluster(n, seed)
    B, Bn = s.b_ia(), s.b_nm()
    xi = np.array(xi)
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, tc_max_ctas=ctas) as p:
        Pi = p.polarizability(xi)
    for g, x in enumerate(xi):
        ref = O.pi_imag(s.eps, s.n_occ, B, x)
        err = np.abs(Pi[g] - ref).max()
        assert err < 2e-5 * np.abs(ref).max(), (g, x, err, np.abs(ref).max())
        assert np.array_equal(Pi[g], Pi[g].T)


@pytest.mark.parametrize("n,ks", [(2, 2), (2, 4), (3, 2), (3, 8), (2, 0), (0, 2)])
def test_fused_pi_split_k(gw, n, ks):
    """The K split of the fused Pi kernel (forced, or ks = 0: autotuned for the shape) against the oracle, and the
    split product against the unsplit one (partials added in a fixed order).  n = 0 is the single water, whose
    N_ov = 95 (3 K blocks) admits no split: the request falls back to one K range."""
    s = synth.workload(0) if n == 0 else synth.water_cluster(n, 9)
    B, Bn = s.b_ia(), s.b_nm()
    xi = np.array([0.0, 0.4, 3.0])
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, pi_ksplit=ks) as p:
        Pi = p.polarizability(xi)
        Pi2 = p.polarizability(xi)
        used = p.stats()["pi_ksplit_last"]
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, pi_ksplit=1) as p:
        Pi1 = p.polarizability(xi)
    if n == 0:
        assert used == 1
    else:
        assert used == ks if ks else used in (1, 2, 4, 8)
    np.testing.assert_array_equal(Pi, Pi2)                       # deterministic
    for g, x in enumerate(xi):
        ref = O.pi_imag(s.eps, s.n_occ, B, x)
        assert np.abs(Pi[g] - ref).max() < 2e-5 * np.abs(ref).max()
        assert np.abs(Pi[g] - Pi1[g]).max() < 2e-6 * np.abs(ref).max()
        assert np.array_equal(Pi[g], Pi[g].T)
