"""Open-shell (spin-unrestricted) G0W0 on the GPU: the closed-shell limit, and a doublet against the oracle's
open-shell CD self-energy."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu
MEV = 3.6749322175655e-5
TIGHT = dict(minres_tol=1e-12, minres_maxit=600, minres_fallback_tol=1e-9)


@pytest.fixture(scope="module")
def gw(gwlib):
    from paper_2107_10423_gb300 import gw as m
    return m


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_equal_spins_give_the_closed_shell(gw, prec):
    s = synth.water_cluster(2, 21, targets=[9, 10, 11])
    B, Bn = s.b_ia(), s.b_nm()
    kw = dict(TIGHT) if prec == "fp64" else {}
    p_ = gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=p_, **kw) as p:
        e_cs, z_cs, _ = p.qp_solve(gw.GW_QP_LINEARISED)
    with gw.Plan.open_shell(s.eps, s.eps, s.n_occ, s.n_occ, B, B, Bn, s.targets, [0, 1, 0], precision=p_, **kw) as p:
        e_os, z_os, _ = p.qp_solve(gw.GW_QP_LINEARISED)
    tol = 1e-9 if prec == "fp64" else 0.5 * MEV      # mixed: B/sqrt(2) and the doubled pair list round differently
    np.testing.assert_allclose(e_os, e_cs, rtol=0, atol=tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-5), ("mixed", 5 * MEV)])
def test_doublet_vs_oracle(gw, prec, tol):
    s = synth.water_cation(2, 61)
    Ba, Bb, Bn = s.b_ia(0), s.b_ia(1), s.b_nm()
    xi, wt = O.mgl_grid(128, 0.5)
    chans = [(s.eps[0], s.n_occ[0], Ba), (s.eps[1], s.n_occ[1], Bb)]
    cd = O.CDSelfEnergyUKS(chans, Bn, s.targets, xi, wt, eta=1e-3)
    ref = []
    for t, (sp, n) in enumerate(s.targets):
        e, Z = O.qp_linearised(s.eps[sp][n], 0.0, lambda w, t=t: cd.sigma_c(t, w))
        ref.append(e)
    kw = dict(TIGHT) if prec == "fp64" else {}
    with gw.Plan.open_shell(s.eps[0], s.eps[1], s.n_occ[0], s.n_occ[1], Ba, Bb, Bn, [n for _, n in s.targets],
                            [sp for sp, _ in s.targets],
                            precision=gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED, **kw) as p:
        e, z, st = p.qp_solve(gw.GW_QP_LINEARISED)
        sc, dsc, sx = p.sigma_cd(np.array([s.eps[sp][n] for sp, n in s.targets]))
    for t in range(len(s.targets)):
        assert abs(sx[t] - cd.sigma_x(t)) < 1e-12
    print("open shell", prec, "|e - oracle| meV:", np.round(np.abs(e - np.array(ref)) / MEV, 4))
    np.testing.assert_allclose(e, ref, rtol=0, atol=tol)
