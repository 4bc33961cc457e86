"""Mixed-precision path (tensor-core Pi, FP32 operator, FP64 recurrences) vs the FP64 oracle: every QP energy
within 5 meV."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu
MEV = 3.6749322175655e-5      # Ha per meV


@pytest.fixture(scope="module")
def gw(gwlib):
    from paper_2107_10423_gb300 import gw as m
    return m


@pytest.mark.parametrize("n,targets", [(2, "valence"), (3, [0, 13, 14, 15, 16])])
def test_mixed_qp_within_5mev(gw, n, targets):
    s = synth.water_cluster(n, 40 + n, targets=targets)
    B, Bn = s.b_ia(), s.b_nm()
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3)
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, minres_tol=1e-8,
                 minres_maxit=200, minres_fallback_tol=1e-6) as p:
        e, z, st = p.qp_solve(gw.GW_QP_STEPTREE)
    err = np.abs(e - ref["e_qp"])
    print("mixed per-state |error| meV:", np.round(err / MEV, 4))
    assert np.all(err < 5 * MEV), err / MEV


def test_mixed_pi_accuracy(gw):
    s = synth.water_cluster(2, 7)
    B, Bn = s.b_ia(), s.b_nm()
    xi = np.array([0.0, 0.1, 3.0])
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED) as p:
        Pi = p.polarizability(xi)
    for g, x in enumerate(xi):
        ref = O.pi_imag(s.eps, s.n_occ, B, x)
        assert np.abs(Pi[g] - ref).max() < 2e-5 * np.abs(ref).max()
