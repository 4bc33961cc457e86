"""Eigenvalue self-consistency (Algorithm 1, outer loop; evGW0 and evGW) on the GPU against the oracle's loop."""
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


@pytest.fixture(scope="module")
def water1():
    s = synth.workload(0)
    return s, s.b_ia(), s.b_nm()


@pytest.mark.parametrize("update_w", [False, True])
@pytest.mark.parametrize("mode", ["linearised", "steptree"])
def test_evgw_fp64_vs_oracle(gw, water1, update_w, mode):
    s, B, Bn = water1
    ref = O.evgw(s.eps, s.n_occ, B, Bn, s.targets, update_w=update_w, mode=mode, tol=1e-7, max_iter=60)
    assert ref["converged"]
    qm = gw.GW_QP_LINEARISED if mode == "linearised" else gw.GW_QP_STEPTREE
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, **TIGHT) as p:
        e0, _, _ = p.qp_solve(qm)
        e, z, st, cycles = p.evgw(update_w=update_w, mode=qm, max_iter=60, tol=1e-7)
        e1, _, _ = p.qp_solve(qm)                  # the plan is back to G0W0 afterwards
    print(f"evGW{'' if update_w else '0'} {mode}: {cycles} cycles (oracle {ref['iterations']}), e_qp {e}")
    np.testing.assert_allclose(e, ref["e_qp"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(z, ref["Z"], rtol=0, atol=1e-5)
    assert abs(cycles - ref["iterations"]) <= 1
    np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-10)
    assert np.max(np.abs(e - e0)) > 0.1              # the cycles moved the energies


@pytest.mark.parametrize("update_w", [False, True])
def test_evgw_mixed_within_5mev(gw, water1, update_w):
    s, B, Bn = water1
    ref = O.evgw(s.eps, s.n_occ, B, Bn, s.targets, update_w=update_w, mode="linearised", tol=1e-7, max_iter=60)
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED) as p:
        e, z, st, cycles = p.evgw(update_w=update_w, mode=gw.GW_QP_LINEARISED, max_iter=60, tol=1e-7)
    err = np.abs(e - ref["e_qp"]) / MEV
    print(f"mixed evGW{'' if update_w else '0'}: {cycles} cycles, |error| meV {np.round(err, 4)}")
    assert np.all(err < 5.0), err
