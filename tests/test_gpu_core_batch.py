"""The core-level batch (ESCA-shaped: 6 C1s states by the step tree, all residue right-hand sides of a QP iteration
in one batched MINRES launch sequence) at a reduced size the oracle finishes in about a minute: mixed precision
against the oracle's step tree, per state."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu
MEV = 3.6749322175655e-5


def test_c1s_batch_steptree_vs_oracle(gwlib):
    from paper_2107_10423_gb300 import gw
    s = synth.esca_like(3, n_virt=40, n_aux=120)
    B, Bn = s.b_ia(), s.b_nm()
    ref = O.g0w0_cd(s.eps, s.n_occ, B, Bn, s.targets, eta=1e-3, qp_tol=1e-6)
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_MIXED, qp_tol=1e-6) as p:
        e, z, st = p.qp_solve(gw.GW_QP_STEPTREE)
        stats = p.stats()
    err = np.abs(e - ref["e_qp"]) / MEV
    print("C1s step tree |mixed - oracle| meV:", np.round(err, 4), " Sigma evaluations:", stats["n_sigma_evals"],
          " MINRES graph launches:", stats["n_graph_launches"])
    # The reduced system couples the C1s levels to each other as strongly as to anything (random B), so they sit
    # among dense satellite poles (|Z| ~ 1e-4) where the QP equation has many roots and neither solver's path is
    # stable against rounding (the oracle itself converges on different states on x86 and Arm).  So, per state
    # the GPU solves: a root of the FP64 QP equation lies within 1 meV of its energy (f from the oracle's Sigma,
    # continuous at finite eta, changes sign inside [e - 1 meV, e + 1 meV]; with Z < 0 it rises through zero);
    # where both solvers converged it is either the oracle's root or another one, and the count is reported.
    cd = ref["cd"]
    conv = st != 1
    assert conv.sum() >= 3, st
    for t, n in enumerate(s.targets):
        if not conv[t]:
            continue
        f = [s.eps[n] + cd.sigma_c(t, w)[0] - w for w in (e[t] - MEV, e[t] + MEV)]
        assert f[0] * f[1] < 0.0, (t, e[t], f)
    same = conv & (ref["status"] == 0) & (err < 5.0)
    print("states on the oracle's own root:", int(same.sum()), "of", int((conv & (ref["status"] == 0)).sum()))
    # one batched MINRES launch sequence (one graph) per QP iteration, shared by every state still active: fewer
    # graph launches than per-state Sigma evaluations, at most one per iteration
    assert 1 <= stats["n_graph_launches"] <= 50
    assert stats["n_sigma_evals"] > 2 * stats["n_graph_launches"]
