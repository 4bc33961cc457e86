"""gw_w_table_noalloc: the W-table triangular solves for callers that cannot allocate device memory
(a process that gives all GPU memory to its own pool, an allocator that forbids cudaMalloc after start-up).
Its output must equal the plan-based W table of gw_w_table and the oracle's dense-LU W^c on the same Pi(i xi),
on two calls in a row.  This file is collected
last so that a stop at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_w_table_matches_plan(gwlib):
    import torch
    from paper_2107_10423_gb300 import gw
    s = synth.water_cluster(2, 21, targets="valence")
    B, Bn = s.b_ia(), s.b_nm()
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets) as p:
        ref = p.w_table()                                  # [n_t][n_bas][n_freq + 1], FP64 path
    xi, _ = gw.grid(128, 0.5)
    xis = np.concatenate([xi, [0.0]])
    n = s.n_aux
    Pis = [O.pi_imag(s.eps, s.n_occ, B, x) for x in xis]
    L = np.stack([np.linalg.cholesky(np.eye(n) - Pi) for Pi in Pis])
    # the oracle's W^c = b^T[(1 - Pi)^-1 - 1]b by dense LU with the same Pi(i xi) the factors come from
    ora = np.stack([np.stack([O.w_corr(Pi, Bn[t].T) for Pi in Pis], axis=-1) for t in range(len(s.targets))])
    dev = torch.device("cuda", 0)
    L_d = torch.from_numpy(np.ascontiguousarray(L)).to(dev)
    rows = np.ascontiguousarray(Bn.reshape(-1, n))
    Bn_d = torch.from_numpy(rows).to(dev)
    R, G = rows.shape[0], len(xis)
    for call in range(2):
        W_d = torch.full((R, G), float("nan"), dtype=torch.float64, device=dev)
        st = gwlib.gw_w_table_noalloc(ctypes.c_void_p(L_d.data_ptr()), n, G, ctypes.c_void_p(Bn_d.data_ptr()), R,
                                      ctypes.c_void_p(W_d.data_ptr()), G, None)
        assert st == gw.GW_OK
        torch.cuda.synchronize()
        W = W_d.cpu().numpy().reshape(ref.shape)
        np.testing.assert_allclose(W, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()), err_msg=f"call {call}")
        # |L^-1 b|^2 - |b|^2 cancels where W is small (large xi): the FP64 bound is a few ulp of |b|^2
        np.testing.assert_allclose(W, ora, rtol=0, atol=1e-12 * max(1.0, np.abs(ora).max()), err_msg=f"oracle {call}")


def test_noalloc_rejects_oversize(gwlib):
    from paper_2107_10423_gb300 import gw
    one = ctypes.c_void_p(16)     # never dereferenced: the size checks come first
    assert gwlib.gw_w_table_noalloc(one, 70000, 3, one, 5, one, 3, None) == gw.GW_ERR_ARG
    assert gwlib.gw_w_table_noalloc(one, 64, 5000, one, 5, one, 5000, None) == gw.GW_ERR_ARG
    assert gwlib.gw_w_table_noalloc(one, 64, 3, one, 5, one, 2, None) == gw.GW_ERR_ARG
