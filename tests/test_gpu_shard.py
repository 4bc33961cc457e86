"""One job split across two ranks through the library (gw_set_shard), both ranks as processes on GPU 0 with gloo
sums on the host between launches (no kernel waits on another rank): every rank returns the single-rank QP
energies."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, prec, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2107_10423_gb300 import gw, shard, synth
    s = synth.water_cluster(2, 21, targets="valence")
    kw = dict(minres_tol=1e-12, minres_maxit=600, minres_fallback_tol=1e-9) if prec == "fp64" else {}
    p = gw.Plan(s.eps, s.n_occ, s.b_ia(), s.b_nm(), s.targets,
                precision=gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED, **kw)
    p.set_shard(rank, world, shard.make_allreduce())
    e, z, st = p.qp_solve(gw.GW_QP_LINEARISED)
    n_rhs = p.stats()["n_rhs_solved"]
    p.close()
    q.put((rank, e.tolist(), int(n_rhs)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 0.05 * 3.6749322175655e-5)])
def test_two_ranks_on_one_gpu_match_single_rank(gwlib, prec, tol):
    from paper_2107_10423_gb300 import gw, synth
    s = synth.water_cluster(2, 21, targets="valence")
    kw = dict(minres_tol=1e-12, minres_maxit=600, minres_fallback_tol=1e-9) if prec == "fp64" else {}
    with gw.Plan(s.eps, s.n_occ, s.b_ia(), s.b_nm(), s.targets,
                 precision=gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED, **kw) as p:
        ref, _, _ = p.qp_solve(gw.GW_QP_LINEARISED)
        n_all = p.stats()["n_rhs_solved"]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, prec, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = dict((r[0], r[1:]) for r in (q.get(timeout=600) for _ in range(2)))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    for r in (0, 1):
        np.testing.assert_allclose(out[r][0], ref, rtol=0, atol=tol)
    assert out[0][1] + out[1][1] == n_all and min(out[0][1], out[1][1]) > 0      # the residues were split
