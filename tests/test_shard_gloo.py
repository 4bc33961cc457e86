"""One job split across two ranks (gloo on CPU): the library's partition of the frequency positions and of the
residue right-hand sides, and the shard module's all-reduce callback, with the oracle standing in for each rank's
GPU work.  The summed W table, the summed residue terms and the QP energies equal the single-rank ones."""
import ctypes
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import gw_oracle as O
    from paper_2107_10423_gb300 import shard, synth
    s = synth.workload(0)
    B, Bn = s.b_ia(), s.b_nm()
    n_freq = 128
    xi, wt = O.mgl_grid(n_freq, 0.5)
    cd = O.CDSelfEnergy(s.eps, s.n_occ, B, Bn, s.targets, xi, wt, eta=1e-3)   # stand-in for this rank's GPU work
    full = np.concatenate([cd.W, cd.W0[:, :, None]], axis=2)                   # [n_t][n_bas][n_freq + 1]
    cb = shard.make_allreduce()
    p0, p1 = shard.shard_columns(n_freq, rank, world)
    mine = np.zeros_like(full)
    for p in range(p0, p1):
        c = shard.position_column(p, n_freq)
        mine[:, :, c] = full[:, :, c]
    buf = np.ascontiguousarray(mine.reshape(-1))
    assert cb(buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), buf.size, None) == 0
    table_ok = np.array_equal(buf.reshape(full.shape), full)
    # residues of every target at omega = e_n, in the library's list order (target-major, then state); this
    # rank's share is every world-th entry
    e_qp = []
    rd = np.zeros(2 * len(s.targets))
    j = 0
    for t, n in enumerate(s.targets):
        for m, sgn, th in O.residue_set(s.eps, s.n_occ, s.eps[n]):
            if shard.owns_residue(j, rank, world):
                w, dw = cd.residue_w(t, m, s.eps[m] - s.eps[n])
                rd[t] += sgn * th * w.real
                rd[len(s.targets) + t] -= sgn * th * dw.real
            j += 1
    assert cb(rd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rd.size, None) == 0
    for t, n in enumerate(s.targets):
        I, dI = cd.i_term(t, s.eps[n])
        sg, dsg = rd[t] - I, rd[len(s.targets) + t] - dI
        e_qp.append(s.eps[n] + sg / (1.0 - dsg))
    q.put((rank, table_ok, (p0, p1), rd.tolist(), e_qp))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_split_matches_single_rank():
    from oracle import gw_oracle as O
    from paper_2107_10423_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r[0], r[1:]) for r in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (ok0, blk0, rd0, e0), (ok1, blk1, rd1, e1) = out[0], out[1]
    assert ok0 and ok1
    assert blk0 == (0, 64) and blk1 == (64, 129)
    np.testing.assert_array_equal(rd0, rd1)
    s = synth.workload(0)
    ref = O.g0w0_cd(s.eps, s.n_occ, s.b_ia(), s.b_nm(), s.targets, eta=1e-3, mode="linearised")
    np.testing.assert_allclose(e0, ref["e_qp"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(e1, e0, rtol=0, atol=0)


def test_shard_columns_partition():
    from paper_2107_10423_gb300 import shard
    for world in (1, 2, 3, 5, 8):
        blocks = [shard.shard_columns(128, r, world) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == 129
        for a, b in zip(blocks, blocks[1:]):
            assert a[1] == b[0] and a[1] - a[0] >= 1
        assert max(b - a for a, b in blocks) - min(b - a for a, b in blocks) <= 1
