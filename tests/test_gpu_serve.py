"""Serving on the GPU: jobs overlapping in the server give the same QP energies as each job run alone."""
import numpy as np
import pytest

from paper_2107_10423_gb300 import serve, synth

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix(gwlib):
    stream = [(0.0, synth.water_cluster(n, 500 + n, targets=t)) for n, t in
              [(2, "homo_lumo"), (3, "o1s"), (1, "homo_lumo"), (4, "homo_lumo"), (2, "o1s")]]
    jobs = serve.make_jobs(stream)
    alone = [serve.run_job(j) for j in jobs]
    srv = serve.Server(max_slots=4)
    mixed = srv.run(serve.make_jobs(stream), time_scale=1.0)
    assert max(len([1 for t, e, _ in srv.log if e == "start" and t <= j.finish]) for j in mixed) >= 2
    for a, m in zip(alone, mixed):
        assert "error" not in m.result, m.result
        np.testing.assert_allclose(m.result["e_qp"], a["e_qp"], rtol=0, atol=1e-8)
    s = serve.summarize(mixed)
    assert s["completed"] == len(jobs)
