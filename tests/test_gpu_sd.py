"""Spectral-decomposition route on the GPU (Sec. 2.2 and 3.2): the Hermitian Casida problem diagonalised by cyclic
Jacobi sweeps in FP64 and Sigma_c summed over its poles, against the oracle's Casida route (LAPACK eigh) for a closed
and an open shell, and against the GPU's own contour-deformation route at eta = 0, where the two are the same
function."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw(gwlib):
    from paper_2107_10423_gb300 import gw as m
    return m


@pytest.mark.parametrize("eta", [0.0, 1e-3])
def test_sd_single_water_vs_oracle(gw, eta):
    """C0 shape (N_ov = 95, odd: one padded index in the Jacobi pairing), HOMO and LUMO, off their KS energies."""
    s = synth.workload(0)
    B, Bn = s.b_ia(), s.b_nm()
    Om, V = O.casida(s.eps, s.n_occ, B)
    om = s.eps[s.targets] + 0.013
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, eta=eta) as p:
        sc, dsc = p.sigma_sd(om)
        # the same values at explicit (target, omega) pairs, repeated
        sc2, _ = p.sigma_sd(np.concatenate([om, om]), target_idx=np.tile(np.arange(len(om)), 2))
    np.testing.assert_array_equal(sc2[:len(om)], sc)
    for t in range(len(s.targets)):
        ref = O.sigma_c_sd(s.eps, s.n_occ, Bn[t], Om, V, om[t], eta)
        assert abs(sc[t] - ref[0]) < 1e-9 * max(1.0, abs(ref[0])), (t, sc[t], ref[0])
        assert abs(dsc[t] - ref[1]) < 1e-8 * max(1.0, abs(ref[1])), (t, dsc[t], ref[1])


def test_sd_equals_cd_at_zero_eta(gw):
    """(H2O)_1 shape, N_ov = 190: Sigma_c at the KS energies by the GPU's SD and CD routes agree to 1e-8 Ha (the CD
    quadrature with static subtraction is exact to that level at eta = 0)."""
    s = synth.water_cluster(1, 9)
    B, Bn = s.b_ia(), s.b_nm()
    om = s.eps[s.targets]
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, eta=0.0, minres_tol=1e-13, minres_maxit=800,
                 minres_fallback_tol=1e-10) as p:
        sd, dsd = p.sigma_sd(om)
        cd, dcd, _ = p.sigma_cd(om)
    print("SD - CD at eta = 0:", np.abs(sd - cd).max(), np.abs(dsd - dcd).max())
    np.testing.assert_allclose(sd, cd, rtol=0, atol=1e-8)
    np.testing.assert_allclose(dsd, dcd, rtol=0, atol=1e-6)


def test_sd_open_shell_vs_oracle(gw):
    """(H2O)_1^+ doublet: two spin blocks in one Casida problem (the plan's 1/sqrt 2 channel scaling gives the
    factor 2 per block), G and the pole weights of each target's own spin."""
    s = synth.water_cation(1, 61)
    Ba, Bb, Bn = s.b_ia(0), s.b_ia(1), s.b_nm()
    Om, V = O.casida_uks([(s.eps[0], s.n_occ[0], Ba), (s.eps[1], s.n_occ[1], Bb)])
    om = np.array([s.eps[sp][n] + 0.011 for sp, n in s.targets])
    with gw.Plan.open_shell(s.eps[0], s.eps[1], s.n_occ[0], s.n_occ[1], Ba, Bb, Bn, [n for _, n in s.targets],
                            [sp for sp, _ in s.targets]) as p:
        sc, dsc = p.sigma_sd(om)
    for t, (sp, n) in enumerate(s.targets):
        ref = O.sigma_c_sd(s.eps[sp], s.n_occ[sp], Bn[t], Om, V, om[t], 1e-3)
        assert abs(sc[t] - ref[0]) < 1e-9 * max(1.0, abs(ref[0])), (t, sc[t], ref[0])
        assert abs(dsc[t] - ref[1]) < 1e-8 * max(1.0, abs(ref[1])), (t, dsc[t], ref[1])


def test_sd_water3_and_bad_index(gw):
    s = synth.water_cluster(3, 9)          # N_ov = 1710: allowed
    B, Bn = s.b_ia(), s.b_nm()
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets) as p:
        sc, _ = p.sigma_sd(s.eps[s.targets] + 0.01)
        assert np.all(np.isfinite(sc))
        with pytest.raises(gw.GWError):
            p.sigma_sd(np.array([0.0]), target_idx=np.array([len(s.targets)]))   # target index out of range
