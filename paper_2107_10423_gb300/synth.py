"""Seeded synthetic G0W0 inputs shaped like water clusters and core-level molecules.

This module holds none of the GW method's arithmetic: it only lays out
orbital energies and draws the fitted three-index tensor B_{P,pq}
(orthonormal auxiliary basis, Sec. 3.1) from a counter-based normal
generator (``csrc/synth.c``).  Both the CUDA path and the CPU oracle take
their inputs from here.

Readings of the workload descriptions (the paper's own systems come from
the Cambridge Cluster Database and GW100/CORE65/ESCA, none available here):

* "levels uniform in [a, b]" are evenly spaced, endpoints included;
* B is i.i.d. normal, symmetric in (p, q): element (P, p, q) is drawn from
  the counter (P, min(p,q), max(p,q)), so the B_ia and B_nm slices agree;
* a water-cluster system (H2O)_n has n O1s-like core levels in
  [-20.6, -20.4] Ha (a single one at -20.5 Ha when n = 1), 4n valence levels
  in [-1.4, -0.4] Ha, 38n virtual levels in [0.03, 8] Ha and 126n auxiliary
  functions with B ~ N(0, (0.6/sqrt(N_aux))^2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth.c")
_LIB_PATH = os.path.join(_HERE, "_synth.so")
_lib = None


def build_synth(force: bool = False) -> str:
    """Compile the generator into ``_synth.so`` (plain C, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_synth())
        lib.synth_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 2 + [ctypes.POINTER(ctypes.c_uint32)]
        lib.synth_b_ia.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p]
        lib.synth_b_ia_rows.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_void_p]
        lib.synth_b_nm.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.c_void_p]
        _lib = lib
    return _lib


def philox4x32_10(counter, key):
    """Raw Philox4x32-10 block (exposed for known-answer tests)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*counter)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def b_ia(seed: int, sigma: float, n_aux: int, n_occ: int, n_virt: int) -> np.ndarray:
    """B_ia as [n_aux, n_occ*n_virt] float64, pair index i*n_virt + a."""
    out = np.empty((n_aux, n_occ * n_virt), dtype=np.float64)
    _load().synth_b_ia(seed, sigma, n_aux, n_occ, n_virt, out.ctypes.data)
    return out


def b_ia_rows(seed: int, sigma: float, p0: int, n_rows: int, n_occ: int, n_virt: int) -> np.ndarray:
    """Rows p0 .. p0 + n_rows - 1 of B_ia (the same values as ``b_ia``), [n_rows, n_occ*n_virt] float64."""
    out = np.empty((n_rows, n_occ * n_virt), dtype=np.float64)
    _load().synth_b_ia_rows(seed, sigma, p0, n_rows, n_occ, n_virt, out.ctypes.data)
    return out


def b_nm(seed: int, sigma: float, n_aux: int, n_bas: int, targets) -> np.ndarray:
    """B_nm rows of the target states as [n_targets, n_bas, n_aux] float64."""
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    out = np.empty((len(t), n_bas, n_aux), dtype=np.float64)
    _load().synth_b_nm(seed, sigma, n_aux, n_bas, t.ctypes.data, len(t), out.ctypes.data)
    return out


@dataclass
class System:
    """A closed-shell G0W0 problem: KS energies, sizes, B generator and targets."""
    name: str
    eps: np.ndarray          # [n_bas] ascending, Ha
    n_occ: int
    n_aux: int
    sigma_b: float
    seed: int
    targets: np.ndarray      # state indices into eps
    meta: dict = field(default_factory=dict)

    @property
    def n_bas(self) -> int:
        return len(self.eps)

    @property
    def n_virt(self) -> int:
        return self.n_bas - self.n_occ

    @property
    def n_ov(self) -> int:
        return self.n_occ * self.n_virt

    def b_ia(self) -> np.ndarray:
        return b_ia(self.seed, self.sigma_b, self.n_aux, self.n_occ, self.n_virt)

    def b_ia_rows(self, p0: int, n_rows: int) -> np.ndarray:
        return b_ia_rows(self.seed, self.sigma_b, p0, n_rows, self.n_occ, self.n_virt)

    def b_nm(self, targets=None) -> np.ndarray:
        return b_nm(self.seed, self.sigma_b, self.n_aux, self.n_bas, self.targets if targets is None else targets)

    def with_targets(self, targets) -> "System":
        return System(self.name, self.eps, self.n_occ, self.n_aux, self.sigma_b, self.seed,
                      np.asarray(targets, dtype=np.int64), dict(self.meta))


def _lin(a, b, n):
    if n <= 0:
        return np.zeros(0)
    if n == 1:
        return np.array([(a + b) / 2.0])
    return np.linspace(a, b, n)


def single_water(seed: int = 0) -> System:
    """Single-water-shaped system: 1 core (-20.5) + 4 valence in [-1.3,-0.45], 19 virtuals in [0.05,3],
    N_aux = 84, sigma_B = 0.15.  Targets HOMO and LUMO."""
    eps = np.concatenate([[-20.5], _lin(-1.3, -0.45, 4), _lin(0.05, 3.0, 19)])
    return System("water1", eps, 5, 84, 0.15, seed, np.array([4, 5]))


def water_cluster(n: int, seed: int, targets="valence") -> System:
    """(H2O)_n-shaped system: N_occ = 5n, N_bas = 43n, N_aux = 126n.

    ``targets``: "valence" = all 4n valence states and the 10 lowest virtuals;
    "homo_lumo" = HOMO and LUMO; "o1s" = the deepest core level; or explicit indices."""
    n_core, n_val, n_virt = n, 4 * n, 38 * n
    eps = np.concatenate([_lin(-20.6, -20.4, n_core), _lin(-1.4, -0.4, n_val), _lin(0.03, 8.0, n_virt)])
    n_occ, n_aux = 5 * n, 126 * n
    if isinstance(targets, str):
        if targets == "valence":
            t = list(range(n_core, n_occ)) + list(range(n_occ, n_occ + min(10, n_virt)))
        elif targets == "homo_lumo":
            t = [n_occ - 1, n_occ]
        elif targets == "o1s":
            t = [0]
        else:
            raise ValueError(targets)
    else:
        t = list(targets)
    return System(f"water{n}", eps, n_occ, n_aux, 0.6 / np.sqrt(n_aux), seed, np.array(t, dtype=np.int64),
                  {"n_water": n})


def water64_mixed(seed: int = 2) -> System:
    """(H2O)_64-shaped system (N_occ 320, N_bas 2752, N_aux 8064); targets HOMO-15..LUMO+5."""
    s = water_cluster(64, seed, targets=list(range(320 - 16, 320 + 6)))
    s.name = "water64"
    return s


def esca_like(seed: int = 3, n_virt: int = 552, n_aux: int = 1800) -> System:
    """ESCA-shaped core-level system: 3 F1s (-25.6 +- 0.05), 3 O1s (-19.3 +- 0.05), 6 C1s in [-11.4,-10.6],
    36 valence in [-1.6,-0.4]; 552 virtuals in [0.03, 8]; N_aux = 1800.  Targets: the 6 C1s levels.
    ``n_virt`` and ``n_aux`` give the same level structure at a smaller size."""
    occ = np.concatenate([_lin(-25.65, -25.55, 3), _lin(-19.35, -19.25, 3), _lin(-11.4, -10.6, 6),
                          _lin(-1.6, -0.4, 36)])
    eps = np.concatenate([occ, _lin(0.03, 8.0, n_virt)])
    return System("esca", eps, 48, n_aux, 0.6 / np.sqrt(n_aux), seed, np.arange(6, 12), {})


@dataclass
class OpenShellSystem:
    """A spin-unrestricted problem: per-spin energies and occupations on a shared orbital and auxiliary basis, B
    drawn per spin (alpha with ``seed``, beta with ``seed + 1``), targets as (spin, state) pairs."""
    name: str
    eps: tuple               # (eps_alpha, eps_beta), each [n_bas] ascending
    n_occ: tuple             # (n_occ_alpha, n_occ_beta)
    n_aux: int
    sigma_b: float
    seed: int
    targets: list            # [(spin, state), ...]

    @property
    def n_bas(self) -> int:
        return len(self.eps[0])

    def b_ia(self, spin: int) -> np.ndarray:
        o = self.n_occ[spin]
        return b_ia(self.seed + spin, self.sigma_b, self.n_aux, o, self.n_bas - o)

    def b_nm(self) -> np.ndarray:
        """Rows of every target in its own spin, [n_targets, n_bas, n_aux]."""
        return np.stack([b_nm(self.seed + sp, self.sigma_b, self.n_aux, self.n_bas, [n])[0] for sp, n in self.targets])


def water_cation(n: int, seed: int) -> OpenShellSystem:
    """(H2O)_n^+-shaped doublet: the levels of ``water_cluster(n)`` for both spins, the beta HOMO emptied and the
    beta levels raised by 0.05 Ha; targets the alpha HOMO and LUMO and the beta HOMO and LUMO."""
    base = water_cluster(n, seed)
    ea = base.eps.copy()
    eb = base.eps + 0.05
    oa, ob = base.n_occ, base.n_occ - 1
    return OpenShellSystem(f"water{n}+", (ea, eb), (oa, ob), base.n_aux, base.sigma_b, seed,
                           [(0, oa - 1), (0, oa), (1, ob - 1), (1, ob)])


def workload(k: int) -> System:
    """The four fixed workloads: 0 single water (FP64, SD and CD), 1 (H2O)_16 valence (FP64 CD+MINRES),
    2 (H2O)_64 (mixed precision), 3 ESCA-shaped C1s batch."""
    if k == 0:
        return single_water(0)
    if k == 1:
        s = water_cluster(16, 1, targets="valence")
        s.name = "water16"
        return s
    if k == 2:
        return water64_mixed(2)
    if k == 3:
        return esca_like(3)
    raise ValueError(k)


def serving_stream(n_jobs: int = 256, rate: float = 4.0, arrival_seed: int = 4, job_seed0: int = 1000,
                   n_max: int = 64, core_fraction: float = 0.3):
    """Job stream for the serving loop: Poisson arrivals at ``rate`` jobs/s; job j is a water cluster with
    n = round(exp(U(0, ln n_max))) waters (seed job_seed0 + j); 70% valence (HOMO, LUMO) and 30% core
    (deepest O1s).  Returns a list of (arrival_time_s, System)."""
    rng = np.random.Generator(np.random.Philox(arrival_seed))
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    t = np.cumsum(gaps)
    ns = np.clip(np.rint(np.exp(rng.uniform(0.0, np.log(n_max), size=n_jobs))), 1, n_max).astype(int)
    kinds = rng.uniform(size=n_jobs) < core_fraction
    jobs = []
    for j in range(n_jobs):
        s = water_cluster(int(ns[j]), job_seed0 + j, targets="o1s" if kinds[j] else "homo_lumo")
        jobs.append((float(t[j]), s))
    return jobs
