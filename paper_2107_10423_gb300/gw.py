"""ctypes binding of libgw.so (include/gw.h).  Argument marshalling only: every step of the
G0W0 path runs in the CUDA library.  Raises if the library is missing (no fallback)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgw.so")

GW_OK, GW_ERR_ARG, GW_ERR_OOM, GW_ERR_CUDA, GW_ERR_NOT_CONVERGED, GW_ERR_TIMEOUT, GW_ERR_UNIMPLEMENTED, \
    GW_ERR_NUMERIC = range(8)
GW_PREC_FP64, GW_PREC_MIXED = 0, 1
GW_QP_LINEARISED, GW_QP_STEPTREE, GW_QP_GRAPHICAL = 0, 1, 2
GW_INPUT_ON_DEVICE, GW_BORROW_DEVICE_PTRS = 1, 2

EXPORTED = ["gw_config_default", "gw_plan_create", "gw_polarizability", "gw_sigma_cd", "gw_residues_minres",
            "gw_qp_solve", "gw_grid", "gw_w_table", "gw_w_table_noalloc", "gw_get_stats", "gw_plan_destroy", "gw_last_error",
            "gw_plan_footprint", "gw_evgw", "gw_set_shard", "gw_shard_columns", "gw_plan_create_uks",
            "gw_sigma_points", "gw_sigma_sd"]


class GWError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gw status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int), ("n_virt", ctypes.c_int), ("n_aux", ctypes.c_int),
                ("n_freq", ctypes.c_int), ("x0", ctypes.c_double), ("eta", ctypes.c_double),
                ("precision", ctypes.c_int), ("minres_maxit", ctypes.c_int), ("minres_tol", ctypes.c_double),
                ("minres_fallback_tol", ctypes.c_double), ("qp_maxit", ctypes.c_int), ("qp_tol", ctypes.c_double),
                ("static_subtraction", ctypes.c_int), ("max_rhs_batch", ctypes.c_int), ("workspace_mb", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("op_parts", ctypes.c_int), ("deriv_fp64", ctypes.c_int), ("refine_df", ctypes.c_int),
                ("tc_max_ctas", ctypes.c_int), ("qp_window", ctypes.c_double), ("qp_window_points", ctypes.c_int),
                ("qp_cluster_gap", ctypes.c_double), ("pi_ksplit", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_screening", ctypes.c_double), ("ms_pi", ctypes.c_double), ("ms_sigma_imag", ctypes.c_double),
                ("ms_residues", ctypes.c_double), ("ms_qp", ctypes.c_double), ("n_rhs_solved", ctypes.c_longlong),
                ("n_minres_iters", ctypes.c_longlong), ("n_fallback", ctypes.c_longlong),
                ("n_sigma_evals", ctypes.c_longlong), ("n_kernel_launches", ctypes.c_longlong),
                ("ms_kernel", ctypes.c_double * 9), ("flops_kernel", ctypes.c_double * 9),
                ("launches_kernel", ctypes.c_longlong * 9), ("n_refine_fp64", ctypes.c_longlong),
                ("bytes_device", ctypes.c_longlong), ("bytes_device_peak", ctypes.c_longlong),
                ("n_graph_launches", ctypes.c_longlong), ("pi_ksplit_last", ctypes.c_int)]


KERNEL_CLASSES = ["pi_tcgen05", "pi_simt", "w_table_factor", "w_table_reduce", "minres_operator_gemm", "minres_recurrence",
                  "fallback_pi_dense", "fallback_lu", "fallback_refine"]


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def load(path: str = LIB_PATH):
    """Load libgw.so; raises FileNotFoundError if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} missing: build it with `python -m paper_2107_10423_gb300.build`")
    lib = ctypes.CDLL(path)
    lib.gw_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.gw_config_default.restype = None
    lib.gw_plan_create.argtypes = [ctypes.POINTER(Config), _P, _P, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_uint,
                                   _P, ctypes.POINTER(_P)]
    lib.gw_plan_create_uks.argtypes = [ctypes.POINTER(Config), _P, _P, ctypes.c_int, _P, _P, _P, _P, _P,
                                       ctypes.c_int, _P, _P, _P, ctypes.c_uint, _P, ctypes.POINTER(_P)]
    lib.gw_plan_create_uks.restype = ctypes.c_int
    lib.gw_polarizability.argtypes = [_P, _P, ctypes.c_int, _P]
    lib.gw_sigma_cd.argtypes = [_P, _P, _P, _P, _P]
    lib.gw_residues_minres.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    lib.gw_sigma_points.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
    lib.gw_sigma_sd.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
    lib.gw_qp_solve.argtypes = [_P, ctypes.c_int, _P, _P, _P]
    lib.gw_evgw.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P, _P]
    lib.gw_evgw.restype = ctypes.c_int
    lib.gw_set_shard.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _P]
    lib.gw_set_shard.restype = ctypes.c_int
    lib.gw_shard_columns.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
    lib.gw_shard_columns.restype = ctypes.c_int
    lib.gw_get_stats.argtypes = [_P, ctypes.POINTER(Stats)]
    lib.gw_w_table_noalloc.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int, _P]
    lib.gw_w_table_noalloc.restype = ctypes.c_int
    lib.gw_w_table.argtypes = [_P, _P]
    lib.gw_w_table.restype = ctypes.c_int
    lib.gw_plan_footprint.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.c_uint,
                                      ctypes.POINTER(ctypes.c_ulonglong)]
    lib.gw_plan_footprint.restype = ctypes.c_int
    lib.gw_grid.argtypes = [ctypes.c_int, ctypes.c_double, _P, _P]
    lib.gw_grid.restype = ctypes.c_int
    lib.gw_plan_destroy.argtypes = [_P]
    lib.gw_plan_destroy.restype = None
    lib.gw_last_error.argtypes = [_P]
    lib.gw_last_error.restype = ctypes.c_char_p
    for f in ["gw_plan_create", "gw_polarizability", "gw_sigma_cd", "gw_residues_minres", "gw_qp_solve",
              "gw_get_stats"]:
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def default_config(**kw) -> Config:
    c = Config()
    load().gw_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def grid(n: int, x0: float = 0.5):
    """The library's built-in modified Gauss-Legendre grid (host only)."""
    xi, wt = np.empty(n), np.empty(n)
    st = load().gw_grid(int(n), float(x0), _ptr(xi), _ptr(wt))
    if st != GW_OK:
        raise GWError(st, "gw_grid")
    return xi, wt


def footprint(n_occ, n_virt, n_aux, n_targets, borrow=False, **config) -> int:
    """Upper bound on a plan's device bytes (gw_plan_footprint; host only)."""
    cfg = default_config(n_occ=int(n_occ), n_virt=int(n_virt), n_aux=int(n_aux), **config)
    out = ctypes.c_ulonglong()
    st = load().gw_plan_footprint(ctypes.byref(cfg), int(n_targets), GW_BORROW_DEVICE_PTRS if borrow else 0,
                                  ctypes.byref(out))
    if st != GW_OK:
        raise GWError(st, "gw_plan_footprint")
    return int(out.value)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class Plan:
    """One G0W0 problem resident on the GPU.

    ``B_ia`` [n_aux, n_occ*n_virt] and ``B_nm`` [n_targets, n_bas, n_aux] are float64 numpy arrays (copied to the
    device) or float64 CUDA torch tensors (borrowed in place when ``borrow`` is true, otherwise copied on device)."""

    def __init__(self, eps, n_occ, B_ia, B_nm, targets, vxc=None, xi=None, wt=None, borrow=True, stream=None,
                 **config):
        lib = load()
        self._lib = lib
        self.eps = np.ascontiguousarray(eps, dtype=np.float64)
        n_bas = len(self.eps)
        n_aux = B_ia.shape[0]
        cfg = default_config(n_occ=int(n_occ), n_virt=int(n_bas - n_occ), n_aux=int(n_aux), **config)
        self.cfg = cfg
        self.targets = np.ascontiguousarray(targets, dtype=np.int32)
        self.n_t = len(self.targets)
        flags = 0
        if _is_torch_cuda(B_ia):
            assert _is_torch_cuda(B_nm) and B_ia.is_contiguous() and B_nm.is_contiguous()
            flags = GW_BORROW_DEVICE_PTRS if borrow else GW_INPUT_ON_DEVICE
            self._keep = (B_ia, B_nm)
            pb, pn = ctypes.c_void_p(B_ia.data_ptr()), ctypes.c_void_p(B_nm.data_ptr())
        else:
            self._keep = (np.ascontiguousarray(B_ia, dtype=np.float64), np.ascontiguousarray(B_nm, dtype=np.float64))
            pb, pn = _ptr(self._keep[0]), _ptr(self._keep[1])
        vx = None if vxc is None else np.ascontiguousarray(vxc, dtype=np.float64)
        xa = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
        wa = None if wt is None else np.ascontiguousarray(wt, dtype=np.float64)
        if xa is not None:
            cfg.n_freq = len(xa)
        self._grid = (vx, xa, wa)
        h = ctypes.c_void_p()
        st = lib.gw_plan_create(ctypes.byref(cfg), _ptr(self.eps), pb, pn, _ptr(self.targets), self.n_t, _ptr(vx),
                                _ptr(xa), _ptr(wa), flags, ctypes.c_void_p(stream) if stream else None,
                                ctypes.byref(h))
        if st != GW_OK:
            raise GWError(st, lib.gw_last_error(None).decode())
        self._h = h

    @classmethod
    def open_shell(cls, eps_a, eps_b, n_occ_a, n_occ_b, B_ia_a, B_ia_b, B_nm, targets, spins, vxc=None, xi=None,
                   wt=None, stream=None, **config):
        """Open-shell plan (gw_plan_create_uks): host float64 arrays (B_ia_a [n_aux, n_occ_a*n_virt_a], B_ia_b
        [n_aux, n_occ_b*n_virt_b], B_nm [n_targets, n_bas, n_aux] in each target's spin), spins 0/1 per target."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self.eps = np.ascontiguousarray(eps_a, dtype=np.float64)
        eb = np.ascontiguousarray(eps_b, dtype=np.float64)
        n_bas = len(self.eps)
        cfg = default_config(n_occ=int(n_occ_a), n_virt=int(n_bas - n_occ_a), n_aux=int(B_ia_a.shape[0]), **config)
        self.cfg = cfg
        self.targets = np.ascontiguousarray(targets, dtype=np.int32)
        sp = np.ascontiguousarray(spins, dtype=np.int32)
        self.n_t = len(self.targets)
        ba = np.ascontiguousarray(B_ia_a, dtype=np.float64)
        bb = np.ascontiguousarray(B_ia_b, dtype=np.float64)
        bn = np.ascontiguousarray(B_nm, dtype=np.float64)
        vx = None if vxc is None else np.ascontiguousarray(vxc, dtype=np.float64)
        xa = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
        wa = None if wt is None else np.ascontiguousarray(wt, dtype=np.float64)
        if xa is not None:
            cfg.n_freq = len(xa)
        self._keep = (ba, bb, bn, eb, sp)
        self._grid = (vx, xa, wa)
        h = ctypes.c_void_p()
        st = lib.gw_plan_create_uks(ctypes.byref(cfg), _ptr(self.eps), _ptr(eb), int(n_occ_b), _ptr(ba), _ptr(bb),
                                    _ptr(bn), _ptr(self.targets), _ptr(sp), self.n_t, _ptr(vx), _ptr(xa), _ptr(wa), 0,
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if st != GW_OK:
            raise GWError(st, lib.gw_last_error(None).decode())
        self._h = h
        return self

    def _check(self, st, allow=()):
        if st != GW_OK and st not in allow:
            raise GWError(st, self._lib.gw_last_error(self._h).decode())
        return st

    def polarizability(self, xi):
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1)
        n = self.cfg.n_aux
        out = np.empty((len(xi), n, n), dtype=np.float64)
        self._check(self._lib.gw_polarizability(self._h, _ptr(xi), len(xi), _ptr(out)))
        return out

    def screening(self):
        self._check(self._lib.gw_polarizability(self._h, None, 0, None))

    def w_table(self):
        out = np.empty((self.n_t, len(self.eps), self.cfg.n_freq + 1))
        self._check(self._lib.gw_w_table(self._h, _ptr(out)))
        return out

    def sigma_cd(self, omega):
        om = np.ascontiguousarray(omega, dtype=np.float64)
        sc, dsc, sx = (np.empty(self.n_t) for _ in range(3))
        self._check(self._lib.gw_sigma_cd(self._h, _ptr(om), _ptr(sc), _ptr(dsc), _ptr(sx)))
        return sc, dsc, sx

    def sigma_points(self, target_idx, omega):
        """Sigma_c and dSigma_c/domega at arbitrary (target, omega) pairs in one batched evaluation."""
        t = np.ascontiguousarray(target_idx, dtype=np.int32)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        sc, dsc = np.empty(len(t)), np.empty(len(t))
        self._check(self._lib.gw_sigma_points(self._h, len(t), _ptr(t), _ptr(om), _ptr(sc), _ptr(dsc)))
        return sc, dsc

    def sigma_sd(self, omega, target_idx=None):
        """Sigma_c and dSigma_c/domega by spectral decomposition (Casida), at omega[t] for every target, or at
        (target_idx[p], omega[p]) pairs."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        t = None if target_idx is None else np.ascontiguousarray(target_idx, dtype=np.int32)
        sc, dsc = np.empty(len(om)), np.empty(len(om))
        self._check(self._lib.gw_sigma_sd(self._h, len(om), None if t is None else _ptr(t), _ptr(om), _ptr(sc),
                                          _ptr(dsc)))
        return sc, dsc

    def residues(self, target_idx, m, x):
        t = np.ascontiguousarray(target_idx, dtype=np.int32)
        mm = np.ascontiguousarray(m, dtype=np.int32)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        k = len(t)
        out = {n: np.empty(k) for n in ("w_re", "w_im", "dw_re", "resnorm")}
        out["iters"] = np.empty(k, dtype=np.int32)
        out["used_fallback"] = np.empty(k, dtype=np.int32)
        self._check(self._lib.gw_residues_minres(self._h, k, _ptr(t), _ptr(mm), _ptr(xx), _ptr(out["w_re"]),
                                                 _ptr(out["w_im"]), _ptr(out["dw_re"]), _ptr(out["iters"]),
                                                 _ptr(out["resnorm"]), _ptr(out["used_fallback"])))
        return out

    def qp_solve(self, mode=GW_QP_STEPTREE, allow_unconverged=True):
        e, z = np.empty(self.n_t), np.empty(self.n_t)
        s = np.empty(self.n_t, dtype=np.int32)
        self._check(self._lib.gw_qp_solve(self._h, mode, _ptr(e), _ptr(z), _ptr(s)),
                    allow=(GW_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return e, z, s

    def evgw(self, update_w=False, mode=GW_QP_STEPTREE, max_iter=30, tol=1e-6, allow_unconverged=False):
        """Eigenvalue self-consistent GW (evGW0, or evGW with ``update_w``): (e_qp, z, status, cycles)."""
        e, z = np.empty(self.n_t), np.empty(self.n_t)
        s = np.empty(self.n_t, dtype=np.int32)
        it = ctypes.c_int()
        self._check(self._lib.gw_evgw(self._h, int(bool(update_w)), mode, int(max_iter), float(tol), _ptr(e), _ptr(z),
                                      _ptr(s), ctypes.byref(it)),
                    allow=(GW_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return e, z, s, it.value

    def set_shard(self, rank, world, allreduce_fn=None):
        """Split this plan's job across ``world`` ranks (gw_set_shard); ``allreduce_fn`` is a
        shard.ALLREDUCE_FN callback (kept alive by the plan)."""
        self._shard_cb = allreduce_fn
        fp = ctypes.cast(allreduce_fn, ctypes.c_void_p) if allreduce_fn is not None else None
        self._check(self._lib.gw_set_shard(self._h, int(rank), int(world), fp, None))

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.gw_get_stats(self._h, ctypes.byref(st)))
        out = {}
        for f, _ in Stats._fields_:
            v = getattr(st, f)
            out[f] = list(v) if f.endswith("_kernel") else v
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def plan_for(system, **kw) -> Plan:
    """Plan for a ``synth.System`` with host inputs."""
    return Plan(system.eps, system.n_occ, system.b_ia(), system.b_nm(), system.targets, **kw)
