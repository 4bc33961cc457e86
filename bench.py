#!/usr/bin/env python
"""Benchmark of the CD-G0W0 hot path on GB300: QP states/s of whole G0W0 jobs on synthetic inputs.

One step = one complete G0W0 job on resident inputs: the imaginary-axis screening (Pi(i xi) on the
128-point grid and xi = 0, factorisation, W table) followed by the QP solve of every target state
(I-term quadrature, residues by batched MINRES with dense fallback, QP update).  Prints one JSON line.

Workloads (seeded synthetic inputs shaped like the paper's systems):
  water64  (H2O)_64-shaped, N_aux 8064, N_ov 778,240, HOMO-15..LUMO+5 (22 states), mixed precision (default)
  water16  (H2O)_16-shaped, N_aux 2016, N_ov 48,640, 64 valence + 10 virtual states
  esca     ESCA-shaped core-level batch, N_aux 1800, the 6 C1s states by the step tree
  water8   (H2O)_8-shaped, a small case for profiler captures

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload W] [--precision mixed|fp64] [--qp ...]
  python bench.py --impl reference     # the FP64 CPU oracle on host cores (bounded sample, extrapolated)
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G0W0 QP states/s, mixed vs FP64 at <=5 meV; Pi TFLOP/s; p50/p99 job latency"
MEV = 3.6749322175655e-5
N_FREQ = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------ workloads
def workload(name):
    from paper_2107_10423_gb300 import synth
    if name == "water64":
        return synth.workload(2), "HOMO-15..LUMO+5"
    if name == "water16":
        return synth.workload(1), "all 64 valence + 10 lowest virtual"
    if name == "esca":
        return synth.workload(3), "the 6 C1s core states"
    if name == "water8":
        return synth.water_cluster(8, 8, targets="valence"), "all 32 valence + 10 lowest virtual"
    raise ValueError(name)


def _config(s, desc, precision, qp, l2):
    return {"workload": f"{s.name}-shaped CD-G0W0: N_occ {s.n_occ}, N_bas {s.n_bas}, N_aux {s.n_aux}, "
                        f"N_ov {s.n_ov}, {len(s.targets)} QP states ({desc}), {N_FREQ}-point imaginary grid + xi=0, "
                        f"eta 1e-3, MINRES 25/5e-5 with dense fallback above 1e-4",
            "precision": precision, "qp_solver": qp, "global_batch": len(s.targets), "l2": l2,
            "parallelism": "replicas"}


def _l2_note(s):
    gb = s.n_aux * s.n_ov * 4 / 1e9
    return (f"inputs larger than L2 (B_ia {s.n_aux * s.n_ov * 8 / 1e9:.1f} GB FP64, {gb:.1f} GB FP32 / BF16 hi+lo "
            f"per operand)")


# ------------------------------------------------------------------------------------------ reference arm
def count_residues(system):
    from oracle import gw_oracle as O
    return sum(len(O.residue_set(system.eps, system.n_occ, system.eps[n])) for n in system.targets)


def oracle_sample(system, n_res_total, r_max=256):
    """Time the FP64 oracle on a bounded sample of one job and extrapolate to the whole job.

    The sample takes the first r = min(N_aux, r_max) auxiliary rows of B_ia and of one target's B_nm: Pi(i xi) of
    that block at one grid frequency (time x (N_aux/r)^2 per frequency, as the work grows with N_aux^2 N_ov), the
    dense W solve of one target's rows with it (x (N_aux/r)^3 x N_targets), and one dense real-axis residue with its
    derivative (x (N_aux/r)^2: the complex Pi(x) build dominates).  Returns (seconds per job, description)."""
    from oracle import gw_oracle as O
    n = system.n_aux
    r = min(n, r_max)
    B = system.b_ia_rows(0, r)
    Bn0 = system.b_nm(system.targets[:1])[0][:, :r]
    xi, wt = O.mgl_grid(N_FREQ, 0.5)
    t0 = time.perf_counter()
    Pi = O.pi_imag(system.eps, system.n_occ, B, xi[N_FREQ // 2])
    t_pi = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.w_corr(Pi, Bn0.T)
    t_w = time.perf_counter() - t0
    nt = system.targets[0]
    m = nt + 1 if nt + 1 < system.n_bas else nt - 1
    x = system.eps[m] - system.eps[nt]
    t0 = time.perf_counter()
    O.w_corr_and_deriv(O.pi_complex(system.eps, system.n_occ, B, x, 1e-3),
                       O.dpi_complex(system.eps, system.n_occ, B, x, 1e-3), Bn0[m])
    t_res = time.perf_counter() - t0
    s2, s3 = (n / r) ** 2, (n / r) ** 3
    job = (N_FREQ + 1) * (t_pi * s2 + t_w * s3 * len(system.targets)) + n_res_total * t_res * s2
    desc = (f"oracle on the first {r} of {n} auxiliary rows: Pi(i xi) at 1 of {N_FREQ + 1} frequencies "
            f"({t_pi:.2f} s, x{s2:.0f}), W solve of 1 of {len(system.targets)} targets ({t_w:.2f} s, x{s3:.0f}), "
            f"1 of {n_res_total} dense residues ({t_res:.2f} s, x{s2:.0f}); extrapolated to one job")
    return job, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s, desc_t = workload(args.workload)
    n_res = count_residues(s)
    vals = []
    desc = ""
    for it in range(args.warmup + args.steps):
        job, desc = oracle_sample(s, n_res)
        if it >= args.warmup:
            vals.append(len(s.targets) / job)
    v = sum(vals) / len(vals)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "QP states/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": len(s.targets) / v * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(s, desc_t, "fp64-oracle", "linearised", _l2_note(s)),
           "cpu_baseline": {"value": v, "unit": "QP states/s", "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "QP states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------------------------------ our arm
def _flops_job(s, n_res, minres_iters, n_fb):
    """Algorithmic flops of one job per kernel class, for the FP64-path estimate (a multiply-add is 2)."""
    n, K, R, G = s.n_aux, s.n_ov, len(s.targets) * s.n_bas, N_FREQ + 1
    return {"pi_simt": G * n * n * K, "w_table_factor": G * n ** 3 / 3.0, "w_table_reduce": G * n * n * R,
            "minres_operator_gemm": 8.0 * n * K * (minres_iters + 1.5 * n_res),
            "fallback_pi_dense": 4.0 * n_fb * n * n * K, "fallback_lu": n_fb * 8.0 / 3.0 * n ** 3}


def fp64_rates(gw, dev, stream):
    """Rates (flop/s) of the FP64 GPU path's kernel classes, measured on an (H2O)_8-shaped job: the screening
    (Pi, Cholesky, triangular-solve W table) and one linearised QP evaluation (MINRES, dense fallback)."""
    import torch
    from paper_2107_10423_gb300 import synth
    s = synth.water_cluster(8, 8, targets=[35, 39, 40])
    B = torch.from_numpy(s.b_ia()).to(dev)
    Bn = torch.from_numpy(s.b_nm()).to(dev)
    with gw.Plan(s.eps, s.n_occ, B, Bn, s.targets, precision=gw.GW_PREC_FP64, stream=stream.cuda_stream) as p:
        p.screening()
        p.qp_solve(gw.GW_QP_LINEARISED)
        st = p.stats()
    rates = {}
    for i, c in enumerate(gw.KERNEL_CLASSES):
        if st["ms_kernel"][i] > 0 and st["flops_kernel"][i] > 0:
            rates[c] = st["flops_kernel"][i] / (st["ms_kernel"][i] / 1e3)
    return rates


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water64", choices=["water64", "water16", "esca", "water8"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--qp", default=None, choices=["linearised", "steptree"],
                    help="default: step tree for the core-level batch (esca), linearised otherwise")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-accuracy", action="store_true", help="same as --accuracy none")
    ap.add_argument("--accuracy", choices=("sample", "all", "none"), default="sample",
                    help="mixed path against the FP64 GPU path on the same job: HOMO, LUMO and the deepest target "
                         "(sample) or every target (all); water16, esca and water8 only (the FP64 path on water64 "
                         "would take hours: its rate is estimated instead)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=32)
    ap.add_argument("--serve-nmax", type=int, default=16)
    ap.add_argument("--workspace-mb", type=int, default=0)
    args = ap.parse_args()
    if args.qp is None:
        args.qp = "steptree" if args.workload == "esca" else "linearised"
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2107_10423_gb300 import gw
    gw.load()

    s, desc_t = workload(args.workload)
    t0 = time.perf_counter()
    B_h, Bn_h = s.b_ia(), s.b_nm()
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", local)
    B_d = torch.from_numpy(B_h).to(dev)
    Bn_d = torch.from_numpy(Bn_h).to(dev)
    prec = gw.GW_PREC_MIXED if args.precision == "mixed" else gw.GW_PREC_FP64
    mode = gw.GW_QP_LINEARISED if args.qp == "linearised" else gw.GW_QP_STEPTREE
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ws = args.workspace_mb if args.workspace_mb else (512 if args.workload == "water8" else 0)
    plan = gw.Plan(s.eps, s.n_occ, B_d, Bn_d, s.targets, precision=prec, stream=stream.cuda_stream, workspace_mb=ws)

    def step():
        plan.screening()
        return plan.qp_solve(mode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st0 = plan.stats()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e_qp, z, status = step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    from paper_2107_10423_gb300 import replicas
    ms, n_states, value = replicas.aggregate(e0.elapsed_time(e1), len(s.targets) * args.steps, device=dev)
    st1 = plan.stats()

    # per-kernel-class rates over the timed region (CUDA events on the plan's stream)
    peaks, peak_src = _peaks()
    classes = gw.KERNEL_CLASSES
    dms = [st1["ms_kernel"][i] - st0["ms_kernel"][i] for i in range(len(classes))]
    dfl = [st1["flops_kernel"][i] - st0["flops_kernel"][i] for i in range(len(classes))]
    dln = [st1["launches_kernel"][i] - st0["launches_kernel"][i] for i in range(len(classes))]
    phases = {classes[i]: {"ms": round(dms[i], 3), "launches": int(dln[i]),
                           "tflops_alg": (round(dfl[i] / dms[i] / 1e9, 3) if dms[i] > 0 and dfl[i] > 0 else None)}
              for i in range(len(classes)) if dln[i] > 0}
    mr = {"rhs_per_step": (st1["n_rhs_solved"] - st0["n_rhs_solved"]) // args.steps,
          "fallback_per_step": (st1["n_fallback"] - st0["n_fallback"]) // args.steps,
          "fp64_refined_per_step": (st1["n_refine_fp64"] - st0["n_refine_fp64"]) // args.steps,
          "iters_per_step": (st1["n_minres_iters"] - st0["n_minres_iters"]) // args.steps}
    # the MINRES operator streams B twice per iteration (B^T z, then B w): algorithmic bytes per launch pair are
    # 2 N_aux N_ov x (4 bytes: BF16 hi + lo in mixed precision, 8 in FP64)
    if "minres_operator_gemm" in phases and dms[4] > 0:
        bpe = 4 if prec == gw.GW_PREC_MIXED else 8
        n_it = dln[4]
        phases["minres_operator_gemm"]["hbm_gbs_alg"] = round(n_it * 2 * s.n_aux * s.n_ov * bpe / (dms[4] / 1e3) / 1e9,
                                                              1)
    dom = max(range(len(classes)), key=lambda i: dms[i])
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    bf16 = peaks["bf16_tflops_sustained"]
    if dom in (0, 2, 3, 4, 6) and prec == gw.GW_PREC_MIXED:
        # tensor-core classes: algorithmic flops against the BF16 peak; the hi/lo split costs three BF16 products
        # per algorithmic multiply-add, so the tensor pipe is busy about 3x the algorithmic fraction
        roof = {"bound": "tensor", "peak": bf16, "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16_tflops_sustained (BF16 hi/lo split: 3 products per algorithmic FMA)"}
    else:
        fp64_cls = dom == 8 or prec != gw.GW_PREC_MIXED
        fp32 = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "peak": 1.0 if fp64_cls else fp32, "unit": "TFLOP/s",
                "peak_source": ("FP64 FMA rate measured on this GB300 (DFMA microbenchmark, 1.0 TFLOP/s)" if fp64_cls
                                else "152 SM x 128 FP32 lanes x 2 x max SM clock")}
    ach = dfl[dom] / dms[dom] / 1e9 if dms[dom] > 0 else 0.0
    roof.update({"kernel": classes[dom], "achieved": round(ach, 3), "frac": round(ach / roof["peak"], 4),
                 "traffic": None, "launches": int(dln[dom]), "ms_per_launch": round(dms[dom] / max(1, dln[dom]), 4)})
    if roof["bound"] == "tensor":
        roof["tensor_pipe_frac_est"] = round(3 * ach / roof["peak"], 4)
    pi_cls = 0 if prec == gw.GW_PREC_MIXED else 1
    pi_tflops = dfl[pi_cls] / dms[pi_cls] / 1e9 if dms[pi_cls] > 0 else None
    launches = int(st1["n_kernel_launches"] - st0["n_kernel_launches"])
    plan.close()
    del plan, B_d, Bn_d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers (pinned in place), H2D + solve + D2H in the region
    cudart = torch.cuda.cudart()
    pinned = []
    for a in (B_h, Bn_h):
        if int(cudart.cudaHostRegister(a.ctypes.data, a.nbytes, 0)) == 0:
            pinned.append(a)
    e2e_ms = []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gw.Plan(s.eps, s.n_occ, B_h, Bn_h, s.targets, precision=prec, stream=stream.cuda_stream,
                     workspace_mb=ws) as p2:
            p2.screening()
            e2, z2, st2 = p2.qp_solve(mode)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    for a in pinned:
        cudart.cudaHostUnregister(a.ctypes.data)
    e2e_val = len(s.targets) * world / (sum(e2e_ms) / len(e2e_ms) / 1e3)
    h2d = B_h.nbytes + Bn_h.nbytes + s.eps.nbytes + 4 * len(s.targets)
    d2h = 3 * 8 * len(s.targets)

    out = {"metric": METRIC, "value": round(value, 4), "unit": "QP states/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3+f32+f64" if prec == gw.GW_PREC_MIXED else "f64", "data": "synthetic",
           "config": _config(s, desc_t, args.precision, args.qp, _l2_note(s)),
           "roofline": roof, "pi_tflops": round(pi_tflops, 3) if pi_tflops else None, "phases": phases,
           "gpu_launches": launches,
           "e2e": {"value": round(e2e_val, 4), "unit": "QP states/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "pinned_in_place": len(pinned) == 2},
           "clocks": clocks, "minres": mr,
           "qp_status_counts": {str(k): int((status == k).sum()) for k in (0, 1, 2)},
           "input_generation_s": round(t_gen, 1)}

    acc_mode = "none" if args.no_accuracy else args.accuracy
    if rank == 0 and prec == gw.GW_PREC_MIXED and args.workload == "water64":
        # FP64 GPU path on this job: its kernel rates measured here on an (H2O)_8-shaped job, applied to this job's
        # algorithmic flops per class (screening, MINRES operator, dense fallback)
        rates = fp64_rates(gw, dev, stream)
        fl = _flops_job(s, mr["rhs_per_step"], mr["iters_per_step"], mr["fallback_per_step"])
        t64 = sum(fl[c] / rates[c] for c in fl if c in rates and fl[c] > 0)
        out["fp64_gpu"] = {"states_per_s_est": round(len(s.targets) / t64, 6), "seconds_per_job_est": round(t64, 1),
                           "speedup_of_mixed_est": round(value / (len(s.targets) / t64), 1),
                           "method": "FP64 kernel-class rates measured in this run on an (H2O)_8-shaped job, applied "
                                     "to this job's algorithmic flops per class",
                           "rates_tflops": {c: round(v / 1e12, 3) for c, v in rates.items()}}
    elif rank == 0 and acc_mode != "none" and prec == gw.GW_PREC_MIXED:
        # per-state error of the mixed path against the FP64 GPU path, same QP solver and MINRES settings
        if acc_mode == "all":
            idx = list(range(len(s.targets)))
        else:
            cand = [int(np.argmin(np.abs(s.targets - (s.n_occ - 1)))), int(np.argmin(np.abs(s.targets - s.n_occ))),
                    0]
            idx = sorted(set(cand))
        sub = s.with_targets(s.targets[idx])
        t0 = time.perf_counter()
        with gw.Plan(sub.eps, sub.n_occ, B_h, Bn_h[idx], sub.targets, precision=gw.GW_PREC_FP64,
                     stream=stream.cuda_stream) as p64:
            e64, z64, st64 = p64.qp_solve(mode)
        t64 = time.perf_counter() - t0
        err = np.abs(e_qp[idx] - e64)
        worst = int(np.argmax(err))
        out["accuracy"] = {"reference": "FP64 GPU path, same solver settings", "mode": acc_mode,
                           "states": [int(v) for v in sub.targets],
                           "abs_err_meV": [round(float(v) / MEV, 4) for v in err],
                           "max_abs_err_meV": round(float(err.max()) / MEV, 4),
                           "median_abs_err_meV": round(float(np.median(err)) / MEV, 4),
                           "worst_state": int(sub.targets[worst]),
                           "within_5meV": bool(err.max() < 5 * MEV),
                           "fp64_seconds": round(t64, 2)}
        if acc_mode == "all":
            out["fp64_gpu"] = {"states_per_s": round(len(idx) / t64, 6),
                               "speedup_of_mixed": round(value / (len(idx) / t64), 1),
                               "method": "the FP64 GPU path on the same job, timed end to end (one job)"}

    if rank == 0 and not args.no_serving:
        # continuous batching on a bounded prefix of the serving stream (Poisson arrivals at 4 jobs/s,
        # (H2O)_n with n log-uniform in [1, 64]; 30% O1s core jobs), same arrival times, versus the same jobs
        # run one after another on the same GPU
        from paper_2107_10423_gb300 import serve, synth
        stream_jobs = synth.serving_stream()
        jobs = serve.make_jobs(stream_jobs, n_max=args.serve_nmax, limit=args.serve_jobs)

        def served(slots, at_zero, keep=None):
            js = serve.make_jobs(stream_jobs, n_max=args.serve_nmax, limit=args.serve_jobs)
            if at_zero:
                for j in js:
                    j.arrival = 0.0
            t0 = time.perf_counter()
            done = serve.Server(max_slots=slots).run(js)
            if keep is not None:
                keep.extend(done)
            return serve.summarize(done, makespan=time.perf_counter() - t0)

        rnd = lambda d: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}
        done4 = []
        live4, live1 = served(4, False, done4), served(1, False)
        cap4, cap1 = served(4, True), served(1, True)
        out["serving"] = {"sample": f"first {len(jobs)} jobs with n <= {args.serve_nmax} of the 256-job stream "
                                    f"(Poisson arrivals over {jobs[-1].arrival:.1f} s), mixed precision, linearised QP",
                          "arrivals_4_slots": rnd(live4), "arrivals_1_slot": rnd(live1),
                          "capacity_jobs_per_s_4_slots": round(cap4["jobs_per_s"], 3),
                          "capacity_jobs_per_s_1_slot": round(cap1["jobs_per_s"], 3),
                          "capacity_p99_latency_s_4_slots": round(cap4["p99_latency_s"], 3)}
        # serial plain-FP64 baseline: the sample's small jobs ((H2O)_n, n <= 3; an FP64 (H2O)_16 job alone takes
        # minutes) solved one after another in FP64, against their latency in the 4-slot mixed run above
        try:
            small = [j for j in done4 if j.system.meta.get("n_water", 99) <= 3 and "error" not in j.result]
            t64 = []
            for j in small:
                t0 = time.perf_counter()
                r = serve.run_job(j, precision="fp64")
                if "error" in r:
                    raise RuntimeError(r["error"])
                t64.append(time.perf_counter() - t0)
            if t64:
                lat = np.array([j.latency for j in small])
                out["serving"]["fp64_serial_small_jobs"] = {
                    "jobs": len(t64), "n_max": 3, "jobs_per_s": round(len(t64) / sum(t64), 3),
                    "p50_s": round(float(np.percentile(t64, 50)), 4), "p99_s": round(float(np.percentile(t64, 99)), 4),
                    "mixed_served_p50_s": round(float(np.percentile(lat, 50)), 4),
                    "mixed_served_p99_s": round(float(np.percentile(lat, 99)), 4)}
        except Exception as e:            # the baseline is a side measurement: report, do not lose the line
            out["serving"]["fp64_serial_small_jobs"] = {"error": repr(e)[:200]}

    if rank == 0 and not args.no_cpu_baseline:
        job, desc = oracle_sample(s, count_residues(s))
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        out["cpu_baseline"] = {"value": round(len(s.targets) / job, 6), "unit": "QP states/s", "cores": cores,
                               "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
