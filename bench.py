#!/usr/bin/env python
"""Benchmark of the CD-G0W0 hot path on GB300: QP states/s for the (H2O)_16-shaped workload.

One step = one complete G0W0 job on resident inputs: the imaginary-axis screening (Pi(i xi) on the
128-point grid and xi = 0, factorisation, W table) followed by the QP solve of all 74 target states
(I-term quadrature, residues by batched MINRES with dense fallback, QP update).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--qp linearised|steptree]
  python bench.py --impl reference     # the FP64 CPU oracle on host cores (bounded sample, extrapolated)
"""
from __future__ import annotations

import argparse
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


# ------------------------------------------------------------------------------------------ reference arm
def oracle_sample(system, B, Bn, n_res_total, n_freq=128):
    """Time the FP64 oracle on a bounded sample of the job: the imaginary-axis stage at one grid frequency
    (Pi, LU solve and W for every target row) and one dense real-axis residue; extrapolate to the whole job
    (n_freq + 1 frequencies, n_res_total residues).  Returns (seconds per job, sample description)."""
    import numpy as np
    from oracle import gw_oracle as O
    xi, wt = O.mgl_grid(n_freq, 0.5)
    t0 = time.perf_counter()
    Pi = O.pi_imag(system.eps, system.n_occ, B, xi[n_freq // 2])
    for t in range(Bn.shape[0]):
        O.w_corr(Pi, Bn[t].T)
    t_freq = time.perf_counter() - t0
    t0 = time.perf_counter()
    n = system.targets[0]
    m = n + 1
    x = system.eps[m] - system.eps[n]
    O.w_corr_and_deriv(O.pi_complex(system.eps, system.n_occ, B, x, 1e-3),
                       O.dpi_complex(system.eps, system.n_occ, B, x, 1e-3), Bn[0, m])
    t_res = time.perf_counter() - t0
    job = (n_freq + 1) * t_freq + n_res_total * t_res
    desc = (f"oracle imaginary-axis stage at 1 of {n_freq + 1} frequencies ({t_freq:.2f} s) + 1 of {n_res_total} "
            f"dense residue solves ({t_res:.2f} s), extrapolated to one job")
    return job, desc


def count_residues(system):
    from oracle import gw_oracle as O
    return sum(len(O.residue_set(system.eps, system.n_occ, system.eps[n])) for n in system.targets)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2107_10423_gb300 import synth
    s = synth.workload(1)
    B, Bn = s.b_ia(), s.b_nm()
    n_res = count_residues(s)
    vals = []
    desc = ""
    for it in range(args.warmup + args.steps):
        job, desc = oracle_sample(s, B, Bn, n_res)
        if it >= args.warmup:
            vals.append(len(s.targets) / job)
    v = sum(vals) / len(vals)
    cores = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "QP states/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": len(s.targets) / v * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(s, "fp64-oracle", "linearised"),
           "cpu_baseline": {"value": v, "unit": "QP states/s", "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "QP states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _config(s, precision, qp):
    return {"workload": f"{s.name}-shaped CD-G0W0: N_occ {s.n_occ}, N_bas {s.n_bas}, N_aux {s.n_aux}, "
                        f"{len(s.targets)} QP states (all valence + 10 lowest virtual), 128-point imaginary grid + xi=0, "
                        f"eta 1e-3, MINRES 25/5e-5 with dense fallback above 1e-4",
            "precision": precision, "qp_solver": qp, "global_batch": len(s.targets),
            "l2": "inputs larger than L2 (B_ia 784 MB FP64 / 392 MB BF16 hi+lo per operand)",
            "parallelism": "replicas"}


# ------------------------------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--qp", default="linearised", choices=["linearised", "steptree"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-accuracy", action="store_true", help="same as --accuracy none")
    ap.add_argument("--accuracy", choices=("sample", "all", "none"), default="sample",
                    help="mixed path against the FP64 GPU path: HOMO, LUMO and the deepest valence state (sample), "
                         "or every target state (all: the FP64 residue solves take about 15 minutes on water16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=32)
    ap.add_argument("--serve-nmax", type=int, default=16)
    ap.add_argument("--workload", default="water16", choices=["water16", "water8"],
                    help="water16: the (H2O)_16-shaped job (default); water8: a smaller case for profiler captures")
    args = ap.parse_args()
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
    from paper_2107_10423_gb300 import gw, synth
    gw.load()

    s = synth.workload(1) if args.workload == "water16" else synth.water_cluster(8, 8, targets="valence")
    B_h, Bn_h = s.b_ia(), s.b_nm()
    dev = torch.device("cuda", local)
    B_d = torch.from_numpy(B_h).to(dev)
    Bn_d = torch.from_numpy(Bn_h).to(dev)
    prec = gw.GW_PREC_MIXED if args.precision == "mixed" else gw.GW_PREC_FP64
    mode = gw.GW_QP_LINEARISED if args.qp == "linearised" else gw.GW_QP_STEPTREE
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ws = 0 if args.workload == "water16" else 512      # the profiling case keeps a few GB on the device
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

    # per-kernel-class rates over the timed region
    peaks, peak_src = _peaks()
    classes = gw.KERNEL_CLASSES
    dms = [st1["ms_kernel"][i] - st0["ms_kernel"][i] for i in range(len(classes))]
    dfl = [st1["flops_kernel"][i] - st0["flops_kernel"][i] for i in range(len(classes))]
    dln = [st1["launches_kernel"][i] - st0["launches_kernel"][i] for i in range(len(classes))]
    phases = {classes[i]: {"ms": round(dms[i], 3), "launches": int(dln[i]),
                           "tflops_alg": (round(dfl[i] / dms[i] / 1e9, 3) if dms[i] > 0 and dfl[i] > 0 else None)}
              for i in range(len(classes)) if dln[i] > 0}
    dom = max(range(len(classes)), key=lambda i: dms[i])
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_cls = dom == 8 or prec != gw.GW_PREC_MIXED   # class 8 time is dominated by its FP64 operator
    if dom in (0, 6) and prec == gw.GW_PREC_MIXED:
        # BF16 hi+lo: three BF16 products per algorithmic multiply-add -> peak = BF16 peak / 3
        roof = {"bound": "tensor", "peak": peaks["bf16_tflops_sustained"] / 3.0, "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16_tflops_sustained / 3 (three BF16 products per FMA)"}
    else:
        # SIMT FMA pipe: 152 SMs x 128 FP32 lanes (FP64: 1 TFLOP/s measured class) x 2 flops x SM clock
        fp32 = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        p = 1.0 if fp64_cls else fp32
        roof = {"bound": "alu", "peak": p, "unit": "TFLOP/s",
                "peak_source": ("FP64 FMA rate measured on this GB300 (DFMA microbenchmark, 1.0 TFLOP/s)" if fp64_cls
                                else "152 SM x 128 FP32 lanes x 2 x max SM clock")}
    ach = dfl[dom] / dms[dom] / 1e9 if dms[dom] > 0 else 0.0
    roof.update({"kernel": classes[dom], "achieved": round(ach, 3), "frac": round(ach / roof["peak"], 4),
                 "traffic": None, "launches": int(dln[dom]), "ms_per_launch": round(dms[dom] / max(1, dln[dom]), 4)})
    pi_cls = 0 if prec == gw.GW_PREC_MIXED else 1
    pi_tflops = dfl[pi_cls] / dms[pi_cls] / 1e9 if dms[pi_cls] > 0 else None

    # end to end through the public API with host buffers (pinned), H2D + solve + D2H inside the region
    B_pin = torch.from_numpy(B_h).pin_memory()
    Bn_pin = torch.from_numpy(Bn_h).pin_memory()
    Bh, Bnh = B_pin.numpy(), Bn_pin.numpy()
    e2e_ms = []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gw.Plan(s.eps, s.n_occ, Bh, Bnh, s.targets, precision=prec, stream=stream.cuda_stream,
                     workspace_mb=ws) as p2:
            p2.screening()
            e2, z2, st2 = p2.qp_solve(mode)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = len(s.targets) * world / (sum(e2e_ms) / len(e2e_ms) / 1e3)
    h2d = B_h.nbytes + Bn_h.nbytes + s.eps.nbytes + 4 * len(s.targets)
    d2h = 3 * 8 * len(s.targets)

    out = {"metric": METRIC, "value": round(value, 4), "unit": "QP states/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3+f32+f64" if prec == gw.GW_PREC_MIXED else "f64", "data": "synthetic",
           "config": _config(s, args.precision, args.qp),
           "roofline": roof, "pi_tflops": round(pi_tflops, 3) if pi_tflops else None, "phases": phases,
           "gpu_launches": int(st1["n_kernel_launches"] - st0["n_kernel_launches"]),
           "e2e": {"value": round(e2e_val, 4), "unit": "QP states/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "clocks": clocks,
           "minres": {"rhs_per_step": (st1["n_rhs_solved"] - st0["n_rhs_solved"]) // args.steps,
                      "fallback_per_step": (st1["n_fallback"] - st0["n_fallback"]) // args.steps,
                      "fp64_refined_per_step": (st1["n_refine_fp64"] - st0["n_refine_fp64"]) // args.steps,
                      "iters_per_step": (st1["n_minres_iters"] - st0["n_minres_iters"]) // args.steps},
           "qp_status_counts": {str(k): int((status == k).sum()) for k in (0, 1, 2)}}

    acc_mode = "none" if args.no_accuracy else args.accuracy
    if rank == 0 and acc_mode != "none" and prec == gw.GW_PREC_MIXED:
        # per-state error of the mixed path against the FP64 GPU path, same QP solver and MINRES settings
        if acc_mode == "all":
            idx = list(range(len(s.targets)))
        else:
            idx = [int(np.where(s.targets == s.n_occ - 1)[0][0]), int(np.where(s.targets == s.n_occ)[0][0]), 0]
        sub = s.with_targets(s.targets[idx])
        Bn_sub = Bn_d[idx].contiguous()
        t0 = time.perf_counter()
        with gw.Plan(sub.eps, sub.n_occ, B_d, Bn_sub, sub.targets, precision=gw.GW_PREC_FP64,
                     stream=stream.cuda_stream) as p64:
            e64, z64, st64 = p64.qp_solve(mode)
        err = np.abs(e_qp[idx] - e64)
        worst = int(np.argmax(err))
        out["accuracy"] = {"reference": "FP64 GPU path, same solver settings", "mode": acc_mode,
                           "states": [int(v) for v in sub.targets],
                           "abs_err_meV": [round(float(v) / MEV, 4) for v in err],
                           "max_abs_err_meV": round(float(err.max()) / MEV, 4),
                           "median_abs_err_meV": round(float(np.median(err)) / MEV, 4),
                           "worst_state": int(sub.targets[worst]),
                           "within_5meV": bool(err.max() < 5 * MEV),
                           "fp64_seconds": round(time.perf_counter() - t0, 2)}

    if rank == 0 and not args.no_serving:
        # continuous batching on a bounded prefix of the serving stream (Poisson arrivals at 4 jobs/s,
        # (H2O)_n with n log-uniform in [1, 64]; 30% O1s core jobs), same arrival times, versus the same jobs
        # run one after another on the same GPU
        from paper_2107_10423_gb300 import serve
        stream = synth.serving_stream()
        jobs = serve.make_jobs(stream, n_max=args.serve_nmax, limit=args.serve_jobs)
        def served(slots, at_zero):
            js = serve.make_jobs(stream, n_max=args.serve_nmax, limit=args.serve_jobs)
            if at_zero:
                for j in js:
                    j.arrival = 0.0
            t0 = time.perf_counter()
            done = serve.Server(max_slots=slots, hbm_budget=120 << 30).run(js)
            return serve.summarize(done, makespan=time.perf_counter() - t0)

        rnd = lambda d: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}
        live4, live1 = served(4, False), served(1, False)
        cap4, cap1 = served(4, True), served(1, True)
        out["serving"] = {"sample": f"first {len(jobs)} jobs with n <= {args.serve_nmax} of the 256-job stream "
                                    f"(Poisson arrivals over {jobs[-1].arrival:.1f} s), mixed precision, linearised QP",
                          "arrivals_4_slots": rnd(live4), "arrivals_1_slot": rnd(live1),
                          "capacity_jobs_per_s_4_slots": round(cap4["jobs_per_s"], 3),
                          "capacity_jobs_per_s_1_slot": round(cap1["jobs_per_s"], 3),
                          "capacity_p99_latency_s_4_slots": round(cap4["p99_latency_s"], 3)}

    if rank == 0 and not args.no_cpu_baseline:
        job, desc = oracle_sample(s, B_h, Bn_h, count_residues(s))
        out["cpu_baseline"] = {"value": round(len(s.targets) / job, 6), "unit": "QP states/s", "cores": os.cpu_count(),
                               "kind": "oracle", "sample": desc}
    plan.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
