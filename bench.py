"""Benchmark of the MRCM / MPM-2P pressure-update hot path (Algorithm 1 steps).

One "step" is one pass of Algorithm 1's loop over the whole workload: upwind transport,
kappa^n and epsilon, an MRCM basis rebuild or an MPM-2P reuse update, the interface
solve and the downscaling.  Metric: fine-cell pressure updates per second
(cells x realisations x timed steps / device time), all on the GPU.

Default workload "gaussian256": 256 x 256 cells, 16 x 16 subdomains of 16 x 16, log-normal
K (Gaussian covariance, variance 4, correlation length 0.05), viscosity ratio 5,
eta = 0.1, piecewise-linear interface spaces on 4-edge segments, alpha = 1, p = 1 / 0 on
the left / right, no flow top and bottom; the run continues Algorithm 1 for W + K steps
after its initial MRCM solve.  Inputs are synthetic and seeded.  The 256^2 working set
fits in L2, so L2 is flushed (a 256 MB write) between timed steps, outside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_11050_gb300 import fields  # noqa: E402

WORKLOAD = "gaussian256"
# dram__bytes_read.sum + dram__bytes_write.sum of one k_downscale_w launch (ncu capture of
# this code, see profiles/); None when the kernel changed since the capture.
TRAFFIC_DOWNSCALE_SOLVE = 8.717824e6
METRIC = "fine-cell pressure updates/s (MRCM & MPM-2P) at <=1e-8 rel flux err vs FP64"
UNIT = "cell-updates/s"
E2E_PASSES = 3
CFL = 0.5
N_SUB = 1


def workload_desc(w):
    return (f"{w['nx']}x{w['ny']} cells, {w['ncx']}x{w['ncy']} subdomains of {w['nx'] // w['ncx']}x"
            f"{w['ny'] // w['ncy']}, log-normal K ({w['cov']} covariance, variance {w['sigma2']}, "
            f"correlation length {w['ell']}), M={w['M']}, eta={w['eta']}, P1 interface spaces on 4-edge "
            f"segments, alpha=1, C_n={N_SUB}, CFL={CFL}")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(w, R=1):
    K, s0, _ = fields.make_workload(WORKLOAD)
    return np.ascontiguousarray(np.broadcast_to(K, (R, w["ny"], w["nx"]))), np.ascontiguousarray(
        np.broadcast_to(s0, (R, w["ny"], w["nx"])))


def setup_ctx(B, w, K, s0, prec, stream, R=1):
    ctx = B.Context(R, w["nx"], w["ny"], 1.0, 1.0, stream=stream)
    mode = {"fp32": B.PREC_FP32_IR, "fp32all": B.PREC_FP32_IR_ALL, "fp64": B.PREC_FP64}[prec]
    ctx.set_precision(mode, 1e-14, 30)
    ctx.set_fluids(w["M"])
    ctx.set_boundary((0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), 1.0)
    sd = w["nx"] // w["ncx"]
    ctx.set_decomposition([sd] * w["ncx"], [w["ny"] // w["ncy"]] * w["ncy"], 4, 1, 1.0)
    ctx.set_permeability(K)
    ctx.set_saturation(s0)
    return ctx


def algorithmic_downscale_solve(w):
    """Algorithmic work of one launch of the downscaling solve (all subdomains).

    Per a x b subdomain: one block-tridiagonal solve with explicit inverse pivots, 2b dense
    a x a matrix-vector products (4 b a^2 flop); one flux-form residual of the refinement
    check (14 flop per cell); the interior fine fluxes (2 faces x 2 flop per cell).  Bytes:
    the stored factor is read once (b a^2 float32), kappa-dependent stencil (32 B/cell), q
    (8 B/cell), the previous solution read and the new one written (16 B/cell), writes p~ and
    the interior fluxes (24 B/cell)."""
    a = w["nx"] // w["ncx"]
    b = w["ny"] // w["ncy"]
    nsub = w["ncx"] * w["ncy"]
    m = a * b
    flops = nsub * (4.0 * b * a * a + 14.0 * m + 4.0 * m)
    byts = nsub * (4.0 * b * a * a + 80.0 * m)
    return flops, byts


def run_gpu(args, w):
    import torch

    from paper_2103_11050_gb300 import binding as B
    from paper_2103_11050_gb300 import build as Bd

    Bd.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    cells = w["nx"] * w["ny"]
    K, s0 = make_inputs(w)
    eta = w["eta"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_run(prec, steps, warmup, profile):
        ctx = setup_ctx(B, w, K, s0, prec, stream.cuda_stream)
        ctx.set_execution(graph=not profile)  # the stage profiler times the eager launch sequence
        ctx.init(eta)
        for _ in range(warmup):
            ctx.step(eta, CFL, N_SUB)
        ctx.sync()
        if profile:
            ctx.profile_read()
            ctx.profile_enable(True)
        launches0 = ctx.get_stats()["kernel_launches"]
        st0 = ctx.get_stats()
        evs = []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step(eta, CFL, N_SUB)
                e1.record(stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        per = [a.elapsed_time(b) for a, b in evs]
        ms = sum(per)
        prof = ctx.profile_read() if profile else None
        st1 = ctx.get_stats()
        res = dict(ms=ms, per=per, launches=st1["kernel_launches"] - launches0,
                   rebuilds=st1["rebuilds"] - st0["rebuilds"], mpm=st1["mpm_updates"] - st0["mpm_updates"], prof=prof,
                   ir=st1["ir_iters_max"])
        ux, uy = ctx.get_flux()
        ctx.close()
        return res, ux

    prec = args.prec
    with ClockSampler(0) as clk:
        main, ux_main = one_run(prec, args.steps, args.warmup, False)
    value = cells * args.steps / (main["ms"] / 1e3)
    # rebuild and MPM-2P steps separately: a rebuild step costs several times an MPM-2P step,
    # so the timed rebuild steps are the slowest ones
    per = sorted(main["per"])
    n_reb = main["rebuilds"]
    mpm_part = per[:len(per) - n_reb] if n_reb < len(per) else per
    reb_part = per[len(per) - n_reb:] if n_reb > 0 else []
    split = {"mpm_step_ms": sum(mpm_part) / len(mpm_part),
             "mpm_step_ms_median": statistics.median(mpm_part),
             "rebuild_step_ms": (sum(reb_part) / len(reb_part)) if reb_part else None,
             "mpm_steps_rate": cells / (sum(mpm_part) / len(mpm_part) / 1e3),
             "rebuild_steps_rate": (cells / (sum(reb_part) / len(reb_part) / 1e3)) if reb_part else None}
    # same steps, eager launches with per-stage CUDA events (for the stage split and roofline)
    prof_run, _ = one_run(prec, args.steps, args.warmup, True)
    main["prof"] = prof_run["prof"]
    # the plain FP64 GPU form on the same steps, and the accuracy of the main form against it
    other = {}
    if prec != "fp64" and not args.no_fp64:
        f64, ux64 = one_run("fp64", args.steps, args.warmup, False)
        f64p, _ = one_run("fp64", args.steps, args.warmup, True)
        other = {"fp64_form_value": cells * args.steps / (f64["ms"] / 1e3),
                 "rel_flux_err_vs_fp64": float(np.linalg.norm(ux_main - ux64) / np.linalg.norm(ux64)),
                 "fp64_form_ms_per_step": f64["ms"] / args.steps,
                 "fp64_form_stage_ms_per_step_eager": {k: v[0] / args.steps for k, v in f64p["prof"].items()}}

    # end to end through the C ABI with host buffers: per step set s (h2d), step, read s (d2h).
    # Each pass replays the timed steps of the device measurement on a fresh context (same
    # initial state, same rebuild steps); the host clock of one pass is exposed to one-off
    # host stalls, so the median of the passes is reported.
    def e2e_pass():
        ctx = setup_ctx(B, w, K, s0, prec, stream.cuda_stream)
        ctx.init(eta)
        for _ in range(args.warmup):
            ctx.step(eta, CFL, N_SUB)
        s_host = torch.empty((1, w["ny"], w["nx"]), dtype=torch.float64).pin_memory().numpy()
        ctx.get_saturation(s_host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_saturation(s_host)
            ctx.step(eta, CFL, N_SUB)
            ctx.get_saturation(s_host)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        ctx.close()
        return t

    e2e_passes = [e2e_pass() for _ in range(E2E_PASSES)]
    e2e_s = statistics.median(e2e_passes)

    pk, pk_kind = peaks()
    prof = main["prof"]
    ds_ms, ds_n = prof["downscale"]
    dom = max(prof, key=lambda k: prof[k][0])
    flops, _bytes = algorithmic_downscale_solve(w)
    ds_avg_s = ds_ms / 1e3 / max(ds_n, 1)
    sm_clock = 2070.0
    fp64_peak = 152 * 2 * 2 * sm_clock * 1e6 / 1e12  # TFLOP/s
    roof = {"kernel": "k_downscale_w", "bound": "alu", "achieved": flops / ds_avg_s / 1e12,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": (flops / ds_avg_s / 1e12) / fp64_peak,
            "traffic": TRAFFIC_DOWNSCALE_SOLVE,
            "peak_kind": "derived: float64 pipe, 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (fallback table's "
                         "nominal 1.25 TFLOP/s; not in MEASURED_PEAKS.json)",
            "avg_launch_us": ds_avg_s * 1e6,
            "dominant_stage": dom,
            "stage_ms_per_step_eager": {k: v[0] / args.steps for k, v in prof.items()},
            "eager_ms_per_step": prof_run["ms"] / args.steps}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64ir" if prec != "fp64" else "f64", "data": "synthetic (seeded log-normal field)",
        "config": {"workload": f"{WORKLOAD}: {workload_desc(w)}", "realisations": 1,
                   "timed_steps_rebuild": main["rebuilds"], "timed_steps_mpm": main["mpm"],
                   "l2": "flushed between timed steps (256 MB write outside the timed region)",
                   "precision": {"fp32": "FP32 downscaling factorisations + FP64 refinement; FP64 Robin factors, "
                                          "interface, fluxes, transport",
                                 "fp32all": "FP32 local factorisations + FP64 refinement; FP64 interface, fluxes, "
                                            "transport",
                                 "fp64": "FP64 throughout"}[prec]},
        "gpu_launches": main["launches"],
        "e2e": {"value": cells * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * cells,
                "d2h_bytes_per_step": 8 * cells, "passes": [cells * args.steps / t for t in e2e_passes],
                "reported": f"median of {E2E_PASSES} passes, each the timed steps on a fresh context"},
        "roofline": roof,
        "clocks": clk.summary(),
        "peaks_source": pk_kind,
        "ir_sweeps_max": main["ir"],
        "step_split": split,
    }
    line.update(other)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    return line


def cpu_baseline(w, budget_s=20.0, max_steps=None):
    """The oracle, as it stands, timed on this host's cores on a bounded prefix of the
    workload (its initial MRCM solve is untimed; the timed steps are Algorithm 1 steps)."""
    from oracle import mpm_oracle as O
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        cores = os.cpu_count() or 1
    K, s0 = make_inputs(w)
    nx, ny = w["nx"], w["ny"]
    prob = O.Problem(nx, ny, 1.0 / nx, (0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), w["M"], 1.0)
    dec = O.uniform_decomposition(nx, ny, w["ncx"], w["ncy"], seg_len=4, degree=1)
    st = O.simulate_init(K[0], s0[0], prob, dec, w["eta"])
    n = 0
    t0 = time.perf_counter()
    reb = 0
    while time.perf_counter() - t0 < budget_s and (max_steps is None or n < max_steps):
        O.simulate_step(st, K[0], prob, dec, w["eta"], CFL, N_SUB)
        reb += st.history[-1]["rebuild"]
        n += 1
    dt = time.perf_counter() - t0
    return {"value": nx * ny * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} Algorithm 1 steps ({reb} rebuilds) of {WORKLOAD} after its initial MRCM solve, "
                      f"{dt:.1f} s of CPU time"}


def combine_ranks(ms_per_step, cells_per_rank, device):
    """Whole-job numbers of replicas on N ranks: the slowest rank's step time and the
    cell updates of all ranks over that time (weak scaling; the only collective is this
    max-reduction of one timing, the hot path itself exchanges nothing)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    t = torch.tensor([ms_per_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * cells_per_rank / (ms / 1e3)


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    budget = 150.0
    cb = cpu_baseline(w, budget_s=budget, max_steps=args.steps + args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": w["nx"] * w["ny"] / cb["value"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded log-normal field)",
            "config": {"workload": f"{WORKLOAD}: {workload_desc(w)}", "realisations": 1},
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=197)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp32all", "fp64"],
                    help="fp32: FP32 downscaling factors + FP64 refinement, FP64 Robin factors; "
                         "fp32all: every local factor FP32 + FP64 refinement; fp64: all FP64")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = fields.WORKLOADS[WORKLOAD]
    if args.impl == "reference":
        line = run_reference(args, w)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        # realisations are independent: each rank runs its own replica; value sums over ranks
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl")
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        args.no_cpu = args.no_cpu or dist.get_rank() != 0
        line = run_gpu(args, w)
        line["ms_per_step"], line["value"] = combine_ranks(line["ms_per_step"], w["nx"] * w["ny"], "cuda")
        line["n_gpus"] = world
        if dist.get_rank() == 0:
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    print(json.dumps(run_gpu(args, w)), flush=True)


if __name__ == "__main__":
    main()
