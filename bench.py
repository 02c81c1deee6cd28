"""Benchmark of the MRCM / MPM-2P pressure-update hot path (Algorithm 1 steps).

One "step" is one pass of Algorithm 1's loop over the whole workload: upwind transport,
kappa^n and epsilon, an MRCM basis rebuild or an MPM-2P reuse update, the interface
solve and the downscaling.  Metric: fine-cell pressure updates per second.

Default workload "channel1024": 1024 x 1024 cells, 64 x 64 subdomains of 16 x 16, binary
permeability with sinusoidal channels (K = 1 in channels of width 8..24 cells covering
30 % of the cells, 1e-4 elsewhere), viscosity ratio 5, eta = 0.1, piecewise-linear
interface spaces on 4-edge segments, alpha = 1, p = 1 / 0 on the left / right, no flow
top and bottom; mixed precision (FP32 downscaling factorisations with FP64 refinement).
Inputs are synthetic and seeded; L2 is flushed (a 256 MB write) before every timed step,
outside the timed region.

A rebuild step costs many MPM-2P steps, so a short window of K steps says little about the
workload's real mix.  The reported value is therefore the blended rate over the workload's
own rebuild mix:
  t_blend = f t_rebuild + (1 - f) t_mpm,  value = cells x R / t_blend,
where t_mpm is the mean device time of the MPM-2P steps of the K timed steps, t_rebuild the
mean of explicitly timed rebuild steps (a context with eta < 0 rebuilds at every step), and
f the fraction of rebuild steps over the workload's whole trajectory (its `steps`), which
this run executes and counts.  The K-window rate itself is reported as window_value.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec P]
                  [--impl reference]
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

METRIC = "fine-cell pressure updates/s (MRCM & MPM-2P) at <=1e-8 rel flux err vs FP64"
UNIT = "cell-updates/s"
E2E_PASSES = 3
CFL = 0.5
N_SUB = 1
FORCED_REBUILDS = 3
IR_TOL = 1e-14  # backward-error target of the FP64 refinement of float32 factors (--ir-tol)
# dram__bytes_read.sum + dram__bytes_write.sum of the step's kernels on the default workload
# (per launch; the interface sweeps: all levels of one solve), from an ncu capture of this
# code (profiles/counters_channel1024.md); a kernel is left out when it changed since.
TRAFFIC = {"k_downscale_w": 161.8e6, "k_mpm_local_w": 260.7e6, "k_upwind_kappa": 55.3e6, "k_nd_up": 309.7e6,
           "k_nd_down": 234.2e6}
PREC = {"fp32": "FP32 downscaling factorisations + FP64 refinement; FP64 Robin factors, interface, fluxes, "
                "transport",
        "fp32all": "FP32 local factorisations + FP64 refinement; FP64 interface, fluxes, transport",
        "fp64": "FP64 throughout"}
DTYPE = {"fp32": "f32+f64ir", "fp32all": "f32+f64ir", "fp64": "f64"}


class Workload:
    """Inputs and run parameters of one benchmark workload (all realisations)."""

    def __init__(self, name):
        self.name = name
        if name == "ensemble":
            Ks, s0, cw, rh, w = fields.make_ensemble()
            self.R = Ks.shape[0]
            self.K = Ks
            self.s0 = np.ascontiguousarray(np.broadcast_to(s0, Ks.shape))
            self.col_w, self.row_h = cw, rh
            self.desc = (f"ensemble: {self.R} realisations of {w['nx']}x{w['ny']}, log-normal K (exponential "
                         f"covariance, variance {w['sigma2']}, correlation length uniform in {w['ell_range']}), "
                         f"uneven decomposition (column widths {cw}, row heights {rh}), M={w['M']}, "
                         f"eta={w['eta']}")
        else:
            K, s0, w = fields.make_workload(name)
            self.R = 1
            self.K = np.ascontiguousarray(K[None])
            self.s0 = np.ascontiguousarray(s0[None])
            a, b = w["nx"] // w["ncx"], w["ny"] // w["ncy"]
            self.col_w, self.row_h = [a] * w["ncx"], [b] * w["ncy"]
            kind = w.get("field", "grf")
            if kind == "grf":
                fdesc = (f"log-normal K ({w['cov']} covariance, variance {w['sigma2']}, correlation length "
                         f"{w['ell']})")
            elif kind == "channelised":
                fdesc = (f"channelised binary K ({w['k_channel']} in sinusoidal channels of width {w['widths'][0]}-"
                         f"{w['widths'][1]} cells covering {w['coverage']:.0%}, {w['k_matrix']} elsewhere)")
            else:
                fdesc = "homogeneous K = 1, fingering initial saturation"
            self.desc = (f"{name}: {w['nx']}x{w['ny']} cells, {w['ncx']}x{w['ncy']} subdomains of {a}x{b}, {fdesc}, "
                         f"M={w['M']}, eta={w['eta']}")
        self.desc += f", P1 interface spaces on 4-edge segments, alpha=1, C_n={N_SUB}, CFL={CFL}"
        self.nx, self.ny = w["nx"], w["ny"]
        self.M, self.eta, self.steps = w["M"], w["eta"], w["steps"]
        self.cells = self.R * self.nx * self.ny


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


def setup_ctx(B, wl, prec, stream, tune=None):
    ctx = B.Context(wl.R, wl.nx, wl.ny, 1.0, wl.ny / wl.nx, stream=stream)
    if tune is not None:
        ctx.set_tuning(tune)
    mode = {"fp32": B.PREC_FP32_IR, "fp32all": B.PREC_FP32_IR_ALL, "fp64": B.PREC_FP64, "tf32": B.PREC_TF32_IR,
            "tf32x3": B.PREC_TF32X3_IR, "bf16": B.PREC_BF16_IR}[prec]
    ctx.set_precision(mode, IR_TOL, 30)
    ctx.set_fluids(wl.M)
    ctx.set_boundary((0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), 1.0)
    ctx.set_decomposition(wl.col_w, wl.row_h, 4, 1, 1.0)
    ctx.set_permeability(wl.K)
    ctx.set_saturation(wl.s0)
    return ctx


def iface_work(nodes):
    """Algorithmic work of one interface solve: (bytes, flops) of the upward step of the level-1
    nodes (done inside the MPM-2P local solve), of the upward sweep kernels (levels 2 and up) and
    of the downward sweep kernels.  An upward step reads the node's separator rows of its
    transposed frontal matrix once (nsep x nf float64) and its gathered right-hand side and
    output (2 nf float64), one multiply-add per matrix entry; a downward step reads the coupling
    block nbnd x nsep (nodes: nd_sizes)."""
    def up(levels):
        sel = [(ns, nf) for ns, nf, lev in nodes if ns > 0 and levels(lev)]
        return sum(8.0 * ns * nf + 16.0 * nf for ns, nf in sel), sum(2.0 * ns * nf for ns, nf in sel)
    # the downward kernels visit the levels between the root (final after the upward sweep) and
    # level 1 (done inside the reconstruction)
    inner = [(ns, nf) for ns, nf, lev in nodes[:-1] if lev >= 2 and ns > 0]
    down = (sum(8.0 * ns * (nf - ns) + 16.0 * ns for ns, nf in inner), sum(2.0 * ns * (nf - ns) for ns, nf in inner))
    return up(lambda lev: lev == 1), up(lambda lev: lev >= 2), down


def local_work(col_w, row_h, R, fp32_factor):
    """Algorithmic work of the single-right-hand-side local kernels over all subdomains:
    (bytes, flops) of the MPM-2P local solve (stored float64 factor read once, b a^2 values;
    the block solve's 2b products of a x a blocks, 4 b a^2 flops; the fine residual, 14 flops
    and 80 bytes of stencil, pressures, conductivities, transmissibilities and source per
    cell) and of the downscaling solve (its factor in the factor type; one block solve; one
    flux-form residual; the interior fluxes; 80 bytes per cell of stencil, source, warm start,
    outputs)."""
    mb = md = fm = fd = 0.0
    fac = 4.0 if fp32_factor else 8.0
    for b in row_h:
        for a in col_w:
            m = a * b
            mb += 8.0 * b * a * a + 80.0 * m
            fm += 4.0 * b * a * a + 14.0 * m
            md += fac * b * a * a + 80.0 * m
            fd += 4.0 * b * a * a + 18.0 * m
    return (R * mb, R * fm), (R * md, R * fd)


def nd_sizes(col_w, row_h, seg_len=4, degree=1):
    """(nsep, nf, level) of every internal nested-dissection node of the interface system, with
    the bisection the library uses (the longer side of each rectangle of subdomains is split in
    half), children before parents (the root last)."""
    ncx, ncy = len(col_w), len(row_h)
    nb = degree + 1
    vdofs = [2 * (row_h[J] // seg_len) * nb for J in range(ncy)]
    hdofs = [2 * (col_w[I] // seg_len) * nb for I in range(ncx)]
    out = []

    def rec(I0, I1, J0, J1):
        if I1 - I0 == 1 and J1 - J0 == 1:
            return 0
        if I1 - I0 >= J1 - J0:
            Im = (I0 + I1) // 2
            lev = 1 + max(rec(I0, Im, J0, J1), rec(Im, I1, J0, J1))
            nsep = sum(vdofs[J] for J in range(J0, J1))
        else:
            Jm = (J0 + J1) // 2
            lev = 1 + max(rec(I0, I1, J0, Jm), rec(I0, I1, Jm, J1))
            nsep = sum(hdofs[I] for I in range(I0, I1))
        bnd = 0
        for J in range(J0, J1):
            bnd += vdofs[J] * ((I0 > 0) + (I1 < ncx))
        for I in range(I0, I1):
            bnd += hdofs[I] * ((J0 > 0) + (J1 < ncy))
        out.append((nsep, nsep + bnd, lev))
        return lev

    rec(0, ncx, 0, ncy)
    return out


def run_gpu(args, wl):
    import torch

    from paper_2103_11050_gb300 import binding as B
    from paper_2103_11050_gb300 import build as Bd

    from paper_2103_11050_gb300 import autotune as AT

    Bd.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cells = wl.cells
    tunes = {}

    def tuning(prec):
        """Launch shapes of this workload and precision: from the cache, or autotuned once on a
        context that has run its initialisation and three steps."""
        if args.no_tune:
            return None
        if prec not in tunes:
            key = AT.shape_key(wl.R, wl.nx, wl.ny, wl.col_w, wl.row_h, prec, torch.cuda.get_device_name())
            hit = AT.cached(key, B.TUNE_KEYS)
            if hit is not None:  # no context needed
                tunes[prec] = (hit, "cache")
                return hit
            ctx = setup_ctx(B, wl, prec, stream.cuda_stream)
            ctx.init(wl.eta)
            for _ in range(3):
                ctx.step(wl.eta, CFL, N_SUB)
            tunes[prec] = AT.tuned(ctx, key)
            ctx.close()
        return tunes[prec][0]

    def timed_steps(ctx, n, eta, flags=None):
        """n steps, each bracketed by CUDA events on the launching stream after an L2 flush;
        with flags (a list), whether any realisation rebuilt in each step is appended."""
        evs = []
        last = ctx.get_stats()["rebuilds"] if flags is not None else 0
        with torch.cuda.stream(stream):
            for _ in range(n):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step(eta, CFL, N_SUB)
                e1.record(stream)
                evs.append((e0, e1))
                if flags is not None:  # a host read between steps, outside the timed region
                    now = ctx.get_stats()["rebuilds"]
                    flags.append(now != last)
                    last = now
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def trajectory(prec, profile=False):
        """init, W warm-up steps, the K timed steps, then the rest of the workload's trajectory."""
        ctx = setup_ctx(B, wl, prec, stream.cuda_stream, tuning(prec))
        # the stage profiler times the eager launch sequence
        ctx.set_execution(graph=not (profile or args.eager))
        ctx.init(wl.eta)
        for _ in range(args.warmup):
            ctx.step(wl.eta, CFL, N_SUB)
        ctx.sync()
        if profile:
            ctx.profile_read()
            ctx.profile_enable(True)
        st0 = ctx.get_stats()
        flags = []
        per = timed_steps(ctx, args.steps, wl.eta, flags)
        st1 = ctx.get_stats()
        prof = ctx.profile_read() if profile else None
        ux, uy = ctx.get_flux()
        res = dict(per=per, flags=flags, launches=st1["kernel_launches"] - st0["kernel_launches"],
                   rebuild_steps=sum(flags), ir=st1["ir_iters_max"], prof=prof, ux=ux, uy=uy,
                   ds_fact=st1["ds_factorisations"] - st0["ds_factorisations"])
        if not profile:
            rest = max(0, wl.steps - args.warmup - args.steps) if not args.no_trajectory else 0
            if rest:
                timed_steps(ctx, rest, wl.eta)
            st2 = ctx.get_stats()
            res["traj_steps"] = args.warmup + args.steps + rest
            res["traj_rebuilds"] = st2["rebuilds"] - wl.R  # realisation rebuilds, the initial build excluded
        ctx.close()
        return res

    def forced(prec, eta, n, profile=False):
        """Steps of one kind timed explicitly: eta < 0 makes every step after the first a rebuild,
        eta = 1e300 makes every step an MPM-2P update."""
        ctx = setup_ctx(B, wl, prec, stream.cuda_stream, tuning(prec))
        ctx.set_execution(graph=not profile)
        ctx.init(eta)
        for _ in range(3):
            ctx.step(eta, CFL, N_SUB)
        ctx.sync()
        if profile:
            ctx.profile_read()
            ctx.profile_enable(True)
        per = timed_steps(ctx, n, eta)
        prof = ctx.profile_read() if profile else None
        ctx.close()
        return per, prof

    def blend(prec, main, reb_per):
        mpm = [t for t, f in zip(main["per"], main["flags"]) if not f]
        src = "the MPM-2P steps of the timed window"
        if not mpm:  # every window step rebuilt some realisation: time MPM-2P steps explicitly
            mpm, _ = forced(prec, 1e300, args.steps)
            src = "explicitly timed MPM-2P steps (eta = 1e300)"
        t_mpm = sum(mpm) / len(mpm)
        t_reb = sum(reb_per) / len(reb_per)
        f = main["traj_rebuilds"] / max(wl.R * main["traj_steps"], 1)
        t = f * t_reb + (1.0 - f) * t_mpm
        return t, dict(mpm_step_ms=t_mpm, mpm_step_ms_median=statistics.median(mpm), mpm_steps_from=src,
                       rebuild_step_ms=t_reb, rebuild_steps_from=f"{len(reb_per)} explicitly timed rebuild steps",
                       rebuild_fraction=f, trajectory_steps=main["traj_steps"],
                       trajectory_rebuilds=main["traj_rebuilds"], mpm_steps_rate=cells / (t_mpm / 1e3),
                       rebuild_steps_rate=cells / (t_reb / 1e3))

    prec = args.prec
    if args.window_only:
        args.no_trajectory = True
        main = trajectory(prec)
        return {"metric": METRIC, "window_value": cells * args.steps / (sum(main["per"]) / 1e3), "unit": UNIT,
                "steps": args.steps, "warmup": args.warmup, "timed_steps_rebuild": main["rebuild_steps"],
                "gpu_launches": main["launches"], "config": {"workload": wl.desc, "precision": PREC[prec], "ir_tol": IR_TOL,
                                                             "tuning": tunes.get(prec)}}
    with ClockSampler(0) as clk:
        main = trajectory(prec)
        reb_per, _ = forced(prec, -1.0, FORCED_REBUILDS)
        t_blend, step_split = blend(prec, main, reb_per)
        # downscaling factorisations computed in the window, as a fraction of subdomains x steps
        # (the rest kept their stored float32 factor, mpm_set_downscale_reuse)
        step_split["downscale_factorised_fraction"] = main["ds_fact"] / (
            len(wl.col_w) * len(wl.row_h) * wl.R * args.steps)
    value = cells / (t_blend / 1e3)
    window_ms = sum(main["per"])
    _, prof_main = forced(prec, 1e300, args.steps, profile=True)
    _, prof_reb = forced(prec, -1.0, FORCED_REBUILDS, profile=True)

    other = {}
    if prec != "fp64" and not args.no_fp64:
        f64 = trajectory("fp64")
        f64_reb, _ = forced("fp64", -1.0, FORCED_REBUILDS)
        t64, split64 = blend("fp64", f64, f64_reb)
        num = np.sqrt(np.sum((main["ux"] - f64["ux"]) ** 2) + np.sum((main["uy"] - f64["uy"]) ** 2))
        den = np.sqrt(np.sum(f64["ux"] ** 2) + np.sum(f64["uy"] ** 2))
        other = {"fp64_form_value": cells / (t64 / 1e3), "fp64_form_ms_per_step": t64,
                 "fp64_form_step_split": split64,
                 "rel_flux_err_vs_fp64": float(num / den),
                 "rel_flux_err_vs_fp64_at": f"after init + {args.warmup + args.steps} steps (ux and uy together)"}

    # Precision study of the rebuild's basis-function solves: a rebuild step (eta < 0) in each
    # mode, its device time, the refinement sweeps it needed, whether every refinement
    # converged, and its fluxes against the plain FP64 form after the same steps.
    def precision_study():
        out, ref = {}, None
        for p in ("fp64", "fp32all", "tf32", "tf32x3", "bf16"):
            ctx = setup_ctx(B, wl, p, stream.cuda_stream)
            ctx.init(-1.0)
            ctx.step(-1.0, CFL, N_SUB)
            ctx.sync()
            per = timed_steps(ctx, 2, -1.0)
            try:
                ctx.sync()
                conv = True
            except B.MPMError as e:
                conv = e.code != B.MPM_ERR_NOT_CONVERGED
            ux, uy = ctx.get_flux() if conv else (None, None)
            st = ctx.get_stats()
            ctx.close()
            rec = {"rebuild_step_ms": min(per), "ir_sweeps_max": st["ir_iters_max"], "converged": conv}
            if p == "fp64":
                ref = (ux, uy)
            elif conv:
                num = np.sqrt(np.sum((ux - ref[0]) ** 2) + np.sum((uy - ref[1]) ** 2))
                rec["rel_flux_err_vs_fp64"] = float(num / np.sqrt(np.sum(ref[0] ** 2) + np.sum(ref[1] ** 2)))
            out[p] = rec
        return out

    study = None if args.no_study else precision_study()

    # Other workloads of the same path, for context: config 1 (64^2, a rebuild at every step:
    # the MRCM cost the RCR model counts), config 2 (256^2) and config 4 (the ensemble):
    # device time per step of each kind (graph launches, L2 flushed before each step).
    # The ensemble (config 4: 256 realisations of 128^2 on the uneven decomposition) gets its
    # own autotuned shapes and its blended rate over its own 500-step trajectory.
    def secondary():
        out = {}
        for name in ("gaussian64", "gaussian256", "ensemble"):
            w2 = Workload(name)
            tune = None
            if name == "ensemble" and not args.no_tune:
                key = AT.shape_key(w2.R, w2.nx, w2.ny, w2.col_w, w2.row_h, prec, torch.cuda.get_device_name())
                ctx = setup_ctx(B, w2, prec, stream.cuda_stream)
                ctx.init(w2.eta)
                for _ in range(3):
                    ctx.step(w2.eta, CFL, N_SUB)
                tune, _ = AT.tuned(ctx, key)
                ctx.close()
            per = {}
            for kind, eta in (("rebuild", -1.0), ("mpm", 1e300)):
                ctx = setup_ctx(B, w2, prec, stream.cuda_stream, tune)
                ctx.init(eta)
                for _ in range(3):
                    ctx.step(eta, CFL, N_SUB)
                t = timed_steps(ctx, 10 if name != "ensemble" else 4, eta)
                ctx.close()
                per[kind] = statistics.median(t)
            rec = {"cells": w2.cells, "rebuild_step_ms": per["rebuild"], "mpm_step_ms": per["mpm"],
                   "rebuild_steps_rate": w2.cells / (per["rebuild"] / 1e3),
                   "mpm_steps_rate": w2.cells / (per["mpm"] / 1e3)}
            if name == "ensemble":
                ctx = setup_ctx(B, w2, prec, stream.cuda_stream, tune)
                ctx.init(w2.eta)
                for _ in range(w2.steps):
                    ctx.step(w2.eta, CFL, N_SUB)
                f = (ctx.get_stats()["rebuilds"] - w2.R) / (w2.R * w2.steps)
                ctx.close()
                t_bl = f * per["rebuild"] + (1 - f) * per["mpm"]
                rec.update({"workload": w2.desc, "rebuild_fraction": f, "blended_rate": w2.cells / (t_bl / 1e3),
                            "tuning": tune})
            out[name] = rec
        return out

    small = None if args.no_study else secondary()

    # End to end through the C ABI with host buffers: per step the saturation is copied in from
    # pinned host memory, the step runs, and the saturation is read back.  MPM-2P steps
    # (eta = 1e300) and rebuild steps (eta < 0) are timed on fresh contexts and blended like
    # the device value; the median of E2E_PASSES passes of each is reported.
    def e2e_pass(eta, nsteps):
        ctx = setup_ctx(B, wl, prec, stream.cuda_stream, tuning(prec))
        ctx.init(eta)
        for _ in range(args.warmup):
            ctx.step(eta, CFL, N_SUB)
        s_host = torch.empty((wl.R, wl.ny, wl.nx), dtype=torch.float64).pin_memory().numpy()
        ctx.get_saturation(s_host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            ctx.set_saturation(s_host)
            ctx.step(eta, CFL, N_SUB)
            ctx.get_saturation(s_host)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        ctx.close()
        return t * 1e3 / nsteps

    e2e_mpm = [e2e_pass(1e300, args.steps) for _ in range(E2E_PASSES)]
    e2e_reb = [e2e_pass(-1.0, FORCED_REBUILDS) for _ in range(E2E_PASSES)]
    f = step_split["rebuild_fraction"]
    e2e_ms = f * statistics.median(e2e_reb) + (1.0 - f) * statistics.median(e2e_mpm)

    # Roofline of the step's kernels: algorithmic bytes and flops per step (iface_work,
    # local_work, the transport's 88 bytes and about 30 flops per cell) over the measured
    # device time per step of each (stage profiler, eager launches, L2 flushed), against the
    # HBM copy bandwidth and the float64 pipe (152 SMs x 2 FMA per clock x 2 flop x 2070 MHz,
    # derived: the measured-peaks file has no float64 figure).  Every kernel here is bound by
    # one of the two; the headline is the kernel with the largest stage time, with the bound
    # whose fraction is larger.
    pk, pk_kind = peaks()
    fp64_peak = 152 * 2 * 2 * 2070e6 / 1e12
    stage = {k: v[0] / max(args.steps, 1) for k, v in prof_main.items()}
    reb_stage = {k: v[0] / FORCED_REBUILDS for k, v in prof_reb.items()}
    (u1b, u1f), (ub, uf), (db, df) = iface_work(nd_sizes(wl.col_w, wl.row_h))
    (lb, lf), (dsb, dsf) = local_work(wl.col_w, wl.row_h, wl.R, prec != "fp64")
    # the MPM-2P local solve also does the upward step of the level-1 nodes
    lb, lf = lb + u1b * wl.R, lf + u1f * wl.R
    work = {"k_mpm_local_w": ("perturb", lb, lf), "k_downscale_w": ("downscale", dsb, dsf),
            "k_upwind_kappa": ("transport", 88.0 * cells, 30.0 * cells),
            "k_nd_up": ("iface_up", ub * wl.R, uf * wl.R), "k_nd_down": ("iface_down", db * wl.R, df * wl.R)}
    kern = {}
    for name, (st_name, byts, flops) in work.items():
        ms = stage.get(st_name, 0.0)
        if ms <= 0:
            continue
        gbs = byts / (ms / 1e3) / 1e9
        tfs = flops / (ms / 1e3) / 1e12
        kern[name] = {"ms_per_step": ms, "bytes": byts, "flops": flops, "gbs": gbs, "frac_hbm": gbs / pk["hbm_gbs"],
                      "tflops": tfs, "frac_fp64": tfs / fp64_peak,
                      "traffic": TRAFFIC.get(name) if wl.name == "channel1024" and prec == "fp32" else None}
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    kd = kern[dom]
    alu = kd["frac_fp64"] >= kd["frac_hbm"]
    roof = {"kernel": dom, "bound": "alu" if alu else "hbm",
            "achieved": kd["tflops"] if alu else kd["gbs"], "peak": fp64_peak if alu else pk["hbm_gbs"],
            "unit": "TFLOP/s" if alu else "GB/s", "frac": kd["frac_fp64"] if alu else kd["frac_hbm"],
            "traffic": kern[dom]["traffic"],
            "peak_kind": ("derived float64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz" if alu
                          else f"{pk_kind} HBM copy bandwidth"),
            "kernels": kern, "stage_ms_per_mpm_step_eager": stage, "stage_ms_per_rebuild_step_eager": reb_stage}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_blend, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic (seeded permeability field)",
        "config": {"workload": wl.desc, "realisations": wl.R,
                   "value": "blended over the workload's rebuild mix: cells / (f t_rebuild + (1-f) t_mpm)",
                   "timed_steps_rebuild": main["rebuild_steps"], "timed_steps_mpm": args.steps - main["rebuild_steps"],
                   "l2": "flushed before every timed step (256 MB write outside the timed region)",
                   "precision": PREC[prec], "ir_tol": IR_TOL,
                   "tuning": None if args.no_tune else {"values": tunes[prec][0], "source": tunes[prec][1]}},
        "window_value": cells * args.steps / (window_ms / 1e3),
        "gpu_launches": main["launches"],
        "e2e": {"value": cells / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * cells,
                "d2h_bytes_per_step": 8 * cells,
                "reported": f"blended like value; median of {E2E_PASSES} passes of {args.steps} MPM-2P steps and of "
                            f"{FORCED_REBUILDS} rebuild steps, each pass on a fresh context",
                "mpm_step_ms": statistics.median(e2e_mpm), "rebuild_step_ms": statistics.median(e2e_reb)},
        "roofline": roof,
        "clocks": clk.summary(),
        "peaks_source": pk_kind,
        "ir_sweeps_max": main["ir"],
        "step_split": step_split,
        "other_workloads": small,
        "precision_study": {"what": "rebuild steps (init + 3 rebuild steps, the last two timed) per precision mode of "
                                    "the local solves; basis-function solves on tensor cores in tf32, tf32x3, bf16",
                            "modes": study},
    }
    line.update(other)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget, gpu_check=(B, stream))
    return line


def oracle_sample(wl):
    """The bounded sample the oracle runs: the workload itself when its grid is at most 256^2
    per realisation (first realisation), else its 256 x 256 lower-left window with the same
    subdomain size, boundary conditions and fluids (the oracle's cost per cell is about
    constant, so the rate of the window stands for the whole grid)."""
    n = 256
    if wl.nx <= n and wl.ny <= n:
        return wl.K[0], wl.s0[0], wl.col_w, wl.row_h, "the workload's first realisation"
    a, b = wl.col_w[0], wl.row_h[0]
    K = np.ascontiguousarray(wl.K[0, :n, :n])
    s0 = np.ascontiguousarray(wl.s0[0, :n, :n])
    return K, s0, [a] * (n // a), [b] * (n // b), f"the lower-left {n}x{n} window of the workload"


def cpu_baseline(wl, budget_s=20.0, max_steps=None, gpu_check=None):
    """The oracle, as it stands, timed on this host's cores on a bounded sample of the
    workload (its initial MRCM solve is untimed; the timed steps are Algorithm 1 steps).
    With gpu_check, the GPU path runs the same sample for the same steps and its relative
    flux error against the oracle is reported."""
    from oracle import mpm_oracle as O
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        cores = os.cpu_count() or 1
    K, s0, cw, rh, what = oracle_sample(wl)
    ny, nx = K.shape
    prob = O.Problem(nx, ny, 1.0 / nx, (0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), wl.M, 1.0)
    dec = O.Decomposition(nx, ny, cw, rh, seg_len=4, degree=1)
    st = O.simulate_init(K, s0, prob, dec, wl.eta)
    n = 0
    t0 = time.perf_counter()
    reb = 0
    while time.perf_counter() - t0 < budget_s and (max_steps is None or n < max_steps):
        O.simulate_step(st, K, prob, dec, wl.eta, CFL, N_SUB)
        reb += st.history[-1]["rebuild"]
        n += 1
    dt = time.perf_counter() - t0
    out = {"value": nx * ny * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{what}: {n} Algorithm 1 steps ({reb} rebuilds) after its initial MRCM solve, "
                     f"{dt:.1f} s of CPU time"}
    if gpu_check is not None:
        B, stream = gpu_check
        errs = {}
        for prec in ("fp32", "fp64"):
            ctx = B.Context(1, nx, ny, 1.0, ny / nx, stream=stream.cuda_stream)
            ctx.set_precision({"fp32": B.PREC_FP32_IR, "fp64": B.PREC_FP64}[prec], IR_TOL, 30)
            ctx.set_fluids(wl.M)
            ctx.set_boundary((0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), 1.0)
            ctx.set_decomposition(cw, rh, 4, 1, 1.0)
            ctx.set_permeability(np.ascontiguousarray(K[None]))
            ctx.set_saturation(np.ascontiguousarray(s0[None]))
            ctx.init(wl.eta)
            for _ in range(n):
                ctx.step(wl.eta, CFL, N_SUB)
            ux, uy = ctx.get_flux()
            ctx.close()
            num = np.sqrt(np.sum((ux[0] - st.step.Fx) ** 2) + np.sum((uy[0] - st.step.Fy) ** 2))
            den = np.sqrt(np.sum(st.step.Fx ** 2) + np.sum(st.step.Fy ** 2))
            errs[prec] = float(num / den)
        out["gpu_rel_flux_err_vs_oracle"] = {"mixed_fp32_ir": errs["fp32"], "fp64": errs["fp64"],
                                             "at": f"{what}, after init + {n} steps"}
    return out


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


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cb = cpu_baseline(wl, budget_s=150.0, max_steps=args.steps + args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wl.cells / cb["value"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded permeability field)",
            "config": {"workload": wl.desc, "realisations": wl.R},
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def breakthrough_study(args, wl):
    """The fingering workload run to breakthrough (water saturation above 0.01 in the outlet
    column, checked every 10 steps, at most the workload's step count) for several rebuild
    thresholds and both GPU forms: steps to breakthrough, rebuilds, device time per step."""
    import torch

    from paper_2103_11050_gb300 import binding as B
    from paper_2103_11050_gb300 import build as Bd

    Bd.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    out = []
    for prec in ("fp32", "fp64"):
        for eta in (0.05, 0.1, 0.2):
            ctx = setup_ctx(B, wl, prec, stream.cuda_stream)
            ctx.init(eta)
            ms, n, bt = 0.0, 0, None
            with torch.cuda.stream(stream):
                while n < wl.steps and bt is None:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(10):
                        ctx.step(eta, CFL, N_SUB)
                    e1.record(stream)
                    s = ctx.get_saturation()
                    ms += e0.elapsed_time(e1)
                    n += 10
                    if s[:, :, -1].max() > 0.01:
                        bt = n
            st = ctx.get_stats()
            eps, reb = ctx.get_eps_history(4096)
            ctx.close()
            out.append({"prec": prec, "eta": eta, "breakthrough_step": bt, "steps_run": n,
                        "rebuilds": st["rebuilds"] - 1, "ms_per_step": ms / n,
                        "eps_max": float(eps.max()) if eps.size else None})
    return {"study": "fingering to breakthrough", "workload": wl.desc, "unit": "steps, ms", "runs": out}


def main():
    global IR_TOL
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=197)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="channel1024",
                    choices=["channel1024", "gaussian256", "finger512", "gaussian64", "ensemble"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp32all", "fp64"],
                    help="fp32: FP32 downscaling factors + FP64 refinement, FP64 Robin factors; "
                         "fp32all: every local factor FP32 + FP64 refinement; fp64: all FP64")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-trajectory", action="store_true",
                    help="do not run the workload's trajectory past the timed window (rebuild mix of the window)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-tune", action="store_true", help="default launch shapes instead of the autotuned ones")
    ap.add_argument("--no-study", action="store_true", help="skip the precision study of the rebuild step")
    ap.add_argument("--breakthrough", action="store_true",
                    help="run the workload to breakthrough for eta = 0.05, 0.1, 0.2 (fingering study) and print that")
    ap.add_argument("--window-only", action="store_true",
                    help="run only init, the warm-up and the timed window and print its rate: the command "
                         "profiled for the kernel launch list")
    ap.add_argument("--eager", action="store_true",
                    help="with --window-only: launch the steps kernel by kernel instead of as one CUDA graph (ncu "
                         "does not profile the kernels of graphs with conditional nodes)")
    ap.add_argument("--ir-tol", type=float, default=IR_TOL,
                    help="backward-error target of the FP64 refinement of the float32 factors")
    args = ap.parse_args()
    IR_TOL = args.ir_tol
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = Workload(args.workload)
    if args.breakthrough:
        print(json.dumps(breakthrough_study(args, wl)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, wl)
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
        line = run_gpu(args, wl)
        line["ms_per_step"], line["value"] = combine_ranks(line["ms_per_step"], wl.cells, "cuda")
        line["n_gpus"] = world
        if dist.get_rank() == 0:
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    print(json.dumps(run_gpu(args, wl)), flush=True)


if __name__ == "__main__":
    main()
