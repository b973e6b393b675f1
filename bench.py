#!/usr/bin/env python
"""Benchmark: seconds per sgn(H) b + d/dU (forward TSL + gauge-force VJP).

Workload (default): 14x14^3 lattice (V = 38416, n = 460992), SU(3) links
U = expm(i 0.2 A), mu = 0.3, m_w = -2, one Gaussian source, k = 800, one
Gaussian cotangent; FP64 throughout (at this point the k-step map amplifies
rounding by ~1e6 and FP32 basis vectors break the recurrence down; the
mixed-precision path is reported separately), pair-periodic
re-biorthogonalisation every 60 steps with one Gram-Schmidt pass (at this
point x stays within 1e-9 and dU within 1e-4 of the result with
re-biorthogonalisation at every step, for any period from 10 to 100, and the
error estimate eps_A is the same; every period pays the same Krylov
truncation error, ~1e-2).  One step = one ov_tsl_sign_vjp call (forward recurrence, sign,
x = V y, Frechet adjoint, reverse sweep, force, dmu) on inputs resident in
HBM; the Krylov bases (5.9 GB) exceed the 129 MB L2, so no flush is needed.

Reported beside the headline: live per-kernel device times (CUDA events on
the library's stream), the roofline of the dominant kernel, the Wilson-Dirac
stencil bandwidth on an L2-busting multi-source batch, the end-to-end time
through host buffers, clocks sampled during the timed region, the FP64 GPU
path's status and its speed and error on a well-conditioned point, and the FP64
oracle timed on a bounded sample on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1604_08057_gb300 import inputs  # noqa: E402

METRIC = "s per sgn(H)b + dsgn/dU at 14^4, k=800"
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
MIXED_SCHEDULES = (20, 10, 1)   # re-biorthogonalisation periods tried by the mixed-path leg


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="14x14^3")
    ap.add_argument("--k", type=int, default=0, help="override the workload's k")
    ap.add_argument("--precision", default="fp64", choices=["mixed", "fp64"])
    ap.add_argument("--rebiorth", type=int, default=None,
                    help="re-biorthogonalisation period P (default 60 for the headline workload, "
                         "20 for the uneven batch)")
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--segment", type=int, default=0,
                    help="two-pass TSL with checkpoints every S steps (needs --rebiorth 0)")
    ap.add_argument("--m-w", type=float, default=None, help="override the workload's Wilson mass")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, stencil, FP64 and CPU legs")
    ap.add_argument("--leg", default="all", choices=["all", "stencil", "batch", "kk", "deflation", "deflation8",
                                                     "nested", "nested_stage"],
                    help="stencil: only the multi-source Wilson-Dirac leg (for kernel profiling); "
                         "batch: the uneven batch of 32 problems (forward + VJP) through ov_tsl_batch; "
                         "kk: one k x k complex product (ov_kk_gemm), FP64 and split, at the workload's k; "
                         "nested: the nested TSL's k x k stage against the full sign at the workload; "
                         "nested_stage: that stage alone on a synthetic tridiagonal of the workload's k")
    args = ap.parse_args()
    # P = 60 at 14x14^3, k = 800: x within 1e-9 and dU within 1e-4 of the P = 1 result
    # (P = 20: 2e-10 and 4e-4), the same eps_A; the uneven batch keeps P = 20
    if args.rebiorth is None:
        args.rebiorth = 20 if args.leg == "batch" else 60
    if args.warmup < 1:
        ap.error("--warmup must be at least 1 (the last warm-up step gives the per-kernel breakdown)")
    return args


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    idx = int(parts[0])
                except ValueError:
                    continue
                rows.append((idx, parts))
        os.unlink(self.path)
        idxs = sorted({i for i, _ in rows})
        use = self.index if self.index in idxs else (idxs[0] if idxs else None)
        rows = [p for i, p in rows if i == use]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(p[1]) for p in rows if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in rows if p[2].replace(".", "").isdigit()]
        power = [float(p[3]) for p in rows if p[3].replace(".", "").isdigit()]
        reasons = set()
        for p in rows:
            for name, val in zip(REASONS, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes (what the method must move), FP32 real size e = 4, FP64 e = 8
# ---------------------------------------------------------------------------
def workload_of(args):
    import dataclasses
    wl = inputs.WORKLOADS[args.workload]
    return wl if args.m_w is None else dataclasses.replace(wl, m_w=args.m_w)


def rebiorth_steps(k, period):
    if period <= 0:
        return []
    return [j for j in range(k - 1) if period == 1 or (j + 1) % period in (0, 1)]


def algorithmic_bytes(kind, k, V, nsrc, e, period, passes):
    """Total algorithmic bytes of one ov_tsl_sign_vjp call for one kernel kind."""
    vec = 24 * e * V            # one spinor field
    links = 72 * e * V
    reb = rebiorth_steps(k, period)
    if kind == "stencil_pair":   # read r, s; write v, w, p, q; links once
        return k * (nsrc * 6 * vec + links)
    if kind == "update":         # read p, q, v_j, w_j, v_j-1, w_j-1; write r, s
        return (k - 1) * nsrc * 8 * vec
    if kind == "proj_dots":      # forward and reverse: read a, b and 2(j+1) basis vectors per pass
        return 2 * passes * nsrc * vec * sum(2 + 2 * (j + 1) for j in reb)
    if kind == "proj_update":    # read 2(j+1) basis vectors and a, b; write a, b
        return 2 * passes * nsrc * vec * sum(4 + 2 * (j + 1) for j in reb)
    if kind == "rev_stencil":    # read g_r, g_s, w_j, v_j, xbar, g_r', g_s'; write Gv, Gw, g_p; links
        acc = 0
        nrec = 0
        for j in range(k - 1, -1, -1):
            if j < k - 1 and j in set(reb):
                nrec += 1
            acc += 2 * nrec
        return k * (nsrc * 10 * vec + links) + nsrc * vec * acc
    if kind == "force":          # read g_p, v_j, w_j, g_q per step (x 4 directions re-read from cache)
        return nsrc * 4 * vec * k + 2 * 72 * 8 * V * ((k + 31) // 32)
    return None


H_FLOP_PER_SITE = 1368   # one Wilson H application on half spinors (8 hops + diagonal)


def algorithmic_flops(kind, k, V, nsrc, period, passes):
    """Algorithmic FP64 flops of one ov_tsl_sign_vjp call for the ALU-bound kinds.

    Gram-Schmidt kinds: 4 FMA (8 flop) per complex element and basis vector.
    stencil_pair: the two H applications and the alpha dot of each step, once
    (replayed segments are extra work, not algorithmic flops).
    rev_stencil, per site and step: H^dag g_p and H (conj(g_alpha) v_j + g_s)
    (2 x 1368), the seven single complex combinations of fields it adds (g_p,
    the H input, xbar, g_r, g_s and the two previous-step terms: 7 x 12 x 8),
    and 2 x 12 x 8 per recorded Gram-Schmidt projection still to be applied."""
    e64 = 8
    if kind in ("proj_dots", "proj_update"):
        basis = 2 * passes * nsrc * 24 * e64 * V * sum(2 * (j + 1) for j in rebiorth_steps(k, period))
        return basis / 16 * 8
    if kind == "stencil_pair":   # H v and H^dag w per step, and alpha = w^dag p (one forward sweep)
        return nsrc * V * k * (2 * H_FLOP_PER_SITE + 12 * 8)
    if kind == "rev_stencil":
        reb = set(rebiorth_steps(k, period))
        nrec, acc = 0, 0
        for j in range(k - 1, -1, -1):
            if j < k - 1 and j in reb:
                nrec += 1
            acc += 2 * 12 * 8 * nrec
        return nsrc * V * (k * (2 * H_FLOP_PER_SITE + 7 * 12 * 8) + acc)
    return None


def job_seconds_per_unit(ms_local, steps, world, device="cpu"):
    """(ms of the timed region, whole-job seconds per unit).  The region's time is
    the MAX over ranks; every rank runs one replica of the workload per step, so
    the job processes steps x world units in that time."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ms / 1e3 / (steps * world)


# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1604_08057_gb300 import binding

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = workload_of(args)
    k = args.k or wl.k
    u, b, xbar = inputs.make_inputs(wl)
    nsrc = b.shape[0]
    V = wl.volume
    ut, bt, xt = (torch.tensor(a, device=dev) for a in (u, b, xbar))
    ctx = binding.context(args.precision, args.rebiorth, args.passes, segment=args.segment)
    tune = binding.autotune(ut, wl.mu, wl.m_w, nsrc, args.precision, args.rebiorth, args.passes,
                            segment=args.segment)

    def step():
        return binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, args.precision, args.rebiorth, args.passes,
                                    return_info=True, segment=args.segment)

    info = None
    for i in range(args.warmup):
        if i == args.warmup - 1:
            # per-kind breakdown from the last warm-up step, every launch group timed
            binding.profile_enable(ctx, True)
            binding.profile_read(ctx, reset=True)
        du, dmu, x, info = step()
    torch.cuda.synchronize()
    prof_w = binding.profile_read(ctx, reset=True)
    e = 4 if args.precision == "mixed" else 8
    lattice = ["stencil_pair", "update", "proj_dots", "proj_update", "rev_stencil", "force"]
    dom = max(lattice, key=lambda kd: prof_w[kd][1])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # inside the timed region only the dominant kind carries event pairs
    binding.profile_select(ctx, [dom])
    binding.profile_read(ctx, reset=True)
    l0 = binding.launch_count(ctx)
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        du, dmu, x, info = step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = binding.launch_count(ctx) - l0
    prof = binding.profile_read(ctx, reset=True)
    binding.profile_select(ctx, None)
    binding.profile_enable(ctx, False)
    ms_total, value = job_seconds_per_unit(e0.elapsed_time(e1), args.steps, world, dev)

    # roofline of the dominant lattice kernel
    hbm, peak_src = hbm_peak()
    bytes_dom = algorithmic_bytes(dom, k, V, nsrc, e, args.rebiorth, args.passes) * args.steps
    gbs = bytes_dom / (prof[dom][1] / 1e3) / 1e9
    per_launch = {"launches": prof[dom][0], "avg_launch_us": round(1e3 * prof[dom][1] / max(1, prof[dom][0]), 2),
                  "algorithmic_bytes_per_launch": int(bytes_dom / max(1, prof[dom][0]))}
    if args.precision == "fp64" and dom in ("proj_dots", "proj_update", "rev_stencil", "stencil_pair"):
        flops = algorithmic_flops(dom, k, V, nsrc, args.rebiorth, args.passes) * args.steps
        achieved = flops / (prof[dom][1] / 1e3) / 1e12
        # FP64 ALU peak from unit counts and clock: 152 SMs x 2 FP64 FMA (4 flop) per
        # SM per clock (1.25 TFLOP/s nominal at 2070 MHz), at the median SM clock sampled
        sm_mhz = clk.get("sm_mhz") or 2070.0
        peak_alu = 152 * 4 * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak_alu, 4),
                    "unit": "TFLOP/s", "frac": round(achieved / peak_alu, 3),
                    "peak_source": f"derived: 152 SMs x 4 FP64 flop/clk x {sm_mhz:.0f} MHz (sampled)",
                    "fp64_gemm_measured_tflops": round(fp64_peak(dev) / 1e3, 3),
                    "frac_of_fp64_gemm": None,
                    "hbm_view": {"achieved_GB_s": round(gbs, 1), "peak": hbm, "frac": round(gbs / hbm, 3)},
                    **per_launch}
        roofline["frac_of_fp64_gemm"] = round(achieved / roofline["fp64_gemm_measured_tflops"], 3)
        if dom == "rev_stencil":
            # ncu: DRAM bytes of k_rev_stencil launches at 14x14^3, k = 120 = 0.845 x their
            # algorithmic bytes; launches differ only in how many fields they stream
            roofline["traffic"] = int(REV_STENCIL_TRAFFIC_RATIO * per_launch["algorithmic_bytes_per_launch"])
            roofline["traffic_source"] = ("ncu dram bytes of two k_rev_stencil launches at 14x14^3, k=120 "
                                          f"(ratio {REV_STENCIL_TRAFFIC_RATIO} to algorithmic), scaled to this "
                                          "launch average")
        elif dom == "proj_dots":
            # ncu: DRAM bytes of a two-sided k_proj_dots launch = 1.050 x its algorithmic
            # bytes (14x14^3, k = 120, nb = 101); traffic grows with the fields streamed
            roofline["traffic"] = int(PROJ_DOTS_TRAFFIC_RATIO * per_launch["algorithmic_bytes_per_launch"])
            roofline["traffic_source"] = ("ncu dram bytes of one k_proj_dots launch at 14x14^3, k=120, nb=101 "
                                          f"(ratio {PROJ_DOTS_TRAFFIC_RATIO} to algorithmic), scaled to this "
                                          "launch average")
        else:
            roofline["traffic"] = None
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(gbs / hbm, 3), "peak_source": peak_src, "traffic": None, **per_launch}
    kernels_ms = {kd: round(v[1], 3) for kd, v in prof_w.items() if v[0]}

    out = {"metric": METRIC, "value": round(value, 6), "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": f"{args.workload} lattice, k={k}, mu={wl.mu}, m_w={wl.m_w}, "
                                  f"{nsrc} source(s), forward + gauge-force VJP",
                      "precision": args.precision, "rebiorth_period": args.rebiorth, "segment": args.segment,
                      "gs_passes": args.passes,
                      "l2": "working set (Krylov bases) > L2; no flush", "parallelism": f"replicas x{world}"},
           "gpu_launches": launches // args.steps * args.steps, "kernels_ms_per_step": kernels_ms,
           "kernels_ms_source": "last warm-up step, every launch group event-timed",
           "phase_ms": [round(t, 3) for t in info["t_ms"][:6]], "newton_iters": [info["newton_iters"],
                                                                                  info["newton_iters_adj"]],
           "roofline": roofline, "clocks": clk, "autotune": tune}

    if not args.no_extras and rank == 0:
        out["forward_only"] = forward_leg(args, ut, bt, wl, k)
        out["e2e"] = e2e_leg(args, ut, bt, xt, wl, k)
        out["dw_stencil"] = stencil_leg(args, ut, wl, hbm, peak_src)
        out["mixed_path"] = mixed_leg(args, ut, bt, xt, wl, k, u, b, xbar)
        out["schedule_compare"] = schedule_leg(args, ut, bt, xt, wl, k, du, dmu, x)
        out["diagnostics"] = diagnostics_leg(args, ut, bt, xt, wl, k, ms_total / args.steps)
        out["kk_products"] = kk_products_leg(args, ut, bt, xt, wl, k, du, dmu, x, ms_total / args.steps)
        try:
            out["nested_tsl"] = nested_leg(args, ut, bt, wl, k)
        except Exception as exc:   # reported, not fatal: the leg is beside the headline
            out["nested_tsl"] = {"error": str(exc)}
        try:
            out["deflation"] = deflation_leg(ut.device.index)
        except Exception as exc:   # reported, not fatal: the leg is beside the headline
            out["deflation"] = {"error": str(exc)}
        out["basis_in_host_memory"] = host_basis_leg(args, ut, bt, xt, wl, k, du, dmu, x)
        out["other_workloads"] = other_workloads_leg(args)
        if world == 1:
            out["cpu_baseline"], out["parity"] = cpu_leg(args, k, ut)
    return out


PROJ_DOTS_TRAFFIC_RATIO = 1.050
REV_STENCIL_TRAFFIC_RATIO = 0.845


def hbm_peak():
    """(HBM copy bandwidth in GB/s, its source): the measured figure of
    MEASURED_PEAKS.json when present, else the profiling fallback of 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fp64_peak(dev, n=4096, reps=3):
    """cuBLAS float64 GEMM rate (context for the FP64 ALU roofline), GFLOP/s."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b)
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def forward_leg(args, ut, bt, wl, k, reps=2):
    """Seconds per sgn(H)b alone (ov_tsl_sign, same workload and schedule), device-timed."""
    import torch
    from paper_1604_08057_gb300 import binding
    opts = (args.precision, args.rebiorth, args.passes)
    binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, *opts, segment=args.segment)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        _, info = binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, *opts, return_info=True, segment=args.segment)
    e1.record()
    torch.cuda.synchronize()
    return {"value": round(e0.elapsed_time(e1) / 1e3 / reps, 6), "unit": "s per sgn(H)b", "steps": reps,
            "newton_iters": info["newton_iters"]}


def nested_leg(args, ut, bt, wl, k, inner=(60, 100, 150), reps=2):
    """The k x k stage of sgn(H) b by the nested TSL (Sec. 4.1: one nesting level,
    inner Krylov size m) against the full Newton sign of T_k, at this workload and
    schedule: seconds per ov_tsl_sign call and its k x k phase (device events), the
    relative difference of x from the full-sign x, eps_A (Eq. error_est) with and
    without nesting, and the k x k stage alone on the call's own T_k
    (ov_tridiag_sign_nested; host-timed, including the T_k upload and y download)."""
    import time
    import torch
    from paper_1604_08057_gb300 import binding
    opts = (args.precision, args.rebiorth, args.passes)

    def call(m):
        binding.nested_sign(m, *opts)
        binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, *opts)        # warm-up: capture, workspace
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            x, info = binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, *opts, return_info=True)
        e1.record()
        torch.cuda.synchronize()
        return x, {"s_per_call": round(e0.elapsed_time(e1) / 1e3 / reps, 4), "kk_ms": round(info["t_ms"][1], 3),
                   "newton_iters": info["newton_iters"]}

    def stage(a, b, d, m, n=3):
        binding.tridiag_sign_nested(a, b, d, m)
        t0 = time.perf_counter()
        for _ in range(n):
            y, _ = binding.tridiag_sign_nested(a, b, d, m)
        return y, round((time.perf_counter() - t0) / n * 1e3, 3)

    out = {"inner_sizes": list(inner), "reps": reps}
    try:
        x0, out["full"] = call(0)
        a, b, d = binding.tsl_coefficients(k, 0, *opts)
        y0, out["full"]["stage_ms"] = stage(a, b, d, 0)
        out["full"]["eps_a"] = float(binding.tsl_eps(ut, wl.mu, wl.m_w, bt, k, *opts)[0])
        for m in inner:
            x, r = call(m)
            r["rel_diff_x_vs_full"] = float((x - x0).norm() / x0.norm())
            y, r["stage_ms"] = stage(a, b, d, m)
            r["stage_rel_diff_y_vs_full"] = float(abs(y - y0).max() / abs(y0).max())
            if m == 100:
                r["eps_a"] = float(binding.tsl_eps(ut, wl.mu, wl.m_w, bt, k, *opts)[0])
            out[f"m{m}"] = r
    finally:
        binding.nested_sign(0, *opts)
    return out


def nested_stage_leg(k, inner=(60, 100, 150), reps=5, seed=11):
    """The k x k stage alone on a seeded synthetic tridiagonal of size k (no lattice):
    ms per ov_tridiag_sign_nested call for the full Newton sign (m = 0) and the nested
    form (host-timed, including the upload of T and the download of y)."""
    import time
    from paper_1604_08057_gb300 import binding
    a, b, d = inputs.tridiagonal_coefficients(k, np.random.default_rng(seed))
    out = {"k": k, "reps": reps}
    for m in (0,) + tuple(inner):
        binding.tridiag_sign_nested(a, b, d, m)
        t0 = time.perf_counter()
        for _ in range(reps):
            _, it = binding.tridiag_sign_nested(a, b, d, m)
        out[f"m{m}"] = {"ms": round((time.perf_counter() - t0) / reps * 1e3, 3), "newton_iters": it}
    return out


def schedule_leg(args, ut, bt, xt, wl, k, du, dmu, x, periods=(20,)):
    """The same call with other re-biorthogonalisation periods: device time and the
    distance of x, dU and dmu from the headline step's results."""
    import torch
    from paper_1604_08057_gb300 import binding
    res = {"headline_period": args.rebiorth}
    rel = lambda a, c: float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
    for period in periods:
        if period == args.rebiorth:
            continue
        try:
            binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, args.precision, period, args.passes)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            du_p, dmu_p, x_p = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, args.precision, period, args.passes)
            e1.record()
            torch.cuda.synchronize()
            res[f"P={period}"] = {"s_per_call": round(e0.elapsed_time(e1) / 1e3, 4),
                                  "rel_x_vs_headline": rel(x_p, x), "rel_dU_vs_headline": rel(du_p, du),
                                  "rel_dmu_vs_headline": abs(dmu_p - dmu) / abs(dmu)}
        except binding.OVError as exc:
            res[f"P={period}"] = f"status {exc.status}"
        except RuntimeError as exc:   # e.g. device memory: the headline line must still print
            res[f"P={period}"] = f"error: {exc}"
    return res


def other_workloads_leg(args, reps=3):
    """Seconds per forward + VJP call on the 4x4^3 (k = 200, one source) and 8x8^3
    (k = 400, four sources) workloads, FP64, projections every 20 steps, one pass,
    after autotuning and one warm-up call (device time over `reps` calls)."""
    import torch
    from paper_1604_08057_gb300 import binding
    res = {}
    dev = torch.device("cuda", torch.cuda.current_device())
    for name in ("4x4^3", "8x8^3"):
        wl = inputs.WORKLOADS[name]
        u, b, xbar = inputs.make_inputs(wl)
        ut, bt, xt = (torch.tensor(a, device=dev) for a in (u, b, xbar))
        opts = ("fp64", 20, 1)
        try:
            binding.autotune(ut, wl.mu, wl.m_w, b.shape[0], *opts)
            binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, wl.k, xt, *opts)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, wl.k, xt, *opts)
            e1.record()
            torch.cuda.synchronize()
            res[name] = {"s_per_call": round(e0.elapsed_time(e1) / 1e3 / reps, 4), "k": wl.k,
                         "sources": int(b.shape[0]), "rebiorth_period": 20}
        except binding.OVError as exc:
            res[name] = {"status": exc.status, "error": str(exc)}
    return res


def host_basis_leg(args, ut, bt, xt, wl, k, du, dmu, x):
    """The headline call with the Krylov bases in pinned host memory (read over the
    CPU-GPU link instead of HBM): seconds per call and whether the results equal
    the headline's bit for bit."""
    import torch
    from paper_1604_08057_gb300 import binding
    opts = (args.precision, args.rebiorth, args.passes)
    binding.basis_memory("host", *opts, segment=args.segment)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        du2, dmu2, x2 = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, *opts, segment=args.segment)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"s_per_call": round(dt, 4), "basis_bytes": 2 * k * 24 * 8 * wl.volume,
                "identical_to_headline": bool(torch.equal(du2, du) and torch.equal(x2, x) and dmu2 == dmu)}
    except (binding.OVError, RuntimeError) as exc:
        return {"error": str(exc)}
    finally:
        binding.basis_memory("device", *opts, segment=args.segment)


def deflation_leg(dev_index, dims=(3, 3, 3, 3), mu=0.3, m_w=-2.0, l=40, ks=(40, 80, 120)):
    """Deflation (Sec. 3) on a lattice small enough for a dense eigendecomposition
    (3^4, n = 972): H is assembled on the GPU (ov_apply_H on the 972 unit vectors),
    its eigen-triples come from scipy (LAPACK zgeev), and sgn(H) b from them is the
    exact reference.  Reported per k: the error of the plain and of the deflated TSL
    (l eigenvalues smallest in |lambda|) and the seconds per call of each."""
    import numpy as np
    import scipy.linalg as sla
    import torch
    from paper_1604_08057_gb300 import binding
    dev = torch.device("cuda", dev_index)
    rng = np.random.default_rng(31)
    u = torch.tensor(inputs.su3_links(dims, 0.3, rng), device=dev)
    b = torch.tensor(inputs.gaussian_spinors(dims, 1, rng), device=dev)
    n = 12 * int(np.prod(dims))
    unit = torch.eye(n, dtype=torch.complex128, device=dev).reshape((n,) + tuple(dims) + (4, 3))
    h = binding.apply_H(u, mu, m_w, unit).reshape(n, n).T.cpu().numpy()    # column j = H e_j
    lam, vl, vr = sla.eig(h, left=True, right=True)
    order = np.argsort(np.abs(lam), kind="stable")
    lam, vl, vr = lam[order], vl[:, order], vr[:, order]
    vr = vr / np.linalg.norm(vr, axis=0, keepdims=True)
    vl = vl / np.einsum("ij,ij->j", vl.conj(), vr).conj()[None, :]
    exact = (vr * np.sign(lam.real)) @ (vl.conj().T @ b.cpu().numpy().ravel())
    shape = (l,) + tuple(dims) + (4, 3)
    rf = torch.tensor(np.ascontiguousarray(vr[:, :l].T).reshape(shape), device=dev)
    lf = torch.tensor(np.ascontiguousarray(vl[:, :l].T).reshape(shape), device=dev)
    out = {"lattice": "x".join(map(str, dims)), "n": n, "deflated": l, "min_abs_re_lambda": float(np.min(np.abs(lam.real))),
           "lambda_l_abs": float(abs(lam[l - 1])), "per_k": {}}
    rel = lambda a: float(np.linalg.norm(a.cpu().numpy().ravel() - exact) / np.linalg.norm(exact))
    for k in ks:
        row = {}
        for name, call in (("plain", lambda: binding.tsl_sign(u, mu, m_w, b, k)),
                           ("deflated", lambda: binding.tsl_sign_deflated(u, mu, m_w, b, k, lam[:l], rf, lf))):
            x = call()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x = call()
            torch.cuda.synchronize()
            row[name] = {"rel_err": rel(x), "s_per_call": round(time.perf_counter() - t0, 5)}
        out["per_k"][str(k)] = row
    return out


def deflation_scale_leg(dev_index, l=30, m=90, ks=(100, 200, 400)):
    """Deflation at the 8x8^3 workload (n = 49152, the lattice size of the paper's
    Sec. 4 test, 30 deflated eigenvalues there too), where no dense reference
    exists: the 30 eigen-triples smallest in |lambda| by shift-and-invert Arnoldi
    (ov_eigen_smallest, m steps per side), then per k the a-posteriori error
    eps = ||sgn(H)^2 b - b|| / (2 ||b||) (Eq. error_est) of the plain and of the
    deflated TSL, and the seconds per sgn(H) b of each."""
    import numpy as np
    import torch
    from paper_1604_08057_gb300 import binding
    dev = torch.device("cuda", dev_index)
    wl = inputs.WORKLOADS["8x8^3"]
    u, b, _ = inputs.make_inputs(wl, nsrc=1)
    ut, bt = torch.tensor(u, device=dev), torch.tensor(b[0], device=dev)
    start = torch.tensor(inputs.gaussian_spinors(wl.dims, 1, np.random.default_rng(71))[0], device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, R, L, res = binding.eigen_smallest(ut, wl.mu, wl.m_w, l, m, start, tol=1e-10)
    torch.cuda.synchronize()
    out = {"lattice": "8x8^3", "n": 12 * wl.volume, "requested": l, "arnoldi_steps_per_side": m,
           "found": int(len(lam)), "eigen_s": round(time.perf_counter() - t0, 2),
           "max_residual": float(res.max()) if len(res) else None,
           "abs_lambda_range": [float(np.abs(lam).min()), float(np.abs(lam).max())] if len(lam) else None,
           "per_k": {}}
    bn = float(torch.linalg.vector_norm(bt))
    for k in ks:
        row = {}
        for name in ("plain", "deflated"):
            def sgn(v):
                if name == "plain":
                    return binding.tsl_sign(ut, wl.mu, wl.m_w, v, k)
                return binding.tsl_sign_deflated(ut, wl.mu, wl.m_w, v, k, lam, R, L)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x = sgn(bt)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t1
            x2 = sgn(x)
            row[name] = {"eps": float(torch.linalg.vector_norm(x2 - bt)) / (2 * bn), "s_per_call": round(dt, 4)}
        out["per_k"][str(k)] = row
    return out


def kk_leg(args, dev_index, reps=5):
    """One complex k x k product C = A^H B of the Frechet adjoint's kind through
    ov_kk_gemm, in FP64 arithmetic and by the tensor-core digit splitting: ms per
    product (CUDA events, after one warm-up each), the rate in FP64-equivalent
    TFLOP/s (8 k^3 flop), and the largest difference between the two relative to
    max |C|."""
    import torch
    from paper_1604_08057_gb300 import binding
    k = args.k or workload_of(args).k
    g = torch.Generator().manual_seed(7)
    dev = torch.device("cuda", dev_index)
    a = torch.randn(k, k, dtype=torch.complex128, generator=g).to(dev)
    b = torch.randn(k, k, dtype=torch.complex128, generator=g).to(dev)
    out = {"leg": "kk_product", "k": k, "op": "A^H B, complex128"}
    res = {}
    for mode in ("fp64", "split"):
        if mode == "split" and k > 1024:
            continue
        res[mode] = binding.kk_gemm(a, b, True, False, mode)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            binding.kk_gemm(a, b, True, False, mode)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[mode] = {"ms_per_product": round(ms, 4), "tflops_fp64_equivalent": round(8 * k**3 / ms / 1e9, 3)}
    if len(res) == 2:
        out["max_rel_diff"] = float((res["split"] - res["fp64"]).abs().max() / res["fp64"].abs().max())
    return out


def kk_products_leg(args, ut, bt, xt, wl, k, du, dmu, x, ms_step):
    """The headline call with the Frechet adjoint's k x k products in FP64 arithmetic
    instead of the tensor-core digit splitting: its seconds per call and how far its
    results lie from the headline's (x is the same: the forward pass forms no
    products); and, for scale, the map's rounding floor with FP64 products: the
    same call with b scaled by 1 + 2^-52 (one ulp), against the unscaled one."""
    import torch
    from paper_1604_08057_gb300 import binding
    opts = (args.precision, args.rebiorth, args.passes)
    binding.kk_products("fp64", *opts, segment=args.segment)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        du2, dmu2, x2 = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, *opts, segment=args.segment)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rel = lambda a, c: float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
        du3, dmu3, _ = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt * (1.0 + 2.0**-52), k, xt, *opts,
                                            segment=args.segment)
        return {"fp64_products_s_per_call": round(dt, 4), "split_products_s_per_call": round(ms_step / 1e3, 4),
                "x_identical": bool(torch.equal(x2, x)), "rel_dU_fp64_vs_split": rel(du2, du),
                "rel_dmu_fp64_vs_split": abs(dmu2 - dmu) / abs(dmu2),
                "fp64_floor_one_ulp_in_b": {"rel_dU": rel(du3, du2), "rel_dmu": abs(dmu3 - dmu2) / abs(dmu2)}}
    except (binding.OVError, RuntimeError) as exc:
        return {"error": str(exc)}
    finally:
        binding.kk_products("auto", *opts, segment=args.segment)


def diagnostics_leg(args, ut, bt, xt, wl, k, ms_step):
    """The headline call once more with the run diagnostics on: the sampled loss of
    biorthogonality of the bases, min |Re| of the Ritz values and ||T_k||, and
    what the diagnostics cost."""
    import torch
    from paper_1604_08057_gb300 import binding
    opts = (args.precision, args.rebiorth, args.passes)
    binding.diagnostics_mode(True, *opts, segment=args.segment)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, info = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, *opts, return_info=True,
                                             segment=args.segment)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"biorth_loss": info["biorth_loss"], "min_abs_re_ritz": info["min_abs_re_ritz"],
                "t_norm": info["t_norm"], "s_per_call_with_diagnostics": round(dt, 4),
                "s_per_call_without": round(ms_step / 1e3, 4)}
    except binding.OVError as exc:
        return {"status": exc.status, "error": str(exc)}
    finally:
        binding.diagnostics_mode(False, *opts, segment=args.segment)


def e2e_leg(args, ut, bt, xt, wl, k):
    """Same metric through the public API with host (pinned) inputs and outputs."""
    import torch
    from paper_1604_08057_gb300 import binding
    uh = ut.cpu().pin_memory()
    bh = bt.cpu().pin_memory()
    xh = xt.cpu().pin_memory()
    du_h = torch.empty_like(uh).pin_memory()
    x_h = torch.empty_like(bh).pin_memory()
    dev = ut.device
    ud, bd, xd = torch.empty_like(ut), torch.empty_like(bt), torch.empty_like(xt)
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ud.copy_(uh, non_blocking=True)
        bd.copy_(bh, non_blocking=True)
        xd.copy_(xh, non_blocking=True)
        du, dmu, x = binding.tsl_sign_vjp(ud, wl.mu, wl.m_w, bd, k, xd, args.precision, args.rebiorth,
                                          args.passes, segment=args.segment)
        du_h.copy_(du, non_blocking=True)
        x_h.copy_(x, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h2d = uh.numel() * 16 + bh.numel() * 16 + xh.numel() * 16
    d2h = du_h.numel() * 16 + x_h.numel() * 16 + 8
    del dev
    return {"value": round(ms / 1e3, 6), "unit": "s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps}


def batch_leg(args, workers=(1, 4), nprob=32):
    """Uneven batch: 32 problems on 8^4, 6x12^3 and 14^4 lattices with mu in
    {0.1, 0.3, 0.5} and k in 300..1000, forward + VJP each, through
    ov_tsl_batch; one warm-up and one timed batch per worker count."""
    import torch
    from paper_1604_08057_gb300 import binding
    links, probs = inputs.uneven_batch(nprob)
    dev = torch.device("cuda", torch.cuda.current_device())
    ut = {d: torch.tensor(u, device=dev) for d, u in links.items()}
    problems = [dict(u=ut[p["dims"]], mu=p["mu"], m_w=p["m_w"], b=torch.tensor(p["b"], device=dev), k=p["k"],
                     xbar=torch.tensor(p["xbar"], device=dev)) for p in probs]
    ctx = binding.context(args.precision, args.rebiorth, args.passes)
    out = {"problems": nprob, "k_total": int(sum(p["k"] for p in probs)),
           "lattices": ["8x8x8x8", "12x12x12x6", "14x14x14x14"], "work": "forward + VJP per problem"}
    for nw in workers:
        binding.tsl_batch(problems, nworkers=nw, precision=args.precision, rebiorth=args.rebiorth,
                          passes=args.passes, check=False)
        torch.cuda.synchronize()
        l0 = binding.launch_count(ctx)
        t0 = time.perf_counter()
        res = binding.tsl_batch(problems, nworkers=nw, precision=args.precision, rebiorth=args.rebiorth,
                                passes=args.passes, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = [r["status"] for r in res]
        out[f"workers_{nw}"] = {"s": round(dt, 3), "s_per_problem": round(dt / nprob, 4),
                                "gpu_launches": binding.launch_count(ctx) - l0,
                                "ok": sum(1 for x in st if x == 0), "statuses": sorted(set(st))}
    return out


def stencil_leg(args, ut, wl, hbm, peak_src, nsrc=32, reps=20):
    """ov_apply_H on nsrc sources sharing the links (working set > L2): live kernel time."""
    import torch
    from paper_1604_08057_gb300 import binding
    res = {}
    V = wl.volume
    g = torch.Generator(device=ut.device).manual_seed(5)
    psi = torch.randn((nsrc,) + tuple(ut.shape[:4]) + (4, 3), dtype=torch.complex128, device=ut.device,
                      generator=g)
    for prec, e in (("mixed", 4), ("fp64", 8)):
        ctx = binding.context(prec)
        tune = binding.autotune(ut, wl.mu, wl.m_w, nsrc, prec)
        binding.apply_H(ut, wl.mu, wl.m_w, psi, precision=prec)
        torch.cuda.synchronize()
        binding.profile_enable(ctx, True)
        binding.profile_read(ctx, reset=True)
        for _ in range(reps):
            binding.apply_H(ut, wl.mu, wl.m_w, psi, precision=prec)
        prof = binding.profile_read(ctx, reset=True)
        binding.profile_enable(ctx, False)
        n, ms = prof["apply_h"]
        nbytes = (nsrc * 2 * 24 * e + 72 * e) * V        # in + out per source, links once
        gbs = nbytes * n / (ms / 1e3) / 1e9
        flops = 1368 * V * nsrc * n / (ms / 1e3) / 1e12
        res[prec] = {"GB_s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 3), "tflops": round(flops, 2),
                     "us_per_launch": round(1e3 * ms / n, 2), "bytes_per_launch": nbytes,
                     "variant": tune["apply_variant"], "variant_us": tune["apply_us"]}
    res.update({"nsrc": nsrc, "peak": hbm, "peak_source": peak_src, "unit": "GB/s",
                "bytes": "algorithmic: spinor in + out per source, links once (480 B/site FP32 at 1 source)"})
    return res


def mixed_leg(args, ut, bt, xt, wl, k, u, b, xbar):
    """The mixed-precision path: at the workload point, and at m_w = -1 where the
    k-step map is well conditioned (timed against the FP64 path there, on the same
    schedule).  FP32 bases need two Gram-Schmidt passes and frequent projections:
    at m_w = -1 one pass breaks down at P = 20 and two passes break down at P = 60,
    while two passes at P = 20 complete.  The schedules MIXED_SCHEDULES are tried
    in turn (the first that completes is timed) and every failure is reported."""
    import torch
    from paper_1604_08057_gb300 import binding
    passes = 2
    res = {"gs_passes": passes}
    rel = lambda a, c: float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
    # at the workload point: projections at every step (the most the schedule can do),
    # against the FP64 path on the same schedule
    wp = {}
    for prec in ("mixed", "fp64"):
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            du, dmu, x = binding.tsl_sign_vjp(ut, wl.mu, wl.m_w, bt, k, xt, prec, 1, passes)
            torch.cuda.synchronize()
            wp[prec] = (time.perf_counter() - t0, du, dmu, x)
        except binding.OVError as exc:
            wp[prec] = f"status {exc.status}: {exc}"
    if all(isinstance(v, tuple) for v in wp.values()):
        (t32, du32, dmu32, x32), (t64, du64, dmu64, x64) = wp["mixed"], wp["fp64"]
        res["workload_point"] = {"rebiorth_period": 1, "mixed_s": round(t32, 3), "fp64_s": round(t64, 3),
                                 "mixed_vs_fp64_rel_x": rel(x32, x64), "mixed_vs_fp64_rel_dU": rel(du32, du64),
                                 "mixed_vs_fp64_rel_dmu": abs(dmu32 - dmu64) / abs(dmu64)}
    else:
        res["workload_point"] = {p: (v if isinstance(v, str) else "ok") for p, v in wp.items()}
        res["workload_point"]["rebiorth_period"] = 1
    m_w = -1.0
    tried = {}
    for reb in MIXED_SCHEDULES:
        out = {}
        for prec in ("fp64", "mixed"):
            try:
                binding.tsl_sign_vjp(ut, wl.mu, m_w, bt, k, xt, prec, reb, passes)
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record()
                du, dmu, x = binding.tsl_sign_vjp(ut, wl.mu, m_w, bt, k, xt, prec, reb, passes)
                t1.record()
                torch.cuda.synchronize()
                out[prec] = (t0.elapsed_time(t1) / 1e3, du, dmu, x)
            except binding.OVError as exc:
                out[prec] = f"status {exc.status}"
        if all(isinstance(v, tuple) for v in out.values()):
            (t64, du64, dmu64, x64), (t32, du32, dmu32, x32) = out["fp64"], out["mixed"]
            res["m_w=-1"] = {"rebiorth_period": reb, "fp64_s": round(t64, 4), "mixed_s": round(t32, 4),
                             "speedup": round(t64 / t32, 2), "mixed_vs_fp64_rel_x": rel(x32, x64),
                             "mixed_vs_fp64_rel_dU": rel(du32, du64),
                             "mixed_vs_fp64_rel_dmu": abs(dmu32 - dmu64) / abs(dmu64)}
            break
        tried[f"P={reb}"] = {p: (v if isinstance(v, str) else "ok") for p, v in out.items()}
    if tried:
        res["m_w=-1_schedules_not_completed"] = tried
    return res


CPU_SMALL_K = 6   # Lanczos steps of the oracle's full-size samples


def oracle_time(fn, reps=1):
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    return (time.perf_counter() - t0) / reps, out


def cpu_composed(args, k, period, passes):
    """The FP64 oracle's seconds per forward + VJP call at the workload, composed
    from pieces timed on the host (the oracle as it stands):

      * t_step: one Lanczos step of the forward and reverse sweeps at full size,
        from a forward + VJP run with CPU_SMALL_K steps and no projections;
      * t_proj(j): the projections of step j (forward Gram-Schmidt and its
        adjoint, both linear in j), from the same run with projections at every
        step minus the first, divided by sum (j + 1);
      * the k x k sign (Newton) and its Frechet adjoint (block Newton), timed on
        the T_k of the 4x4^3 workload's oracle run at k = 200 and scaled by
        (k / 200)^3 (dense O(k^3) iterations);
      * the 4x4^3 workload itself (k = 200, period 20, one pass), run end to end.

    Returns (estimate in s, details, the 4x4^3 oracle result)."""
    from oracle import ksign, tsl, vjp
    wl = workload_of(args)
    u, b, xbar = inputs.make_inputs(wl, nsrc=1)
    ks = CPU_SMALL_K

    def run(reb):
        fwd = tsl.tsl_forward(u, b[0], wl.mu, wl.m_w, ks, rebiorth=reb, passes=passes)
        return vjp.tsl_vjp(u, b[0], wl.mu, wl.m_w, ks, xbar[0], rebiorth=reb, passes=passes, fwd=fwd)

    t_plain, _ = oracle_time(lambda: run(0))
    t_proj_all, _ = oracle_time(lambda: run(1))
    t_step = t_plain / ks
    proj_units_small = sum(j + 1 for j in rebiorth_steps(ks, 1))
    t_unit = max(0.0, t_proj_all - t_plain) / proj_units_small
    proj_units = sum(j + 1 for j in rebiorth_steps(k, period))
    # the 4x4^3 workload end to end (also the parity reference of the GPU path)
    w0 = inputs.WORKLOADS["4x4^3"]
    u0, b0, x0 = inputs.make_inputs(w0)

    def small():
        f = tsl.tsl_forward(u0, b0[0], w0.mu, w0.m_w, w0.k, rebiorth=20, passes=1)
        d, m, _ = vjp.tsl_vjp(u0, b0[0], w0.mu, w0.m_w, w0.k, x0[0], rebiorth=20, passes=1, fwd=f)
        return f, d, m

    t_small, (f0, du0, dmu0) = oracle_time(small)
    g = np.zeros_like(f0.t)
    g[:, 0] = f0.beta0 * np.arange(1, w0.k + 1)
    t_sign, _ = oracle_time(lambda: ksign.sign_newton(f0.t))
    t_frechet, _ = oracle_time(lambda: ksign.frechet_adjoint_sign(f0.t, g))
    scale = (k / w0.k) ** 3
    est = k * t_step + proj_units * t_unit + scale * (t_sign + t_frechet)
    details = {"t_step_s": round(t_step, 4), "t_proj_per_basis_vector_s": round(t_unit, 5),
               "proj_basis_vectors": proj_units, "t_sign_k200_s": round(t_sign, 3),
               "t_frechet_k200_s": round(t_frechet, 3), "dense_scale": round(scale, 1),
               "workload_4x4^3_k200_s": round(t_small, 3)}
    return est, details, (w0, u0, b0, x0, f0, du0, dmu0)


def cpu_leg(args, k, ut):
    """The FP64 oracle on the host cores: the 4x4^3 workload measured end to end, and
    the benchmark's workload composed from timed pieces (``cpu_composed``).  The
    same 4x4^3 oracle run is the reference of the GPU path's errors there (x, dU,
    dmu of the FP64 path, period 20, one pass)."""
    import torch
    from paper_1604_08057_gb300 import binding
    t0 = time.perf_counter()
    est, details, (w0, u0, b0, x0, f0, du0, dmu0) = cpu_composed(args, k, args.rebiorth, args.passes)
    wall = time.perf_counter() - t0
    dev = ut.device
    du, dmu, x = binding.tsl_sign_vjp(torch.tensor(u0, device=dev), w0.mu, w0.m_w, torch.tensor(b0[0], device=dev),
                                      w0.k, torch.tensor(x0[0], device=dev), "fp64", 20, 1)
    rel = lambda a, c: float(np.linalg.norm(a - c) / np.linalg.norm(c))
    parity = {"workload": "4x4^3 lattice, k=200, mu=0.3, m_w=-2, period 20, one pass (FP64 GPU vs FP64 oracle)",
              "rel_x": rel(x.cpu().numpy(), f0.x), "rel_dU": rel(du.cpu().numpy(), du0),
              "rel_dmu": abs(dmu - dmu0) / abs(dmu0),
              "oracle_rounding_floor": {"x": 1.0e-10, "dU": 7.4e-7, "dmu": 2.7e-7}}
    cpu = {"value": round(est, 2), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"composed from oracle pieces timed on the host ({wall:.1f} s of CPU work): "
                      f"{CPU_SMALL_K}-step forward + VJP runs at {args.workload} with and without projections, "
                      f"the k x k sign and Frechet adjoint at k=200 scaled by (k/200)^3, and the 4x4^3 "
                      f"workload end to end ({details['workload_4x4^3_k200_s']} s per call)"),
           "pieces": details}
    return cpu, parity


def run_reference(args, rank):
    if rank != 0:
        return None
    wl = workload_of(args)
    k = args.k or wl.k
    from oracle import tsl
    w0 = inputs.WORKLOADS["4x4^3"]
    u0, b0, _ = inputs.make_inputs(w0)
    for _ in range(args.warmup):   # warm-up: the oracle's stencil and recurrence on a small lattice
        tsl.tsl_forward(u0, b0[0], w0.mu, w0.m_w, 40, rebiorth=20, passes=1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        est, details, _ = cpu_composed(args, k, args.rebiorth, args.passes)
        vals.append(est)
    dt = (time.perf_counter() - t0) / args.steps
    value = statistics.median(vals)
    desc = (f"FP64 numpy oracle, composed per step from pieces timed on the host ({dt:.1f} s of CPU work per "
            f"step): {CPU_SMALL_K}-step forward + VJP runs at {args.workload} with and without projections, the "
            f"k x k sign and Frechet adjoint at k=200 scaled by (k/200)^3")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload} lattice, k={k}, mu={wl.mu}, m_w={wl.m_w}, "
                                   f"1 source, forward + gauge-force VJP",
                       "rebiorth_period": args.rebiorth, "gs_passes": args.passes},
            "cpu_baseline": {"value": round(value, 2), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc, "pieces": details},
            "e2e": {"value": round(value, 2), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.leg == "batch":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"leg": "uneven_batch", "precision": args.precision, "rebiorth_period": args.rebiorth,
                          "segment": args.segment,
                          "gs_passes": args.passes, **batch_leg(args)}))
        return
    if args.leg == "deflation8":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"leg": "deflation_8x8^3", **deflation_scale_leg(local_rank)}))
        return
    if args.leg == "deflation":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"leg": "deflation", **deflation_leg(local_rank)}))
        return
    if args.leg == "kk":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps(kk_leg(args, local_rank)))
        return
    if args.leg == "nested_stage":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"leg": "nested_stage", **nested_stage_leg(args.k or workload_of(args).k)}))
        return
    if args.leg == "nested":
        import torch
        torch.cuda.set_device(local_rank)
        wl = workload_of(args)
        k = args.k or wl.k
        u, b, _ = inputs.make_inputs(wl)
        dev = f"cuda:{local_rank}"
        print(json.dumps({"leg": "nested_tsl", "workload": f"{args.workload}, k={k}, mu={wl.mu}, m_w={wl.m_w}",
                          "rebiorth_period": args.rebiorth, "gs_passes": args.passes,
                          **nested_leg(args, torch.tensor(u, device=dev), torch.tensor(b, device=dev), wl, k)}))
        return
    if args.leg == "stencil":
        import torch
        torch.cuda.set_device(local_rank)
        wl = workload_of(args)
        u, _, _ = inputs.make_inputs(wl)
        hbm, peak_src = hbm_peak()
        out = stencil_leg(args, torch.tensor(u, device=f"cuda:{local_rank}"), wl, hbm, peak_src)
        print(json.dumps(out))
        return
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
