#!/usr/bin/env python
"""Benchmark: density-matrix RT-TDDFT steps per second on GB300.

Workload (the precision configuration): 4096-atom periodic diamond cell
(8x8x8 conventional cells, a = 5.43 A, jitter 0.05 A), 13 functions per atom
(n = 53,248), r_S = r_H = 7 A, truncation radii r_Sinv = r_T = r_U = r_K =
r_M = 10 A (--radius selects another point of the 6/8/10/12 A sweep), K0 from
a Chebyshev Fermi-operator expansion (order 200, kT = 0.01 Ha, untimed), x
delta kick kappa = 1e-3, dt = 0.05 a.u., exponential-midpoint propagator with
6 Taylor terms, U rebuilt at every step's midpoint.

A step is one pass of the whole path: U(t + dt/2), the sandwich
K <- U K U^dagger and the traces Tr(KS), Tr(KD_xyz).

GPU paths timed from the same K(0+):
  * the plain FP64 path (the literal step: T = S^-1 H, Taylor powers, sandwich);
  * the headline, mixed precision in the reference split: K = K_ref + dK, the
    part acting on K_ref and U itself in FP64 (polynomials in the field value,
    exact for H = H0 - E D), FP32 block products on dK;
  * the literal mixed path (FP32 products on the whole K), reported with its
    dipole error, which grows with the step count;
  * the propagation step (U built once) in FP64 and in the reference split.
`value` is the reference split when its dipole error relative to the induced
swing, max_t |P_mixed - P_fp64| / max_t |P_fp64(t) - P_fp64(t_1)|, is within
1e-6 over the compared steps, else the FP64 path.

--impl reference times the CPU oracle (plain C, all host cores) on a row
sample of the same step and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--radius", type=float, default=10.0)
    ap.add_argument("--ncell", type=int, default=8)
    ap.add_argument("--basis", default="spd13")
    ap.add_argument("--atom-order", default="lattice", choices=["lattice", "morton"],
                    help="numbering of the atoms of the benchmark cell (morton: along a Morton curve)")
    ap.add_argument("--prop", default="em", choices=["em", "cn", "etrs", "m4"])
    ap.add_argument("--foe-order", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the nvidia-smi clock samples of the timed region (default: a temp dir)")
    ap.add_argument("--fp64-steps", type=int, default=4, help="timed FP64 steps (an FP64 step takes seconds)")
    ap.add_argument("--gate-steps", type=int, default=12,
                    help="steps over which the mixed dipole is compared with the FP64 run")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the mixed-precision context (FOE ground state, kick, warm-up, steps) and print "
                         "its per-kernel-class times: a small resident set for kernel captures, no benchmark line")
    ap.add_argument("--literal", action="store_true", help="--kernel-case: the literal FP32 path")
    ap.add_argument("--only-split", action="store_true",
                    help="time only the FP64 step and the reference-split mixed step (less device memory, e.g. "
                         "for larger radii)")
    ap.add_argument("--scalar-fma", action="store_true",
                    help="reference split: the row-layout complex products with scalar FMAs instead of packed ones")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="FP32 contexts run the sandwich's 13-function products on the tensor cores (tcgen05)")
    ap.add_argument("--study", default=None, choices=["truncation", "scaling", "batching", "propagators",
                                                       "propagator-timing"],
                    help="run a study instead of the benchmark and print its JSON line")
    ap.add_argument("--precision-study", type=int, default=0, metavar="NSTEPS",
                    help="instead of timing: run both paths NSTEPS steps and report their agreement")
    return ap.parse_args()


def workload(args):
    import synth
    s = synth.diamond_system(args.ncell, args.basis, 7.0, 7.0, order=args.atom_order)
    return s


def model_spectrum(args):
    """mu (mid-gap at valence filling) and spectral bounds from a 2x2x2 cell of
    the same model (dense generalised diagonalisation; input preparation)."""
    import synth
    small = synth.diamond_system(2, args.basis, 7.0, 7.0)
    _, w, _ = synth.ground_state_dense(small, 2 * small.n_atoms)
    n_occ = 2 * small.n_atoms
    mu = 0.5 * (w[n_occ - 1] + w[n_occ])
    return mu, float(w.min()) - 0.5, float(w.max()) + 0.5


def cfg_name(args):
    return (f"diamond {args.ncell ** 3 * 8} atoms x {synth_nfunc(args.basis)} functions, r_S=r_H=7A, "
            f"r_Sinv=r_T=r_U=r_K=r_M={args.radius:g}A, dt=0.05, {args.prop.upper()} 6 terms, x-kick 1e-3"
            + (", atoms in Morton order" if args.atom_order == "morton" else ""))


def synth_nfunc(basis):
    return {"sp4": 4, "spd13": 13, "h1": 1}[basis]


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------
# peaks
# ----------------------------------------------------------------------------
def measured_peaks():
    p = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            p = json.load(open(path))
        except Exception:
            p = {}
    return p


# DRAM bytes (read + write) per launch of the dominant kernel from an ncu capture of
# the same kernel and workload, keyed by (path, kernel class); None when the kernel
# changed after the capture.
TRAFFIC = {("diamond 4096 atoms x 13 functions, r_S=r_H=7A, r_Sinv=r_T=r_U=r_K=r_M=10A, dt=0.05, EM 6 terms, "
            "x-kick 1e-3", "fp32", "gemm_M=UK"): 24.574e9 + 2.604e9}  # k_gemm13_c32<EPI_STORE, packed>


def derived_alu_peaks(torch, sm_max_mhz):
    """ALU peaks from unit counts and the maximum SM clock, TFLOP/s: FP32 is
    128 FMA lanes per SM x 2 flops; FP64 is GB300's nominal 1.25 TFLOP/s at
    2070 MHz scaled to the clock (2 FP64 FMA per clock per SM on 152 SMs)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ghz = (sm_max_mhz or 2070.0) / 1e3
    return {"fp32": sms * 128 * 2 * ghz / 1e3, "fp64": sms * 2 * 2 * ghz / 1e3, "sms": sms, "sm_max_ghz": ghz}


def alu_peaks(torch):
    """FP64 and FP32 (no TF32) GEMM throughput measured with cuBLAS through torch
    (denominators for the ALU-bound block products), TFLOP/s."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in [("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)]:
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            best = 1e9
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# ranks (one process per GPU, independent replicas; no data-path collective)
# ----------------------------------------------------------------------------
def nvtx_push(torch, name):
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:  # NVTX markers are optional
        pass


def nvtx_pop(torch):
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (timings are reported as the max over ranks)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps_per_rank: int, max_ms: float, world: int) -> float:
    """Whole-job steps/s: every rank runs its own replica of the workload, so
    the job advances world * steps_per_rank steps in the slowest rank's time."""
    return world * steps_per_rank / (max_ms / 1e3)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def _dipole_errors(o_mixed, o64):
    """Dipole (Re Tr(K Dx)) error of a mixed run against the FP64 run from the
    same K(0+), over the steps both ran: relative to the induced swing
    max_t |P_FP64(t) - P_FP64(t_1)| (the bar) and to max_t |P_FP64|."""
    m = min(len(o_mixed), len(o64))
    if m < 2:
        return {"induced": None, "abs_P": None, "trks": None, "compared_steps": m}
    p64, p32 = o64[:m, 3], o_mixed[:m, 3]
    err = float(np.abs(p32 - p64).max())
    ind = float(np.abs(p64 - p64[0]).max())
    return {"induced": err / ind if ind > 0 else None, "abs_P": err / float(np.abs(p64).max()),
            "trks": float(np.abs(o_mixed[:m, 1] - o64[:m, 1]).max() / abs(o64[0, 1])), "compared_steps": m}


def run_gpu(args):
    import torch

    import paper_1404_5776_gb300 as rtm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    rtm.build()
    dev_name = torch.cuda.get_device_name()

    s = workload(args)
    mu, e_lo, e_hi = model_spectrum(args)
    R = args.radius
    radii = dict(r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    common = dict(dt=0.05, prop=args.prop, n_kick=1, obs_capacity=8192, tensor_cores=1 if args.tensor_cores else 0,
                  packed_fma=0 if args.scalar_fma else 1, **radii)
    split_ok = args.prop == "em" and args.basis in ("spd13", "sp4")

    # --- FP64 context (the plain FP64 GPU path): ground state (untimed set-up), kick
    c64 = rtm.RT(s, precision="fp64", **common)
    it64, res64 = c64.inverse()
    c64.ground_state(0, args.foe_order, mu, 0.01, e_lo, e_hi)
    c64.kick(0, 0, 0, 1e-3)
    K1 = c64.matrix(0, rtm.RT_MAT_K)  # K(0+), seeds every other path

    # --- headline: mixed precision in the reference split, full step (EM with
    # the field polynomial: U(E) and R(E) = U K_ref U^dagger - K_ref formed in
    # FP64 from coefficients set up once, FP32 products on dK = K - K_ref).
    # One-time set-up, host wall clock: rt_create, rt_inverse (Hotelling S^-1
    # and the V_m), and the reference (K_ref, the B_p) formed by the first step.
    setup_s = {}
    launch_shapes, launch_shape_ms = None, None
    c32s = None
    if split_ok:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c32s = rtm.RT(s, precision="fp32", incremental=1, field_poly=1, **common)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        c32s.inverse()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        c32s.set_density(0, 0, K1)
        c32s.step(1)
        c32s.synchronize()
        t3 = time.perf_counter()
        setup_s = {"create": round(t1 - t0, 3), "inverse": round(t2 - t1, 3), "reference": round(t3 - t2, 3),
                   "what": "mixed reference-split context, host wall clock: rt_create (patterns by cell lists, "
                           "triple lists, block maps, allocations); rt_inverse (Hotelling S^-1, the field "
                           "polynomial V_m of U: FP64 block products); the first rt_step (K_ref and the "
                           "coefficients B_p of R(E): 2 (taylor_terms)^2 + taylor_terms FP64 complex products, "
                           "then one step)"}
        # launch shapes of the two products (stages per warp, one-shot or
        # persistent grid): timed on this context's own products, fastest kept
        if not args.tensor_cores:
            t4 = time.perf_counter()
            tuned = c32s.autotune(reps=2)
            setup_s["autotune"] = round(time.perf_counter() - t4, 3)
            launch_shapes = {c32s.STAGES[st]: {"stages_per_warp": v[0], "persistent": v[1]}
                             for st, v in tuned["chosen"].items()}
            launch_shape_ms = {f"{r['what']}: stages {r['stages_per_warp']}, persistent {r['persistent']}":
                               round(r["ms"], 3) for r in tuned["rows"]}
    # the literal mixed path (FP32 block products on the whole K): faster set-up,
    # but its dipole error grows with the step count (reported, not the headline)
    c32l = c64p = c32p = None
    if not args.only_split:
        c32l = rtm.RT(s, precision="fp32", **common)
        c32l.inverse()
        c32l.set_density(0, 0, K1)
        # propagation step (the delta kick leaves H constant: U built once, FP64):
        # FP64 and the reference split
        c64p = rtm.RT(s, precision="fp64", full_step=0, **common)
        c64p.inverse()
        c64p.set_density(0, 0, K1)
        c64p.propagator(0.0)
    if args.basis in ("spd13", "sp4") and not args.only_split:
        c32p = rtm.RT(s, precision="fp32", full_step=0, incremental=1, **common)
        c32p.inverse()
        c32p.set_density(0, 0, K1)
        c32p.propagator(0.0)
        if c32s is not None and launch_shapes is not None:  # same products: the headline's tuned shapes
            for st, v in tuned["chosen"].items():
                c32p.set_launch_shape(st, v[0], v[1])

    n64 = args.fp64_steps if args.fp64_steps is not None else args.steps

    def timed(ctx, nsteps, warm, label):
        ctx.step(warm)
        ctx.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        # an NVTX range marks the timed launches (ncu --nvtx-include "timed_<label>/")
        nvtx_push(torch, "timed_" + label)
        ctx.step(nsteps)
        nvtx_pop(torch)
        ev1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        return ms / max(nsteps, 1)

    clocks_dir = args.clocks_dir or tempfile.gettempdir()
    clocks = Clocks(os.path.join(clocks_dir, f"clocks_r{rank}.csv"))
    clocks.start()
    ms64 = timed(c64, n64, args.warmup, "fp64")
    ms32s = timed(c32s, args.steps, args.warmup, "fp32_split") if c32s else float("nan")
    ms32l = timed(c32l, args.steps, args.warmup, "fp32_literal") if c32l else float("nan")
    ms64p = timed(c64p, n64, args.warmup, "fp64_propagation") if c64p else float("nan")
    ms32p = timed(c32p, args.steps, args.warmup, "fp32_split_propagation") if c32p else float("nan")
    clk = clocks.stop()
    # the FP64 reference run continues to --gate-steps for the dipole comparison
    extra = args.gate_steps - (args.warmup + n64)
    if extra > 0:
        c64.step(extra)
        if c64p:
            c64p.step(extra)

    flops64, _ = c64.step_work()
    flops32l, _ = c32l.step_work() if c32l else (float("nan"), 0.0)
    flops32s, _ = c32s.step_work() if c32s else (float("nan"), 0.0)
    o64, o64p = c64.observables(0, 0), (c64p.observables(0, 0) if c64p else None)
    gate_s = _dipole_errors(c32s.observables(0, 0), o64) if c32s else None
    gate_l = _dipole_errors(c32l.observables(0, 0), o64) if c32l else None
    gate_p = _dipole_errors(c32p.observables(0, 0), o64p) if c32p else None
    BAR = 1e-6
    headline_ok = bool(gate_s and gate_s["induced"] is not None and gate_s["induced"] <= BAR)
    head = c32s if headline_ok else c64
    ms_head = ms32s if headline_ok else ms64
    hp = "fp32" if headline_ok else "fp64"

    # per-kernel-class times (CUDA events on the library stream), a short extra pass
    prof = {}
    for name, ctx, n in (("fp64", c64, 2), ("fp32", c32s, 5), ("fp32_literal", c32l, 5)):
        if ctx is None:
            continue
        ctx.profile(True)
        ctx.step(n)
        prof[name] = ctx.profile_read()
        ctx.profile(False)

    # e2e through the public API with host buffers: set K(0+) from pinned host
    # memory (the reference split keeps its K_ref and carries it as dK), run
    # the steps, read the observables back
    n_e2e = args.steps if headline_ok else n64
    K1_pinned = torch.empty(K1.shape, dtype=torch.complex128, pin_memory=True)
    K1_host = K1_pinned.numpy()
    K1_host[:] = K1
    head.observables(0, 0)  # drain the earlier records
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    head.set_density(0, 0, K1_host)
    head.step(n_e2e)
    obs_e2e = head.observables(0, 0)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    h2d = K1_host.nbytes / n_e2e
    d2h = obs_e2e.nbytes / n_e2e

    # roofline of the dominant kernel class of the headline path
    pr = prof[hp]
    dom = max(pr, key=lambda k: pr[k]["ms"])
    d = pr[dom]
    per_launch_flops = d["flops"] / max(d["launches"], 1)
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    peaks = alu_peaks(torch) if rank == 0 else {}
    derived = derived_alu_peaks(torch, clk.get("sm_max_mhz") if isinstance(clk, dict) else None)
    mp = measured_peaks()
    if d["flops"] > 0:
        achieved = per_launch_flops / (per_launch_ms / 1e3) / 1e12
        peak = derived[hp]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 3),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": TRAFFIC.get((cfg_name(args), hp, dom)),
                "peak_source": (f"derived: {derived['sms']} SMs x "
                                f"{'128 FP32 lanes x 2 flops' if hp == 'fp32' else '2 FP64 FMA x 2 flops'}"
                                f" x {derived['sm_max_ghz']:.3f} GHz"),
                "cublas_gemm_tflops": {k: round(v, 3) for k, v in peaks.items()},
                "frac_of_cublas_gemm": round(achieved / peaks[hp], 4) if peaks.get(hp) else None,
                "per_launch_flops": per_launch_flops, "per_launch_ms": round(per_launch_ms, 4)}
    else:
        achieved = d["bytes"] / max(d["launches"], 1) / (per_launch_ms / 1e3) / 1e9
        peak = mp.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None}

    launches_per_step = head.step_kernels()
    line = {
        "metric": "TDDFT steps/sec & block GFLOP/s vs plain FP64 GPU path at dipole err<=1e-6",
        "value": round(job_rate(1, ms_head, world), 4),
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_head, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if headline_ok else "f64",
        "data": "synthetic (seeded diamond-lattice Gaussian model; no paper data)",
        "config": {"workload": cfg_name(args), "n_atoms": s.n_atoms, "n": int(s.n), "radius_A": R,
                   "path": ("mixed precision, reference split (EM, U(E) and U K_ref U^dagger from FP64 "
                            "field polynomials, FP32 products on K - K_ref)") if headline_ok else "FP64",
                   "l2": "inputs larger than L2 (K alone %.2f GB > 129 MB)" % (K1.nbytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "paths": {
            "fp64": {"ms_per_step": round(ms64, 3), "steps_per_s": round(1e3 / ms64, 4),
                     "tflops": round(flops64 / (ms64 / 1e3) / 1e12, 4), "step_tflop": round(flops64 / 1e12, 4),
                     "timed_steps": n64,
                     "what": "literal EM step in FP64: T = cut(S^-1 H), 4 Taylor powers, M = cut(U K), K' = M U^dagger"},
            "mixed_reference_split": {
                "ms_per_step": round(ms32s, 3), "steps_per_s": round(1e3 / ms32s, 4),
                "tflops": round(flops32s / (ms32s / 1e3) / 1e12, 4), "step_tflop": round(flops32s / 1e12, 4),
                "timed_steps": args.steps, "dipole_err": gate_s,
                "what": ("per step: U(E) - I stochastically rounded to FP32 and R(E) by Horner passes over FP64 "
                         "coefficients; M = cut(dU dK), K' = dK + R + M + cut((dK + M) dU^dagger) with FP32 "
                         "products; the Taylor powers and T = S^-1 H are in the coefficients, formed once")}
            if c32s else None,
            "mixed_literal": {"ms_per_step": round(ms32l, 3), "steps_per_s": round(1e3 / ms32l, 4),
                              "tflops": round(flops32l / (ms32l / 1e3) / 1e12, 4),
                              "step_tflop": round(flops32l / 1e12, 4), "timed_steps": args.steps,
                              "dipole_err": gate_l,
                              "what": ("T = T0 - E T_D, Taylor powers and the delta-form sandwich as FP32 block "
                                       "products on the whole K; its error grows with the step count")}
            if c32l else None,
            "speedup_split_vs_fp64": round(ms64 / ms32s, 2) if c32s else None,
            "speedup_literal_vs_fp64": round(ms64 / ms32l, 2) if c32l else None,
            "propagation_step": {
                "what": "delta kick: H is constant for t > 0, U built once (FP64) and reused; sandwich + traces",
                "fp64": {"ms_per_step": round(ms64p, 3), "steps_per_s": round(1e3 / ms64p, 4)},
                "mixed_reference_split": {"ms_per_step": round(ms32p, 3), "steps_per_s": round(1e3 / ms32p, 4),
                                          "dipole_err": gate_p} if c32p else None,
                "speedup": round(ms64p / ms32p, 2) if c32p else None} if c64p else None,
            "hotelling": {"iters": it64, "residual": res64},
            "setup_s": setup_s,
            "launch_shapes": launch_shapes,
            "launch_shape_ms": launch_shape_ms,
        },
        "roofline": roof,
        "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in prof[hp].items() if v["launches"]},
        "e2e": {"value": round(job_rate(n_e2e, e2e_s * 1e3, world), 4), "unit": "steps/s",
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "what": "rt_set_density(K(0+) from pinned host memory) + rt_step(n) + rt_observables, timed on the host"},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "device": dev_name,
        "device_mem_gb": round(torch.cuda.max_memory_allocated() / 1e9, 2),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, s, budget_s=20.0)
    line["gate"] = {
        "reading": ("dipole error relative to the induced swing, max_t |P_mixed - P_fp64| / "
                    "max_t |P_fp64(t) - P_fp64(t_1)| <= 1e-6 (P = Re Tr(K Dx), FP64 run from the same K(0+)); "
                    "the error relative to |P| is reported beside it"),
        "headline_passes": headline_ok,
        "compared_steps": gate_s["compared_steps"] if gate_s else None,
        "mixed_reference_split": gate_s, "mixed_literal": gate_l, "propagation_step_split": gate_p}
    for ctx in (c64, c32s, c32l, c64p, c32p):
        if ctx:
            ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
def oracle_step_sample(args, s, rows):
    """Times the oracle's truncated products of one EM step for output block
    rows [0, rows) and returns (seconds, rows).  Operand values do not change
    the work of the plain C product, so S stands in for S^-1 on its pattern."""
    import oracle
    R = args.radius
    pat = oracle.pattern(s.pos, s.cell, R)
    S = oracle.BlockMatrix(s.bsize, oracle.Pattern(s.s_rowptr, s.s_col), s.s_val)
    H = oracle.BlockMatrix(s.bsize, oracle.Pattern(s.h_rowptr, s.h_col), s.h_val)
    Sinv = oracle.restrict(S, pat)
    K = oracle.zeros(s.bsize, pat)
    K.val[:] = 0.01 + 0.002j
    t0 = time.perf_counter()
    T = oracle.spgemm(Sinv, H, pat, rows=(0, rows))
    P = T
    for _ in range(2, 6):
        P = oracle.spgemm(T, P, pat, rows=(0, rows))
    U = P  # U = I + sum c_n T^n: an O(nnz) vector update, left out of the row sample
    M = oracle.spgemm(U, K, pat, rows=(0, rows))
    Kn = oracle.zeros(s.bsize, pat)
    oracle.spgemm(M, U, pat, b_dag=True, upper_only=True, out=Kn, rows=(0, rows))
    return time.perf_counter() - t0


def cpu_baseline(args, s, budget_s=20.0):
    import oracle
    oracle.build()
    # calibrate the row sample to about budget_s of CPU work
    rows = 4
    t = oracle_step_sample(args, s, rows)
    rows = int(max(4, min(s.n_atoms, rows * budget_s / max(t, 1e-3))))
    t = oracle_step_sample(args, s, rows)
    step_s = t * s.n_atoms / rows
    return {"value": 1.0 / step_s, "unit": "steps/s", "cores": oracle.lib().or_num_threads(), "kind": "oracle",
            "sample": f"oracle truncated products of one literal EM step (T, 4 Taylor powers, U K, M U^dagger) "
                      f"for {rows} of {s.n_atoms} block rows ({t:.1f} s), extrapolated linearly to all rows; "
                      f"placeholder operand values (S on P_Sinv for S^-1, a constant K: the plain C product "
                      f"does the same work for any values)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    s = workload(args)
    rows = 4
    t = oracle_step_sample(args, s, rows)
    rows = int(max(4, min(s.n_atoms, rows * 3.0 / max(t, 1e-3))))  # ~3 s per sampled step
    for _ in range(args.warmup):
        oracle_step_sample(args, s, rows)
    tot = 0.0
    for _ in range(args.steps):
        tot += oracle_step_sample(args, s, rows)
    step_s = (tot / max(args.steps, 1)) * s.n_atoms / rows
    v = 1.0 / step_s
    cores = oracle.lib().or_num_threads()
    sample = (f"each step: oracle truncated products of one literal EM step for {rows} of {s.n_atoms} block "
              f"rows, extrapolated linearly to all rows; placeholder operand values (S on P_Sinv for S^-1, "
              f"a constant K: the plain C product does the same work for any values)")
    line = {"metric": "TDDFT steps/sec & block GFLOP/s vs plain FP64 GPU path at dipole err<=1e-6",
            "value": v, "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "sampled_ms_per_step": tot / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded diamond-lattice Gaussian model)",
            "config": {"workload": cfg_name(args), "n_atoms": s.n_atoms, "n": int(s.n), "radius_A": args.radius},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def precision_study(args):
    """The mixed paths against the FP64 path over many steps from the same K(0+):
    dipole error relative to the induced swing and to |P|, charge difference
    and drift, and the S-unitarity error of the propagators; the reference
    split (the mixed mode with the accuracy bar) and the literal FP32 path."""
    import paper_1404_5776_gb300 as rtm
    rtm.build()
    s = workload(args)
    mu, e_lo, e_hi = model_spectrum(args)
    R = args.radius
    n = args.precision_study
    common = dict(dt=0.05, prop=args.prop, n_kick=1, obs_capacity=n + 8, r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R,
                  tensor_cores=1 if args.tensor_cores else 0, packed_fma=0 if args.scalar_fma else 1)
    c64 = rtm.RT(s, precision="fp64", **common)
    c64.inverse()
    c64.ground_state(0, args.foe_order, mu, 0.01, e_lo, e_hi)
    c64.kick(0, 0, 0, 1e-3)
    K1 = c64.matrix(0, rtm.RT_MAT_K)
    t0 = time.perf_counter()
    c64.step(n)
    o64 = c64.observables(0, 0)
    wall = {"fp64": time.perf_counter() - t0}
    u64 = c64.unitarity(0, True)
    c64.close()
    out = {"study": "precision", "workload": cfg_name(args), "steps": n,
           "induced_amplitude_rel_P": float(np.abs(o64[:, 3] - o64[0, 3]).max() / np.abs(o64[:, 3]).max()),
           "trks_drift_fp64_rel": float(np.abs(o64[:, 1] - o64[0, 1]).max() / abs(o64[0, 1])),
           "unitarity_fp64": {"max": u64[0], "mean": u64[1]}}
    paths = [("mixed_literal", dict(precision="fp32"))]
    if args.prop == "em" and args.basis in ("spd13", "sp4"):
        paths.insert(0, ("mixed_reference_split", dict(precision="fp32", incremental=1, field_poly=1)))
    for name, kw in paths:
        c = rtm.RT(s, **kw, **common)
        c.inverse()
        c.set_density(0, 0, K1)
        t0 = time.perf_counter()
        c.step(n)
        o = c.observables(0, 0)
        wall[name] = time.perf_counter() - t0
        u = c.unitarity(0, True)
        c.close()
        e = _dipole_errors(o, o64)
        err = np.abs(o[:, 3] - o64[:, 3])
        ind = np.abs(o64[:, 3] - o64[0, 3]).max()
        # the error relative to the induced swing at checkpoints of the run
        marks = sorted({m for m in (10, 25, 50, 100, 200, 500, 1000, 1500, 2000, 5000) if m <= n} | {n})
        out[name] = {"dipole_err_rel_induced": e["induced"], "dipole_err_rel_P": e["abs_P"],
                     "trks_diff_rel": e["trks"],
                     "trks_drift_rel": float(np.abs(o[:, 1] - o[0, 1]).max() / abs(o[0, 1])),
                     "unitarity": {"max": u[0], "mean": u[1]}, "unitarity_excess_max": u[0] - u64[0],
                     "err_rel_induced_by_step": {str(m): float(err[:m].max() / ind) for m in marks}}
    out["wall_s"] = wall
    out["dipole_trace_every_100"] = [float(a) for a in o64[::100, 3]]
    print(json.dumps(out))


def truncation_study(args):
    """The paper's truncation experiments (Sec. IV-V) on synthetic diamond cells,
    every matrix from the library: S^-1 and S^-1 H errors and U unitarity vs
    range, S^-1 H error vs system size, unitarity vs time step and Taylor terms,
    and the spectrum vs the density-matrix range."""
    import synth

    import paper_1404_5776_gb300 as rtm
    from paper_1404_5776_gb300 import spectra, studies
    rtm.build()
    t_start = time.perf_counter()
    out = {"study": "truncation", "data": "synthetic (seeded diamond-lattice Gaussian model)", "r_S": 7.0,
           "r_H": 7.0}
    # range sweeps (r_Sinv = r_T = r_U = r); the last radius covers every pair (dense)
    for ncell, basis, radii in ((3, "spd13", [3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 10.0, 12.0, 15.0]),
                                (4, "sp4", [3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 10.0, 12.0, 19.0])):
        s = synth.diamond_system(ncell, basis, 7.0, 7.0)
        out[f"range_{basis}_{s.n_atoms}"] = studies.truncation_sweep(rtm, s, radii)
    # size dependence at fixed ranges
    systems = [synth.diamond_system(nc, "sp4", 7.0, 7.0) for nc in (2, 3, 4, 5)]
    out["size_sp4_rSinv6_rT6"] = studies.size_sweep(rtm, systems, r_Sinv=6.0, r_T=6.0)
    # time step and Taylor terms (64 atoms, every pair kept)
    s = synth.diamond_system(2, "sp4", 7.0, 7.0)
    out["unitarity_dt_terms"] = studies.unitarity_vs_dt_terms(
        rtm, s, [0.01, 0.02, 0.05, 0.1, 0.15, 0.2], [2, 3, 4, 5, 6, 7, 8], r=12.0)
    # density-matrix range: delta kick, U built once (H constant after the kick), 2000 steps
    s = synth.diamond_system(3, "sp4", 7.0, 7.0)
    K0, _, gap = synth.ground_state_dense(s, s.n // 2)
    steps, kappa, dt = 2000, 1e-3, 0.05
    omegas = np.linspace(0.0, 3.0, 601)[1:]
    spec = {}
    for rk in (4.0, 6.0, 8.0, 10.0, 15.0):
        ctx = rtm.RT(s, dt=dt, full_step=0, obs_capacity=steps + 8, r_Sinv=10.0, r_T=10.0, r_U=10.0, r_K=rk,
                     r_M=rk)
        ctx.inverse()
        ctx.set_density_dense(0, 0, K0)
        q0 = float(np.sum(K0 * s.to_dense("S").T))
        ctx.kick(0, 0, 0, kappa)
        ctx.propagator(0.0)
        ctx.step(steps)
        obs = ctx.observables(0, 0)
        blocks = ctx.pattern(0, rtm.RT_PAT_K)[1].size / s.n_atoms
        ctx.close()
        t = obs[:, 0]
        alpha = spectra.polarizability(t, obs[:, 3] - obs[0, 3], kappa, omegas, damping=0.05)
        Sw = spectra.strength_function(omegas, [alpha, 0 * alpha, 0 * alpha])
        spec[rk] = (Sw, {"r_K": rk, "blocks_per_atom_K": blocks,
                         "charge_step1_minus_exact_K0": float(obs[0, 1] - q0),
                         "charge_drift": float(np.abs(obs[:, 1] - obs[0, 1]).max()),
                         "f_sum": spectra.f_sum(omegas, Sw), "peaks": spectra.peaks(omegas, Sw, 4).tolist()})
    ref = spec[15.0][0]
    out["spectrum_vs_r_K"] = {
        "system": f"{s.n_atoms} atoms sp4, gap {gap:.4f} Ha, kick {kappa} x, dt {dt}, {steps} steps, damping 0.05",
        "runs": [dict(v[1], rel_l2_vs_dense=float(np.linalg.norm(v[0] - ref) / np.linalg.norm(ref)))
                 for v in spec.values()]}
    out["wall_s"] = round(time.perf_counter() - t_start, 1)
    print(json.dumps(out))


def scaling_study(args):
    """Linear-scaling sweep (4-function diamond cells from 4096 to 32768 atoms,
    r = 8 A, x, y and z kicks batched in one context): time per full step of
    the FP64 and mixed paths, device memory and the mixed path's dipole
    agreement, against the atom count."""
    import torch

    import synth

    import paper_1404_5776_gb300 as rtm
    rtm.build()
    basis = "sp4"
    R = args.radius
    small = argparse.Namespace(basis=basis)
    mu, e_lo, e_hi = model_spectrum(small)
    common = dict(dt=0.05, prop=args.prop, n_kick=3, obs_capacity=64, r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    recs = []
    t_start = time.perf_counter()
    for ncell in (8, 10, 12, 14, 16):
        t0 = time.perf_counter()
        s = synth.diamond_system(ncell, basis, 7.0, 7.0)
        t_build = time.perf_counter() - t0
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base_mem = torch.cuda.memory_allocated()
        c64 = rtm.RT(s, precision="fp64", **common)
        c64.inverse()
        c64.ground_state(0, args.foe_order, mu, 0.01, e_lo, e_hi)
        for k in range(3):
            c64.kick(0, k, k, 1e-3)
        K1 = [c64.matrix(0, rtm.RT_MAT_K, k) for k in range(3)]
        mem64 = (torch.cuda.max_memory_allocated() - base_mem) / 1e9
        c32 = rtm.RT(s, precision="fp32", **common)
        c32.inverse()
        for k in range(3):
            c32.set_density(0, k, K1[k])
        mem_both = (torch.cuda.max_memory_allocated() - base_mem) / 1e9
        res = {}
        for name, ctx in (("fp64", c64), ("mixed", c32)):
            ctx.step(args.warmup)
            ctx.synchronize()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.step(args.steps)
            e1.record()
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / args.steps
        err_P = err_ind = 0.0
        for k in range(3):
            o64, o32 = c64.observables(0, k), c32.observables(0, k)
            p64, p32 = o64[:, 3 + 2 * k], o32[:, 3 + 2 * k]
            ind = np.abs(p64 - p64[0]).max()
            err_P = max(err_P, float(np.abs(p32 - p64).max() / np.abs(p64).max()))
            err_ind = max(err_ind, float(np.abs(p32 - p64).max() / ind) if ind > 0 else 0.0)
        f64, _ = c64.step_work()
        recs.append({"n_atoms": s.n_atoms, "n": int(s.n), "blocks_per_atom_K": c64.pattern(0, rtm.RT_PAT_K)[1].size / s.n_atoms,
                     "ms_per_step_fp64": round(res["fp64"], 3), "ms_per_step_mixed": round(res["mixed"], 3),
                     "us_per_atom_step_mixed": round(1e3 * res["mixed"] / s.n_atoms, 4),
                     "gflops_fp64": round(f64 / res["fp64"] / 1e6, 1), "gflops_mixed": round(f64 / res["mixed"] / 1e6, 1),
                     "device_gb_fp64_context": round(mem64, 3), "device_gb_both_contexts": round(mem_both, 3),
                     "dipole_err_rel_P_max_over_kicks": err_P, "dipole_err_rel_induced_max_over_kicks": err_ind,
                     "compared_steps": int(args.steps + args.warmup), "host_build_s": round(t_build, 1)})
        c64.close()
        c32.close()
        del K1
        torch.cuda.empty_cache()
    out = {"study": "scaling", "workload": f"diamond cells, {basis}, r_S=r_H=7A, all step radii {R:g}A, EM, "
                                           "x, y and z kicks 1e-3 batched (3 K per system)",
           "steps": args.steps, "warmup": args.warmup, "runs": recs, "wall_s": round(time.perf_counter() - t_start, 1)}
    print(json.dumps(out))


def kernel_case(args):
    """The headline mixed step alone (reference split, or with --literal the
    literal FP32 path) on the given cell, for ncu captures that must hold only a
    few GB: FOE ground state, x kick, W warm-up steps, K steps with per-class
    CUDA-event times."""
    import torch

    import paper_1404_5776_gb300 as rtm
    rtm.build()
    s = workload(args)
    mu, e_lo, e_hi = model_spectrum(args)
    R = args.radius
    kw = dict(precision="fp32", tensor_cores=1 if args.tensor_cores else 0, packed_fma=0 if args.scalar_fma else 1)
    if not args.literal and args.prop == "em":
        kw.update(incremental=1, field_poly=1)
    ctx = rtm.RT(s, dt=0.05, prop=args.prop, obs_capacity=args.steps + args.warmup + 8,
                 r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R, **kw)
    ctx.inverse()
    ctx.ground_state(0, args.foe_order, mu, 0.01, e_lo, e_hi)
    ctx.kick(0, 0, 0, 1e-3)
    ctx.step(args.warmup)
    ctx.synchronize()
    ctx.profile(True)
    nvtx_push(torch, "timed_kernel_case")
    ctx.step(args.steps)
    nvtx_pop(torch)
    pr = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    print(json.dumps({"kernel_case": cfg_name(args), "path": "literal" if args.literal else "reference split",
                      "steps": args.steps, "warmup": args.warmup,
                      "device_mem_gb": round(torch.cuda.max_memory_allocated() / 1e9, 2),
                      "per_launch_ms": {k: round(v["ms"] / v["launches"], 4) for k, v in pr.items() if v["launches"]}}))


def batching_study(args):
    """Several systems of uneven size and block size in one context, each with
    x, y and z kicks, advanced together (one graph per step): diamond cells of
    512 ... 8000 atoms (13 functions for 512, 1728, 4096, 8000; 4 for 1000,
    2744, 5832) and the H-terminated Si cluster (4 and 1 functions), r = 8 A.
    Mixed precision (reference split) timed over K steps; the FP64 run over the
    same steps for the dipole agreement.  The two contexts run one after the
    other (together they would not fit in device memory)."""
    import torch

    import synth

    import paper_1404_5776_gb300 as rtm
    rtm.build()
    R = 8.0  # the batching workload's radius
    spec = [(4, "spd13"), (5, "sp4"), (6, "spd13"), (7, "sp4"), (8, "spd13"), (9, "sp4"), (10, "spd13")]
    t0 = time.perf_counter()
    systems = [synth.diamond_system(nc, b, 7.0, 7.0) for nc, b in spec]
    pos, species = synth.si_h_cluster(target=1200)
    systems.append(synth.build_system(pos, None, species, 7.0, 7.0))
    t_build = time.perf_counter() - t0
    cl = systems[-1]
    K0c, _, gap_c = synth.ground_state_dense(cl, int(np.sum(cl.bsize)) // 2)
    spectra_by_basis = {b: model_spectrum(argparse.Namespace(basis=b)) for b in ("sp4", "spd13")}
    common = dict(dt=0.05, prop="em", n_kick=3, obs_capacity=args.steps + args.warmup + 16,
                  r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)

    # FP64 context: ground states (FOE; the cluster by dense diagonalisation), x/y/z kicks
    torch.cuda.reset_peak_memory_stats()
    c64 = rtm.RT(systems, precision="fp64", **common)
    c64.inverse()
    for si, (nc, b) in enumerate(spec):
        mu, e_lo, e_hi = spectra_by_basis[b]
        c64.ground_state(si, args.foe_order, mu, 0.01, e_lo, e_hi)
    for k in range(3):
        c64.set_density_dense(len(spec), k, K0c)
    for si in range(len(systems)):
        for k in range(3):
            c64.kick(si, k, k, 1e-3)
    K1 = {(si, k): c64.matrix(si, rtm.RT_MAT_K, k) for si in range(len(systems)) for k in range(3)}
    # the FP64 run over every step the mixed run takes, then its context is freed
    n64 = 1 + args.warmup + args.steps
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c64.step(n64)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / n64
    o64s = {(si, k): c64.observables(si, k) for si in range(len(systems)) for k in range(3)}
    mem64 = torch.cuda.max_memory_allocated() / 1e9
    c64.close()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    # mixed context (reference split, EM field polynomial) from the same K(0+);
    # its grouped products (one launch per product and block size) tuned
    c32 = rtm.RT(systems, precision="fp32", incremental=1, field_poly=1, **common)
    c32.inverse()
    for (si, k), Kv in K1.items():
        c32.set_density(si, k, Kv)
    del K1
    c32.step(1)  # the reference (K_ref, the B_p of every system)
    tuned = c32.autotune(reps=2)
    c32.step(args.warmup)
    c32.synchronize()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    nvtx_push(torch, "timed_batch_fp32")
    c32.step(args.steps)
    nvtx_pop(torch)
    e1.record()
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1) / args.steps
    launches = c32.step_kernels()
    flops, _ = c32.step_work()
    mem32 = torch.cuda.max_memory_allocated() / 1e9
    runs = []
    for si, (nc, b) in enumerate(spec + [(None, "si_h")]):
        for k in range(3):
            o64 = o64s[(si, k)]
            o32 = c32.observables(si, k)[:len(o64)]
            p64, p32 = o64[:, 3 + 2 * k], o32[:, 3 + 2 * k]
            ind = np.abs(p64 - p64[0]).max()
            runs.append({"system": si, "atoms": int(systems[si].n_atoms), "basis": b, "kick": "xyz"[k],
                         "dipole_err_rel_P": float(np.abs(p32 - p64).max() / np.abs(p64).max()),
                         "dipole_err_rel_induced": float(np.abs(p32 - p64).max() / ind) if ind > 0 else None})
    c32.close()
    n_atoms = sum(int(x.n_atoms) for x in systems)
    out = {"study": "batching", "systems": [{"atoms": int(x.n_atoms), "functions": int(x.n)} for x in systems],
           "total_atoms": n_atoms, "kicks": 3, "radius_A": R, "steps": args.steps, "warmup": args.warmup,
           "cluster_gap_Ha": gap_c, "host_build_s": round(t_build, 1),
           "mixed": {"path": "reference split, EM field polynomial; one launch per product and block size",
                     "ms_per_step": round(ms32, 3), "batch_steps_per_s": round(1e3 / ms32, 3),
                     "atom_kick_steps_per_s": round(3 * n_atoms * 1e3 / ms32, 1),
                     "algorithmic_tflops": round(flops / ms32 / 1e9, 2), "kernels_per_step": int(launches),
                     "launch_shapes": {c32.STAGES[st]: {"stages_per_warp": v[0], "persistent": v[1]}
                                       for st, v in tuned["chosen"].items()},
                     "tuning_ms": [{k: r[k] for k in ("what", "stages_per_warp", "persistent", "ms")}
                                   for r in tuned["rows"]]},
           "device_gb": {"fp64_context": round(mem64, 2), "mixed_context": round(mem32, 2)},
           "fp64": {"ms_per_step": round(ms64, 1), "timed_steps": n64},
           "speedup_mixed_vs_fp64": round(ms64 / ms32, 2),
           "dipole_agreement_over_fp64_steps": runs}
    print(json.dumps(out))


def propagators_study(args, timing_only=False):
    """EM, ETRS, M4 and CN (Sec. II.A) under a Gaussian pulse on a 512-atom cell
    (13 functions, r = 8 A): dipole error against an M4 run at dt/8, charge
    drift, S-unitarity of the last U and time per step, for several dt, FP64
    and mixed.  timing_only: time per step of each propagator over the first
    20 steps (dt = 0.05), FP64 and mixed, and their dipole difference."""
    import torch

    import synth

    import paper_1404_5776_gb300 as rtm
    rtm.build()
    s = synth.diamond_system(4, "spd13", 7.0, 7.0)
    K0, _, gap = synth.ground_state_dense(s, 2 * s.n_atoms)
    R = 8.0
    radii = dict(r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    t_end = 4.0
    field = dict(kind=rtm.RT_FIELD_GAUSSIAN, dir=0, E0=5e-3, t0=1.0, sigma=0.3, omega=0.6)

    def run(prop, dt, precision="fp64"):
        n = int(round((1.0 if timing_only else t_end) / dt))
        ctx = rtm.RT(s, dt=dt, prop=prop, precision=precision, obs_capacity=n + 8, **radii)
        ctx.set_field(**field)
        ctx.inverse()
        ctx.set_density_dense(0, 0, K0)
        ctx.step(2)  # warm-up (graph capture), then restart from K0
        ctx.set_density_dense(0, 0, K0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(n)
        e1.record()
        torch.cuda.synchronize()
        obs = ctx.observables(0, 0)
        u = ctx.unitarity(0, True)
        ctx.close()
        return obs, e0.elapsed_time(e1) / n, u

    if timing_only:
        # time per step of every propagator, FP64 and mixed, over the first
        # 20 steps of the same run (dt = 0.05), and the mixed run's dipole
        # against the FP64 run of the same propagator
        recs = []
        for prop in ("em", "etrs", "m4", "cn"):
            o64, ms64, u64 = run(prop, 0.05, "fp64")
            o32, ms32, u32 = run(prop, 0.05, "fp32")
            recs.append({"prop": prop, "ms_per_step_fp64": round(ms64, 3), "ms_per_step_mixed": round(ms32, 3),
                         "speedup": round(ms64 / ms32, 2),
                         "dipole_mixed_vs_fp64_rel_P": float(np.abs(o32[:, 3] - o64[:, 3]).max()
                                                             / np.abs(o64[:, 3]).max()),
                         "unitarity_max_fp64": u64[0], "unitarity_max_mixed": u32[0]})
        print(json.dumps({"study": "propagator-timing", "system": f"{s.n_atoms} atoms x 13, r = 8 A",
                          "field": "gaussian E0 5e-3, t0 1.0, sigma 0.3, omega 0.6, along x",
                          "dt": 0.05, "steps": 20, "runs": recs}))
        return
    ref_obs, _, _ = run("m4", 0.05 / 8)
    t_ref = ref_obs[:, 0]
    p_ref = ref_obs[:, 3]
    recs = []
    for dt in (0.05, 0.1, 0.2):
        for prop in ("em", "etrs", "m4", "cn"):
            for precision in ("fp64", "fp32"):
                obs, ms, u = run(prop, dt, precision)
                idx = np.searchsorted(t_ref, obs[:, 0] - 1e-9)
                ok = idx < len(t_ref)
                err = np.abs(obs[ok, 3] - p_ref[idx[ok]]).max()
                swing = np.abs(p_ref - p_ref[0]).max()
                recs.append({"prop": prop, "dt": dt, "precision": precision, "ms_per_step": round(ms, 3),
                             "dipole_err_vs_ref_rel_swing": float(err / swing),
                             "charge_drift_rel": float(np.abs(obs[:, 1] - obs[0, 1]).max() / abs(obs[0, 1])),
                             "unitarity_max": u[0]})
    print(json.dumps({"study": "propagators", "system": f"{s.n_atoms} atoms x 13, r = 8 A, gap {gap:.3f} Ha",
                      "field": "gaussian E0 5e-3, t0 1.0, sigma 0.3, omega 0.6, along x", "t_end": t_end,
                      "reference": "M4 at dt = 0.05/8, FP64", "runs": recs}))


def main():
    args = parse()
    if args.study in ("propagators", "propagator-timing"):
        propagators_study(args, timing_only=args.study == "propagator-timing")
        return
    if args.study == "batching":
        batching_study(args)
        return
    if args.kernel_case:
        kernel_case(args)
        return
    if args.study == "truncation":
        truncation_study(args)
        return
    if args.study == "scaling":
        scaling_study(args)
        return
    if args.precision_study:
        precision_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
