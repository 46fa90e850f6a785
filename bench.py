#!/usr/bin/env python
"""Benchmark of the C-PCM / ISWIG hot path on one GB300 (or N, as replicas).

One step is one pass of the whole path over one synthetic molecule:
surface build (points, switching, Bz and the solver's operator), basis and
primitive-pair list with screening, ESP c, rhs, PCG solve (RBJ, threshold of
Eq. 21 for a 1e-6 Eh energy error), Fock correction dF and the Eq. 13 energy.

Metric: ESP + Fock equivalent Cartesian primitive integrals per second
(kept primitive pairs x ncart(a) ncart(b) x M, summed over the ESP and the
Fock call of a step) divided by the step time; the PCG solve time is
reported beside it.  Default workload: the 1000-atom H:C:N:O:S =
50:31:9:9:1 cluster with 6-31G*-like s/sp/d shells (nbf ~ 8.5k), 2000
occupied orbitals, 110 points per sphere at 1.2 x Bondi (M ~ 46k).  The
timed path is PCM_MIXED (FP32 integrals, FP64 accumulation, refinement with
double-float residuals) unless --precision fp64; the PCM_FP64 step is timed
beside it, and the energy of the timed solve is compared with an FP64 solve
at delta = 1e-10.  The 300-atom s/sp cluster (nbf ~ 1.66k, M ~ 12k) is
timed the same way as a sub-record.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cluster1000_spd|cluster300_sp|cluster300_spd|water|batch]

With N > 1 (torchrun) every rank runs its own conformation (seed offset by
rank): independent problems, no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "ESP+Fock integrals/s & PCG solve ms: mixed/batched vs FP64, at 1e-6 Eh"
UNIT = "integrals/s"
# Eq. 21: Err(delta) = 0.01 delta^1.07 = 1e-6 Eh
DELTA_1E6 = (1e-6 / 0.01) ** (1.0 / 1.07)
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz


# --------------------------------------------------------------------------
# algorithmic FP64 operation counts per pair-point interaction
# --------------------------------------------------------------------------
def _nherm(L):
    return (L + 1) * (L + 2) * (L + 3) // 6


def _hermite_ops(L):
    ops = 0
    for n in range(L, -1, -1):
        D = L - n
        for d in range(1, D + 1):
            for t in range(d, -1, -1):
                for u in range(d - t, -1, -1):
                    v = d - t - u
                    k = t if t > 0 else (u if u > 0 else v)
                    ops += 1 + (2 if k > 1 else 0)
    return ops


def flops_per_interaction(L, kind):
    """Operations of the algorithm (an FMA counts 2): distance and T (9),
    Boys F_0..F_L by 7-term Taylor (7 + 12 (L+1)), (-2 rho)^n scaling (2L),
    Hermite recurrence, then the ESP dot (2 nherm + 2) or the Fock
    accumulation (1 + nherm)."""
    base = 9 + 7 + 12 * (L + 1) + 2 * L + _hermite_ops(L)
    if kind == "esp":
        return base + 2 * _nherm(L) + 2
    return base + 1 + _nherm(L)


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz

# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels (profiles/); a kernel missing here reports traffic null.  The ESP ps
# class of the 1000-atom cluster: its packed kernel esp_kernel_f32x2<1, 2>
# read 105,000,704 and wrote 6,144,768 bytes in one launch (the class's
# one-centre kernel and reduction add a few MB more).
NCU_TRAFFIC_BYTES = {
    ("cluster1000_spd", "ESP ps class: esp_kernel_f32x2<L=1> + same-atom pairs (esp_kernel_f32) + reduction"):
        105000704 + 6144768,
}

CLASS_L = [0, 1, 2, 2, 3, 4]
CLASS_NAME = ["ss", "ps", "pp", "ds", "dp", "dd"]


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU)
# --------------------------------------------------------------------------
def dist_init(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return rank, world, local


def dist_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units, ms, world, device):
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time.  Returns (units/s, max ms)."""
    ms_max = dist_max(ms, world, device)
    return dist_sum(units, world, device) / (ms_max * 1e-3), ms_max


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


WORKLOADS = {"water": 0, "cluster300_sp": 1, "cluster1000_spd": 2, "cluster300_spd": 3}
DEFAULT_WORKLOAD = "cluster1000_spd"
# oracle points per sample: about 10-30 s of host work on 16 cores (cpu_baseline),
# and a few seconds per step of the reference arm
CPU_POINTS = {"water": 252, "cluster300_sp": 320, "cluster1000_spd": 16, "cluster300_spd": 96}
REF_POINTS = {"water": 252, "cluster300_sp": 16, "cluster1000_spd": 2, "cluster300_spd": 8}


def workload_for(name, rank):
    i = WORKLOADS[name]
    if rank == 0:
        return workloads.config(i)
    w0 = workloads.config(i)
    seed = w0.seed + 1000 * rank
    return workloads.cluster(w0.mol.natom, seed, workloads.GLOBULE_RADIUS_A[w0.mol.natom],
                             d_shells=name.endswith("_spd"), nocc=w0.nocc, name=w0.name + "_r%d" % rank)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def _timed_steps(pcm, w, precision, args, dev, stream, flush, delta, steps, warmup):
    """Warm up, then time `steps` whole-path steps with CUDA events on the
    library's stream; L2 is flushed between steps outside the events."""
    import torch
    ctx = pcm.Context(precision=precision, device=dev.index, stream=stream.cuda_stream, timing=True,
                      seed=args.seed, autotune=(precision == "mixed" and args.autotune),
                      fp32x2=not args.scalar_fp32, operator=args.operator)
    b = w.basis
    Pd = torch.tensor(w.P, dtype=torch.float64, device=dev)
    bufs = {}

    phase = {k: 0.0 for k in ("surface", "basis", "esp", "solve", "fock", "energy")}

    def mark(ev):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        ev.append(e)

    def step(timed=False):
        ev = []
        mark(ev)
        M = ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
        mark(ev)
        nbf = ctx.set_basis(b.shell_atom, b.shell_l, b.shell_nprim, b.exps, b.coefs)
        mark(ev)
        if "c" not in bufs or bufs["c"].numel() != M:
            bufs["c"] = torch.empty(M, dtype=torch.float64, device=dev)
            bufs["q"] = torch.empty(M, dtype=torch.float64, device=dev)
            bufs["dF"] = torch.empty((nbf, nbf), dtype=torch.float64, device=dev)
        ctx.esp(Pd, out=bufs["c"])
        mark(ev)
        q, st = ctx.solve(delta=delta, q=bufs["q"])
        mark(ev)
        ctx.fock(q, out=bufs["dF"])
        mark(ev)
        E = ctx.energy(q)
        mark(ev)
        if timed:
            ev[-1].synchronize()
            for k, a, b_ in zip(phase, ev[:-1], ev[1:]):
                phase[k] += a.elapsed_time(b_)
        return E, st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.stats()["launches"]
    out = {"times": [], "solve_ms": [], "iters": [], "E": [], "ints": 0.0, "esp_cls": np.zeros(6),
           "fock_cls": np.zeros(6)}
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E, st = step(timed=True)
        e1.record(stream)
        e1.synchronize()
        out["times"].append(e0.elapsed_time(e1))
        s = ctx.stats()
        out["solve_ms"].append(s["ms_solve"])
        out.setdefault("precond_ms", []).append(s["ms_precond"])
        out["iters"].append(st["iterations"])
        out["E"].append(E)
        out["ints"] += s["integrals_esp"] + s["integrals_fock"]
        out["esp_cls"] += np.array(s["ms_esp_class"])
        out["fock_cls"] += np.array(s["ms_fock_class"])
    s = ctx.stats()
    out["phase_ms"] = {k: v / max(1, steps) for k, v in phase.items()}
    out["launches"] = s["launches"] - launches0
    out["stats"] = s
    out["ctx"] = ctx
    out["bufs"] = bufs
    out["Pd"] = Pd
    return out


def _time_gradient(res, q, flush, stream, steps):
    """Nuclear gradient (Eq. 14) on the step's final state: CUDA-event time
    per call, L2 flushed before each call.  Returns (ms, gradient, stats)."""
    import torch
    ctx, Pd = res["ctx"], res["Pd"]
    g = torch.empty((ctx.natom, 3), dtype=torch.float64, device=Pd.device)
    ctx.gradient(q, Pd, out=g)                      # warm-up
    ts = []
    for _ in range(max(1, steps)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.gradient(q, Pd, out=g)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts), g.cpu().numpy(), ctx.stats()


def _dominant(res, precision, steps, packed=True, measured=None):
    """The step's longest integral class: its algorithmic flops (the per-
    interaction figures of flops_per_interaction, the same in both precisions
    and for near and far pairs) over its CUDA-event time, against the nominal
    pipe peak of its precision (unit counts x maximum clock) and, when given,
    the pipe rate pcm_pipe_peak measured on this GPU."""
    s = res["stats"]
    M = s["M"]
    tag = "f64" if precision == "fp64" else ("f32x2" if packed else "f32")
    cand = []
    for k in range(6):
        for kind, ms in (("esp", res["esp_cls"][k]), ("fock", res["fock_cls"][k])):
            if ms > 0:
                n = s["%s_class_pairs" % kind][k] * M
                if precision == "fp64":
                    label = "%s %s class: %s_kernel_f64<L=%d>" % (kind.upper(), CLASS_NAME[k], kind, CLASS_L[k])
                else:
                    rest = "same-atom pairs (esp_kernel_f32) + reduction" if kind == "esp" else "epilogue"
                    label = ("%s %s class: %s_kernel_%s<L=%d> + %s"
                             % (kind.upper(), CLASS_NAME[k], kind, tag, CLASS_L[k], rest))
                cand.append((label, ms / steps, n * flops_per_interaction(CLASS_L[k], kind)))
    name, ms_k, flops_k = max(cand, key=lambda t: t[1])
    peak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = flops_k / (ms_k * 1e-3) / 1e12
    src = ("nominal FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz" if precision == "fp64" else
           "nominal FP32 pipe: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz")
    out = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "peak_source": src, "kernel_ms": ms_k,
           "flops": "algorithmic: flops_per_interaction (Hermite form with Boys F_0..F_L) x pair-point "
                    "interactions; far pairs run a cheaper multipole form and count the same"}
    out["classes"] = {lab.split(" class")[0]: {"ms": round(t, 3), "achieved": round(f / (t * 1e-3) / 1e12, 3),
                                              "frac": round(f / (t * 1e-3) / 1e12 / peak, 3)}
                      for lab, t, f in cand}
    if measured:
        key = "fp64" if precision == "fp64" else ("fp32x2" if packed else "fp32")
        out["peak_measured"] = measured[key]
        out["peak_measured_source"] = "pcm_pipe_peak(%s): independent FMA chains, CUDA events" % key
        out["frac_of_measured"] = achieved / measured[key]
    return out


def _reference_energy(pcm, w, dev, stream):
    """The FP64 path with a tight solve (delta = 1e-10), not timed."""
    with pcm.Context(precision="fp64", device=dev.index, stream=stream.cuda_stream) as ref:
        ref.setup(w.mol, w.basis)
        ref.esp(w.P)
        qr, _ = ref.solve(delta=1e-10)
        return ref.energy(qr)


def _measure(pcm, w, args, dev, stream, flush, delta, steps, warmup, fp64_steps):
    """Time `steps` steps of the requested precision and, for PCM_MIXED,
    `fp64_steps` PCM_FP64 steps of the same workload; energies against the
    FP64 delta = 1e-10 solve."""
    E_ref = _reference_energy(pcm, w, dev, stream)
    main = _timed_steps(pcm, w, args.precision, args, dev, stream, flush, delta, steps, warmup)
    torch_sync()
    other = None
    if args.precision == "mixed" and fp64_steps > 0:
        other = _timed_steps(pcm, w, "fp64", args, dev, stream, flush, delta, fp64_steps, 1)
    return E_ref, main, other


def torch_sync():
    import torch
    torch.cuda.synchronize()


def _fp64_record(other, E_ref, world, pipe=None):
    n = len(other["times"])
    return {"value": other["ints"] * world / (sum(other["times"]) * 1e-3), "unit": UNIT,
            "ms_per_step": sum(other["times"]) / n, "steps": n,
            "pcg_solve_ms": statistics.mean(other["solve_ms"]), "pcg_iterations": statistics.mean(other["iters"]),
            "esp_kernel_ms": float(other["esp_cls"].sum() / n),
            "fock_kernel_ms": float(other["fock_cls"].sum() / n),
            "energy_err_Eh": abs(other["E"][-1] - E_ref), "phase_ms": other["phase_ms"],
            "roofline": _dominant(other, "fp64", n, measured=pipe)}


def _small_record(pcm, args, dev, stream, flush, delta, pipe=None):
    """The 300-atom s/sp cluster (nbf ~ 1.66k, M ~ 12k), timed as the main
    workload: mixed steps, one FP64 step, energies against delta = 1e-10."""
    w = workloads.config(WORKLOADS["cluster300_sp"])
    E_ref, main, other = _measure(pcm, w, args, dev, stream, flush, delta, max(3, args.steps), 3, 1)
    n = len(main["times"])
    s = main["stats"]
    rec = {"workload": w.name, "natom": w.mol.natom, "nbf": s["nbf"], "M": s["M"], "precision": args.precision,
           "value": main["ints"] / (sum(main["times"]) * 1e-3), "unit": UNIT, "steps": n,
           "ms_per_step": sum(main["times"]) / n, "pcg_solve_ms": statistics.mean(main["solve_ms"]),
           "pcg_iterations": statistics.mean(main["iters"]), "energy_err_Eh": abs(main["E"][-1] - E_ref),
           "phase_ms": main["phase_ms"], "roofline": _dominant(main, args.precision, n, packed=not args.scalar_fp32, measured=pipe)}
    if other is not None:
        rec["fp64"] = _fp64_record(other, E_ref, 1, pipe)
        rec["speedup_vs_fp64"] = rec["fp64"]["ms_per_step"] / rec["ms_per_step"]
    main["ctx"].close()
    if other is not None:
        other["ctx"].close()
    return rec


def run_ours(args):
    import torch
    rank, world, local = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1505_07851_gb300 as pcm

    w = workload_for(args.workload, rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    delta = args.delta if args.delta else DELTA_1E6
    b = w.basis
    E_ref = _reference_energy(pcm, w, dev, stream)

    barrier(world)
    with ClockSampler(local) as clk:
        main = _timed_steps(pcm, w, args.precision, args, dev, stream, flush, delta, args.steps, args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    other = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        other = _timed_steps(pcm, w, "fp64", args, dev, stream, flush, delta, args.fp64_steps, 1)

    value, total_ms_max = replica_throughput(main["ints"], sum(main["times"]), world, dev)
    pipe = {k: pcm.pipe_peak(k, local) for k in ("fp32", "fp32x2", "fp64")}
    roofline = _dominant(main, args.precision, args.steps, packed=not args.scalar_fp32, measured=pipe)
    roofline["traffic"] = args.traffic if args.traffic is not None else \
        NCU_TRAFFIC_BYTES.get((w.name, roofline["kernel"]))
    s = main["stats"]
    ctx = main["ctx"]

    # end-to-end through the public API with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Ph = np.ascontiguousarray(w.P)
        h2d = Ph.nbytes + w.mol.xyz.nbytes + w.mol.Z.nbytes + w.mol.radius.nbytes + \
            b.shell_atom.nbytes + b.shell_l.nbytes + b.shell_nprim.nbytes + b.exps.nbytes + b.coefs.nbytes
        et = []
        for it in range(max(1, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
            ctx.set_basis(b.shell_atom, b.shell_l, b.shell_nprim, b.exps, b.coefs)
            ch = ctx.esp(Ph)
            qh, _ = ctx.solve(delta=delta)
            Fh = ctx.fock(qh)
            ctx.energy(qh)
            et.append(time.perf_counter() - t0)
        d2h = ch.nbytes + qh.nbytes + Fh.nbytes + 8
        e_val, e_ms = replica_throughput(main["ints"] * len(et) / args.steps, sum(et) * 1e3, world, dev)
        e2e = {"value": e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms / len(et)}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(w, args.cpu_points or CPU_POINTS.get(w.name, 16))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32/f64",
            "data": "synthetic (seeded protein-shaped cluster; no PDB/basis data in this container)",
            "config": {"workload": w.name, "natom": w.mol.natom, "nbf": s["nbf"], "M": s["M"],
                       "pts_per_sphere": 110, "precision": args.precision, "delta": delta,
                       "fp32_instructions": "scalar" if args.scalar_fp32 else "packed x2",
                       "precond": "rbj-100" if s["M"] >= 1000 else "jacobi",
                       "l2": "flushed between timed steps (512 MB write, not timed)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "pcg_solve_ms": statistics.mean(main["solve_ms"]), "pcg_iterations": statistics.mean(main["iters"]),
            "operator_build_ms_side_stream": statistics.mean(main["precond_ms"]),
            "energy_Eh": main["E"][-1], "energy_ref_fp64_Eh": E_ref,
            "energy_err_Eh": abs(main["E"][-1] - E_ref),
            "esp_kernel_ms": float(main["esp_cls"].sum() / args.steps),
            "fock_kernel_ms": float(main["fock_cls"].sum() / args.steps),
            "esp_class_ms": [float(x) / args.steps for x in main["esp_cls"]],
            "fock_class_ms": [float(x) / args.steps for x in main["fock_cls"]],
            "integrals_per_step": main["ints"] / args.steps, "pairs_kept": s["pairs_kept"],
            "phase_ms": main["phase_ms"],
            "roofline": roofline, "pipe_peaks_measured_tflops": pipe,
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": main["launches"],
            "autotune": pcm.autotune_table(),
            "cpu_baseline": cpu,
        }
        if other is not None:
            line["fp64"] = _fp64_record(other, E_ref, world, pipe)
            line["speedup_vs_fp64"] = line["fp64"]["ms_per_step"] / line["ms_per_step"]
        if not args.no_grad:
            q = main["bufs"]["q"]
            g_ms, g_main, gst = _time_gradient(main, q, flush, stream, args.steps)
            grad = {"ms": g_ms, "integrals_per_s": gst["integrals_grad"] / (g_ms * 1e-3),
                    "precision": args.precision}
            if other is not None:
                # the FP64 gradient with the same charges
                g64_ms, g64, _ = _time_gradient(other, q, flush, stream, 1)
                grad.update(fp64_ms=g64_ms, speedup_vs_fp64=g64_ms / g_ms,
                            max_abs_diff_vs_fp64_Eh_per_bohr=float(np.max(np.abs(g_main - g64))))
            line["gradient"] = grad
        if other is not None:
            other["ctx"].close()
            other = None
        if not args.no_precond:
            # Section 4b-ii: CG steps and solve time per preconditioner (FP64, fixed delta = 1e-6) on the
            # step's own right-hand side -f (Bz + c)
            f = (78.39 - 1.0) / 78.39
            Bz = torch.empty_like(main["bufs"]["c"])
            ctx.esp(main["Pd"], out=main["bufs"]["c"], bz_out=Bz)
            rhs = -f * (Bz + main["bufs"]["c"])
            pc = {}
            for name, kw in (("jacobi", {"precond": "jacobi"}), ("rbj-100", {"precond": "rbj", "rbj_block": 100}),
                             ("rbj-800", {"precond": "rbj", "rbj_block": 800}),
                             ("octree-800", {"precond": "octree", "octree_leaf": 800})):
                with pcm.Context(precision="fp64", timing=True, device=dev.index, stream=stream.cuda_stream,
                                 **kw) as pctx:
                    pctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
                    _, pst = pctx.solve(rhs=rhs, delta=1e-6)
                    pc[name] = {"cg_steps": pst["iterations"], "converged": bool(pst["converged"]),
                                "solve_ms_incl_setup": pst["ms_solve"], "setup_ms": pst["ms_precond"]}
            line["preconditioners"] = pc
        if not args.no_scf:
            # Section 4b-i: CG steps and solve time along a synthetic SCF history
            from paper_1505_07851_gb300.scf import run_sequence
            seq = workloads.scf_sequence(w, 14)
            sc = {}
            for scheme in ("fixed", "2delta", "dynamic"):
                rec = run_sequence(main["ctx"], seq, scheme, delta_tight=1e-6)
                sc[scheme] = {"cg_steps": [r["cg_steps"] for r in rec],
                              "total_cg_steps": sum(r["cg_steps"] for r in rec),
                              "total_solve_ms": sum(r["solve_ms"] for r in rec),
                              "final_energy_Eh": rec[-1]["energy"]}
            sc["workload"] = "%s, 14 iterations, DIIS error 0.1 x 0.4^n, warm start, delta_2 = 1e-6" % w.name
            line["scf_sequence"] = sc
        main["ctx"].close()
        if not args.no_small and w.name != "cluster300_sp":
            line["cluster300_sp"] = _small_record(pcm, args, dev, stream, flush, delta, pipe)
        if not args.no_batch:
            line["batch"] = measure_batch(pcm, args, dev, stream, flush, delta, steps=2, warmup=1,
                                          operator=args.batch_operator)
        print(json.dumps(line))
    else:
        main["ctx"].close()
        if other is not None:
            other["ctx"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# the oracle, timed on the host cores
# --------------------------------------------------------------------------
def _oracle_sample(w, npts, seed=0):
    import oracle
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(s["zeta"]), size=min(npts, len(s["zeta"])), replace=False))
    # equivalent Cartesian primitive integrals the oracle evaluates per point
    nc = (eb.sh_l + 1) * (eb.sh_l + 2) // 2
    w_sh = eb.sh_nprim * nc
    tot = float(w_sh.sum())
    per_point = 0.5 * (tot * tot + float((w_sh * w_sh).sum()))     # shell pairs A <= B
    return oracle, s, eb, idx, per_point


def cpu_baseline(w, npts):
    oracle, s, eb, idx, per_point = _oracle_sample(w, npts)
    t0 = time.perf_counter()
    oracle.esp(eb, w.P, s["r"][idx], s["zeta"][idx])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": per_point * len(idx) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle ESP (Obara-Saika, no screening) at %d of %d surface points over all "
                      "%d shell pairs; %.1f s" % (len(idx), len(s["zeta"]), eb.nshell * (eb.nshell + 1) // 2, dt)}


def run_reference(args):
    rank, world, local = dist_init("gloo")
    if rank != 0:
        return
    w = workloads.config(WORKLOADS[args.workload])
    npts = args.ref_points or REF_POINTS.get(w.name, 4)
    oracle, s, eb, idx_all, per_point = _oracle_sample(w, 10 ** 9)
    rng = np.random.default_rng(1)
    times = []
    ints = 0.0
    for it in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(s["zeta"]), size=npts, replace=False))
        t0 = time.perf_counter()
        oracle.esp(eb, w.P, s["r"][idx], s["zeta"][idx])
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            ints += per_point * len(idx)
    total = sum(times)
    value = ints / total
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = ("oracle ESP at %d random surface points per step over all %d shell pairs (the full "
              "step would need %d points)" % (npts, eb.nshell * (eb.nshell + 1) // 2, len(s["zeta"])))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "natom": w.mol.natom, "nbf": w.basis.nbf, "M": len(s["zeta"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _single_pass(pcm, w, precision, dev, stream, flush, delta):
    """One molecule through single-molecule calls (surface and basis set up
    and one warm pass untimed): the CUDA-event time of ESP + solve + Fock +
    energy, with L2 flushed before it.  Returns (ms, energy)."""
    import torch
    with pcm.Context(precision=precision, device=dev.index, stream=stream.cuda_stream) as ctx:
        M, nbf = ctx.setup(w.mol, w.basis)
        Pd = torch.tensor(w.P, dtype=torch.float64, device=dev)
        c = torch.empty(M, dtype=torch.float64, device=dev)
        q = torch.empty_like(c)
        F = torch.empty((nbf, nbf), dtype=torch.float64, device=dev)

        def once():
            ctx.esp(Pd, out=c)
            ctx.solve(delta=delta, q=q)
            ctx.fock(q, out=F)
            return ctx.energy(q)
        once()
        torch.cuda.synchronize()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E = once()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), E


def measure_batch(pcm, args, dev, stream, flush, delta, rank=0, world=1, nmol=None, steps=None, warmup=None,
                  operator="auto"):
    """The batch of conformations (150-600 atoms, s/sp shells): ESP + solve +
    Fock + energy for every molecule per step through pcm_batch_run (the
    packed integral blocks of all molecules in one launch per angular class,
    lockstep PCG), inputs resident on the device; beside it the same molecules
    one at a time through single-molecule calls (mixed), and a sample in FP64
    (time and energy error)."""
    import torch
    nmol = nmol or args.nmol
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    t0 = time.time()
    confs = workloads.conformations(nmol, seed=150507851 + 4 + 1000 * rank, workers=os.cpu_count() or 1)
    gen_s = time.time() - t0
    b = pcm.Batch(len(confs), precision=args.precision, device=dev.index, stream=stream.cuda_stream,
                  fp32x2=not args.scalar_fp32, operator=operator)
    t0 = time.time()
    for i, w in enumerate(confs):
        b.set_molecule(i, w.mol, w.basis)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    Pd = [torch.tensor(w.P, dtype=torch.float64, device=dev) for w in confs]
    Fd = [torch.empty((w.basis.nbf, w.basis.nbf), dtype=torch.float64, device=dev) for w in confs]
    for _ in range(warmup):
        b.run(Pd, delta, dF_out=Fd)
    torch.cuda.synchronize()
    launches0 = b.stats()["launches"]
    times, ints = [], 0.0
    with ClockSampler(dev.index) as clk:
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E, _, _ = b.run(Pd, delta, dF_out=Fd)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            tot = b.stats()
            ints += tot["integrals_esp"] + tot["integrals_fock"]
    torch.cuda.synchronize()
    tot = b.stats()
    launches = tot["launches"] - launches0
    per = [b.stats(i) for i in range(len(confs))]
    E = list(E)
    e2e = None
    if not args.no_e2e:
        Ph = [np.ascontiguousarray(w.P) for w in confs]
        Fh = [np.empty_like(P) for P in Ph]
        et = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            b.run(Ph, delta, dF_out=Fh)
            et.append(time.perf_counter() - t1)
        e2e = {"ms_per_step": 1e3 * statistics.mean(et), "h2d_bytes_per_step": int(sum(P.nbytes for P in Ph)),
               "d2h_bytes_per_step": int(sum(F.nbytes for F in Fh)) + 8 * len(confs)}
    b.close()
    ms = sum(times) / len(times)
    # the same molecules one at a time (PCM_MIXED single-molecule calls)
    seq = [_single_pass(pcm, w, args.precision, dev, stream, flush, delta) for w in confs]
    seq_ms = sum(t for t, _ in seq)
    # a sample in FP64: time per molecule and the error of the batch energies
    nref = min(args.ref_mols, len(confs))
    fp64 = []
    for i in range(nref):
        w = confs[i]
        t64, _ = _single_pass(pcm, w, "fp64", dev, stream, flush, delta)
        with pcm.Context(precision="fp64", device=dev.index, stream=stream.cuda_stream) as ctx:
            ctx.setup(w.mol, w.basis)
            ctx.esp(w.P)
            qt, _ = ctx.solve(delta=1e-10)
            fp64.append((t64, abs(E[i] - ctx.energy(qt))))
    Ms = [p["M"] for p in per]
    mixed_sample = sum(seq[i][0] for i in range(nref))
    fp64_sample = sum(t for t, _ in fp64)
    return {
        "workload": "batch%d_conformations_150to600_sp" % len(confs), "nmol": len(confs),
        "M_min": min(Ms), "M_max": max(Ms), "M_total": sum(Ms), "precision": args.precision, "delta": delta,
        "operator": operator, "steps": len(times), "ms_per_step": ms, "solves_per_s": len(confs) / (ms * 1e-3),
        "integrals_per_s": ints / (sum(times) * 1e-3), "gpu_launches_per_step": launches / len(times),
        "pcg_iterations_max": max(p["iterations"] for p in per),
        "pcg_iterations_mean": statistics.mean(p["iterations"] for p in per),
        "all_converged": all(p["converged"] for p in per),
        "sequential_mixed": {"ms_total": seq_ms, "solves_per_s": len(confs) / (seq_ms * 1e-3),
                             "batched_speedup": seq_ms / ms,
                             "what": "the same molecules one at a time: ESP + solve + Fock + energy through "
                                     "single-molecule contexts (set-up untimed), L2 flushed before each"},
        "fp64_sample": {"n": nref, "ms_total": fp64_sample, "mixed_ms_same_molecules": mixed_sample,
                        "fp64_over_mixed": fp64_sample / mixed_sample if mixed_sample else None,
                        "batch_energy_err_vs_fp64_Eh_max": max(e for _, e in fp64) if fp64 else None},
        "l2": "flushed between timed steps (512 MB write, not timed)",
        "setup_s": setup_s, "workload_generation_s": gen_s, "clocks": clk.summary(), "e2e": e2e,
        "M_range_note": "150-600 atoms at the density of the 300-atom cluster give 6.4k-22k points; "
                        "denser globules cannot place the atoms",
    }


def run_batch(args):
    """The batch workload alone: one JSON line with the batch record."""
    import torch
    rank, world, local = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1505_07851_gb300 as pcm
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    delta = args.delta if args.delta else DELTA_1E6
    rec = measure_batch(pcm, args, dev, stream, flush, delta, rank, world, operator=args.batch_operator)
    value, ms_max = replica_throughput(rec["integrals_per_s"] * rec["ms_per_step"] * 1e-3 * rec["steps"],
                                       rec["ms_per_step"] * rec["steps"], world, dev)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": rec["steps"],
                "warmup": args.warmup, "ms_per_step": ms_max / rec["steps"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32/f64",
                "data": "synthetic (seeded peptide-like clusters of 150-600 atoms)",
                "config": {"workload": rec["workload"], "nmol": rec["nmol"], "precision": args.precision,
                           "parallelism": "replicas" if world > 1 else "single", "l2": rec["l2"]},
                "batch": rec, "clocks": rec["clocks"], "e2e": None, "gpu_launches": rec["gpu_launches_per_step"]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batch"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="PCM_FP64 steps timed beside a mixed run (0: none)")
    ap.add_argument("--delta", type=float, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-points", type=int, default=None, help="oracle points of the cpu_baseline sample")
    ap.add_argument("--ref-points", type=int, default=None, help="oracle points per step of the reference arm")
    ap.add_argument("--traffic", type=float, default=None, help="DRAM bytes per launch of the dominant kernel (ncu)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-grad", action="store_true", help="skip the nuclear-gradient timing")
    ap.add_argument("--no-small", action="store_true", help="skip the 300-atom sub-record")
    ap.add_argument("--nmol", type=int, default=64, help="conformations in the batch workload")
    ap.add_argument("--operator", default="auto", choices=["auto", "stored", "free"],
                    help="PCM_MIXED operator of the single-molecule contexts (auto: matrix-free above 24576 points)")
    ap.add_argument("--batch-operator", default="auto", choices=["auto", "stored", "free"],
                    help="operator of the batch members (auto: stored, lockstep solver)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch sub-record")
    ap.add_argument("--ref-mols", type=int, default=4, help="batch members checked against the FP64 path")
    ap.add_argument("--no-scf", action="store_true", help="skip the SCF-sequence threshold comparison")
    ap.add_argument("--no-precond", action="store_true", help="skip the preconditioner comparison")
    ap.add_argument("--autotune", action="store_true", help="pick tile shapes by timed trials in the warm-up")
    ap.add_argument("--scalar-fp32", action="store_true",
                    help="scalar FP32 instructions in the mixed kernels instead of packed two-lane ones")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
