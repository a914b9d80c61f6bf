#!/usr/bin/env python
"""Benchmark of the fixed-point solver's hot path: voxel-iterations per second.

Workload (the 256^3 polycrystal of the paper's method at scale): 256^3 voxels,
Voronoi polycrystal of 500 grains (seeds uniform in the box, seed 2), cubic
elasticity C11 = 168, C12 = 121, C44 = 75 GPa with orientations uniform on
SO(3) (seed 3), small strain, double-tetrahedron (TETRA2) scheme, B0 Green
operator with lambda0 = C12 and mu0 = (C44 + (C11 - C12)/2)/2, Dirichlet on
the x faces (all components, eps_xx = 1e-3), Neumann y, periodic z,
equilibrium tolerance 1e-6, Anderson depth 4 every 3 iterations.

One step = one load step of Algorithm 1 from u^f = 0 to convergence (every
row of the hot path: gradient, law, divergence and norms, Anderson,
forward DTs, Green operator, inverse DTs).  value = voxels x iterations / time.

The device-resident number (`value`) times the steps with the phase map
already on the GPU; `e2e` times the same steps through the C ABI with host
buffers (phase map in, displacement field out, pinned memory).  The oracle
(CPU, FP64) is timed on a bounded sample beside it (`cpu_baseline`);
`--impl reference` times only the oracle.

Multi-GPU: each rank solves its own replica (replicas only; no collective on
the data path); value = all ranks' voxel-iterations / max rank time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s"
UNIT = "voxel-it/s"
def workload_name(n, grains):
    return (f"voronoi_polycrystal_{n}: {n}^3 voxels, {grains}-grain Voronoi, cubic elastic C11/C12/C44="
            "168/121/75 GPa, random orientations, TETRA2, B0, x Dirichlet / y Neumann / z periodic, "
            "eps_xx=1e-3, tol=1e-6, Anderson 4/3")
REF_SLAB = 32  # z-planes of the oracle's bounded sample


# ----------------------------------------------------------------------------------------
def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--grains", type=int, default=500)
    ap.add_argument("--precision", choices=["fp32", "fp32_tc", "fp32_tf32", "fp64"], default="fp32_tf32",
                    help="the headline path (default: FP32 fields with TF32 tensor-core transforms, the precision "
                         "form); the others are timed beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1, help="FP64 path steps timed beside (0 = skip)")
    ap.add_argument("--tc-steps", type=int, default=3,
                    help="tensor-core (FP32_TC) path steps timed beside the FP32 path (0 = skip)")
    ap.add_argument("--tf32-steps", type=int, default=3,
                    help="TF32 tensor-core (FP32_TF32) path steps timed beside the headline (0 = skip)")
    ap.add_argument("--fp32-steps", type=int, default=3,
                    help="FP32 path (FFT transforms) steps timed beside the headline (0 = skip)")
    ap.add_argument("--workload", choices=["polycrystal", "sphere_inclusion", "sphere_bending", "cp_torsion_bending"],
                    default="polycrystal",
                    help="polycrystal: the headline step; the others print one line per precision arm for the "
                         "32^3 sphere inclusion (FP64, tol 1e-8), the 128^3 J2 sphere composite under 20 bending "
                         "steps and the 128^3 crystal-plasticity polycrystal under 30 torsion-bending increments")
    ap.add_argument("--arms", default="",
                    help="comma-separated precisions of a --workload scenario (default: per scenario) or of "
                         "--serve (one line each, same requests; default: --precision)")
    ap.add_argument("--residual-passes", type=int, choices=[0, 1, 2], default=0,
                    help="residual form: 0 = chosen by the library's launch-shape tuner, 1 = one pass, "
                         "2 = two passes (FFTM_OPT_RESIDUAL_PASSES)")
    ap.add_argument("--residual-tile", type=int, choices=[0, 8, 16], default=0,
                    help="one-pass residual tile height: 0 = tuned, 8 or 16 voxel rows (FFTM_OPT_RESIDUAL_TILE)")
    ap.add_argument("--graph", type=int, choices=[0, 1], default=0,
                    help="1: device-decided steps replayed from CUDA graphs (FFTM_OPT_CUDA_GRAPH)")
    ap.add_argument("--device-loop", type=int, choices=[0, 1], default=1,
                    help="1: convergence test on the device (default); 0: the host reads the norms every iteration")
    ap.add_argument("--serve", action="store_true",
                    help="serving stream (mixed sizes/BCs/laws, Poisson arrivals): solves/s and p50/p99 latency")
    ap.add_argument("--requests", type=int, default=96, help="requests of the serving stream (--serve)")
    ap.add_argument("--slots", type=int, default=4, help="resident solves of the server (--serve)")
    return ap.parse_args(argv)


def workload(n, grains):
    """The synthetic workload; the phase map is cached in the temp dir (generation is exact and seeded)."""
    import synthetic as syn

    key = hashlib.sha1(f"voronoi-{n}-{grains}-2-3-v1".encode()).hexdigest()[:16]
    path = os.path.join(tempfile.gettempdir(), f"fftm_phase_{key}.npy")
    phase = None
    if os.path.exists(path):
        try:
            phase = np.load(path)
        except Exception:
            phase = None
    if phase is None:
        phase, _ = syn.voronoi((n, n, n), grains, 2)
        try:
            tmp = f"{path}.{os.getpid()}.npy"
            np.save(tmp, phase)
            os.replace(tmp, path)
        except OSError:
            pass
    quats = syn.shoemake_quaternions(grains, 3)
    mats = [syn.Material(1, (168.0, 121.0, 75.0), tuple(q)) for q in quats]
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    C11, C12, C44 = 168.0, 121.0, 75.0
    return syn.Workload(name=f"voronoi_polycrystal_{n}", n=(n, n, n), phase=phase, materials=mats,
                        bc=[[["D"] * 3] * 2, [["N"] * 3] * 2, [["P"] * 3] * 2], scheme="TETRA2", green="B0",
                        lambda0=C12, mu0=0.5 * (C44 + 0.5 * (C11 - C12)), tol=1e-6, A=A, max_iter=1000)


# ---- distributed harness (replicas) ------------------------------------------------------
class Dist:
    def __init__(self, use_cuda):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("nccl" if use_cuda else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value, op):
        """All-reduce of a float over ranks ('max' or 'sum')."""
        if not self.pg:
            return value
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def timed_steps(step, steps, warmup, dist, sync, start_timer, stop_timer):
    """W untimed steps, then K steps bracketed by barrier + sync; returns (seconds, units)."""
    for _ in range(warmup):
        step()
    dist.barrier()
    sync()
    start_timer()
    units = 0.0
    for _ in range(steps):
        units += step()
    sync()
    sec = stop_timer()
    dist.barrier()
    return sec, units


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def element_counts(wl):
    """Stored nodes, and per axis the field elements (all components) one pass over it moves:
    a component's transform along an axis covers n+1 (Neumann/Neumann), n (periodic, or mixed
    Neumann/Dirichlet) or n-1 (Dirichlet/Dirichlet) node positions (Table 1)."""
    N = [wl.n[a] if wl.bc[a][0][0] == "P" else wl.n[a] + 1 for a in range(3)]
    nodes = N[0] * N[1] * N[2]
    per_axis = []
    for a in range(3):
        tot = 0
        for q in range(3):
            l, r = wl.bc[a][0][q], wl.bc[a][1][q]
            L = wl.n[a] + (0 if l == "P" else (1 if (l, r) == ("N", "N") else (-1 if (l, r) == ("D", "D") else 0)))
            tot += L * int(np.prod([N[b] for b in range(3) if b != a]))
        per_axis.append(tot)
    return nodes, per_axis


def traffic_record(kernel):
    """ncu DRAM bytes per launch recorded in profiles/, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        h = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return rec if h == rec.get("source_sha1") else None


# ---- the oracle's bounded sample ------------------------------------------------------------
def oracle_sample(wl, iterations):
    """Time `iterations` fixed-point iterations of the FP64 oracle on a 256 x 256 x REF_SLAB z-slab
    of the workload (same microstructure planes, same per-voxel work); returns voxel-it/s."""
    import copy

    from oracle.solver import Problem

    w = copy.copy(wl)
    w.n = (wl.n[0], wl.n[1], min(REF_SLAB, wl.n[2]))
    w.phase = np.ascontiguousarray(wl.phase[:, :, : w.n[2]])
    pr = Problem(w)
    Gs = pr.grad_ustar()
    u = np.zeros(pr.grid.node_shape)
    t0 = time.perf_counter()
    for _ in range(iterations):
        p, D, P, G, SD, SP = pr.residual(u, Gs)
        u = pr.green_update(p)
    sec = time.perf_counter() - t0
    vox = w.n[0] * w.n[1] * w.n[2]
    return vox * iterations / sec, sec, f"{iterations} fixed-point iteration(s) of the FP64 oracle on a " \
        f"{w.n[0]}x{w.n[1]}x{w.n[2]} z-slab of the workload (same phase map planes, same per-voxel work)"


def reference_arm(args):
    dist_rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if dist_rank != 0:
        return 0
    wl = workload(args.n, args.grains)
    for _ in range(args.warmup):
        oracle_sample(wl, 1)
    total_vox_it = 0.0
    total_sec = 0.0
    sample = None
    for _ in range(args.steps):
        v, sec, sample = oracle_sample(wl, 1)
        total_sec += sec
        total_vox_it += v * sec
    value = total_vox_it / total_sec
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n, args.grains), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "threads_note": "scipy.fft with workers=-1; NumPy elementwise on one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- the GPU arm ----------------------------------------------------------------------------
def gpu_arm(args):
    import torch

    from paper_2607_05929_gb300 import build as libbuild
    from paper_2607_05929_gb300 import fftm as F

    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the GPU arm has no CPU fallback")
    dist = Dist(True)
    torch.cuda.set_device(dist.local)
    if dist.rank == 0:
        libbuild.build()
    dist.barrier()
    F.load_library()
    wl = workload(args.n, args.grains)
    stream = torch.cuda.Stream()
    ctx = F.fftm_ctx_create(dist.local, stream)
    mats = [(m.law, m.params, m.quat) for m in wl.materials]

    def make(precision):
        desc, keep = F.make_desc(wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green,
                                 lambda0=wl.lambda0, mu0=wl.mu0, precision=precision, tol=wl.tol,
                                 max_iter=wl.max_iter)
        p = F.fftm_problem_create(ctx, desc)
        F.fftm_set_option(p, F.FFTM_OPT_DEVICE_LOOP, args.device_loop)
        F.fftm_set_option(p, F.FFTM_OPT_CUDA_GRAPH, args.graph)
        if args.residual_passes:
            F.fftm_set_option(p, F.FFTM_OPT_RESIDUAL_PASSES, args.residual_passes)
        if args.residual_tile:
            F.fftm_set_option(p, F.FFTM_OPT_RESIDUAL_TILE, args.residual_tile)
        F.fftm_set_load(p, wl.A)
        return p

    prob = make(args.precision)
    nvox = wl.n[0] * wl.n[1] * wl.n[2]
    last = {}

    def step():
        F.fftm_reset_state(prob)
        st, r, _, _ = F.fftm_solve_step(prob)
        if not r["converged"]:
            raise RuntimeError(f"solve did not converge: {r}")
        last.update(r)
        return float(nvox * r["iterations"])

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dist.local)

    def start_timer():
        ev0.record(stream)
        F.fftm_set_profiling(prob, True)
        L0[0] = F.fftm_kernel_launches(prob)
        clocks.start()

    def stop_timer():
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1000.0

    L0 = [0]
    sec, units = timed_steps(step, args.steps, args.warmup, dist, torch.cuda.synchronize, start_timer, stop_timer)
    clk = clocks.stop()
    launches = F.fftm_kernel_launches(prob) - L0[0]
    ktimes = F.fftm_kernel_times(prob)
    F.fftm_set_profiling(prob, False)
    sec_max = dist.reduce(sec, "max")
    units_all = dist.reduce(units, "sum")
    value = units_all / sec_max
    iters = last["iterations"]

    # ---- roofline of the dominant kernel (algorithmic bytes / CUDA-event time) ----
    # algorithmic bytes of the method (the pass model): every pass reads and writes the field
    # once (a node of 3 components: 12 B each way in FP32), the residual reads u^f and the phase
    # and writes D; the low part of the FP32 displacement and the transforms' extra launches
    # (the TF32 path's separate z inverse) are implementation traffic and not counted
    esz = 8 if args.precision == "fp64" else 4
    nodes, per_axis = element_counts(wl)
    it_total = iters * args.steps
    acc_total = last["n_accelerated"] * args.steps
    bytes_cat = {
        "residual": it_total_plus1(args.steps, iters) * (nodes * 3 * esz * 2 + nvox * 2),
        "pass_x": it_total * per_axis[0] * esz * 4,  # forward and inverse, read + write each
        "pass_y": it_total * per_axis[1] * esz * 4,
        "pass_z_fused": it_total * per_axis[2] * esz * 2,  # z forward, Green factor, z inverse
        # Gram: 4 D reads; combination: 4 D + 4 u reads, one u write
        "anderson": acc_total * nodes * 3 * esz * (4 + 4 + 4 + 1),
    }
    rows = {}
    for k, b in bytes_cat.items():
        ms, n = ktimes.get(k, (0.0, 0))
        if ms > 0:
            rows[k] = {"ms": ms, "launches": n, "GBps": b / (ms * 1e-3) / 1e9}
    dom = max(rows, key=lambda k: rows[k]["ms"])
    peaks, peak_src = measured_peaks()
    achieved = rows[dom]["GBps"]
    traffic = traffic_record(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                "algorithmic_bytes_per_launch": bytes_cat[dom] / max(1, rows[dom]["launches"]),
                "per_category": rows,
                # the whole iteration against the 4-pass model (96 B per node + 2 B phase in FP32) and
                # against the compulsory bytes (u^f read and written once, 24 B, + 2 B phase)
                "pass_model_frac": (nodes * 24 * esz + nvox * 2) * (value / nvox) / (peaks["hbm_gbs"] * 1e9 * dist.world),
                "compulsory_frac": (nodes * 6 * esz + nvox * 2) * (value / nvox) / (peaks["hbm_gbs"] * 1e9 * dist.world)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n, args.grains), "precision": args.precision,
                       "convergence_test": "device" if args.device_loop else "host",
                       "iterations_per_step": iters, "anderson_steps_per_step": last["n_accelerated"],
                       "l2": "inputs larger than L2 (working set several GB; no flush needed)",
                       "parallelism": f"replicas x{dist.world}"},
            "roofline": roofline, "gpu_launches": launches, "clocks": clk,
            "tuning": [t for t in F.fftm_tuning_table().splitlines() if t]}

    # ---- measured FMA rates (the arithmetic roof of the FP64 path) ----
    line["fma_peak_tflops"] = {"fp64": F.fftm_device_fma_rate(dist.local, True) / 1e12,
                               "fp32": F.fftm_device_fma_rate(dist.local, False) / 1e12}

    # ---- the other precisions beside it (same workload, device-resident), and every path's
    # converged stresses against the FP64 path's (relative L2, computed on the device) ----
    def stress_dev(pp):
        prec = F.fftm_problem_layout(pp)[1]
        nb = F.fftm_field_bytes(pp, F.FFTM_FIELD_STRESS)
        t = torch.empty(nb // (8 if prec == F.FFTM_FP64 else 4),
                        dtype=torch.float64 if prec == F.FFTM_FP64 else torch.float32, device="cuda")
        torch.cuda.synchronize()
        F.fftm_get_field(pp, F.FFTM_FIELD_STRESS, t)
        return t.double()

    def side(prec, nsteps, note):
        nonlocal prob
        F.fftm_problem_destroy(prob)
        prob = make(prec)
        step()  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        F.fftm_set_profiling(prob, True)
        e0.record(stream)
        un = sum(step() for _ in range(nsteps))
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        kt = F.fftm_kernel_times(prob)
        F.fftm_set_profiling(prob, False)
        rec = {"value": un / sec, "unit": UNIT, "iterations_per_step": last["iterations"], "steps": nsteps,
               "ms_per_step": 1000.0 * sec / nsteps,
               "ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in kt.items()}, "note": note}
        return rec, stress_dev(prob)

    notes = {"fp64": "FP64 fields, transforms and residual",
             "fp32": "FP32 fields (hi + lo displacement) and residual, mixed-radix FFT transforms",
             "fp32_tf32": "per-axis transforms as tcgen05 TF32 contractions, FP32 fields and residual",
             "fp32_tc": "per-axis transforms as tcgen05 BF16 contractions, FP32 fields and residual"}
    keys = {"fp64": "fp64_path", "fp32": "fp32_path", "fp32_tf32": "fp32_tf32_path", "fp32_tc": "fp32_tc_path"}
    counts = {"fp64": args.fp64_steps, "fp32": args.fp32_steps, "fp32_tf32": args.tf32_steps, "fp32_tc": args.tc_steps}
    stresses = {args.precision: stress_dev(prob)}
    for prec in ("fp64", "fp32", "fp32_tf32", "fp32_tc"):
        if prec == args.precision or counts[prec] <= 0:
            continue
        line[keys[prec]], stresses[prec] = side(prec, counts[prec], notes[prec])
    if "fp64" in stresses:
        ref = stresses["fp64"]
        nref = float(torch.linalg.vector_norm(ref))
        line["stress_rel_l2_vs_fp64"] = {p_: float(torch.linalg.vector_norm(t - ref)) / nref
                                         for p_, t in stresses.items() if p_ != "fp64"}
    del stresses
    F.fftm_problem_destroy(prob)
    prob = make(args.precision)

    # ---- end to end through the C ABI with host buffers ----
    if not args.no_e2e:
        ph_host = torch.empty(nvox * 2, dtype=torch.uint8, pin_memory=True)
        ph_np = ph_host.numpy().view(np.uint16)
        ph_np[:] = np.ascontiguousarray(wl.phase.transpose(2, 1, 0)).ravel()
        ubytes = F.fftm_field_bytes(prob, F.FFTM_FIELD_U)
        u_host = torch.empty(ubytes, dtype=torch.uint8, pin_memory=True)

        def e2e_step():
            F.fftm_set_phase_raw(prob, ph_host.data_ptr())
            F.fftm_set_load(prob, wl.A)
            F.fftm_reset_state(prob)
            st, r, _, _ = F.fftm_solve_step(prob)
            F.fftm_get_field(prob, F.FFTM_FIELD_U, u_host)
            return float(nvox * r["iterations"])

        t = [0.0]
        es, eu = timed_steps(e2e_step, args.steps, 1, dist, torch.cuda.synchronize,
                             lambda: t.__setitem__(0, time.perf_counter()),
                             lambda: time.perf_counter() - t[0])
        es = dist.reduce(es, "max")
        eu = dist.reduce(eu, "sum")
        line["e2e"] = {"value": eu / es, "unit": UNIT, "h2d_bytes_per_step": nvox * 2 + 96,
                       "d2h_bytes_per_step": ubytes + 128}

    # ---- CPU baseline (oracle), rank 0 at N = 1 only ----
    if not args.no_cpu_baseline and dist.world == 1:
        v, s, sample = oracle_sample(wl, 2)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample, "seconds": s,
                                "threads_note": "scipy.fft with workers=-1; NumPy elementwise on one thread"}
    F.fftm_problem_destroy(prob)
    F.fftm_ctx_destroy(ctx)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def it_total_plus1(steps, iters):
    """Residual evaluations: one per iteration plus the final converged check, per step."""
    return steps * (iters + 1)


def _serve_request(k):
    from synthetic.serving import request_spec, request_workload
    spec = request_spec(k)
    wl, loads = request_workload(spec)
    return spec, wl, loads


def serve_requests(count):
    """The first `count` requests of the serving stream (generation is exact and seeded), built
    by a spawned process pool on the host cores; call before any GPU work."""
    import multiprocessing as mp

    workers = max(1, min(16, os.cpu_count() or 1, count))
    if workers == 1:
        return [_serve_request(k) for k in range(count)]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_serve_request, range(count), chunksize=1)


def serve_arm(args):
    """Continuous-batching server over one GPU: a closed-loop pass measures the capacity C,
    then the same requests arrive as a Poisson stream at 0.8 C; latency = completion - arrival."""
    from paper_2607_05929_gb300 import build as libbuild
    from paper_2607_05929_gb300 import fftm as F

    reqs = serve_requests(args.requests)  # before any GPU call
    libbuild.build()
    F.load_library()
    arms = [a.strip() for a in args.arms.split(",") if a.strip()] if args.arms else [args.precision]
    for prec in arms:
        serve_one(args, F, reqs, prec)
    return 0


def serve_one(args, F, reqs, precision):
    descs = []
    for spec, wl, loads in reqs:
        mats = [(m.law, m.params, m.quat) for m in wl.materials]
        descs.append(F.make_desc(wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green, lambda0=wl.lambda0,
                                 mu0=wl.mu0, precision=precision, tol=wl.tol, max_iter=wl.max_iter))

    def run(arrivals):
        srv = F.fftm_server_create(0, 0, args.slots)
        F.fftm_server_set_option(srv, F.FFTM_OPT_CUDA_GRAPH, args.graph)
        done = {}
        t0 = time.monotonic()
        ids = {}
        try:
            def submitter():
                for i, at in arrivals:
                    wait = t0 + at - time.monotonic()
                    if wait > 0:
                        time.sleep(wait)
                    ids[F.fftm_server_submit(srv, descs[i][0], reqs[i][2])] = i
            th = threading.Thread(target=submitter)
            th.start()
            while len(done) < len(arrivals):
                for r in F.fftm_server_poll(srv, wait=True):
                    done[r["id"]] = r
                if th.is_alive() and not F.fftm_server_pending(srv)[0] and not F.fftm_server_pending(srv)[1]:
                    time.sleep(0.001)  # nothing queued or running: the next arrival is still to come
            th.join()
        finally:
            F.fftm_server_destroy(srv)
        return [(ids[k], r) for k, r in done.items()]

    warm = [i for i, (spec, _, _) in enumerate(reqs) if spec["n"] <= 48][:4]
    run([(i, 0.0) for i in warm])  # warm-up: first launches, module loading
    closed = run([(i, 0.0) for i in range(len(reqs))])
    span = max(r["t_end"] for _, r in closed) - min(r["t_submit"] for _, r in closed)
    capacity = len(reqs) / span
    rate = 0.8 * capacity
    gaps = np.random.default_rng(7).exponential(1.0 / rate, size=len(reqs))
    arrivals = [(i, float(t)) for i, t in zip(range(len(reqs)), np.cumsum(gaps) - gaps[0])]
    opened = run(arrivals)
    lat = np.array([r["t_end"] - r["t_submit"] for _, r in opened])
    t_first = min(r["t_submit"] for _, r in opened)
    t_last = max(r["t_end"] for _, r in opened)
    vox_it = sum(reqs[i][1].phase.size * r["iterations"] for i, r in opened)
    bad = [r["status"] for _, r in opened if r["status"] != 0]
    line = {"metric": "solves/s", "value": len(opened) / (t_last - t_first), "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "capacity_solves_per_s": capacity, "arrival_rate_per_s": rate,
            "voxel_iterations_per_s": vox_it / (t_last - t_first), "requests": len(reqs), "slots": args.slots,
            "not_converged_or_failed": len(bad), "dtype": "f64" if precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": f"serving stream: {len(reqs)} requests (seeds 1000..{999 + len(reqs)}), sides "
                                   "32/48/64/96/128, per-axis P/D/N, isotropic or J2 matrix, HEX1 or TETRA2, "
                                   "spheres or Voronoi; Poisson arrivals at 0.8x the measured capacity",
                       "precision": precision, "cuda_graph": args.graph}}
    print(json.dumps(line), flush=True)


def scenario(name, n=None):
    """(workload, loads, default arms, description) of a --workload scenario."""
    import synthetic as syn

    if name == "sphere_inclusion":
        wl = syn.sphere_inclusion_32(n=n or 32)
        return wl, [(wl.A, wl.b, wl.Q)], ["fp64"], (
            f"sphere_inclusion_{wl.n[0]}: {wl.n[0]}^3, centred sphere r = n/4, E 1 / 10, nu 0.3, HEX1, B0, "
            "x Dirichlet / y Neumann / z periodic, eps_xx = 1e-3, tol 1e-8")
    if name == "sphere_bending":
        wl, loads = syn.sphere_composite_bending(n or 128)
        return wl, loads, ["fp64", "fp32", "fp32_tf32", "fp32_tc"], (
            f"sphere_composite_bending_{wl.n[0]}: {wl.n[0]}^3, random spheres 30 %, r in [4, 10], J2 matrix "
            "(E 200 GPa, nu 0.3, sigma_y 0.3 GPa, H 2 GPa), elastic particles, HEX1, B0, 20 bending steps "
            "(theta up to 0.012), x Dirichlet / y, z Neumann, tol 1e-6")
    if name == "cp_torsion_bending":
        wl, loads = syn.cp_polycrystal_torsion_bending(n or 128)
        return wl, loads, ["fp32", "fp32_tf32"], (
            f"cp_polycrystal_torsion_bending_{wl.n[0]}: {wl.n[0]}^3, 200-grain Voronoi FCC crystal plasticity "
            "(12 {111}<110> systems, n 20, gdot0 1e-3/s, Voce 30/90/300 MPa), TETRA2, B0, 30 torsion-bending "
            "increments (phi 0.05, theta 0.02), x Dirichlet / y, z Neumann, tol 1e-6, finite strain")
    raise ValueError(name)


def scenario_arm(args):
    """A whole load history of one scenario per precision arm on one GPU: voxel-iterations/s over
    the history (CUDA events on the library's stream), iterations per step, and each FP32 arm's
    final stresses against the FP64 arm's (relative L2) when both ran."""
    import torch

    from paper_2607_05929_gb300 import build as libbuild
    from paper_2607_05929_gb300 import fftm as F

    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the GPU arm has no CPU fallback")
    wl, loads, arms, desc = scenario(args.workload, args.n if args.n != 256 else None)
    if args.arms:
        arms = [a.strip() for a in args.arms.split(",") if a.strip()]
    libbuild.build()
    F.load_library()
    stream = torch.cuda.Stream()
    ctx = F.fftm_ctx_create(0, stream)
    mats = [(m.law, m.params, m.quat) for m in wl.materials]
    nvox = wl.n[0] * wl.n[1] * wl.n[2]
    npp = 2 if wl.scheme == "TETRA2" else 1
    results = {}
    for prec in arms:
        d, keep = F.make_desc(wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green, lambda0=wl.lambda0,
                              mu0=wl.mu0, precision=prec, tol=wl.tol, max_iter=wl.max_iter, h=wl.h)
        p = F.fftm_problem_create(ctx, d)
        its, accs, conv = [], [], []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for A, b, Q in loads:
            F.fftm_set_load(p, A, b, Q)
            st, r, _, _ = F.fftm_solve_step(p)
            its.append(r["iterations"])
            accs.append(r["n_accelerated"])
            conv.append(bool(r["converged"]))
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        nb = F.fftm_field_bytes(p, F.FFTM_FIELD_STRESS)
        S = np.zeros(nb // (8 if prec == "fp64" else 4), dtype=np.float64 if prec == "fp64" else np.float32)
        F.fftm_get_field(p, F.FFTM_FIELD_STRESS, S)
        F.fftm_problem_destroy(p)
        results[prec] = S.astype(np.float64)
        line = {"metric": METRIC, "value": nvox * sum(its) / sec, "unit": UNIT, "n_gpus": 1,
                "higher_is_better": True, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
                "precision": prec, "seconds": sec, "steps": len(loads), "iterations_total": int(sum(its)),
                "iterations_per_step": its, "anderson_steps_per_step": accs, "all_converged": all(conv),
                "voxel_points": nvox * npp, "config": {"workload": desc}}
        if "fp64" in results and prec != "fp64":
            ref = results["fp64"]
            line["final_stress_rel_l2_vs_fp64"] = float(np.linalg.norm(results[prec] - ref) / np.linalg.norm(ref))
        print(json.dumps(line), flush=True)
    F.fftm_ctx_destroy(ctx)
    if not args.no_cpu_baseline:
        print(json.dumps(scenario_oracle(args.workload, wl, loads, desc)), flush=True)
    return 0


def scenario_oracle(name, wl, loads, desc):
    """The FP64 oracle on the host cores for a scenario: the whole first load step on the full grid
    for the 32^3 sphere inclusion; two fixed-point iterations of the first load step on the full
    grid for the larger scenarios (a bounded sample, scaled to voxel-it/s)."""
    from oracle.solver import Problem

    pr = Problem(wl)
    A, b, Q = loads[0]
    nvox = wl.n[0] * wl.n[1] * wl.n[2]
    if name == "sphere_inclusion":
        t0 = time.perf_counter()
        _, rep = pr.solve_step(A=A, b=b, Q=Q)
        sec = time.perf_counter() - t0
        its = rep.iterations
        sample = f"the whole first load step ({its} iterations) of the FP64 oracle on the full grid"
    else:
        its = 2
        Gs = pr.grad_ustar(A, b, Q)
        u = np.zeros(pr.grid.node_shape)
        t0 = time.perf_counter()
        for _ in range(its):
            p_, D, P, G, SD, SP = pr.residual(u, Gs)
            u = pr.green_update(p_)
        sec = time.perf_counter() - t0
        sample = f"{its} fixed-point iterations of the first load step of the FP64 oracle on the full grid"
    return {"impl": "reference", "metric": METRIC, "value": nvox * its / sec, "unit": UNIT, "dtype": "f64",
            "data": "synthetic", "seconds": sec,
            "cpu_baseline": {"value": nvox * its / sec, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "config": {"workload": desc}}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)
    if args.serve:
        return serve_arm(args)
    if args.workload != "polycrystal":
        return scenario_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
