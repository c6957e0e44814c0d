#!/usr/bin/env python3
"""Benchmark of the DFPT Hubbard-parameter hot path on GB300.

Workloads (--workload):
  precision (default)  the rocksalt-like cube (8.4 bohr, 4 H + 4 L, 40 electrons, collinear nspin = 2
                       with an antiferromagnetic start) at 50 Ry, FFT 45^3, k 4x4x4, q 2x2x2: the
                       mixed-precision form's workload;
  medium               the same cell at 35 Ry, FFT 36^3;
  batch                the batching form (cells per hour over a batch of cells).
The H species' projector strength is D = -4.0 Ha in every workload (the insulating reading of the
model; +1.5 Ha leaves the cells metallic).  Ground states are computed on the GPU before timing.

One step = one (q, J) self-consistent Sternheimer response (the per-q set-up a1 and a3-a10): every
(spin, k, band) system of that pair, in the mixed-precision form (FP32 FFTs, grid work and
projections; FP64 step lengths, norms, mixing and inversion).  value = H.psi/s over the K timed
steps (single-band applications of the Sternheimer operator, summed over ranks).

Beside the timed steps, on the same ground state and GPU:
  * the full chi matrix in the mixed form, measured: every (q, J) pair and hp_hubbard, wall time
    from a ready ground state to U and V in host memory (chi_matrix.mixed_s);
  * the FP64 form on --fp64-steps pairs (H.psi/s and seconds per pair), and with --fp64-full the
    whole FP64 chi matrix, measured, with max |U_mixed - U_FP64| and |V_mixed - V_FP64| in meV;
  * with --companion medium (the default for the precision workload): the 35 Ry cell's ground state
    and full mixed chi matrix, measured, and the declared oracle column of that cell (q = (1/2,0,0),
    J = the first H; stored by the oracle under tests/golden/) against this run's FP64 and mixed
    responses, element by element.
e2e: the same response through the C ABI with the ground state copied in from pinned host memory
and Delta n copied out, every step.  cpu_baseline: the oracle's Sternheimer operator on the host
cores, one thread and one process per core.

N > 1 (torchrun): the (q, J) pairs are sharded round-robin over ranks (weak scaling, no collective
on the data path); timing is the max over ranks between barriers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "full χ-matrix wall time & H·ψ/s, mixed vs FP64 on 1 GB300 at |ΔU|≤1 meV"
UNIT = "Hpsi/s"
_CELL = "rocksalt cube a=8.4 bohr, 4 H + 4 L (H projector D=-4.0 Ha), 40 electrons, nspin=2 (AFM start), "
WORKLOADS = {
    "precision": "precision: " + _CELL + "ecutwfc 50 Ry (npw<=3575), FFT 45^3, k 4x4x4, q 2x2x2",
    "medium": "medium: " + _CELL + "ecutwfc 35 Ry (npw<=2103), FFT 36^3, k 4x4x4, q 2x2x2",
    "batch": "batch: 16 synthetic cells from seed 15684, 2-12 atoms, orthorhombic 7-12 bohr, "
             "25-45 Ry, k 2-4 and q 1-2 per axis, nspin=1, occupied bands at the largest bare gap, mixed form",
}
STEP = ("one (q, J) self-consistent Sternheimer response (set-up a1, a3-a10) over every (spin, k, band) system of "
        "the pair, mixed form")
GOLDEN_MEDIUM = os.path.join(ROOT, "tests", "golden", "medium_column.json")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--fp64-warmup", type=int, default=1)
    p.add_argument("--fp64-full", action="store_true", help="also measure the whole FP64 chi matrix (minutes)")
    p.add_argument("--no-chi-matrix", action="store_true", help="skip the measured full mixed chi matrix")
    p.add_argument("--companion", default=None, choices=["none", "medium"],
                   help="second workload measured beside the headline (default: medium for precision)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--band-batch", type=int, default=0, help="grids per FFT batch (0 = automatic)")
    p.add_argument("--workload", default="precision", choices=sorted(WORKLOADS))
    p.add_argument("--tc-accuracy", action="store_true",
                   help="print the tensor-core building block's accuracy table (hp_selftest_tc) and exit")
    p.add_argument("--cg-adapt", type=float, default=None,
                   help="CG threshold factor for outer iterations after the first (library default if omitted)")
    a = p.parse_args()
    if a.companion is None:
        a.companion = "medium" if a.workload == "precision" else "none"
    return a


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + QUERY, "--format=csv",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path).read().splitlines()[1:]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------------
def _oracle_sample(seconds, workload="precision", seed=2203):
    """The oracle's Sternheimer operator (H_k+q + alpha O_k+q - eps, Eq. LRKSeq_lp) applied to blocks of
    nocc bands on the workload's k spheres and grid, with the oracle's own starting-density potential
    and seeded orthonormal occupied states, for about ``seconds``; returns (H.psi count, elapsed)."""
    import numpy as np

    import workloads as W
    from oracle import groundstate as G
    from oracle.model import Model
    from oracle.response import sternheimer_operator

    w = getattr(W, workload)()
    m = Model(w)
    vr = m.vloc_r() + G.hxc_potential(m, G.initial_density(m))[0]
    rng = np.random.default_rng(seed)
    n, t0, ik = 0, time.perf_counter(), seed % len(m.kpts)
    while True:
        kd = m.kdata(m.kpts[ik % len(m.kpts)])
        U = np.linalg.qr(rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc)))[0]
        X = rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc))
        Y = sternheimer_operator(m, kd, vr, U, 2.0, np.full(m.nocc, 0.5), X)
        n += X.shape[1]
        ik += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el, float(np.abs(Y).max())


def _oracle_procs(seconds, workload, nproc):
    """nproc one-thread oracle processes at once (different k points); -> (total H.psi, max elapsed)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for i in range(nproc):
        code = ("import json,sys; sys.path.insert(0, %r); import bench; n, el, _ = bench._oracle_sample(%f, %r, %d); "
                "print(json.dumps(dict(n=n, el=el)))" % (ROOT, seconds, workload, 2203 + i))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True))
    n, el = 0, 0.0
    for p in procs:
        out, _ = p.communicate(timeout=900)
        d = json.loads(out.strip().splitlines()[-1])
        n += d["n"]
        el = max(el, d["el"])
    return n, el


def host_cpu():
    """(model name, logical cores) of the host, read at run time."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    return model or "unknown", os.cpu_count() or 1


def cpu_baseline(seconds, workload="precision"):
    model, ncores = host_cpu()
    n1, el1 = _oracle_procs(seconds, workload, 1)
    nall, elall = _oracle_procs(seconds, workload, ncores)
    return {"value": nall / elall, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu_model": model,
            "one_thread": {"value": n1 / el1, "cores": 1},
            "sample": "the oracle's Sternheimer operator (numpy FP64) on blocks of 20 bands cycling over the %s "
                      "workload's k spheres: %d one-thread processes at once for %.1f s (%d H.psi), and one process "
                      "alone (%d H.psi in %.1f s)" % (workload, ncores, elall, nall, n1, el1)}


def _oracle_tiny():
    """The oracle's full chi of the tiny workload (ground state, then the one (q, J) column and
    U); returns (ground-state seconds, chi seconds from the ready ground state, U in eV)."""
    import numpy as np

    import workloads as W
    from oracle import groundstate as G, hubbard as HB, response as R
    from oracle.model import Model

    m = Model(W.tiny())
    t0 = time.perf_counter()
    gs = G.scf(m, tol=1e-12)
    t1 = time.perf_counter()
    r = R.solve_column(m, gs, 0, m.hub_atoms[0])
    c0 = HB.trace_column(m, r["dn0"]).real
    c = HB.trace_column(m, r["dn"]).real
    U = HB.hubbard_matrix(np.array([[c0[0]]]), np.array([[c[0]]]))[0, 0]
    return t1 - t0, time.perf_counter() - t1, float(U)


def oracle_tiny_chi(ncores):
    """Oracle chi time for the tiny workload in a subprocess with all host cores available to its BLAS."""
    env = dict(os.environ, OMP_NUM_THREADS=str(ncores), OPENBLAS_NUM_THREADS=str(ncores))
    code = ("import json,sys; sys.path.insert(0, %r); import bench; g, c, u = bench._oracle_tiny(); "
            "print(json.dumps(dict(gs=g, chi=c, U=u)))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    return json.loads(r.stdout.strip().splitlines()[-1])


def gpu_tiny_chi(P, W, stream):
    """The library's full chi of the tiny workload (FP64 and mixed) from its own ground state: seconds and U."""
    import torch

    w = W.tiny()
    out = {}
    ctx = P.Context.from_workload(w, cuda_stream=stream.cuda_stream)
    ctx.ground_state(w["nelec"], w["nspin"])
    atoms, _ = ctx.hubbard_atoms()
    for prec, tag in ((0, "fp64"), (1, "mixed")):
        ctx.set_precision(prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.response(0, int(atoms[0]))
        hp = ctx.hubbard_parameters()
        torch.cuda.synchronize()
        out[tag] = {"chi_s": time.perf_counter() - t0, "U_eV": float(hp["U"][0])}
    ctx.destroy()
    return out


def static_config(workload, world=1):
    return {"workload": WORKLOADS[workload], "step": STEP,
            "l2": "inputs larger than L2 (response working set of several GB)",
            "parallelism": "(q, J) pairs round-robin over %d rank(s)" % world}


def reference_arm(args, rank):
    """The oracle as it stands, timed on the host cores (one process per core) on this arm's workload
    and metric; each step is a bounded sample of the workload."""
    if rank != 0:
        return
    if args.workload == "batch":
        print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no oracle arm"}))
        return
    model, ncores = host_cpu()
    per = 4.0
    for _ in range(args.warmup):
        _oracle_procs(0.5, args.workload, ncores)
    n_tot, el_tot = 0, 0.0
    for _ in range(args.steps):
        n, el = _oracle_procs(per, args.workload, ncores)
        n_tot += n
        el_tot += el
    value = n_tot / el_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": static_config(args.workload, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu_model": model,
                             "sample": "each step: %d one-thread oracle processes applying the Sternheimer operator for "
                                       "about %.0f s; %d H.psi in %.1f s over %d steps"
                                       % (ncores, per, n_tot, el_tot, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
FAMILY_KERNELS = {"fft_pass": ("fft_fixed_kernel / fft_axis_kernel (FP32 Stockham pass)", "fft.cu"),
                  "column": ("col_inv_reg_kernel + col_fwd_reg_kernel (fused z-column transforms)", "fused.cu"),
                  "plane": ("plane_reg_kernel (fused x/y plane transforms + real-space product)", "fused.cu"),
                  "project": ("proj_kernel + proj_reduce_kernel (FP32 projections)", "kernels.cu"),
                  "expand": ("expand_kernel (FP32 projector expansion)", "kernels.cu")}
# what bounds each family on GB300 (ncu summaries under profiles/): FP32 instruction issue for the
# in-register FFTs and the projector contractions, HBM for the data-movement passes
FAMILY_BOUND = {"fft_pass": "hbm", "column": "hbm", "plane": "alu", "project": "alu", "expand": "alu"}
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def ncu_traffic(family, alg_bytes_per_launch, workload="medium"):
    """DRAM bytes per launch of a kernel family: the DRAM/algorithmic byte ratio of a committed ncu
    capture (profiles/traffic_<family>_<workload>.json) times this run's algorithmic bytes per launch;
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.json" % (family, workload))
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    src = open(os.path.join(ROOT, "paper_2203_15684_gb300", "csrc", FAMILY_KERNELS[family][1]), "rb").read()
    if d.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return d["dram_over_algorithmic"] * alg_bytes_per_launch


def shard_pairs(pairs, rank, world):
    """The (q, J) pairs one rank runs: round-robin over ranks, disjoint, together all pairs."""
    return pairs[rank::world]


def reduce_over_ranks(elapsed, units, dist, device):
    """Whole-job timing: (max elapsed over ranks, sum of the units all ranks processed).  dist is
    torch.distributed (or None for one process)."""
    if dist is None:
        return elapsed, float(units)
    import torch

    t = torch.tensor([elapsed, float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax[0:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def tensor_peak():
    """Dense TF32 tensor peak for the contractions: the measured bf16 burst peak x the nominal
    TF32/BF16 ratio (1.1 / 2.25)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 burst (MEASURED_PEAKS.json) x 1.1/2.25 (TF32)"
    return 1900.0 * 1.1 / 2.25, "fallback 1.9 PFLOP/s bf16 x 1.1/2.25 (TF32)"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    return 6800.0, "fallback (no MEASURED_PEAKS.json)"


def batch_arm(args):
    """Batching form: the seeded batch of 16 uneven synthetic cells (2-12 atoms, 7-12 bohr, 25-45 Ry,
    k meshes 2-4 per axis, q meshes 1-2 per axis), occupied bands from the largest gap of each cell's
    bare spectrum at k = 0, nspin = 1, mixed form.  After every cell's ground state: the full chi
    matrix and U/V of every cell one cell after the other, then all cells at once (hp_batch_run: one
    host thread and CUDA stream per cell, kernels of different cells overlapping); cells per hour of
    each (the ground states are not timed)."""
    import torch

    import paper_2203_15684_gb300 as P
    import workloads as W

    cells, ctxs, skipped, bare_gap = W.batch_cells(), [], [], {}
    for w in cells:
        stream = torch.cuda.Stream()
        ctx = P.Context.from_workload(w, cuda_stream=stream.cuda_stream, precision=1)
        b, gap = P.batch_band_choice(ctx, w)
        bare_gap[w["name"]] = gap
        nelec = 2.0 * b
        try:
            ctx.ground_state(nelec, 1)
        except P.HPError as e:
            skipped.append("%s: %s" % (w["name"], str(e)[:200]))
            ctx.destroy()
            continue
        ctxs.append((w, ctx, stream, nelec))

    def alone():
        for _, ctx, _, _ in ctxs:
            atoms, _ = ctx.hubbard_atoms()
            for J in atoms:
                for iq in range(ctx.query_sizes()["nq"]):
                    ctx.response(iq, int(J))
            ctx.hubbard()

    def together():
        P.batch_run([c for _, c, _, _ in ctxs])

    times_a, times_b = [], []
    l0 = P.launch_count()
    for rep in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        alone()
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        t0 = time.perf_counter()
        together()
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        if rep >= args.warmup:
            times_a.append(ta)
            times_b.append(tb)
    ta, tb = sum(times_a) / len(times_a), sum(times_b) / len(times_b)
    n = len(ctxs)
    line = {"metric": "cells/hour, seeded batch of synthetic cells (full chi and U/V per cell, mixed form)",
            "value": n * 3600.0 / tb, "unit": "cells/h", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"], "cells": n, "skipped": skipped,
                       "step": "one batch: every (q, J) response and chi/U/V of every cell, ground states before timing",
                       "nelec": {w["name"]: e for w, _, _, e in ctxs},
                       "bare_gap_ha": bare_gap,
                       "one_after_another_cells_per_hour": n * 3600.0 / ta,
                       "speedup_batch_vs_one_after_another": ta / tb},
            "gpu_launches": P.launch_count() - l0}
    print(json.dumps(line), flush=True)


def _traces(dn, nh):
    import numpy as np

    return np.array([np.trace(dn[a].sum(0)) for a in range(nh)])


class Engine:
    """One workload's context and ground state on this rank's GPU, and the timed pieces run on it."""

    def __init__(self, P, W, name, stream, args, rank, world):
        import torch

        self.P, self.torch, self.name, self.stream = P, torch, name, stream
        self.w = getattr(W, name)()
        opts = dict(cuda_stream=stream.cuda_stream, band_batch=args.band_batch)
        if args.cg_adapt is not None:
            opts["cg_adapt"] = args.cg_adapt
        self.ctx = P.Context.from_workload(self.w, **opts)
        t0 = time.perf_counter()
        self.gs = self.ctx.ground_state(self.w["nelec"], self.w["nspin"], self.w["moments"])
        torch.cuda.synchronize()
        self.gs_seconds = time.perf_counter() - t0
        self.atoms, _ = self.ctx.hubbard_atoms()
        self.sizes = self.ctx.query_sizes()
        self.pairs = [(iq, int(J)) for J in self.atoms for iq in range(self.sizes["nq"])]
        self.mine = shard_pairs(self.pairs, rank, world)

    def event_time(self, fn):
        """fn() between CUDA events on the context's stream; -> (result, seconds)."""
        torch = self.torch
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        out = fn()
        e1.record(self.stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1000.0

    def chi_matrix(self, precision):
        """Every (q, J) response and hp_hubbard from the ready ground state: -> dict with the measured
        wall time, H.psi, U (eV) and the V list."""
        self.ctx.set_precision(precision)

        def run():
            hpsi = 0
            for iq, J in self.pairs:
                _, _, info = self.ctx.response(iq, J)
                hpsi += info["hpsi"]
            return hpsi, self.ctx.hubbard_parameters()

        (hpsi, hp), el = self.event_time(run)
        return {"seconds": el, "hpsi": hpsi, "hpsi_per_s": hpsi / el, "pairs": len(self.pairs),
                "U_eV": [float(u) for u in hp["U"]], "V": [(int(a), int(b), float(d), float(v)) for a, b, d, v in hp["V"]]}


    def chi_matrix_reduced(self, precision, full, find_atpert=1):
        """The same chi with the symmetry reductions (Sec. 2.4, Sec. 3.2): find_atpert = 1 (hp.x's
        default: one atom per class of equal occupations, the other columns rebuilt by hp_hubbard) or
        3 (space-group orbits and the star of q), and time reversal; only hp_irreducible_pairs' (q, J)
        responses are computed.  -> dict as chi_matrix plus the perturbed atoms and |U - U_full|,
        |V - V_full| in meV."""
        self.ctx.set_precision(precision)

        def run():
            atoms, _, _ = self.ctx.perturbed_atoms(find_atpert)
            hpsi, n = 0, 0
            for iq, J in self.ctx.irreducible_pairs():
                _, _, info = self.ctx.response(iq, J)
                hpsi += info["hpsi"]
                n += 1
            return hpsi, n, atoms, self.ctx.hubbard_parameters()

        try:
            (hpsi, n, atoms, hp), el = self.event_time(run)
        except self.P.HPError as e:
            return {"unavailable": str(e)[:200]}
        finally:
            self.ctx.perturbed_atoms(4)  # every atom its own column again
        out = {"seconds": el, "hpsi": hpsi, "hpsi_per_s": hpsi / el, "pairs": n, "perturbed_atoms": atoms,
               "U_eV": [float(u) for u in hp["U"]], "V": [(int(a), int(b), float(d), float(v)) for a, b, d, v in hp["V"]]}
        out["u_err_mev_vs_full"], out["v_err_mev_vs_full"] = uv_error_mev(out, full)
        out["speedup_vs_full"] = full["seconds"] / el
        return out


def uv_error_mev(a, b):
    """max |U_a - U_b| and max |V_a - V_b| over the pairs, in meV."""
    du = max(abs(x - y) for x, y in zip(a["U_eV"], b["U_eV"])) * 1000.0
    dv = max(abs(x[3] - y[3]) for x, y in zip(a["V"], b["V"])) * 1000.0 if a["V"] else None
    return du, dv


def golden_check(eng):
    """The oracle's stored column of the medium cell (tests/golden/) against this GPU's FP64 and mixed
    responses of the same (q, J) on its own ground state: max |Delta n_GPU - Delta n_oracle| /
    max |Delta n_oracle| for Delta n^0 and Delta n, and the ground-state eigenvalues."""
    import numpy as np

    if not os.path.exists(GOLDEN_MEDIUM):
        return None
    g = json.load(open(GOLDEN_MEDIUM))
    iq, J = int(g["iq"]), int(g["J"])
    hub = [int(a) for a in g["hub_atoms"]]
    mm = eng.sizes["mmax"]

    def pad(d):
        out = np.zeros((len(hub), eng.sizes["nspin"], mm, mm), dtype=complex)
        for i, a in enumerate(hub):
            re, im = d[str(a)]
            x = np.array(re) + 1j * np.array(im)
            out[i, :, : x.shape[1], : x.shape[2]] = x
        return out

    r0, r1 = pad(g["dn0"]), pad(g["dn"])
    eps, _, _ = eng.ctx.get_ground_state()
    out = {"column": {"qfrac": g["qfrac"], "J": J},
           "eps_max_abs_diff_ha": float(np.abs(eps - np.array(g["eps"])).max())}
    for prec, tag in ((0, "fp64"), (1, "mixed")):
        eng.ctx.set_precision(prec)
        dn0, dn, _ = eng.ctx.response(iq, J)
        out[tag] = {"dn0_rel_err": float(np.abs(dn0 - r0).max() / np.abs(r0).max()),
                    "dn_rel_err": float(np.abs(dn - r1).max() / np.abs(r1).max())}
    return out


def tc_accuracy():
    """Accuracy of the tcgen05 kind::tf32 building block (three-product TF32 split, hp_selftest_tc)
    on D = A B^T, A (128 x K), B (16 x K) from PCG64 seed K, normal or absolute-normal entries, in four
    modes (3 or 4 products, with or without draining the TMEM accumulator every 32 values of K):
    max |D - D_exact| / sqrt(sum_k (a b)^2) and its signed mean, beside the same sum taken
    sequentially in FP32."""
    import numpy as np

    import paper_2203_15684_gb300 as P

    out = {}
    for kind in ("normal", "positive"):
        for K in (32, 256, 2048):
            rng = np.random.default_rng(K)
            A = rng.standard_normal((128, K)).astype(np.float32)
            B = rng.standard_normal((16, K)).astype(np.float32)
            if kind == "positive":
                A, B = np.abs(A), np.abs(B)
            ref = A.astype(np.float64) @ B.astype(np.float64).T
            scale = np.sqrt((A.astype(np.float64) ** 2) @ (B.astype(np.float64) ** 2).T)
            seq = np.cumsum((A[:, None, :] * B[None, :, :]).astype(np.float32), axis=2, dtype=np.float32)[:, :, -1]
            row = {"fp32_seq": float(np.abs(seq - ref).max() / scale.max()),
                   "fp32_seq_mean_signed": float(((seq - ref) / scale).mean())}
            for mode, name in ((0, "3"), (2, "4"), (4, "3drain"), (6, "4drain")):
                e = (P.selftest_tc(A, B, four=bool(mode & 2), drain=bool(mode & 4)) - ref) / scale
                row[name] = float(np.abs(e).max())
                row[name + "_mean_signed"] = float(e.mean())
            out["%s_K%d" % (kind, K)] = row
    print(json.dumps(out, indent=1))


def main():
    args = parse()
    if args.tc_accuracy:
        tc_accuracy()
        return
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no oracle arm"}))
            return
        batch_arm(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    import numpy as np
    import torch

    import paper_2203_15684_gb300 as P
    import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream()
    eng = Engine(P, W, args.workload, stream, args, rank, world)
    ctx, mine, nh = eng.ctx, eng.mine, len(eng.atoms)

    def barrier():
        if dist is not None:
            dist.barrier()

    def leg(precision, first, warmup, steps, profile=False, clocks=None):
        """warm-up and timed (q, J) responses of one precision form; returns timings and traces."""
        ctx.set_precision(precision)
        traces = {}
        k = first
        for _ in range(warmup):
            iq, J = mine[k % len(mine)]
            _, dn, _ = ctx.response(iq, J)
            traces[(iq, J)] = _traces(dn, nh)
            k += 1
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if profile:
            P.profile_begin()
        l0 = P.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hpsi, iters = 0, []
        for _ in range(steps):
            iq, J = mine[k % len(mine)]
            torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed launches
            _, dn, info = ctx.response(iq, J)
            torch.cuda.nvtx.range_pop()
            traces[(iq, J)] = _traces(dn, nh)
            hpsi += info["hpsi"]
            iters.append(info["iterations"])
            k += 1
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        out = dict(launches=P.launch_count() - l0, prof=P.profile_end() if profile else None,
                   clocks=clocks.stop() if clocks else None, elapsed=e0.elapsed_time(e1) / 1000.0,
                   hpsi=hpsi, iters=iters, traces=traces, k=k)
        out["elapsed"], out["hpsi_all"] = reduce_over_ranks(out["elapsed"], hpsi, dist, "cuda")
        out["value"] = out["hpsi_all"] / out["elapsed"] if steps else None
        out["ms_per_step"] = 1000.0 * out["elapsed"] / steps if steps else None
        return out

    # the headline: mixed form, K timed (q, J) responses
    mix = leg(1, 0, args.warmup, args.steps, profile=True, clocks=ClockSampler(torch.cuda.current_device()))

    # end to end through the C ABI (mixed form): ground state from pinned host memory, response,
    # Delta n back to the host, every step
    eps, rho, vhxc = ctx.get_ground_state()
    psi = ctx.get_wavefunctions()
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in (vhxc, rho, eps)]
    psi_h = torch.from_numpy(psi.view(np.float64)).pin_memory().numpy().view(np.complex128)
    h2d = sum(a.nbytes for a in host) + psi_h.nbytes
    d2h = 2 * eng.sizes["nhub_atoms"] * eng.sizes["nspin"] * eng.sizes["mmax"] ** 2 * 16
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    hpsi_e, k = 0, mix["k"]
    for _ in range(args.e2e_steps):
        iq, J = mine[k % len(mine)]
        ctx.set_ground_state_packed(eng.w["nspin"], eng.w["nelec"], host[0], host[1], host[2], psi_h)
        _, _, info = ctx.response(iq, J)
        hpsi_e += info["hpsi"]
        k += 1
    torch.cuda.synchronize()
    e2e_el = max(time.perf_counter() - te, 1e-9)
    barrier()

    # FP64 form on the same ground state and pairs (comparison), the measured chi matrices
    f64 = leg(0, 0, args.fp64_warmup, args.fp64_steps)
    common = [p for p in f64["traces"] if p in mix["traces"]]
    chi_rel = max(float(np.abs(mix["traces"][p] - f64["traces"][p]).max() / np.abs(f64["traces"][p]).max())
                  for p in common) if common else None
    chi = {"pairs_per_matrix": len(eng.pairs)}
    if rank == 0 and world == 1 and not args.no_chi_matrix:
        chi["mixed"] = eng.chi_matrix(1)
        chi["mixed_reduced"] = eng.chi_matrix_reduced(1, chi["mixed"])
        chi["mixed_star"] = eng.chi_matrix_reduced(1, chi["mixed"], find_atpert=3)
        if args.fp64_full:
            chi["fp64"] = eng.chi_matrix(0)
            chi["u_err_mev_mixed_vs_fp64"], chi["v_err_mev_mixed_vs_fp64"] = uv_error_mev(chi["mixed"], chi["fp64"])
            chi["speedup_mixed_vs_fp64"] = chi["fp64"]["seconds"] / chi["mixed"]["seconds"]
        elif args.fp64_steps > 0:
            # the FP64 matrix through the star of q (its reconstruction is exact), and the mixed form's
            # error on every U and V against it
            chi["fp64_star"] = eng.chi_matrix_reduced(0, chi["mixed"], find_atpert=3)
            if "U_eV" in chi["fp64_star"]:
                chi["u_err_mev_mixed_vs_fp64"], chi["v_err_mev_mixed_vs_fp64"] = uv_error_mev(chi["mixed"], chi["fp64_star"])
                chi["u_err_mev_mixed_star_vs_fp64"], chi["v_err_mev_mixed_star_vs_fp64"] = uv_error_mev(
                    chi["mixed_star"], chi["fp64_star"])
            eng.ctx.set_precision(1)
    companion = None
    if rank == 0 and world == 1 and args.companion != "none":
        del ctx, eng.ctx
        eng2 = Engine(P, W, args.companion, stream, args, 0, 1)
        companion = {"workload": WORKLOADS[args.companion], "ground_state_s": eng2.gs_seconds, "gap_ha": eng2.gs["gap"]}
        companion["chi_matrix"] = {"mixed": eng2.chi_matrix(1)}
        if args.fp64_full:
            companion["chi_matrix"]["fp64"] = eng2.chi_matrix(0)
            u, v = uv_error_mev(companion["chi_matrix"]["mixed"], companion["chi_matrix"]["fp64"])
            companion["chi_matrix"]["u_err_mev_mixed_vs_fp64"], companion["chi_matrix"]["v_err_mev_mixed_vs_fp64"] = u, v
        if args.companion == "medium":
            companion["oracle_column"] = golden_check(eng2)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family (largest summed event time in the timed region)
    prof = mix["prof"]
    peak, peak_src = measured_peaks()
    fam = max(prof, key=lambda f: prof[f]["ms"])
    p = prof[fam]
    avg_s = p["ms"] / p["launches"] / 1000.0
    alg = p["bytes"] / p["launches"]
    achieved = alg / avg_s / 1e9
    bound = FAMILY_BOUND[fam]
    tflops = p["flops"] / p["ms"] * 1e-9
    if bound == "alu":
        roofline = {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tflops / FP32_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (nominal flops: 5 n log2 n "
                                   "per transformed line, 8 per complex multiply-add)",
                    "hbm_achieved_gbs": achieved, "hbm_peak_gbs": peak, "hbm_frac": achieved / peak}
    elif bound == "tensor":
        tpeak = tensor_peak()
        roofline = {"bound": "tensor", "achieved": tflops, "peak": tpeak[0], "unit": "TFLOP/s",
                    "frac": tflops / tpeak[0], "peak_source": tpeak[1],
                    "hbm_achieved_gbs": achieved, "hbm_peak_gbs": peak, "hbm_frac": achieved / peak}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_src, "achieved_tflops": tflops}
    roofline.update({"traffic": ncu_traffic(fam, alg, args.workload), "kernel": FAMILY_KERNELS[fam][0],
                     "launches": p["launches"], "avg_launch_ms": avg_s * 1000.0, "algorithmic_bytes_per_launch": alg,
                     "share_of_step": p["ms"] / 1000.0 / mix["elapsed"]})
    roofline["families"] = {f: {"share_of_step": round(q["ms"] / 1000.0 / mix["elapsed"], 4),
                                "launches": q["launches"], "bound": FAMILY_BOUND[f],
                                "gbs": round(q["bytes"] / q["ms"] * 1e-6, 1) if q["ms"] else None,
                                "tflops": round(q["flops"] / q["ms"] * 1e-9, 3) if q["ms"] else None,
                                "traffic_per_launch": (ncu_traffic(f, q["bytes"] / q["launches"], args.workload)
                                                       if q["launches"] else None)}
                            for f, q in prof.items()}
    line = {"metric": METRIC, "value": mix["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mix["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 grids and projections, FP64 step lengths, norms, "
                                      "mixing and chi)",
            "data": "synthetic", "config": static_config(args.workload, world),
            "outer_iterations_per_step": mix["iters"],
            "chi_matrix": chi,
            "fp64": {"hpsi_per_s": f64["value"], "ms_per_pair": f64["ms_per_step"], "steps": args.fp64_steps,
                     "warmup": args.fp64_warmup, "outer_iterations_per_step": f64["iters"],
                     "gpu_launches": f64["launches"],
                     "speedup_mixed_vs_fp64_per_pair": (f64["ms_per_step"] / mix["ms_per_step"]
                                                        if f64["ms_per_step"] else None),
                     "chi_column_max_rel_diff_mixed_vs_fp64": chi_rel},
            "ground_state_s": eng.gs_seconds, "gap_ha": eng.gs["gap"],
            "companion": companion,
            "clocks": mix["clocks"],
            "e2e": {"value": hpsi_e / e2e_el, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": mix["launches"], "roofline": roofline}
    if args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.workload)
        # the tiny workload end to end: the oracle's chi time on the host cores against this GPU's
        ref0 = oracle_tiny_chi(line["cpu_baseline"]["cores"])
        gpu0 = gpu_tiny_chi(P, W, stream)
        line["cpu_baseline"]["tiny_chi"] = {
            "workload": "tiny: two-atom cube a=8 bohr, 20 Ry, FFT 20^3, k 2x2x2, q 1x1x1",
            "oracle_chi_s": ref0["chi"], "oracle_ground_state_s": ref0["gs"], "oracle_U_eV": ref0["U"],
            "gpu": gpu0, "u_err_mev_fp64_vs_oracle": 1000.0 * abs(gpu0["fp64"]["U_eV"] - ref0["U"]),
            "u_err_mev_mixed_vs_oracle": 1000.0 * abs(gpu0["mixed"]["U_eV"] - ref0["U"])}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
