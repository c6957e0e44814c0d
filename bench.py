#!/usr/bin/env python3
"""Benchmark of the DFPT Hubbard-parameter hot path on GB300.

Workload (--workload): "medium" (default), the rocksalt-like cell (8.4 bohr cube, 4 H + 4 L,
40 electrons, collinear nspin = 2 with an antiferromagnetic start, 35 Ry, FFT 36^3, k 4x4x4,
q 2x2x2); "precision", the same cell at 50 Ry (FFT 45^3).  The ground state is computed on the GPU
before timing.  One step = one (q, J) self-consistent Sternheimer response
(the per-q set-up a1 and a3-a10): every (spin, k, band) system of that pair, to the FP64
tolerances the parity tests use.  The 64 (q, J) pairs of the full chi matrix are independent and
alike, so the full-matrix wall time is reported as steps-per-matrix x time per step.  The headline
is the mixed-precision form (FP32 FFTs, grid work and projections; FP64 vectors, CG scalars,
mixing and inversion); the FP64 form is timed on the same ground state and pairs for comparison.

Metric: H.psi/s (single-band applications of the Sternheimer operator, summed over ranks).
N > 1 (torchrun): the (q, J) pairs are sharded round-robin over ranks (weak scaling, no collective
on the data path); timing is the max over ranks between barriers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload medium|precision]
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
WORKLOADS = {
    "medium": "medium: rocksalt cube a=8.4 bohr, 4 H + 4 L, 40 electrons, nspin=2 (AFM start), "
              "ecutwfc 35 Ry (npw<=2103), FFT 36^3, k 4x4x4, q 2x2x2",
    "precision": "precision: the medium cell at ecutwfc 50 Ry (npw<=3575), FFT 45^3, k 4x4x4, q 2x2x2, "
                 "nspin=2 (AFM start)",
    "batch": "batch: 6 small insulating cells of uneven sizes (two-atom cube at 8/10/20 Ry, q meshes of 1-8 "
             "points, rocksalt cell at 6 Ry with nspin=2), mixed form",
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--fp64-warmup", type=int, default=1)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--band-batch", type=int, default=0, help="grids per FFT batch (0 = automatic)")
    p.add_argument("--workload", default="medium", choices=sorted(WORKLOADS))
    p.add_argument("--cg-adapt", type=float, default=None,
                   help="CG threshold factor for outer iterations after the first (library default if omitted)")
    return p.parse_args()


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
def _oracle_sample(seconds, workload="medium"):
    """The oracle's Sternheimer operator (H + alpha P_v - eps) applied to blocks of 20 bands on the
    workload's spheres and grid, with the oracle's own starting-density potential, for about
    ``seconds``; returns (H.psi count, elapsed)."""
    import numpy as np

    import workloads as W
    from oracle import groundstate as G
    from oracle.hamiltonian import apply_h
    from oracle.model import Model

    w = getattr(W, workload)()
    m = Model(w)
    vr = m.vloc_r() + G.hxc_potential(m, G.initial_density(m))[0]
    rng = np.random.default_rng(2203)
    n, t0, ik = 0, time.perf_counter(), 0
    while True:
        kd = m.kdata(m.kpts[ik % len(m.kpts)])
        U = np.linalg.qr(rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc)))[0]
        X = rng.standard_normal((kd.npw, m.nocc)) + 1j * rng.standard_normal((kd.npw, m.nocc))
        Y = apply_h(m, kd, vr, X) + 2.0 * (U @ (U.conj().T @ X)) - X * 0.5
        n += X.shape[1]
        ik += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el, float(np.abs(Y).max())


def run_oracle_subprocess(seconds, workload="medium"):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; n, el, _ = bench._oracle_sample(%f, %r); "
            "print(json.dumps(dict(n=n, el=el)))" % (ROOT, seconds, workload))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["n"], d["el"]


def cpu_baseline(seconds, workload="medium"):
    n, el = run_oracle_subprocess(seconds, workload)
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle Sternheimer operator (H + alpha P_v - eps) on %d single-band vectors of the %s "
                      "workload (20-band blocks cycling over its 64 k spheres), %.1f s, 1 thread" % (n, workload, el)}


def reference_arm(args, rank):
    if rank != 0:
        return
    vals = []
    n_tot, el_tot = 0, 0.0
    for _ in range(args.warmup):
        run_oracle_subprocess(2.0, args.workload)
    for _ in range(args.steps):
        n, el = run_oracle_subprocess(5.0, args.workload)
        vals.append(n / el)
        n_tot += n
        el_tot += el
    value = n_tot / el_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "step": "about 5 s of the oracle's Sternheimer operator on the "
                                                          "workload's spheres (1 thread)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d H.psi in %.1f s over %d steps" % (n_tot, el_tot, args.steps)},
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


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    return 6800.0, "fallback (no MEASURED_PEAKS.json)"


def batch_arm(args):
    """Batching form: the full chi matrices of a batch of small cells, one cell after the other and
    all at once (hp_batch_run: one host thread and CUDA stream per cell); cells per hour of each."""
    import torch

    import paper_2203_15684_gb300 as P
    import workloads as W

    cells = W.batch_small()

    def ready(w):
        stream = torch.cuda.Stream()
        ctx = P.Context.from_workload(w, cuda_stream=stream.cuda_stream, precision=1)
        ctx.ground_state(w["nelec"], w["nspin"], w.get("moments"))
        return ctx, stream

    def alone(ctxs):
        for ctx, _ in ctxs:
            atoms, _ = ctx.hubbard_atoms()
            for J in atoms:
                for iq in range(ctx.query_sizes()["nq"]):
                    ctx.response(iq, int(J))
            ctx.hubbard()

    times_a, times_b = [], []
    l0 = P.launch_count()
    for rep in range(args.warmup + args.steps):
        ctxs = [ready(w) for w in cells]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        alone(ctxs)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        ctxs = [ready(w) for w in cells]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.batch_run([c for c, _ in ctxs])
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        if rep >= args.warmup:
            times_a.append(ta)
            times_b.append(tb)
    ta, tb = sum(times_a) / len(times_a), sum(times_b) / len(times_b)
    n = len(cells)
    line = {"metric": "cells/hour, batch of small cells (full chi and U/V per cell, mixed form)",
            "value": n * 3600.0 / tb, "unit": "cells/h", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"], "step": "one batch: every (q, J) response and chi/U/V of every "
                                                                "cell, ground states computed before timing",
                       "one_after_another_cells_per_hour": n * 3600.0 / ta,
                       "speedup_batch_vs_one_after_another": ta / tb},
            "gpu_launches": P.launch_count() - l0}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch mode has no reference arm"}))
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
    w = getattr(W, args.workload)()
    opts = dict(cuda_stream=stream.cuda_stream, band_batch=args.band_batch)
    if args.cg_adapt is not None:
        opts["cg_adapt"] = args.cg_adapt
    ctx = P.Context.from_workload(w, **opts)
    t0 = time.perf_counter()
    gs = ctx.ground_state(w["nelec"], w["nspin"], w["moments"])
    gs_seconds = time.perf_counter() - t0
    atoms, _ = ctx.hubbard_atoms()
    s = ctx.query_sizes()
    pairs = [(iq, int(J)) for J in atoms for iq in range(s["nq"])]
    mine = shard_pairs(pairs, rank, world)

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
            traces[(iq, J)] = np.array([np.trace(dn[a].sum(0)) for a in range(len(atoms))])
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
            torch.cuda.nvtx.range_push("timed_step")
            _, dn, info = ctx.response(iq, J)
            torch.cuda.nvtx.range_pop()
            traces[(iq, J)] = np.array([np.trace(dn[a].sum(0)) for a in range(len(atoms))])
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

    # FP64 form (comparison) then the mixed form (headline), on the same ground state and pairs
    f64 = leg(0, 0, args.fp64_warmup, args.fp64_steps)
    mix = leg(1, 0, args.warmup, args.steps, profile=True, clocks=ClockSampler(torch.cuda.current_device()))
    common = [p for p in f64["traces"] if p in mix["traces"]]
    chi_rel = max(float(np.abs(mix["traces"][p] - f64["traces"][p]).max() / np.abs(f64["traces"][p]).max())
                  for p in common) if common else None

    # end to end through the C ABI (mixed form): ground state from pinned host memory, response,
    # Delta n back to the host, every step
    eps, rho, vhxc = ctx.get_ground_state()
    psi = ctx.get_wavefunctions()
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in (vhxc, rho, eps)]
    psi_h = torch.from_numpy(psi.view(np.float64)).pin_memory().numpy().view(np.complex128)
    h2d = sum(a.nbytes for a in host) + psi_h.nbytes
    d2h = 2 * s["nhub_atoms"] * s["nspin"] * s["mmax"] ** 2 * 16
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    hpsi_e, k = 0, mix["k"]
    for _ in range(args.e2e_steps):
        iq, J = mine[k % len(mine)]
        ctx.set_ground_state_packed(w["nspin"], w["nelec"], host[0], host[1], host[2], psi_h)
        _, _, info = ctx.response(iq, J)
        hpsi_e += info["hpsi"]
        k += 1
    torch.cuda.synchronize()
    e2e_el = max(time.perf_counter() - te, 1e-9)
    barrier()
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
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_src, "achieved_tflops": tflops}
    roofline.update({"traffic": ncu_traffic(fam, alg, args.workload), "kernel": FAMILY_KERNELS[fam][0],
                     "launches": p["launches"], "avg_launch_ms": avg_s * 1000.0, "algorithmic_bytes_per_launch": alg,
                     "share_of_step": p["ms"] / 1000.0 / mix["elapsed"]})
    roofline.update({
                "families": {f: {"share_of_step": round(q["ms"] / 1000.0 / mix["elapsed"], 4),
                                 "launches": q["launches"], "bound": FAMILY_BOUND[f],
                                 "gbs": round(q["bytes"] / q["ms"] * 1e-6, 1) if q["ms"] else None,
                                 "tflops": round(q["flops"] / q["ms"] * 1e-9, 3) if q["ms"] else None,
                                 "traffic_per_launch": (ncu_traffic(f, q["bytes"] / q["launches"], args.workload)
                                                        if q["launches"] else None)}
                             for f, q in prof.items()}})
    line = {"metric": METRIC, "value": mix["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mix["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 grids and projections, FP64 vectors and scalars)",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "step": "one (q, J) self-consistent Sternheimer response, %d band systems"
                               % (s["nspin"] * s["nk"] * s["nocc"]),
                       "pairs_per_chi_matrix": len(pairs),
                       "chi_matrix_s": mix["ms_per_step"] * len(pairs) / 1000.0 / world,
                       "outer_iterations_per_step": mix["iters"],
                       "fp64": {"hpsi_per_s": f64["value"], "ms_per_step": f64["ms_per_step"],
                                "chi_matrix_s": (f64["ms_per_step"] * len(pairs) / 1000.0 / world
                                                 if f64["ms_per_step"] else None),
                                "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                                "outer_iterations_per_step": f64["iters"], "gpu_launches": f64["launches"]},
                       "chi_matrix_speedup_mixed_vs_fp64": (f64["ms_per_step"] / mix["ms_per_step"]
                                                            if f64["ms_per_step"] else None),
                       "chi_max_rel_diff_mixed_vs_fp64": chi_rel,
                       "ground_state_s": gs_seconds, "gap_ha": gs["gap"],
                       "l2": "inputs larger than L2 (response working set about 1.7 GB mixed, 2.6 GB FP64)",
                       "parallelism": "(q, J) pairs round-robin over %d rank(s)" % world},
            "clocks": mix["clocks"],
            "e2e": {"value": hpsi_e / e2e_el, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": mix["launches"], "roofline": roofline}
    if args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.workload)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
