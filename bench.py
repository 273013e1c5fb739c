"""Benchmark: seconds to a 1e-10 relative residual on the unit sphere, dx = 1/256.

One step = one complete solve of (1 - Lap_S) u = f on the unit sphere band at
dx = 1/256 (6.79 M band points; f from 23 seeded spherical harmonics,
l in {2, 3, 5}) from u = 0 until ||f - A u||_inf <= 1e-10 ||f||_inf, with the
FP32 V-cycle preconditioning the FP64 outer loop (the headline form).  The
plain FP64 V-cycle solve of the same system is timed beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cpm|reference]
For N > 1 it runs under torchrun, one independent replica per GPU (the solve
does not shard); rank 0 prints one JSON line.

``--impl reference`` times the CPU FP64 oracle (assembled sparse operators,
CPU V-cycle) on a bounded sample of the same workload (the sphere at
dx = 1/64 solved to 1e-10, scaled to dx = 1/256 by the band-size ratio).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DX = 1.0 / 256
METRIC = "s to 1e-10 rel residual, sphere Δx=1/256: FP32-IR/learned vs FP64; HBM GB/s"
SAMPLE_DX = 1.0 / 64
# Outer residual in FP32 pairs (cpm_residual): algorithmic bytes per point of
# B+ (pair weights 96, record 4, delta 8, ref 4) and per point of B (u staged
# 8; the stencil's neighbour indices 24, u 8, f 8, r 8, own delta and ref 12).
RESID_PAIR_BYTES_BPLUS = 96 + 4 + 8 + 4
RESID_PAIR_BYTES_B = 8 + 24 + 8 + 8 + 8 + 12
# FP32 extension bytes: per point of B+ its record 4 + fractions 12 + w 4; per
# point of B its value u 4 (the tile tables, ~2 B per point, are not counted).
EXTEND32_BYTES_BPLUS = 20
EXTEND32_BYTES_B = 4
# DRAM bytes (read + write) of one FP32 extension launch over B+ of the unit
# sphere at dx = 1/256, from one ncu capture of the same kernel and workload.
EXTEND32_TRAFFIC = 165.824768e6 + 21.474048e6


def _sphere_rhs(y):
    import synth
    return synth.sphere_harmonics(y)[1]


def _mixed_rhs(y):
    import synth
    return synth.mixed_rhs(y)


# sphere256 is the headline; the others are the mixed-precision workloads at dx = 1/512
WORKLOADS = {
    "sphere256": {"kind": "sphere", "params": (), "dx": 1 / 256, "coarsest": 1 / 8, "rhs": _sphere_rhs,
                  "desc": "unit sphere dx=1/256, 23 N(0,1) harmonics l in {2,3,5}"},
    "sphere512": {"kind": "sphere", "params": (), "dx": 1 / 512, "coarsest": 1 / 8, "rhs": _mixed_rhs,
                  "desc": "unit sphere dx=1/512, f = (1 + 0.5 x y) u_rand"},
    "torus512": {"kind": "torus", "params": (1.0, 0.4), "dx": 1 / 512, "coarsest": 1 / 16,
                 "rhs": _mixed_rhs, "desc": "torus R=1 r=0.4 dx=1/512, f = (1 + 0.5 x y) u_rand"},
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def band_size(kind: str, inv_dx: int) -> int:
    """|B| of the oracle's band, from tests/golden/band_sizes.txt (make_band_sizes.py)."""
    with open(os.path.join(ROOT, "tests", "golden", "band_sizes.txt")) as fh:
        for line in fh:
            p = line.split()
            if p and not line.startswith("#") and p[0] == kind and int(p[2]) == inv_dx:
                return int(p[3])
    raise KeyError((kind, inv_dx))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest per-rank value (the slowest replica sets the job's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _oracle_worker(barrier, queue, repeats):
    """One oracle process: build the sample hierarchy, wait for the others,
    then time `repeats` solves (seconds each)."""
    import warnings

    warnings.simplefilter("ignore")
    import synth
    from oracle.geometry import sphere
    from oracle.multigrid import MGOptions, build_hierarchy, solve

    t0 = time.perf_counter()
    H = build_hierarchy(sphere(), SAMPLE_DX, 1 / 8,
                        opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8))
    build_s = time.perf_counter() - t0
    b = H.fine.band
    _, f = synth.sphere_harmonics(b.cp[: b.nb])
    barrier.wait()
    times, iters = [], 0
    for _ in range(repeats):
        t = time.perf_counter()
        _, rep = solve(H, f, tol=1e-10, max_iter=60)
        times.append(time.perf_counter() - t)
        iters = rep.iters
    queue.put({"times": times, "iters": iters, "nb": int(b.nb), "build_s": build_s})


def oracle_timing(procs: int, repeats: int):
    """Time the oracle (as it stands, single-threaded numpy/scipy) on the bounded
    sample: the unit sphere at dx = 1/64 solved to 1e-10.  `procs` independent
    spawned processes, each pinned to one BLAS thread, build the sample, meet at
    a barrier and time their solves together: procs = 1 is the one-core time,
    procs = nproc the whole host's throughput (seconds per solve = the slowest
    process's time / procs)."""
    import multiprocessing as mp

    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier, queue = ctx.Barrier(procs), ctx.Queue()
        ps = [ctx.Process(target=_oracle_worker, args=(barrier, queue, repeats)) for _ in range(procs)]
        for p in ps:
            p.start()
        res = [queue.get() for _ in ps]
        for p in ps:
            p.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    # per repeat: the slowest process sets the wall time of `procs` solves
    per_rep = [max(r["times"][k] for r in res) for k in range(repeats)]
    wall = statistics.median(per_rep)
    scale = band_size("sphere", 256) / res[0]["nb"]
    return {"procs": procs, "wall_s": wall, "s_per_solve": wall / procs, "scale": scale,
            "value": wall / procs * scale, "iters": res[0]["iters"], "nb_sample": res[0]["nb"],
            "build_s": max(r["build_s"] for r in res)}


def cpu_baseline_line(one, many):
    sample = (f"oracle FP64 defect correction with its V-cycle (Jacobi nu=3/3, omega=0.8) on the "
              f"unit sphere at dx=1/64 ({one['nb_sample']} band points) to 1e-10: measured "
              f"{one['s_per_solve']:.2f} s per solve on 1 core"
              + (f", {many['s_per_solve']:.2f} s per solve on {many['procs']} cores "
                 f"({many['procs']} independent solves at once, {many['wall_s']:.2f} s wall)"
                 if many else "")
              + f"; value = the 1-core time scaled x{one['scale']:.2f} by the band-size ratio to "
              f"dx=1/256 (an estimate); hierarchy assembly excluded")
    line = {"value": one["value"], "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
            "measured": {"dx": SAMPLE_DX, "points": one["nb_sample"], "iters": one["iters"],
                         "s_1core": one["s_per_solve"]}}
    if many:
        line["nproc"] = {"cores": many["procs"], "s_per_solve": many["s_per_solve"],
                         "wall_s": many["wall_s"], "value_scaled": many["value"]}
    return line


def run_reference(args, world, rank):
    if rank != 0:
        return
    one = oracle_timing(1, max(1, args.steps))
    sample = (f"oracle FP64 defect correction with its V-cycle (Jacobi nu=3/3, omega=0.8) on the "
              f"unit sphere at dx=1/64 ({one['nb_sample']} band points) to 1e-10, median of "
              f"{args.steps} solves = {one['s_per_solve']:.2f} s on 1 core, scaled by the band-size "
              f"ratio {one['scale']:.2f} to dx=1/256; assembly excluded")
    line = {"impl": "reference", "metric": METRIC, "value": one["value"], "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": one["s_per_solve"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "unit sphere dx=1/256 (bounded sample dx=1/64)", "tol": 1e-10},
            "cpu_baseline": {"value": one["value"], "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": one["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cpm(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1307_4354_gb300 as pkg
    import synth

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    t0 = time.perf_counter()
    wl = WORKLOADS[args.workload]
    band = pkg.Band(wl["kind"], wl["params"], wl["dx"])
    H = pkg.Hierarchy(band, coarsest_dx=wl["coarsest"], nu1=args.nu, nu2=args.nu, omega=args.omega,
                      residual=args.residual)
    setup_s = time.perf_counter() - t0
    _, cp, _ = band.export()
    f_np = wl["rhs"](cp[: band.nb])
    nb = band.nb
    f = torch.from_numpy(f_np).to(dev)
    u = torch.zeros(nb, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    tol = wl.get("tol", 1e-10)

    def solve(mode):
        _, rep = H.solve(f, u, tol=tol, max_iter=200, mode=mode, zero_init=True,
                         inner_cycles=args.inner)
        assert rep["converged"], rep
        return rep

    # warm-up (also captures the CUDA graphs)
    for _ in range(args.warmup):
        solve("mixed")
        if not args.only_mixed:
            solve("f64")
    torch.cuda.synchronize()

    # timed: mixed precision (headline)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = pkg.capi.cpm_kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_mixed")  # the range a launch-list capture selects
        ev0.record(st)
        reps = [solve("mixed") for _ in range(args.steps)]
        ev1.record(st)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    mixed_ms = ev0.elapsed_time(ev1) / args.steps
    launches = pkg.capi.cpm_kernel_launches() - launches0
    u_mixed = u.clone()
    mixed_ms = max_over_ranks(mixed_ms, world, dev)
    iters_mixed = reps[-1]["iters"]

    if args.only_mixed:
        print(json.dumps({"mixed_ms": mixed_ms, "iters": iters_mixed, "gpu_launches": int(launches)}),
              flush=True)
        return
    # plain FP64 solve (context)
    k64 = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    ev0.record(st)
    reps64 = [solve("f64") for _ in range(k64)]
    ev1.record(st)
    torch.cuda.synchronize()
    f64_ms = ev0.elapsed_time(ev1) / k64
    u_f64 = u.clone()

    def rel_diff(a, b):
        return float((a - b).abs().max() / b.abs().max())

    accuracy = {"mixed_vs_f64": rel_diff(u_mixed, u_f64)}
    if args.workload == "sphere256":  # closed-form solution sum a_lm Y_lm at cp
        uex = torch.from_numpy(synth.sphere_harmonics(cp[:nb])[0]).to(dev)
        accuracy["f64_vs_exact"] = rel_diff(u_f64, uex)
        accuracy["mixed_vs_exact"] = rel_diff(u_mixed, uex)

    # learned smoother: trained on the GPU (own kernels) on V-cycle residuals of
    # seeded ellipsoids and tori at dx = 1/64, then judged against Jacobi
    learned = None
    if not args.no_learned and args.workload == "sphere256":
        from paper_1307_4354_gb300 import train as tr
        t0 = time.perf_counter()
        sets = tr.training_set(seed=0, spacings=(1 / 64, 1 / 96, 1 / 128))
        data_s = time.perf_counter() - t0
        sm = pkg.Smoother(0)
        trep = tr.train(sm, sets, steps=args.train_steps, lr=2e-3, lr_final=2e-4)
        loss0, loss1 = trep["loss_first"], trep["loss_last"]
        train_s = trep["seconds"]
        train_points = [h.nb for h, _ in sets]
        del sets
        H.set_smoother(sm)

        def solve_learned():
            _, rep = H.solve(f, u, tol=1e-10, max_iter=200, mode="mixed", zero_init=True,
                             inner_cycles=args.inner, learned=True)
            assert rep["converged"], rep
            return rep

        for _ in range(2):
            solve_learned()
        torch.cuda.synchronize()
        ev0.record(st)
        repsL = [solve_learned() for _ in range(args.steps)]
        ev1.record(st)
        torch.cuda.synchronize()
        learned_ms = ev0.elapsed_time(ev1) / args.steps
        accuracy["learned_vs_f64"] = rel_diff(u, u_f64)
        # held-out evaluation: torus R = 1, r = 0.35, dx = 1/256, c = 1 + 0.5 sin(2 pi z)
        Ht, _ = tr.residual_fields("torus", (1.0, 0.35), DX, seed=7, iters=(0,),
                                   c_fn=lambda y: 1.0 + 0.5 * np.sin(2 * np.pi * y[:, 2]))
        Ht.set_smoother(sm)
        ut = torch.zeros_like(Ht._f)
        ev = {}
        for name, flag in (("jacobi", False), ("learned", True)):
            Ht.solve(Ht._f, ut, tol=1e-10, max_iter=200, mode="mixed", zero_init=True,
                     inner_cycles=args.inner, learned=flag)
            torch.cuda.synchronize()
            ev0.record(st)
            _, rp = Ht.solve(Ht._f, ut, tol=1e-10, max_iter=200, mode="mixed", zero_init=True,
                             inner_cycles=args.inner, learned=flag)
            ev1.record(st)
            torch.cuda.synchronize()
            ev[name] = {"s": ev0.elapsed_time(ev1) / 1e3, "iters": rp["iters"],
                        "converged": rp["converged"], "fallback": rp["fallback"],
                        "jacobi_factor": rp["jacobi_factor"], "learned_factor": rp["learned_factor"]}
        learned = {"s": learned_ms / 1e3, "iters": repsL[-1]["iters"],
                   "fallback": repsL[-1]["fallback"], "jacobi_factor": repsL[-1]["jacobi_factor"],
                   "learned_factor": repsL[-1]["learned_factor"], "train_s": train_s,
                   "train_data_s": data_s, "train_points": train_points,
                   "train_steps": args.train_steps, "train_loss": [loss0, loss1],
                   "torus_r035_dx256_variable_c": ev, "torus_points": Ht.nb}
        H.set_smoother(None)
        del Ht

    # end to end through the C ABI with host buffers
    f_host = torch.from_numpy(f_np).pin_memory()
    u_host = torch.empty(nb, dtype=torch.float64).pin_memory()
    fd = torch.empty(nb, dtype=torch.float64, device=dev)
    ud = torch.empty(nb, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(st)
    for _ in range(args.steps):
        fd.copy_(f_host, non_blocking=True)
        H.solve(fd, ud, tol=tol, max_iter=200, mode="mixed", zero_init=True,
                inner_cycles=args.inner)
        u_host.copy_(ud, non_blocking=True)
    ev1.record(st)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1) / args.steps

    # dominant kernel: the FP32 extension over B+ (one launch = nB + nG points),
    # CUDA events on the launching stream; and the outer residual in FP32 pairs.
    w32 = torch.empty(nb + band.ng, dtype=torch.float32, device=dev)
    r64 = torch.empty_like(u)
    u32 = u.float()
    for _ in range(3):
        H.residual(f, u, out=r64)
        H.extend(u32, with_ghost=True, out=w32)
    reps_k = 20
    torch.cuda.synchronize()
    ev0.record(st)
    for _ in range(reps_k):
        H.residual(f, u, out=r64)
    ev1.record(st)
    torch.cuda.synchronize()
    resid_ms = ev0.elapsed_time(ev1) / reps_k
    ev0.record(st)
    for _ in range(reps_k):
        H.extend(u32, with_ghost=True, out=w32)
    ev1.record(st)
    torch.cuda.synchronize()
    ext32_ms = ev0.elapsed_time(ev1) / reps_k
    npl = nb + band.ng
    bytes_res = RESID_PAIR_BYTES_BPLUS * npl + RESID_PAIR_BYTES_B * nb
    ach_res = bytes_res / (resid_ms * 1e-3) / 1e9
    bytes32 = EXTEND32_BYTES_BPLUS * npl + EXTEND32_BYTES_B * nb
    ach32 = bytes32 / (ext32_ms * 1e-3) / 1e9
    pk = peaks()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and args.workload == "sphere256":
        one = oracle_timing(1, 1)
        many = oracle_timing(os.cpu_count() or 1, 1) if (os.cpu_count() or 1) > 1 else None
        cpu = cpu_baseline_line(one, many)
    nl = H.n_levels
    sizes = [H.level_size(l) for l in range(nl)]
    sweeps = 2 * args.nu * args.inner  # Jacobi sweeps per level per outer iteration
    updates = sum(sizes[:-1]) * sweeps * iters_mixed
    line = {
        "metric": METRIC if args.workload == "sphere256" else
                  f"s to {tol:g} rel residual, {wl['desc']}: FP32-IR vs FP64",
        "value": mixed_ms / 1e3, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed_ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"{wl['desc']} ({nb} band points, {band.ng} ghost), c=1, tol {tol:g}, "
                               "mixed FP32 V-cycle in FP64 defect correction",
                   "levels": sizes, "smoother": f"jacobi nu={args.nu}/{args.nu} omega={args.omega}",
                   "residual": args.residual, "inner_cycles": args.inner, "transfers": "linear",
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "iters_mixed": iters_mixed, "fp64_s": f64_ms / 1e3, "iters_fp64": reps64[-1]["iters"],
        "history_mixed": reps[-1]["history"], "f64_checks": reps[-1]["f64_checks"],
        "pair_floor": reps[-1]["pair_floor"],
        "accuracy": dict(accuracy, note="max-norm differences relative to max |u_f64| (or |u_exact|)"),
        "learned": learned,
        "band_point_updates_per_s": updates / (mixed_ms * 1e-3),
        "vcycles_per_s": {"mixed_fp32": iters_mixed * args.inner / (mixed_ms * 1e-3),
                          "fp64": reps64[-1]["iters"] / f64_ms * 1e3},
        "setup_s": setup_s,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": nb * 8,
                "d2h_bytes_per_step": nb * 8},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_extend_tiles<float,3> (FP32 extension over B+, the largest "
                               "share of the mixed solve's kernel time)", "bound": "hbm",
                     "achieved": ach32, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": ach32 / pk.get("hbm_gbs", 6800.0),
                     "traffic": EXTEND32_TRAFFIC if wl["kind"] == "sphere" and wl["dx"] == DX else None,
                     "algorithmic_bytes": bytes32, "points": npl, "ms": ext32_ms,
                     "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"},
        "roofline_outer_residual": {"kernel": "cpm_residual in FP32 pairs (k_extend_pair over B+, "
                                              "k_resid_pair over B, norms)", "bound": "hbm",
                                    "achieved": ach_res, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                                    "frac": ach_res / pk.get("hbm_gbs", 6800.0), "traffic": None,
                                    "algorithmic_bytes": bytes_res, "ms": resid_ms,
                                    "note": "the pair extension is FP32-pipe and latency bound "
                                            "(pair arithmetic, 72 registers); see profiles"},
        "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_batch(args, world, rank, local):
    """Batched workload: 64 ellipsoids (semi-axes ~ U[0.6, 1.2]^3, dx drawn from
    {1/64, 1/96, 1/128}) x 4 right-hand sides, all solved to 1e-10 by one
    cpm_solve_batch call (one graph launch per outer iteration, autotuned
    concurrency).  The same systems solved one after another with cpm_solve are
    timed beside it."""
    import numpy as np
    import torch

    import paper_1307_4354_gb300 as pkg
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    inst = synth.ellipsoid_batch(seed=0, count=args.batch_count)
    n_rhs = 4
    t0 = time.perf_counter()
    hs, fs = [], []
    for i, (ax, dx) in enumerate(inst):
        g = pkg.Band("ellipsoid", ax, dx)
        H = pkg.Hierarchy(g, nu1=args.nu, nu2=args.nu, omega=args.omega, residual=args.residual,
                          coarse_f64_max=4096, coarse_dense_max=65536)
        _, cp, _ = g.export()
        for fk in synth.harmonic_fields(cp[: g.nb], [100 * i + k for k in range(n_rhs)]):
            fs.append(torch.from_numpy(fk).to(dev))
        hs.append(H)
        del g
    B = pkg.Batch(hs, n_rhs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    us = [torch.zeros_like(f) for f in fs]
    st = torch.cuda.current_stream()

    def solve():
        _, reps = B.solve(fs, us, tol=1e-10, max_iter=200, mode="mixed", inner_cycles=args.inner,
                          zero_init=True, raise_on_fail=False)
        return reps

    for _ in range(args.warmup):  # the first solve also runs the autotuner
        solve()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = pkg.capi.cpm_kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(st)
        reps = [solve() for _ in range(args.steps)]
        ev1.record(st)
        torch.cuda.synchronize()
    batch_ms = ev0.elapsed_time(ev1) / args.steps
    launches = pkg.capi.cpm_kernel_launches() - launches0
    last = reps[-1]
    # the same systems one after another (cpm_solve per system)
    torch.cuda.synchronize()
    ev0.record(st)
    seq_iters = []
    for s, f in enumerate(fs):
        _, r = hs[s // n_rhs].solve(f, us[s], tol=1e-10, max_iter=200, mode="mixed",
                                    inner_cycles=args.inner, zero_init=True, raise_on_fail=False)
        seq_iters.append(r["iters"])
    ev1.record(st)
    torch.cuda.synchronize()
    seq_ms = ev0.elapsed_time(ev1)
    K, tune = B.info()
    iters = [r["iters"] for r in last]
    sizes = [h.nb for h in hs]
    coarse = [h.level_size(h.n_levels - 1) for h in hs]
    pts = sum(sizes) * n_rhs
    if rank != 0:
        return
    line = {
        "metric": "s to 1e-10 rel residual, batch of 64 ellipsoids x 4 RHS (mixed FP32/FP64)",
        "value": batch_ms / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"{len(hs)} ellipsoids, semi-axes U[0.6,1.2]^3 (seed 0), dx in "
                               "{1/64,1/96,1/128}, 4 harmonic right-hand sides each, c=1, tol 1e-10",
                   "band_points": sizes, "coarsest_points": coarse, "inner_cycles": args.inner,
                   "smoother": f"jacobi nu={args.nu}/{args.nu} omega={args.omega}",
                   "residual": args.residual, "l2": "inputs larger than L2 (no flush)"},
        "systems": len(fs), "points_x_rhs": pts,
        "converged": sum(1 for r in last if r["converged"]),
        "status": sorted({r["status"] for r in last}),
        "iters": {"min": min(iters), "max": max(iters), "mean": float(np.mean(iters))},
        "autotune": {"concurrency": K, "ms_per_iteration_by_K": tune},
        "sequential_s": seq_ms / 1e3, "sequential_iters_equal": seq_iters == iters,
        "band_point_updates_per_s": sum(sizes[s // n_rhs] * iters[s] for s in range(len(fs)))
        * 2 * args.inner * args.nu / (batch_ms * 1e-3),
        "vcycles_per_s": sum(iters) * args.inner / (batch_ms * 1e-3),
        "setup_s": setup_s, "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    B.close()


def run_micro(args):
    """Kernel micro-benchmark on the dx = 1/256 sphere band (also the ncu target):
    each case is one kind of launch, timed with CUDA events on the launching
    stream after `--warmup` untimed launches.  Cases: extend32 / extend64 (the
    extension over B+), extend32_v0 / _v1 / _v2 (the FP32 extension forced to
    one work decomposition), apply32 / apply64 (M u), jacobi32 (one Jacobi
    sweep), resid64 / resid64_f64 (the relative-form outer residual in FP32 pairs
    / in FP64), vcycle32 (one FP32
    V-cycle: transfers and the coarsest solve included), mlp (the learned
    smoother's forward over B).  The timed launches sit in the NVTX range
    "micro", so that ncu can select them with --nvtx-include micro/."""
    import torch

    import paper_1307_4354_gb300 as pkg

    pkg.build()
    band = pkg.Band("sphere", (), DX)
    nb, ng = band.nb, band.ng
    wanted = args.micro.split(",")
    hiers = {}

    def hier(v=None, outer_f64=False):
        if (v, outer_f64) not in hiers:
            hiers[v, outer_f64] = pkg.Hierarchy(band, coarsest_dx=1 / 8, nu1=args.nu, nu2=args.nu,
                                                omega=args.omega, residual=args.residual,
                                                ext_variant=v, outer_f64=outer_f64)
        return hiers[v, outer_f64]

    g = torch.Generator(device="cuda").manual_seed(0)
    u64 = torch.rand(nb, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    u32 = u64.float()
    f64 = torch.rand(nb, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    f32 = f64.float()
    w64 = torch.empty(nb + ng, dtype=torch.float64, device="cuda")
    w32 = torch.empty(nb + ng, dtype=torch.float32, device="cuda")
    m64 = torch.empty_like(u64)
    m32 = torch.empty_like(u32)
    z32 = torch.zeros_like(u32)
    cases = {
        "extend32": lambda: hier().extend(u32, with_ghost=True, out=w32),
        "extend64": lambda: hier().extend(u64, with_ghost=True, out=w64),
        "extend32_v0": lambda: hier(0).extend(u32, with_ghost=True, out=w32),
        "extend32_v1": lambda: hier(1).extend(u32, with_ghost=True, out=w32),
        "extend32_v2": lambda: hier(2).extend(u32, with_ghost=True, out=w32),
        "apply32": lambda: hier().apply(u32, out=m32),
        "apply64": lambda: hier().apply(u64, out=m64),
        "jacobi32": lambda: hier().smooth(f32, u32, sweeps=1),
        "resid64": lambda: hier().residual(f64, u64, out=m64),
        "resid64_f64": lambda: hier(outer_f64=True).residual(f64, u64, out=m64),
        "vcycle32": lambda: hier().vcycle(f32, z32.zero_()),
    }
    if "mlp" in wanted or args.micro == "all":
        sm = pkg.Smoother(0)
        hier().set_smoother(sm)
        cases["mlp"] = lambda: hier().smoother_correction(f32, out=m32)
    out = {}
    st = torch.cuda.current_stream()
    for name, fn in cases.items():
        if args.micro != "all" and name not in wanted:
            continue
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("micro")
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out[name + "_ms"] = e0.elapsed_time(e1) / max(1, args.steps)
    tuning = [hier().ext_tuning(l) for l in range(hier().n_levels)]
    print(json.dumps({"micro": out, "nb": nb, "ng": ng, "ext_tuning": tuning}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cpm", choices=["cpm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner", type=int, default=3, help="FP32 V-cycles per outer iteration")
    ap.add_argument("--residual", default="plain", choices=["extended", "plain"],
                    help="residual restricted in the V-cycle: f - A(E u) (Sec. 4.4) or f - A u")
    ap.add_argument("--nu", type=int, default=4, help="pre- and post-smoothing sweeps")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-smoother form")
    ap.add_argument("--workload", default="sphere256", choices=sorted(WORKLOADS))
    ap.add_argument("--only-mixed", action="store_true",
                    help="time only the mixed-precision solve (profiling runs)")
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--batch", action="store_true",
                    help="batched workload: ellipsoids x 4 right-hand sides in one cpm_solve_batch")
    ap.add_argument("--batch-count", type=int, default=64, help="ellipsoids in the batched workload")
    ap.add_argument("--omega", type=float, default=0.8, help="Jacobi weight")
    ap.add_argument("--micro", default=None,
                    help="kernel micro-benchmark instead of the solve: a comma-separated list of "
                         "extend32, extend64, extend32_v0/_v1/_v2, apply32, apply64, jacobi32, "
                         "resid64, vcycle32, mlp, or all")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.micro:
        run_micro(args)
        return
    if args.batch:
        run_batch(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_cpm(args, world, rank, local)


if __name__ == "__main__":
    main()
