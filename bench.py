"""Benchmark: walker local-energy evaluations per second at pentacene scale.

One step = walkers_energy over one batch of W walkers through the C ABI: the
whole hot path (overlap, LU, log-det, Theta, one-body + Coulomb, LO pair
exchange, FP64 reductions).  Default workload: synthetic acene ribbon,
M = 440 basis functions, N = 73 occupied orbitals (closed shell), X = 1800
Cholesky vectors, W = 1024 walkers, T_SVD = 1e-4, FP16 hi+lo split products.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (bounded sample of the same workload).  Under torchrun
each rank evaluates its own W walkers (independent walker shards, no
collective on the data path); the wall time is the max over ranks.
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

from paper_2202_00832_b300 import synth  # noqa: E402

METRIC = "walker local-energy evals/sec at pentacene scale"
WORKLOADS = {"pentacene": synth.PENTACENE_440, "naphthalene": synth.NAPHTHALENE_250,
             "chain": synth.CHAIN_60, "acene_n73": synth.PROFILE_N73}
UNIT = "walker-energies/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--workload", default="pentacene", choices=sorted(WORKLOADS),
                    help="pentacene (the benchmark) or a smaller system for profiling")
    ap.add_argument("--threshold", type=float, default=1e-4)
    ap.add_argument("--precision", default="fp16x3",
                    choices=["fp16x3", "fp16x3_f64inv", "bf16x3", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=3, help="walkers timed on the oracle")
    ap.add_argument("--full-sample", type=int, default=64, help="walkers of the FP64 full GPU leg")
    ap.add_argument("--no-extras", action="store_true", help="skip accuracy / FP64 / CPU legs")
    ap.add_argument("--screen-report", action="store_true",
                    help="learned pair screen on the open-shell metallocene-scale cage instead of the "
                         "throughput line: train on walkers 0-255, pairs kept and speed at each cutoff, "
                         "energy changes against unscreened LO and full FP64, and a bound screen")
    ap.add_argument("--hetero-report", action="store_true",
                    help="the six-molecule heterogeneous batch (acene ribbons M 100..480) instead of the "
                         "throughput line: aggregate walker energies/s of one multi-system graph launch "
                         "against one walkers_energy call per molecule, per-molecule error, SM budgets")
    ap.add_argument("--tsvd-report", action="store_true",
                    help="the T_SVD sweep on the naphthalene-scale honeycomb instead of the throughput line: "
                         "compression, <M_SVD>, LO-vs-full and mixed-vs-FP64 errors, truncation bound")
    ap.add_argument("--batch-report", action="store_true",
                    help="walker-batching curve at pentacene scale instead of the throughput line: "
                         "walker energies/s against the walkers per call (64 .. 4096)")
    ap.add_argument("--propagator-report", action="store_true",
                    help="propagator operator V_w = sum_g x_wg L_g at pentacene scale instead of the "
                         "throughput line: time per 1024 walkers (split precision and FP64) and its roofline")
    ap.add_argument("--cas-report", action="store_true",
                    help="multi-determinant (CAS) trial energy through SMW updates: timing and oracle check")
    ap.add_argument("--tsvd-workload", default="naphthalene", choices=["naphthalene", "fragments"],
                    help="T_SVD sweep system: the naphthalene-scale honeycomb or four separate fragments")
    ap.add_argument("--screen-workload", default="metallocene", choices=["metallocene", "fragments"],
                    help="screen report system: the metallocene-scale cage (2048 walkers) or four "
                         "separate fragments (1024 walkers)")
    ap.add_argument("--screen-cutoffs", default="1e-6,1e-3,1e-2,1e-1",
                    help="per-pair cutoffs (Ha) of the screen report")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def walker_first(rank: int, W: int) -> int:
    """Each rank evaluates its own W walkers: walker seeds rank*W .. rank*W + W - 1
    (weak scaling: no data-path collective)."""
    return rank * W


def max_over_ranks(x: float, dist) -> float:
    """The slowest rank's time (the job is done when every rank is)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_link_gbs(src, reps: int = 4, pieces: int = 16) -> float:
    """H2D rate of the pinned walker array alone (GB/s): each copy in 16
    pieces taken in turn by two streams, as the library uploads a submitted
    call; the bound on an end-to-end rate that uploads every step's walkers."""
    import torch
    flat = src.view(-1)
    dst = torch.empty(flat.shape, dtype=flat.dtype, device="cuda")
    n = flat.numel()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for i in range(pieces):
            sl = slice(i * n // pieces, (i + 1) * n // pieces)
            with torch.cuda.stream(streams[i % 2]):
                dst[sl].copy_(flat[sl], non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    del dst
    return reps * flat.numel() * flat.element_size() / dt / 1e9


def whole_job_rate(world: int, W: int, steps: int, seconds: float) -> float:
    """Walker energies per second of all ranks together."""
    return world * W * steps / seconds


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names[1:], r[3][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


PROFILE_TRAFFIC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                               "lo_dense_tc_naphthalene_M250_W1024.md")


def chunk_geom(k: int, cap: int = 256):
    """Balanced chunks of at most cap rows, a multiple of 16 (the library's rule)."""
    if k <= 0:
        return 0, 0
    nch = (k + cap - 1) // cap
    return nch, ((k + nch - 1) // nch + 15) // 16 * 16


def lo_work(M: int, N: int, msvd, W: int, ntot=None, cap: int = 256):
    """Work of the LO exchange split as the library splits it: a pair whose dense
    block (M + 1 rows) takes fewer MMA columns than its two factor sides runs in
    the dense kernel.  Flops are real flops per launch over W walkers."""
    nkb = (M + 63) // 64
    n_wt = (W + 127) // 128
    dn, dnc = chunk_geom(M + 1, cap)
    dense_cols = dn * dnc
    out = {p: {"method_flops": 0.0, "performed_flops": 0.0, "issued_flops": 0.0, "pairs": 0,
               "alg_bytes": 0.0} for p in ("dense", "factored")}
    for k in msvd:
        k = int(k)
        fn, fnc = chunk_geom(k, cap)
        if fn > 0 and dense_cols < 2 * fn * fnc:
            d = out["dense"]
            d["performed_flops"] += 4.0 * M * (M + 1) * W
            d["issued_flops"] += dense_cols * 3 * 2 * 64 * nkb * 256 * n_wt
            d["alg_bytes"] += dense_cols * 64 * nkb * 2 * 2 + dn * W * 16  # B tiles hi/lo once, partials
        else:
            d = out["factored"]
            d["performed_flops"] += 8.0 * M * k * W
            d["issued_flops"] += 2 * fn * fnc * 3 * 2 * 64 * nkb * 256 * n_wt
        d["method_flops"] += 8.0 * M * k * W
        d["pairs"] += 1
    if out["dense"]["pairs"]:
        nt = N if ntot is None else ntot
        nrb = 2 * n_wt
        sd = dense_cols + 32
        # Delta tiles (A operand, hi/lo) and the FP32 Delta copy, each read once
        out["dense"]["alg_bytes"] += nt * nrb * nkb * 16384 * 2 + nt * nrb * 128 * sd * 4
    return out


def lo_traffic(wl, alg_bytes):
    """DRAM bytes per launch of the dense LO kernel, scaled from the committed
    naphthalene-scale ncu capture by the ratio of algorithmic bytes (None if the
    summary is missing)."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None, None
    vals = {}
    for line in open(PROFILE_TRAFFIC):
        if "=" in line and line.split("=")[0].strip() in ("traffic_bytes_per_launch",
                                                         "algorithmic_bytes_per_launch"):
            k, v = line.split("=", 1)
            vals[k.strip()] = float(v)
    if len(vals) < 2:
        return None, None
    if wl is synth.NAPHTHALENE_250:
        return vals["traffic_bytes_per_launch"] / 1e9, "GB per launch, ncu capture of this case (profiles/)"
    scaled = vals["traffic_bytes_per_launch"] / vals["algorithmic_bytes_per_launch"] * alg_bytes
    return scaled / 1e9, ("GB per launch, scaled from the naphthalene-scale ncu capture (profiles/) "
                          "by algorithmic bytes")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return {"bf16_tflops": p["bf16_tflops"], "bf16_tflops_sustained": p["bf16_tflops_sustained"],
                "hbm_gbs": p["hbm_gbs"], "source": "measured"}
    return {"bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "hbm_gbs": 6400.0,
            "source": "fallback"}


def blas_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return os.cpu_count()


def time_oracle(mol, walkers):
    """The FP64 oracle (exact Cholesky form) as it stands, per walker."""
    from oracle import energy as E
    t0 = time.perf_counter()
    energies = [E.walker_energy(mol, w)["E"] for w in walkers]
    dt = time.perf_counter() - t0
    return np.array(energies), dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    mol = wl.molecule()
    n = max(1, args.cpu_sample)
    walkers = wl.walkers(mol, W=n)
    cores = blas_threads()
    for _ in range(min(args.warmup, 1)):
        time_oracle(mol, walkers[:1])
    total = 0.0
    for s in range(args.steps):
        _, dt = time_oracle(mol, walkers[:n])
        total += dt
    value = args.steps * n / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "walkers_per_step": n, "mode": "exact Cholesky form",
                   "sample": f"{n} walkers per step of the {wl.W}-walker workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} walkers per step, oracle.energy.walker_energy"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_2202_00832_b300.lo_afqmc import Context, position_operators

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)

    wl = WORKLOADS[args.workload]
    W = args.walkers or wl.W
    t_gen = time.perf_counter()
    mol = wl.molecule()
    walk = wl.walkers(mol, W=W, first=walker_first(rank, W), processes=min(16, os.cpu_count() or 1))
    t_gen = time.perf_counter() - t_gen

    stream = torch.cuda.current_stream()
    ctx = Context(local, stream=stream.cuda_stream)
    t_setup = time.perf_counter()
    ctx.load_molecule(mol)
    pct, msvd = ctx.lo_localize_compress(args.threshold, position_operators(mol), localize=True)
    t_setup = time.perf_counter() - t_setup

    phi_d = torch.from_numpy(walk).to(f"cuda:{local}")
    e_d = torch.zeros(W, dtype=torch.complex128, device=phi_d.device)
    ld_d = torch.zeros_like(e_d)
    st_d = torch.zeros(W, dtype=torch.int32, device=phi_d.device)

    def step():
        ctx.walkers_energy(phi_d, mode="lo", precision=args.precision, e_out=e_d,
                           logdet_out=ld_d, walker_status=st_d)

    t_first = time.perf_counter()
    step()  # builds the split operands once
    t_first = time.perf_counter() - t_first
    for _ in range(max(args.warmup, 3) - 1):
        step()

    def barrier():
        if dist is not None:
            dist.barrier()

    ctx.profile(True)
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # the timed region is also the profiler's range (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        barrier()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(world, W, args.steps, ms / 1e3)

    # ---- end to end through the public API with pinned host buffers ----
    # (more steps than the device-timed loop: a stream of submitted calls
    # fills its pipeline once, on the first call's upload; 30 steps take about
    # a third of a second at pentacene scale)
    e2e_steps = max(args.steps, 30)
    phi_h = torch.from_numpy(walk).pin_memory()
    e_h = torch.zeros(W, dtype=torch.complex128).pin_memory()
    ld_h = torch.zeros_like(e_h).pin_memory()
    st_h = torch.zeros(W, dtype=torch.int32).pin_memory()
    ctx.walkers_energy(phi_h, mode="lo", precision=args.precision, e_out=e_h, logdet_out=ld_h,
                       walker_status=st_h)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.walkers_energy(phi_h, mode="lo", precision=args.precision, e_out=e_h,
                           logdet_out=ld_h, walker_status=st_h)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_blocking = whole_job_rate(world, W, e2e_steps, t_e2e)
    # the same steps as a stream of submitted calls: each step still uploads
    # its walkers and reads back its results, but the upload of step k + 1
    # runs on the copy engines while step k computes
    outs = [(e_h, ld_h, st_h), (torch.zeros_like(e_h).pin_memory(), torch.zeros_like(ld_h).pin_memory(),
                                torch.zeros_like(st_h).pin_memory())]
    ctx.walkers_energy_submit(phi_h, *outs[0], mode="lo", precision=args.precision)
    ctx.walkers_energy_wait()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.walkers_energy_submit(phi_h, *outs[k % 2], mode="lo", precision=args.precision)
    ctx.walkers_energy_wait()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = whole_job_rate(world, W, e2e_steps, t_e2e)
    h2d = W * mol.M * (mol.n_alpha if mol.closed_shell else mol.n_alpha + mol.n_beta) * 16
    d2h = W * (16 + 16 + 4)
    link_gbs = host_link_gbs(phi_h)

    if rank != 0:
        if dist is not None:
            dist.barrier()
        return

    # ---- roofline of the dominant kernel (live stage timers) ----
    peaks = load_peaks()
    M, N, X = mol.M, mol.n_alpha, mol.X
    kernels = {k: v for k, v in prof.items() if k not in ("h2d_walkers", "finalize_d2h")}
    dominant = max(kernels, key=lambda k: kernels[k][0])
    per_launch_ms = {k: v[0] / max(v[1], 1) for k, v in kernels.items()}
    lo = lo_work(M, N, msvd, W, ntot=N if mol.closed_shell else mol.n_alpha + mol.n_beta,
                 cap=ctx.tiles()[0])
    coul_flops = 4.0 * (X + 1) * N * M * W            # dJ_g = sum_ir Lbar_gir Delta_ri (complex)
    theta_flops = (4.0 * N * N * M + 8.0 / 3.0 * N ** 3 + 8.0 * M * N * N) * W
    fp64_peak_tflops = 1.25  # nominal B300 FP64 (2 DFMA / clk / SM class figure)

    def tc_roof(name, flops):
        # the kernel runs for a few ms of each step at the maximum SM clock, so the
        # measured burst rate is its peak (the sustained figure was taken at a
        # power-capped clock)
        t = per_launch_ms[name] / 1e3
        ach = flops / t / 1e12
        pk = peaks["bf16_tflops"]
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": None,
                "peak_source": f"{peaks['source']} bf16 burst (fp16 same rate); of measured",
                "frac_of_sustained": ach / peaks["bf16_tflops_sustained"]}

    rooflines = {}
    for name, part in (("lo_dense_tc", "dense"), ("lo_exchange_tc", "factored")):
        if name not in per_launch_ms:
            continue
        w = lo[part]
        t = per_launch_ms[name] / 1e3
        # achieved: the method's algorithmic work of these pairs, 8 M K per pair and
        # walker (a = Ubar^T Theta_j, b = Vbar Theta_i); performed: the flops of the
        # contraction the kernel runs (dense blocks: 4 M (M + 1)); issued: MMA flops
        # with three hi/lo products and the padding of chunks and basis blocks
        r = tc_roof(name, w["method_flops"])
        r["algorithmic_flops"] = "8 M K per pair and walker (the method's count)"
        r["performed_tflops"] = w["performed_flops"] / t / 1e12
        r["performed_frac_of_burst"] = r["performed_tflops"] / peaks["bf16_tflops"]
        r["issued_tflops"] = w["issued_flops"] / t / 1e12
        r["issued_frac_of_burst"] = r["issued_tflops"] / peaks["bf16_tflops"]
        r["pairs"] = w["pairs"]
        if part == "dense":
            r["traffic"], r["traffic_source"] = lo_traffic(wl, w["alg_bytes"])
            r["algorithmic_bytes"] = w["alg_bytes"]
        rooflines[name] = r
    if "coulomb_tc" in per_launch_ms:
        rooflines["coulomb_tc"] = tc_roof("coulomb_tc", coul_flops)
    if "inverse_df" in per_launch_ms:
        # double-float Gauss-Jordan: N^3 complex FMAs per walker and spin, each four
        # error-free double-float multiply-adds of 15 FP32 operations (60 in all);
        # peak: 148 SMs x 128 FP32 lanes x 2.032 GHz
        t = per_launch_ms["inverse_df"] / 1e3
        n3 = N ** 3 if mol.closed_shell else mol.n_alpha ** 3 + mol.n_beta ** 3
        ach = 60.0 * n3 * W / t / 1e12
        pk = 148 * 128 * 2.032e9 / 1e12
        rooflines["inverse_df"] = {"kernel": "gauss_jordan (double-float)", "bound": "alu",
                                   "achieved": ach, "peak": pk, "unit": "T FP32 lane-ops/s",
                                   "frac": ach / pk, "traffic": None,
                                   "peak_source": "148 SMs x 128 FP32 lanes x 2.032 GHz"}
    if "inverse_f64" in per_launch_ms:
        # FP64 Gauss-Jordan: N^3 complex multiply-adds (8 flops) per walker and spin
        t = per_launch_ms["inverse_f64"] / 1e3
        n3 = N ** 3 if mol.closed_shell else mol.n_alpha ** 3 + mol.n_beta ** 3
        ach = 8.0 * n3 * W / t / 1e12
        rooflines["inverse_f64"] = {"kernel": "gauss_jordan (FP64)", "bound": "alu", "achieved": ach,
                                    "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                                    "frac": ach / fp64_peak_tflops, "traffic": None,
                                    "peak_source": "nominal FP64 ALU peak of B300"}
    if "theta_fp64" in per_launch_ms:
        t = per_launch_ms["theta_fp64"] / 1e3
        ach = theta_flops / t / 1e12
        rooflines["theta_fp64"] = {"kernel": "theta_fp64", "bound": "alu", "achieved": ach,
                                   "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                                   "frac": ach / fp64_peak_tflops, "traffic": None,
                                   "peak_source": "nominal FP64 ALU peak of B300"}
    roof = rooflines.get(dominant) or next(iter(rooflines.values()))

    extras = {}
    cpu = None
    if not args.no_extras:
        # accuracy of every walker of the batch against the FP64 LO path on the GPU
        # (same factors), and of a few walkers against the FP64 oracle's full energy
        e_mixed = e_d.cpu().numpy()
        e64_d = torch.zeros_like(e_d)
        ctx.walkers_energy(phi_d, mode="lo", precision="fp64", e_out=e64_d)
        torch.cuda.synchronize()
        e_lo64 = e64_d.cpu().numpy()
        dev = np.abs(e_mixed - e_lo64)
        n_acc = max(1, args.cpu_sample)
        ref, dt = time_oracle(mol, walk[:n_acc])
        extras["accuracy_mha"] = {
            "walkers": W,
            "mixed_vs_fp64_lo_max": float(dev.max() * 1e3),
            "mixed_vs_fp64_lo_mean": float(dev.mean() * 1e3),
            "oracle_walkers": n_acc,
            "mixed_vs_oracle_full_max": float(np.abs(e_mixed[:n_acc] - ref).max() * 1e3),
            "lo_truncation_vs_oracle_full_max": float(np.abs(e_lo64[:n_acc] - ref).max() * 1e3),
        }
        cpu = {"value": n_acc / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"{n_acc} walkers of the workload through the FP64 oracle "
                         f"(exact Cholesky form, {dt:.1f} s)"}
        # precision variants of the same step: the overlap inverse and log-det on
        # the FP64 pipe (FP16X3_F64INV), and BF16 hi + lo operands (BF16X3)
        if args.precision == "fp16x3":
            variants = {}
            for prec in ("fp16x3_f64inv", "bf16x3", "tf32"):
                ev = torch.zeros_like(e_d)
                ldv = torch.zeros_like(e_d)
                for _ in range(2):
                    ctx.walkers_energy(phi_d, mode="lo", precision=prec, e_out=ev, logdet_out=ldv)
                ctx.profile(True)
                torch.cuda.synchronize()
                v0 = torch.cuda.Event(enable_timing=True)
                v1 = torch.cuda.Event(enable_timing=True)
                v0.record(stream)
                for _ in range(args.steps):
                    ctx.walkers_energy(phi_d, mode="lo", precision=prec, e_out=ev, logdet_out=ldv)
                v1.record(stream)
                torch.cuda.synchronize()
                vprof = ctx.profile_read()
                ctx.profile(False)
                vms = v0.elapsed_time(v1) / args.steps
                dv = np.abs(ev.cpu().numpy() - e_lo64)
                dld = np.abs(ldv.cpu().numpy().real - ld_d.cpu().numpy().real)
                variants[prec] = {
                    "value": W / (vms / 1e3), "unit": UNIT, "ms_per_step": vms,
                    "vs_fp64_lo_max_mha": float(dv.max() * 1e3),
                    "vs_fp64_lo_mean_mha": float(dv.mean() * 1e3),
                    "logdet_vs_fp16x3_max": float(dld.max()),
                    "stage_ms_per_step": {k: v[0] / args.steps for k, v in vprof.items()
                                          if k.startswith("inverse") or k in ("lo_dense_tc", "coulomb_tc")},
                }
            extras["precision_variants"] = variants
        # the plain full-exchange FP64 path on the same GPU (subset of walkers)
        nf = min(args.full_sample, W)
        phi_f = phi_d[:nf].contiguous()
        ef = torch.zeros(nf, dtype=torch.complex128, device=phi_d.device)
        ctx.walkers_energy(phi_f, mode="full", precision="fp64", e_out=ef)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.walkers_energy(phi_f, mode="full", precision="fp64", e_out=ef)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        extras["full_fp64_gpu"] = {"value": nf / tf, "unit": UNIT, "walkers": nf}
        extras["lo_vs_full_fp64_speedup"] = value / world / (nf / tf)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.precision}: 16-bit hi+lo x3 tcgen05 contractions (fp32 acc); overlap and "
                 f"Theta as exact 7-bit slice products on tcgen05; "
                 + ("f64" if args.precision == "fp16x3_f64inv" else "double-float (2 x f32)")
                 + " inverse and log-det; f64 reductions"
                 if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name + (" (pentacene-scale acene ribbon)" if wl is synth.PENTACENE_440
                                          else ""), "M": M, "N_occ": N,
                   "X": X, "walkers_per_gpu": W, "t_svd": args.threshold, "mode": "lo",
                   "compression_pct": pct, "mean_m_svd": float(msvd.mean()),
                   "pairs": int(len(msvd)), "l2": "inputs larger than L2 (walkers "
                   f"{walk.nbytes / 1e6:.0f} MB, LO factors, Delta planes)",
                   "setup_s": t_setup, "first_call_s": t_first, "input_gen_s": t_gen},
        "roofline": roof,
        "rooflines": rooflines,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": int(sum(v[2] for k, v in prof.items())),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps,
                "api": "walkers_energy_submit per step (pinned host walkers in, pinned host energies, "
                       "log-dets and statuses out), walkers_energy_wait after the last",
                "blocking_value": e2e_blocking,
                "host_link_h2d_gbs": link_gbs,
                "host_link_bound": link_gbs * 1e9 / (h2d / W) * world,
                "blocking_api": "one walkers_energy call per step (returns with the outputs written)"},
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()


def screen_report(args):
    """Learned pair screen (a8) on the metallocene-scale cage (M 500, N 48/47, X 2000,
    2048 device-resident walkers timed) or on four separate fragments (M 480, N 80,
    X 960, 1024 walkers): the network is trained on walkers 0-255; at each cutoff
    the screen's kept pairs, the step time of the screened LO energy against the
    unscreened one, and the energy change per walker on held-out walkers
    against unscreened LO (FP16x3) and against the full FP64 energy.  The bound
    screen keeps a pair when max_w sigma_1 |Theta_i(w)| |Theta_j(w)| over the
    training walkers reaches the cutoff (|e_ij| <= sigma_1 |Theta_i| |Theta_j|)."""
    import torch
    from paper_2202_00832_b300.lo_afqmc import Context, init_screen_params, position_operators

    torch.cuda.set_device(0)
    wl = synth.FRAGMENTS_480 if args.screen_workload == "fragments" else synth.METALLOCENE_500
    mol = wl.molecule()
    W = args.walkers or wl.W
    n_train, n_test = 256, 16
    walk = wl.walkers(mol, W=max(W, n_train + n_test), processes=min(16, os.cpu_count() or 1))
    stream = torch.cuda.current_stream()
    ctx = Context(0, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    ctx.load_molecule(mol)
    pct, msvd = ctx.lo_localize_compress(args.threshold, position_operators(mol), localize=True)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = ctx.pair_screen_train(walk[:n_train], init_screen_params(0), epochs=1000, lr=3e-3)
    t_train = time.perf_counter() - t0
    q = ctx.pair_screen_query()
    n_pairs = ctx.num_pairs
    test = walk[n_train:n_train + n_test]

    # pair order and energy weight: spins concatenated, i <= j, weight 1/2 mult (1 or 2)
    pairs, wgt = [], []
    spins = [(0, mol.n_alpha)] if mol.closed_shell else [(0, mol.n_alpha), (mol.n_alpha, mol.n_beta)]
    mult = 2.0 if mol.closed_shell else 1.0
    for col0, n in spins:
        for i in range(n):
            for j in range(i, n):
                pairs.append((col0 + i, col0 + j))
                wgt.append(0.5 * mult * (1.0 if i == j else 2.0))
    pairs, wgt = np.array(pairs), np.array(wgt)
    assert len(pairs) == n_pairs

    # bound screen from the training walkers' Theta column norms (FP64 path)
    th, _, _ = ctx.walkers_theta(walk[:n_train])
    norms = np.linalg.norm(th, axis=2)                       # (W, ntot)
    sigma1 = np.exp(q["features"][:, 4])
    bound = sigma1 * np.max(norms[:, pairs[:, 0]] * norms[:, pairs[:, 1]], axis=0)

    phi_d = torch.from_numpy(walk[:W]).to("cuda")
    e_d = torch.zeros(W, dtype=torch.complex128, device="cuda")

    def step_ms():
        for _ in range(2):
            ctx.walkers_energy(phi_d, mode="lo", precision=args.precision, e_out=e_d)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(3):
            ctx.walkers_energy(phi_d, mode="lo", precision=args.precision, e_out=e_d)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 3

    ctx.pair_screen_set(-1.0)
    t_unscreened = step_ms()
    e_lo, _, _ = ctx.walkers_energy(test, mode="lo", precision=args.precision)
    e_full, _, _ = ctx.walkers_energy(test[:4], mode="full", precision="fp64")
    ep = ctx.walkers_pair_exchange(test, precision="fp64")   # (pairs, walkers)
    rows = []
    # the fixed cutoffs, then cutoffs at the 10 / 25 / 50 % quantiles of the
    # predicted log10 |e_ij| (these synthetic pairs are all large, so the fixed
    # ones keep everything; the quantile ones show the speed / error trade)
    cutoffs = [float(x) for x in args.screen_cutoffs.split(",")]
    cutoffs += [float(10 ** np.quantile(q["pred"], f)) for f in (0.10, 0.25, 0.50)]
    for cut in cutoffs:
        kept = ctx.pair_screen_set(cut)
        t_s = step_ms()
        e_s, _, _ = ctx.walkers_energy(test, mode="lo", precision=args.precision)
        keep_b = bound >= cut
        # E_K loses the dropped pairs' values: E rises by their weighted sum
        e_b = e_lo + (wgt[~keep_b, None] * ep[~keep_b]).sum(axis=0)
        rows.append({
            "cutoff_ha": cut, "pairs_kept": kept, "pairs_total": n_pairs,
            "ms_per_step": t_s, "speedup_vs_unscreened": t_unscreened / t_s,
            "max_abs_dE_vs_unscreened_mha": float(np.abs(e_s - e_lo).max() * 1e3),
            "max_abs_dE_vs_full_fp64_mha": float(np.abs(e_s[:4] - e_full).max() * 1e3),
            "bound_screen": {"pairs_kept": int(keep_b.sum()),
                             "max_abs_dE_vs_unscreened_mha": float(np.abs(e_b - e_lo).max() * 1e3)},
        })
    ctx.pair_screen_set(-1.0)
    out = {"screen_report": {
        "workload": wl.name, "walkers_timed": W, "train_walkers": n_train, "test_walkers": n_test,
        "t_svd": args.threshold, "precision": args.precision, "compression_pct": pct,
        "setup_s": t_setup, "train_s": t_train, "train_loss_first_last": [float(hist[0]), float(hist[-1])],
        "pred_target_corr": float(np.corrcoef(q["pred"], q["target"])[0, 1]),
        "target_log10_max_abs_e_min_median_max": [float(np.min(q["target"])), float(np.median(q["target"])),
                                                  float(np.max(q["target"]))],
        "unscreened_ms_per_step": t_unscreened,
        "unscreened_vs_full_fp64_max_mha": float(np.abs(e_lo[:4] - e_full).max() * 1e3),
        "cutoffs": rows}}
    print(json.dumps(out), flush=True)


def hetero_report(args):
    """Six acene ribbons of different sizes (M 100..480, N 14..80, W 512..128;
    LO, T_SVD = 1e-4, FP16x3): the aggregate rate of one walkers_energy_multi
    graph launch (autotuned SM budgets) against one walkers_energy call per
    molecule in turn, both on device-resident walkers, and each molecule's
    energy error against its FP64 LO path on 4 walkers."""
    import torch
    from paper_2202_00832_b300.lo_afqmc import Context, position_operators, walkers_energy_multi

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctxs, phis, walks, info = [], [], [], []
    t0 = time.perf_counter()
    for wl in synth.HETERO_BATCH:
        mol = wl.molecule()
        walk = wl.walkers(mol, processes=min(16, os.cpu_count() or 1))
        c = Context(0, stream=stream.cuda_stream)
        c.load_molecule(mol)
        pct, msvd = c.lo_localize_compress(args.threshold, position_operators(mol), localize=True)
        ctxs.append(c)
        walks.append(walk)
        phis.append(torch.from_numpy(walk).cuda())
        info.append({"workload": wl.name, "M": mol.M, "N": mol.n_alpha, "X": mol.X, "W": len(walk),
                     "pairs": int(len(msvd)), "compression_pct": pct})
    t_setup = time.perf_counter() - t0
    total_w = sum(p.shape[0] for p in phis)
    e = [torch.zeros(p.shape[0], dtype=torch.complex128, device="cuda") for p in phis]

    def timed(fn, reps=5):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    def sequential():
        for c, p, x in zip(ctxs, phis, e):
            c.walkers_energy(p, mode="lo", precision=args.precision, e_out=x)

    # the graph with the library's default tile shapes and SM budgets, then with
    # the autotuner's choices (tile shapes per system, then SM budgets)
    walkers_energy_multi(ctxs, phis, e, precision=args.precision, autotune=False)
    t_default = timed(lambda: walkers_energy_multi(ctxs, phis, e, precision=args.precision, autotune=False))
    t1 = time.perf_counter()
    caps = walkers_energy_multi(ctxs, phis, e, precision=args.precision, autotune=True)
    t_tune = time.perf_counter() - t1
    t_multi = timed(lambda: walkers_energy_multi(ctxs, phis, e, precision=args.precision, autotune=True))
    t_seq = timed(sequential)
    walkers_energy_multi(ctxs, phis, e, precision=args.precision, autotune=True)
    for k, c in enumerate(ctxs):
        got = e[k][:4].cpu().numpy()
        e64, _, _ = c.walkers_energy(walks[k][:4], mode="lo", precision="fp64")
        info[k]["max_abs_dE_vs_fp64_lo_mha"] = float(np.abs(got - e64).max() * 1e3)
        info[k]["sm_budget"] = caps[k]
        info[k]["lo_chunk_cap"], info[k]["coulomb_split"] = c.tiles()
    out = {"hetero_report": {
        "molecules": info, "walkers_total": total_w, "setup_s": t_setup, "autotune_s": t_tune,
        "multi_graph_default_tiles": {"ms_per_batch": t_default,
                                      "walker_energies_per_s": total_w / (t_default / 1e3)},
        "multi_graph": {"ms_per_batch": t_multi, "walker_energies_per_s": total_w / (t_multi / 1e3)},
        "sequential_calls": {"ms_per_batch": t_seq, "walker_energies_per_s": total_w / (t_seq / 1e3)},
        "speedup": t_seq / t_multi,
        "sm_budget_note": "0 = the persistent kernels may fill all 148 SMs",
        "tile_note": "lo_chunk_cap: largest LO chunk (MMA N); coulomb_split 0 = the library's rule"}}
    print(json.dumps(out), flush=True)


def tsvd_report(args):
    """T_SVD sweep on the naphthalene-scale honeycomb (M 250, N 34, X 1000; 64
    walkers) or four separate fragments: per threshold the compression, <M_SVD>
    and the M_SVD histogram (Boys-localized and canonical orbitals), the LO-vs-full error of the FP64 path, the mixed-vs-FP64 LO error,
    and the closed-form truncation bound |E_K^LO - E_K| < (mult/2) sum_sigma
    T (sum_i |Theta_i|)^2 (every dropped singular value is below T), checked per
    walker."""
    from paper_2202_00832_b300.lo_afqmc import Context, position_operators

    wl = synth.FRAGMENTS_480 if args.tsvd_workload == "fragments" else synth.NAPHTHALENE_250
    mol = wl.molecule()
    walk = wl.walkers(mol, W=64, processes=min(16, os.cpu_count() or 1))
    ctx = Context(0)
    ctx.load_molecule(mol)
    e_full, _, _ = ctx.walkers_energy(walk, mode="full", precision="fp64")
    # M_SVD histograms (the paper's compression figure, localized against canonical
    # orbitals): ten bins of M / 10 kept ranks
    edges = np.linspace(0, mol.M, 11)

    def hist(m):
        return np.histogram(np.asarray(m), bins=edges)[0].tolist()
    canon = Context(0)
    canon.load_molecule(mol)
    mult = 2.0 if mol.closed_shell else 1.0
    rows = []
    for T in [1e-2, 1e-3, 1e-4, 1e-5]:
        pct, msvd = ctx.lo_localize_compress(T, position_operators(mol), localize=True)
        pct_c, msvd_c = canon.lo_localize_compress(T, position_operators(mol), localize=False)
        th, _, _ = ctx.walkers_theta(walk)                   # localized trial: (W, ntot, M)
        nrm = np.linalg.norm(th, axis=2)
        if mol.closed_shell:
            bound = mult / 2 * T * nrm.sum(axis=1) ** 2
        else:
            na = mol.n_alpha
            bound = mult / 2 * T * (nrm[:, :na].sum(axis=1) ** 2 + nrm[:, na:].sum(axis=1) ** 2)
        e64, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
        e16, _, _ = ctx.walkers_energy(walk, mode="lo", precision=args.precision)
        etf, _, _ = ctx.walkers_energy(walk, mode="lo", precision="tf32")
        err = np.abs(e64 - e_full)
        rows.append({
            "t_svd": T, "compression_pct": pct, "mean_m_svd": float(msvd.mean()),
            "canonical_compression_pct": pct_c, "canonical_mean_m_svd": float(msvd_c.mean()),
            "m_svd_histogram": {"bin_edges": edges.tolist(), "localized": hist(msvd),
                                "canonical": hist(msvd_c)},
            "lo_vs_full_fp64_mean_mha": float(err.mean() * 1e3), "lo_vs_full_fp64_max_mha": float(err.max() * 1e3),
            "mixed_vs_fp64_lo_max_mha": float(np.abs(e16 - e64).max() * 1e3),
            "tf32_vs_fp64_lo_max_mha": float(np.abs(etf - e64).max() * 1e3),
            "tf32_vs_fp64_lo_mean_mha": float(np.abs(etf - e64).mean() * 1e3),
            "tf32_vs_full_fp64_max_mha": float(np.abs(etf - e_full).max() * 1e3),
            "bound_max_mha": float(bound.max() * 1e3), "bound_holds_all_walkers": bool(np.all(err <= bound)),
        })
    print(json.dumps({"tsvd_report": {"workload": wl.name, "walkers": len(walk), "precision": args.precision,
                                      "rows": rows}}), flush=True)


def batch_report(args):
    """Throughput against the batch size at pentacene scale (LO, T_SVD = 1e-4,
    FP16x3, device-resident walkers): one walkers_energy call per batch of W
    walkers, W = 64 .. 4096 (walkers beyond the 1024 generated ones repeat)."""
    import torch
    from paper_2202_00832_b300.lo_afqmc import Context, position_operators

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    wl = synth.PENTACENE_440
    mol = wl.molecule()
    walk = wl.walkers(mol, processes=min(16, os.cpu_count() or 1))
    ctx = Context(0, stream=stream.cuda_stream)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(args.threshold, position_operators(mol), localize=True)
    rows = []
    for W in [64, 128, 256, 512, 1024, 2048, 4096]:
        reps = -(-W // len(walk))
        phi = torch.from_numpy(np.concatenate([walk] * reps)[:W]).cuda()
        e = torch.zeros(W, dtype=torch.complex128, device="cuda")
        for _ in range(3):
            ctx.walkers_energy(phi, mode="lo", precision=args.precision, e_out=e)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(3, 8192 // W)
        ev0.record(stream)
        for _ in range(n):
            ctx.walkers_energy(phi, mode="lo", precision=args.precision, e_out=e)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / n
        rows.append({"walkers_per_call": W, "ms_per_call": ms, "walker_energies_per_s": W / (ms / 1e3)})
        del phi, e
    print(json.dumps({"batch_report": {"workload": wl.name, "precision": args.precision, "rows": rows}}),
          flush=True)


def propagator_report(args):
    """V_w = sum_g x_wg L_g for W = 1024 pentacene-scale walkers (M 440, X 1800),
    fields and outputs resident in HBM (3.2 GB of V): time per batch in the split
    precision, algorithmic work 4 W X M^2 flops (complex field times real L),
    and the FP64 (cuBLAS) path on 64 walkers for comparison."""
    import torch
    from paper_2202_00832_b300.lo_afqmc import Context

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    mol = synth.PENTACENE_440.molecule()
    ctx = Context(0, stream=stream.cuda_stream)
    ctx.load_molecule(mol)
    rng = np.random.default_rng(4)
    out = {"workload": synth.PENTACENE_440.name, "M": mol.M, "X": mol.X}

    def timed(W, precision, reps):
        x = torch.from_numpy(rng.standard_normal((W, mol.X)) * 0.1
                             + 1j * rng.standard_normal((W, mol.X)) * 0.05).cuda()
        v = torch.zeros((W, mol.M, mol.M), dtype=torch.complex128, device="cuda")
        ctx.walkers_propagator(x, precision=precision, out=v)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            ctx.walkers_propagator(x, precision=precision, out=v)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        del x, v
        return ms

    W = 1024
    ms = timed(W, args.precision, 5)
    flops = 4.0 * W * mol.X * mol.M ** 2
    peaks = load_peaks()
    out[args.precision] = {"walkers": W, "ms_per_batch": ms, "walkers_per_s": W / (ms / 1e3),
                           "algorithmic_tflops": flops / (ms / 1e3) / 1e12,
                           "frac_of_bf16_sustained": flops / (ms / 1e3) / 1e12 / peaks["bf16_tflops_sustained"]}
    ms64 = timed(64, "fp64", 2)
    out["fp64"] = {"walkers": 64, "ms_per_batch": ms64, "walkers_per_s": 64 / (ms64 / 1e3),
                   "tflops": 4.0 * 64 * mol.X * mol.M ** 2 / (ms64 / 1e3) / 1e12}
    print(json.dumps({"propagator_report": out}), flush=True)


def cas_report(args):
    """Mixed-estimate energies with a multi-determinant (CAS) trial through SMW
    updates of the reference (FP64): an acene ribbon M 100, N 14, X 400 with 10
    inactive + 12 active orbitals and 64 determinants (up to 4 changed slots),
    T_SVD = 1e-4, 256 device-resident walkers; timing with CUDA events, the
    largest |dE| against the oracle's SMW route on 2 walkers, the oracle's time
    per walker, and the single-determinant FP64 LO energy on the same walkers."""
    import time
    import torch
    from oracle import multidet as MD
    from paper_2202_00832_b300.lo_afqmc import Context, position_operators

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    mol = synth.make_molecule("acene_M100_N14_X400", 100, 400, 14, 14, "acene", 1006)
    cas = synth.make_cas_trial(mol, 10, 12, 64, 4, 77)
    t_svd = 1e-4
    prep = MD.prepare_cas(mol, cas, t_svd)
    W = 256
    walk = synth.make_walkers(mol, W, 0.1, 3006)
    ctx = Context(0, stream=stream.cuda_stream)
    ctx.ao_load_cholesky(mol.h, mol.L, np.ascontiguousarray(prep.C))
    _, msvd = ctx.lo_localize_compress(t_svd, localize=False)
    dphi = torch.from_numpy(walk).cuda()
    e = torch.zeros(W, dtype=torch.complex128, device="cuda")
    lov = torch.zeros(W, dtype=torch.complex128, device="cuda")
    st = torch.zeros(W, dtype=torch.int32, device="cuda")
    dets = np.array(cas.dets, dtype=np.int32)
    for _ in range(3):
        ctx.walkers_energy_cas(dphi, dets, cas.coeffs, e_out=e, logov_out=lov, walker_status=st)
    torch.cuda.synchronize()
    reps = 5
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        ctx.walkers_energy_cas(dphi, dets, cas.coeffs, e_out=e, logov_out=lov, walker_status=st)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    e_host = e.cpu().numpy()
    # oracle with the library's kept ranks (identical truncation)
    from oracle import energy as E
    from oracle import lo as LO
    fac = LO.truncate(LO.pair_svds(prep.Lbar), t_svd, keep=msvd)
    prep_lib = MD.CASPrep(prep.C, prep.Lbar, prep.hbar, fac, {p: n for n, p in enumerate(fac.pairs)})
    t0 = time.perf_counter()
    ref = [MD.energy_multidet_lo(mol, cas, prep_lib, walk[w])[0] for w in range(2)]
    t_or = (time.perf_counter() - t0) / 2
    err = max(abs(e_host[w] - ref[w]) for w in range(2))
    # the single-determinant (reference) energy on a context with the reference trial
    ctx1 = Context(0, stream=stream.cuda_stream)
    ctx1.load_molecule(mol)
    ctx1.lo_localize_compress(t_svd, position_operators(mol))
    e1 = torch.zeros(W, dtype=torch.complex128, device="cuda")
    ctx1.walkers_energy(dphi, mode="lo", precision="fp64", e_out=e1)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        ctx1.walkers_energy(dphi, mode="lo", precision="fp64", e_out=e1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms1 = ev0.elapsed_time(ev1) / reps
    out = {"workload": "acene_M100_N14_X400, CAS 10 inactive + 12 active, 64 determinants, up to 4 changed slots",
           "t_svd": t_svd, "walkers": W, "ms_per_call": ms, "walker_energies_per_s": W / (ms / 1e3),
           "max_abs_dE_vs_oracle_Ha": float(err), "oracle_s_per_walker": t_or,
           "single_det_lo_fp64_ms_per_call": ms1,
           "mean_m_svd": float(np.mean(msvd)), "pairs": int(len(msvd))}
    print(json.dumps({"cas_report": out}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.propagator_report:
        if rank == 0:
            propagator_report(args)
        return
    if args.cas_report:
        if rank == 0:
            cas_report(args)
        return
    if args.batch_report:
        if rank == 0:
            batch_report(args)
        return
    if args.tsvd_report:
        if rank == 0:
            tsvd_report(args)
        return
    if args.hetero_report:
        if rank == 0:
            hetero_report(args)
        return
    if args.screen_report:
        if rank == 0:
            screen_report(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
