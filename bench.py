"""Benchmark of the KBE hot path on GB300.

One step = one KBE step of the last row n = N_t - 1 of the 8-orbital
Hubbard-chain workload (N_t = 1024 nonuniform points, orders 1..5, Gaussian
pulse): predictor, then P = 2 fixed-point sweeps of self-energy row,
history slice (Eq. KBE2), right-hand side and corrector, all on the GPU
(host FP64 weights are computed once per grid).  The history of rows
0..n-1 is the non-interacting propagator of the chain; the stored
right-hand-side rows n-K..n-1 are rebuilt by the library from that history
before timing (the restart reconstruction).

Metric: history-slice TFLOP/s = P * 8 M^3 (n+1)(3n+2) / step time, and ms
per KBE step.  Inputs (1.07 GB of history) are larger than L2.

--impl reference times the CPU oracle (test infrastructure) on the host
cores instead: one oracle KBE step of the same row per step.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "chain_m8_n1024"
# FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA per clock x 2 flops
# x 2.070 GHz (the nominal 1.25 TFLOP/s of the part); a DFMA probe kernel
# reached 1.199 TFLOP/s (95%) and the persistent batched contraction 1.247.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes of one FP64 contraction launch of the bench slice (ncu capture,
# profiles/history_partial_fp64_chain_m8_n1024.md)
FP64_SLICE_TRAFFIC = 1.989e9
# DRAM bytes of one split contraction launch (split_main2) of the bench slice
# (ncu capture, profiles/split_main2_chain_m8_n1024.md)
SPLIT_SLICE_TRAFFIC = 2.263e9
SPLIT_TRAFFIC_SOURCE = ("ncu dram__bytes_read+write of the launch at n=767 (18432 units), scaled by units to "
                        "n=1023 (32768 units)")
SPLIT_KERNEL = "split_main2 (tcgen05 contraction fed by bulk copies of fp16 digit planes)"


def split_stream_bytes(M, n):
    """Bytes the split contraction streams for slice n: per (column tile of
    128/M columns, chunk of 16 complex history entries, 8-orbital part) one
    66560-byte unit of digit planes (PL, Q, column exponents)."""
    ct = 128 // M
    cpt = ((n + 1) * M + 15) // 16
    return ((n + 1 + ct - 1) // ct) * cpt * ((M + 7) // 8) * 66560
METRIC = "history-slice TFLOP/s and ms per KBE step vs plain FP64 GPU path at stated error"


def slice_flops(M, n):
    """Algorithmic flops of one history slice of row n: complex multiply-adds
    (8 flops each) of the 2n+1 required output blocks."""
    return 8.0 * M ** 3 * (n + 1) * (3 * n + 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--P", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-m32", action="store_true", help="skip the 32-orbital precision-form measurement")
    ap.add_argument("--n-t", type=int, default=None,
                    help="truncate the grid to this many points (smaller profiling case)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-system batching form")
    ap.add_argument("--no-window", action="store_true", help="skip the differentiation form")
    ap.add_argument("--no-selfenergy", action="store_true", help="skip the whole-triangle self-energy timing")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the adaptive history-order run")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-interaction self-energy and step")
    ap.add_argument("--no-controller", action="store_true", help="skip the adaptive time-stepping runs")
    ap.add_argument("--no-thermal", action="store_true", help="skip the thermal-branch step")
    ap.add_argument("--no-seeds", action="store_true", help="skip the main step at the other input seeds")
    ap.add_argument("--no-runs", action="store_true", help="skip the whole-run measurements")
    ap.add_argument("--sharded", action="store_true",
                    help="time the row-band sharded step (the N-GPU line) also on one GPU")
    ap.add_argument("--profile-run", default=None, choices=["dimer_m2_n64"],
                    help="only the FP64 whole run of this workload, twice, with one JSON line (the launches a "
                         "profiler captures)")
    ap.add_argument("--profile-slice", default=None, choices=["fp64", "split", "split-fused", "df64"],
                    help="only run three history slices of row n_t - 1 with this contraction (a small case "
                         "for ncu with --n-t; split-fused: the split path without its plane buffer) and exit")
    ap.add_argument("--workload", default=None, choices=["chain_m8_n1024", "goe_m32_n1024"],
                    help="workload of --profile-slice (default: the main one)")
    ap.add_argument("--dense-norb", default="2,8,16,32",
                    help="comma-separated orbital counts of the dense self-energy rows")
    return ap.parse_args()


def dist_setup(args):
    rank, world = 0, 1
    if args.gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if world > 1:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
    return rank, world


class Clocks:
    """nvidia-smi samples during the timed region, written to the CSV file
    named by KBE_CLOCKS_CSV (a temporary file when unset)."""

    def __init__(self, idx):
        self.proc = None
        self.path = os.environ.get("KBE_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     "kbe_clocks_%d.csv" % os.getpid())
        try:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(idx),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def setup_workload(kbe, seed, n_t_override=None, name=None):
    import torch
    import workloads as W
    cfg = W.CONFIGS[name or WORKLOAD]
    M, n_t = cfg["M"], cfg["n_t"]
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], seed)
    if n_t_override:
        n_t = int(n_t_override)
        t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, seed)
    rho0 = W.half_filled_rho(h)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    run = kbe.Run(ctx)
    L, R = W.free_triangles_torch(h, rho0, t, n_t, "cuda")
    run.L.copy_(L)
    run.R.copy_(R)
    del L, R
    n = n_t - 1
    K = int(order[1:].max())
    for j in range(max(0, n - K), n):  # restart: rebuild the stored right-hand sides
        ctx.rhs_row(j, run.L, run.R, run.Sl, run.Sg, run.I, run.F)
    ctx.sync_status()
    torch.cuda.synchronize()
    return cfg, t, order, h, U, v, pulse, ctx, run, n


def time_steps(ctx, run, n, P, steps, warmup, stream, precision="fp64"):
    import torch
    for _ in range(warmup):
        run.step(n, P=P, precision=precision, stream=stream)
    torch.cuda.synchronize()
    launches = 0
    ctx.set_profiling(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run.step(n, P=P, precision=precision, stream=stream)
        launches += ctx.last_launch_count
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    k_count, k_ms = ctx.read_profiling()
    ctx.set_profiling(False)
    ctx.sync_status()
    return ms, launches, k_count, k_ms


def e2e_steps(ctx, run, n, P, steps, warmup, stream):
    """The same step through the public API with host buffers
    (kbe_step_host): every step copies the history rows 0..n-1 and the
    stored right-hand sides from pinned host memory, runs the step (the
    first history slice contracts each chunk of columns as its rows arrive)
    and reads the new row back."""
    import torch
    L_h = run.L.cpu().pin_memory()
    R_h = run.R.cpu().pin_memory()
    F_h = run.F.cpu().pin_memory()
    M = ctx.M
    out_L = torch.empty((n + 1, M, M), dtype=torch.complex128).pin_memory()
    out_R = torch.empty_like(out_L).pin_memory()
    h2d = 2 * W_tri(n) * M * M * 16 + F_h.numel() * 16
    d2h = 2 * (n + 1) * M * M * 16

    def one():
        run.step_host(n, L_h, R_h, F_h, out_L, out_R, P=P, stream=stream)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, h2d, d2h


def oracle_step_inputs(t, order, h, U, v, pulse, L_rows, R_rows, n, threads):
    """Inputs of one oracle KBE step of row n: the history rows 0..n-1 and the
    right-hand-side rows n-K..n-1 rebuilt by the oracle itself from them."""
    import oracle
    M = h.shape[0]
    L = np.zeros((W_tri(n + 1), M, M), np.complex128)
    R = np.zeros_like(L)
    L[: W_tri(n)] = L_rows
    R[: W_tri(n)] = R_rows
    F = {}
    for j in oracle.f_rows_needed(order, n, n + 1):
        F[j] = oracle.rhs_row(j, t, order, h, U, v, pulse, L[: W_tri(j + 1)], R[: W_tri(j + 1)], nthreads=threads)
    return L, R, F


def W_tri(n):
    return n * (n + 1) // 2


def cpu_baseline(run, t, order, h, U, v, pulse, n, M, P, gpu_rows):
    """The oracle's own KBE step of row n (P sweeps) from the same history on
    the host cores: its time, and the deviation of each GPU step in
    ``gpu_rows`` ({name: (row L, row R, history slice)}) from it."""
    import oracle
    threads = oracle.threads_available()
    L_rows = run.L[: W_tri(n)].cpu().numpy()
    R_rows = run.R[: W_tri(n)].cpu().numpy()
    L, R, F = oracle_step_inputs(t, order, h, U, v, pulse, L_rows, R_rows, n, threads)
    t0 = time.perf_counter()
    Lo, Ro, Io = oracle.run(t[: n + 1], order[: n + 1], h, U, v, pulse, P, L, R, F, n, n + 1, nthreads=threads)
    dt = time.perf_counter() - t0
    p = W_tri(n)
    errs = {}
    for name, (gl, gr, gi) in gpu_rows.items():
        errs[name] = {"row_L": float(np.abs(gl - Lo[p:]).max() / np.abs(Lo[p:]).max()),
                      "row_R": float(np.abs(gr - Ro[p:]).max() / np.abs(Ro[p:]).max()),
                      "history_slice": float(np.abs(gi - Io).max() / np.abs(Io).max())}
    tflops = P * slice_flops(M, n) / dt / 1e12
    sample = ("one oracle KBE step of row n=%d (P=%d: self-energy, history slice, corrector), "
              "%.2f s wall on %d threads" % (n, P, dt, threads))
    return tflops, threads, sample, errs, dt


def cpu_thread_scaling(run, t, order, U, n_s=255):
    """The oracle's history slice of row n_s (bounded sample) on one thread
    and on all host threads: seconds and FP64 GFLOP/s each."""
    import oracle
    threads = oracle.threads_available()
    L = run.L[: W_tri(n_s + 1)].cpu().numpy()
    R = run.R[: W_tri(n_s + 1)].cpu().numpy()
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n_s, L, R)
    M = L.shape[-1]
    out = {"sample": "oracle history slice of row n=%d, M=%d" % (n_s, M), "threads": threads}
    for key, nt in (("one_thread", 1), ("all_threads", threads)):
        t0 = time.perf_counter()
        oracle.history_slice(t, order, n_s, L, R, Sl, Sg, nthreads=nt)
        dt = time.perf_counter() - t0
        out[key + "_s"] = round(dt, 3)
        out[key + "_gflops"] = round(slice_flops(M, n_s) / dt / 1e9, 3)
    return out


def batch_bench(kbe, seed, P, stream, rank=0, world=1):
    """The batching form on 64 independent chains (M in {4,8,12,16,24},
    N_t in [256,1536], U in [0.5,3]): one batched KBE step advances every
    system at its last row n_i = N_t,i - 1.  Times the plain FP64 path (one
    kbe_step per system, in sequence), the batched graph in FP64 and with
    the split-precision contraction, and reports the deviation of the new
    rows from the plain path's.  Histories are the non-interacting
    propagators; the stored right-hand sides are their exact t-derivatives.
    With several ranks each takes a cost-balanced share of the 64 systems
    (no communication on the data path) and times are the max over ranks."""
    import torch
    import workloads as W
    from paper_2405_08737_gb300 import parallel
    all_systems = W.batch_systems(64, seed)
    costs = [parallel.slice_cost(sy["M"], sy["n_t"] - 1) for sy in all_systems]
    mine = parallel.shard_systems(costs, world)[rank]
    systems = [all_systems[i] for i in mine]
    need = 0
    for sy in systems:
        M, nt = sy["M"], sy["n_t"]
        need += (2 * W.tri_size(nt) + (2 * 13 + 2 + 2 + 35) * nt) * M * M * 16 + 200e6
    free, _ = torch.cuda.mem_get_info()
    if parallel.max_over_ranks(1.0 if need > free - 16e9 else 0.0) > 0:
        return {"skipped": "needs %.1f GB of device memory, %.1f GB free" % (need / 1e9, free / 1e9)}
    t_setup = time.perf_counter()
    runs, rows = [], []
    for sy in systems:
        t, order, h, U, v, pulse = W.batch_model(sy)
        M, nt = sy["M"], sy["n_t"]
        ctx = kbe.Context(M, nt)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        W.free_triangles_torch(h, W.half_filled_rho(h), t, nt, "cuda", out=(run.L, run.R))
        n = nt - 1
        hd = torch.as_tensor(h, device="cuda")
        for j in range(max(0, n - int(order[1:].max())), n):
            p = W.tri_size(j)
            Lj, Rj = run.L[p:p + j + 1], run.R[p:p + j + 1]
            run.F[j % 13, 0, : j + 1] = -1j * torch.matmul(hd, Lj)
            run.F[j % 13, 1, : j + 1] = -1j * torch.matmul(hd, Rj + Lj)
        runs.append(run)
        rows.append(n)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    setup_s = time.perf_counter() - t_setup
    total_flops = sum(P * slice_flops(sy["M"], sy["n_t"] - 1) for sy in all_systems)
    batch = kbe.Batch(runs)
    t0 = time.perf_counter()
    tune_rows = [max(1, r // 4) for r in rows]
    blk, work, tune_ms = batch.autotune(tune_rows, reps=1, stream=stream)
    tune_s = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def new_rows():
        return [r.L[W.tri_size(n):W.tri_size(n) + n + 1].clone() for r, n in zip(runs, rows)]

    # plain FP64 path: one kbe_step per system
    plain_launches = 0
    e0.record(stream)
    for r, n in zip(runs, rows):
        r.step(n, P=P, stream=stream)
        plain_launches += r.ctx.last_launch_count
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = parallel.max_over_ranks(e0.elapsed_time(e1))
    ref = new_rows()
    out = {"workload": "64 chains, M in {4,8,12,16,24}, N_t in [256,1536], U in [0.5,3] (seed %d); "
                       "one batched step = every system steps its last row, P=%d" % (seed, P),
           "history_GB": round(sum(2 * W.tri_size(sy["n_t"]) * sy["M"] ** 2 * 16 for sy in all_systems) / 1e9, 1),
           "ranks": world, "scaling": "strong (the 64 systems are split across ranks)" if world > 1 else None,
           "setup_s": round(setup_s, 1), "plain_fp64_ms_per_step": round(plain_ms, 2),
           "plain_fp64_launches": plain_launches,
           "autotune": {"block": blk, "item_work_log2": work, "history_ms_at_quarter_rows": round(tune_ms, 3),
                        "seconds": round(tune_s, 2)}}
    for prec in ("fp64", "split", "df64"):
        batch.step(rows, P=P, precision=prec, stream=stream)  # warm-up (graph capture)
        torch.cuda.synchronize()
        e0.record(stream)
        batch.step(rows, P=P, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        batch.sync_status()
        ms = parallel.max_over_ranks(e0.elapsed_time(e1))
        got = new_rows()
        err = parallel.max_over_ranks(max(float((a - b).abs().max() / b.abs().max()) for a, b in zip(got, ref)))
        out["batched_" + prec] = {"ms_per_step": round(ms, 2), "speedup_vs_plain_fp64": round(plain_ms / ms, 3),
                                  "value": round(total_flops / (ms * 1e-3) / 1e12, 4),
                                  "unit": "TFLOP/s (history slices, FP64-equivalent)",
                                  "graph_launches_per_step": 1, "kernels_per_step": batch.last_launch_count,
                                  "max_rel_dev_from_plain_fp64": err}
    out["batched_split"]["contraction"] = ("one persistent tensor-core launch per sweep over every system's "
                                           "(column tile, history chunk) units, digits formed in the kernel")
    # the same split steps, one system at a time, with the same contraction (no plane buffer):
    # what batching itself gains
    for r in runs:
        r.ctx.set_split_planes(False)
    for r, n in zip(runs, rows):  # warm-up
        r.step(n, P=P, precision="split", stream=stream)
    torch.cuda.synchronize()
    seq_launches = 0
    e0.record(stream)
    for r, n in zip(runs, rows):
        r.step(n, P=P, precision="split", stream=stream)
        seq_launches += r.ctx.last_launch_count
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = parallel.max_over_ranks(e0.elapsed_time(e1))
    got = new_rows()
    err = parallel.max_over_ranks(max(float((a - b).abs().max() / b.abs().max()) for a, b in zip(got, ref)))
    out["split_one_system_at_a_time"] = {
        "ms_per_step": round(seq_ms, 2), "kernels_per_step": seq_launches,
        "batched_split_speedup": round(seq_ms / out["batched_split"]["ms_per_step"], 3),
        "note": "64 kbe_step calls with KBE_SPLIT_BF16 and the same fused contraction (kbe_set_split_planes(0))",
        "max_rel_dev_from_plain_fp64": err}
    out["batched_fp64"]["roofline_frac_of_fp64_peak"] = round(out["batched_fp64"]["value"] / FP64_PEAK_TFLOPS, 4)
    batch.close()
    for r in runs:
        r.ctx.close()
    del runs, batch
    torch.cuda.empty_cache()
    return out


def split_roofline(M, n, k_avg_ms):
    """Roofline of the split contraction of slice n.  Bound: the larger of
    the HBM time of the algorithmic bytes (the FP64 L and R triangles read
    once, 16 M^2 (n+1)(n+2) B) and the tensor time of the digit products
    (13 digit pairs x 4 real products x 2 flops per complex multiply-add,
    (n+1)(3n+2) M^3 of them) at the sustained fp16 peak (the measured bf16
    figure: fp16 and bf16 share the nominal dense rate).  achieved/frac are
    on the binding one; the bytes the kernel actually streams are reported
    beside it."""
    hbm = hbm_peak_gbs()
    alg_bytes = 16.0 * M * M * (n + 1) * (n + 2)
    digit_flops = 13 * 4 * 2 * (n + 1) * (3 * n + 2) * M ** 3
    tc = bf16_peak_tflops(sustained=True)
    t_hbm = alg_bytes / (hbm * 1e9)
    t_tc = digit_flops / (tc * 1e12)
    sec = k_avg_ms * 1e-3
    out = {"kernel": SPLIT_KERNEL, "avg_ms": round(k_avg_ms, 4), "algorithmic_bytes": alg_bytes,
           "digit_product_flops": digit_flops, "streamed_bytes": split_stream_bytes(M, n),
           "hbm_frac_on_algorithmic_bytes": round(alg_bytes / sec / 1e9 / hbm, 4),
           "tensor_frac_on_digit_flops": round(digit_flops / sec / 1e12 / tc, 4)}
    if t_hbm >= t_tc:
        out.update({"bound": "hbm", "achieved": round(alg_bytes / sec / 1e9, 1), "peak": hbm, "unit": "GB/s",
                    "frac": out["hbm_frac_on_algorithmic_bytes"], "peak_source": "MEASURED_PEAKS.json hbm_gbs"})
    else:
        out.update({"bound": "tensor", "achieved": round(digit_flops / sec / 1e12, 2), "peak": tc,
                    "unit": "TFLOP/s", "frac": out["tensor_frac_on_digit_flops"],
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained x 1 (fp16 digits; fp16 and bf16 "
                                   "share the nominal dense tensor rate)"})
    return out


def slice_sweep(kbe, ctx, run, M, stream, rows=(255, 511, 767, 1023), reps=3):
    """The history slice alone at several rows n of the main workload's
    history, each precision's contraction kernel timed by the library's
    events: FP64 against the FP64 peak, split against HBM (its digit planes),
    double-float as FP64-equivalent TFLOP/s."""
    import torch
    out = {}
    I = torch.empty_like(run.I)
    hbm = hbm_peak_gbs()
    for n in rows:
        ctx.selfenergy_slice(n, run.L, run.R, run.Sl, run.Sg, stream=stream)
        res = {}
        for prec in ("fp64", "split", "df64"):
            ctx.history_slice(n, run.L, run.R, run.Sl, run.Sg, I, precision=prec, stream=stream)  # warm-up
            torch.cuda.synchronize()
            ctx.set_profiling(True)
            for _ in range(reps):
                ctx.history_slice(n, run.L, run.R, run.Sl, run.Sg, I, precision=prec, stream=stream)
            torch.cuda.synchronize()
            k, ms = ctx.read_profiling()
            ctx.set_profiling(False)
            res[prec + "_contraction_ms"] = round(ms / max(k, 1), 4)
        f = slice_flops(M, n)
        res["fp64_frac_of_fp64_peak"] = round(f / (res["fp64_contraction_ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4)
        sr = split_roofline(M, n, res["split_contraction_ms"])
        res["split_bound"] = sr["bound"]
        res["split_frac"] = sr["frac"]
        res["df64_tflops_fp64_equivalent"] = round(f / (res["df64_contraction_ms"] * 1e-3) / 1e12, 4)
        out[str(n)] = res
    ctx.sync_status()
    return out


def band_split(kbe, ctx, run, n, stream, worlds=(2, 4, 8), reps=2):
    """The one-system split by row bands (parallel.row_bands): each band's
    partial slice of row n timed on this GPU (CUDA events), against the whole
    slice divided by the band count -- the compute each of N devices would
    do, without the all-reduce of the 2 (n+1) M^2 partials."""
    import torch
    from paper_2405_08737_gb300 import parallel
    out = {}
    part = torch.empty_like(run.I)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ctx.selfenergy_slice(n, run.L, run.R, run.Sl, run.Sg, stream=stream)
    full = timed(lambda: ctx.history_slice(n, run.L, run.R, run.Sl, run.Sg, part, stream=stream))
    out["whole_slice_ms"] = round(full, 4)
    for w in worlds:
        ms = [round(timed(lambda lo=lo, hi=hi: ctx.history_slice_band(n, lo, hi, run.L, run.R, run.Sl, run.Sg, part,
                                                                      stream=stream)), 4)
              for lo, hi in parallel.row_bands(n + 1, w)]
        out[str(w)] = {"band_ms": ms, "max_over_ideal": round(max(ms) / (full / w), 3)}
    ctx.sync_status()
    return out


def sigma_bench(kbe, ctx, run, n_t, stream, reps=10):
    """The self-energy kernel over the whole stored triangle (kbe_selfenergy_all):
    32 B read and 32 B written per complex entry, 2.15 GB for the chain
    workload (far above L2).  Returns GB/s against the measured HBM peak."""
    import torch
    Sl = torch.empty_like(run.L)
    Sg = torch.empty_like(run.L)
    for _ in range(3):
        ctx.selfenergy_all(n_t, run.L, run.R, Sl, Sg, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.selfenergy_all(n_t, run.L, run.R, Sl, Sg, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.sync_status()
    ms = e0.elapsed_time(e1) / reps
    nbytes = 64.0 * n_t * (n_t + 1) // 2 * ctx.M * ctx.M
    peak = hbm_peak_gbs()
    del Sl, Sg
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"kernel": "sigma_kernel over the whole triangle (kbe_selfenergy_all)", "bound": "hbm",
            "arithmetic": "double-float (hi + lo FP32 pairs, about 2^-47 per operation) for the products of "
                          "Eq. SE; G^> = R + L and the final hi + lo sums in FP64; rows within 1e-13 of the "
                          "FP64 oracle",
            "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "avg_ms": round(ms, 4), "bytes_per_launch": nbytes,
            "note": "algorithmic bytes: L, R read and S^<, S^> written once (64 B per complex entry)"}


def dense_bench(kbe, seed, stream, n_t=1024, norbs=(2, 8, 16, 32)):
    """The self-energy of Eq. (SE) with a dense four-index interaction
    (synthetic Coulomb tensors with the symmetries of real-orbital
    integrals): row n = n_t-1 of random two-time data, one kernel per call.
    Algorithmic work: 12 M^5 FP64 multiply-adds per block and component,
    2 n_t (block, component) units per row."""
    import torch
    import workloads as W
    out = {"kernel": "sigma_dense_kernel (FP64 DFMA)", "n": n_t - 1, "bound": "alu", "unit": "TFLOP/s",
           "peak": round(FP64_PEAK_TFLOPS, 4), "rows": []}
    n = n_t - 1
    for M in norbs:
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(*W.grid(n_t, 0.02, 0.4, seed))
        ctx.set_model(W.chain_h(M), np.ones(M), W.site_potential(M), None)
        ctx.set_interaction(W.coulomb_tensor(M, seed, U=1.0))
        Lr, Rr = W.random_rows(M, n, seed + M)
        Rr[n] = -1j * np.eye(M)
        L = torch.zeros((W.tri_size(n_t), M, M), dtype=torch.complex128, device="cuda")
        R = torch.zeros_like(L)
        L[W.tri_index(n, 0):] = torch.as_tensor(Lr, device="cuda")
        R[W.tri_index(n, 0):] = torch.as_tensor(Rr, device="cuda")
        Sl = torch.empty((n_t, M, M), dtype=torch.complex128, device="cuda")
        Sg = torch.empty_like(Sl)
        flops = 24.0 * M ** 5 * 2 * n_t
        reps = max(2, min(20, int(2e11 / flops)))
        for _ in range(2):
            ctx.selfenergy_slice(n, L, R, Sl, Sg, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.selfenergy_slice(n, L, R, Sl, Sg, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.sync_status()
        ms = e0.elapsed_time(e1) / reps
        tf = flops / (ms * 1e-3) / 1e12
        out["rows"].append({"norb": M, "ms": round(ms, 4), "achieved": round(tf, 4),
                            "frac": round(tf / FP64_PEAK_TFLOPS, 4), "reps": reps})
        del L, R, Sl, Sg
        ctx.close()
        torch.cuda.empty_cache()
    return out


def controller_bench(kbe, seed, stream, t_end=8.0, n_max=2048):
    """Adaptive time stepping (Sec. 3.1): the 8-orbital chain from the
    uncorrelated state through its pulse (t0 = 5) to t_end, with the run
    choosing its own grid and orders (history order 5 on every interval).
    FP64 at rtol 1e-6 and 1e-8 (the difference of their final density
    matrices shows the accuracy reached at 1e-6) and the split contraction
    at 1e-6."""
    import torch
    import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    M = cfg["M"]
    h, U, v, pulse = W.build_model(cfg, seed)
    rho = W.half_filled_rho(h)
    out = {"workload": "%s model, t = 0 .. %.1f, grid chosen by the run (atol = 1e-2 rtol)" % (WORKLOAD, t_end),
           "runs": []}
    finals = {}
    for rtol, precision in ((1e-6, "fp64"), (1e-8, "fp64"), (1e-6, "split"), (1e-8, "df64")):
        ctx = kbe.Context(M, n_max)
        ctx.set_model(h, U, v, pulse)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = ctx.run_controlled(rho, rtol, rtol * 1e-2, 0.01, t_end, precision=precision, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.sync_status()
        n = g["n"]
        finals[(rtol, precision)] = g["L"][W.tri_index(n - 1, n - 1)].cpu().numpy()
        steps, nerr, nconv, nfev, nrec = g["stats"]
        dt = np.diff(g["t"])
        out["runs"].append({"rtol": rtol, "precision": precision, "status": g["status"], "rows": n,
                            "ms": round(e0.elapsed_time(e1), 2), "steps": steps, "error_test_failures": nerr,
                            "convergence_failures": nconv, "rhs_evaluations": nfev, "reconstructed_blocks": nrec,
                            "max_order": int(g["q"].max()), "dt_min": float(dt.min()), "dt_max": float(dt.max()),
                            "t_end": float(g["t"][-1])})
        ctx.close()
        del g
        torch.cuda.empty_cache()
    ref = finals[(1e-8, "fp64")]
    out["final_density_diff_rtol1e-6_vs_1e-8"] = float(np.abs(finals[(1e-6, "fp64")] - ref).max())
    out["final_density_diff_split_vs_fp64_1e-8"] = float(np.abs(finals[(1e-6, "split")] - ref).max())
    out["final_density_diff_df64_vs_fp64_at_1e-8"] = float(np.abs(finals[(1e-8, "df64")] - ref).max())
    return out


def thermal_bench(kbe, ctx, run, n, P, stream, t, h, steps, beta=10.0, n_tau=128):
    """The KBE step of the main workload with the thermal branch (Eq. KBE3):
    mixed rows of the non-interacting state at inverse temperature beta on
    n_tau tau points, the mixed right-hand sides of the last rows rebuilt,
    then the same timed steps.  Algorithmic FP64 work of the thermal terms
    per sweep: the KBE2 mixed term (n+1) M^2 n_tau M and the KBE3 right-hand
    side n_tau M^2 (n+1+n_tau) M complex multiply-adds (8 flops each)."""
    import torch
    import workloads as W
    M = ctx.M
    GM, _, mix = W.thermal_free(h, beta, n_tau, t[:n + 1])
    ctx.set_thermal(beta, GM, k_tau=5)
    ctx.set_mixed_rows(torch.as_tensor(mix, device="cuda"))
    del mix
    for j in range(max(0, n - 6), n):
        ctx.rhs_row(j, run.L, run.R, run.Sl, run.Sg, run.I, run.F, stream=stream)
    out = {"workload": "%s step of row n=%d with a thermal branch: beta=%.1f, %d tau points, tau order 5"
                       % (WORKLOAD, n, beta, n_tau), "n_tau": n_tau}
    for precision in ("fp64", "split"):
        ms, launches, _, _ = time_steps(ctx, run, n, P, steps, 2, stream, precision)
        out[precision + "_ms_per_step"] = round(ms / steps, 4)
        out[precision + "_gpu_launches"] = launches
    ctx.set_thermal(beta, None)
    out["thermal_flops_per_step"] = 8.0 * P * (M ** 3 * n_tau * (n + 1) + M ** 3 * n_tau * (n + 1 + n_tau))
    return out


def bf16_peak_tflops(sustained=True):
    """Measured dense bf16 peak (MEASURED_PEAKS.json): the sustained figure
    for kernels timed inside a long step, else the burst figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained" if sustained else "bf16_tflops"])
    except Exception:
        return 1700.0 if sustained else 1900.0


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k])
    except Exception:
        pass
    return 6800.0


def adaptive_bench(kbe, seed, stream, n_rows=256, K=6):
    """Adaptive history orders (Sec. 3.2): the first n_rows steps of the
    8-orbital chain from the uncorrelated state, with the history order of
    every interval chosen on the device (orders up to K) and with the grid's
    orders; reports the time of both runs and the chosen orders."""
    import torch
    import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    M = cfg["M"]
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], seed)
    t, order = t[:n_rows], order[:n_rows]
    h, U, v, pulse = W.build_model(cfg, seed)
    out = {"workload": "%s: first %d steps from the uncorrelated state, P=2, FP64" % (WORKLOAD, n_rows), "K": K}
    for mode in ("grid", "adaptive"):
        ctx = kbe.Context(M, n_rows)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        if mode == "adaptive":
            ctx.set_adaptive_orders(K)
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for n in range(1, n_rows):
            run.step(n, P=2, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.sync_status()
        out[mode + "_ms"] = round(e0.elapsed_time(e1), 2)
        if mode == "adaptive":
            ko = ctx.history_orders(n_rows)
            out["chosen_orders_histogram"] = {int(k): int(c) for k, c in zip(*np.unique(ko[1:], return_counts=True))}
        ctx.close()
    out["overhead_vs_grid_orders"] = round(out["adaptive_ms"] / out["grid_ms"] - 1.0, 4)
    return out


def window_bench(kbe, seed, stream):
    """The differentiation form: gradient of the final site-0 density
    2 Im L(N-1,N-1)_00 with respect to U (uniform) and E0 through the last 32
    steps of the 16-orbital, 512-point chain (pulse centred inside the
    window), restarted from the non-interacting history.  Times the window
    forward (FP64 steps keeping every right-hand-side row) and the reverse
    sweep, and checks dF/dU and dF/dE0 against central differences (h=1e-5)."""
    import torch
    import workloads as W
    cfg = W.CONFIGS["chain_m16_n512_w32"]
    M, nt, Wn = cfg["M"], cfg["n_t"], cfg["window"]
    n_start = nt - Wn
    t, order = W.grid(nt, cfg["dt0"], cfg["sig"], seed)
    h, U, v, pulse = W.build_model(cfg, seed)
    pulse = dict(pulse, t0=float(t[-1] - 0.35))
    L, R, F = W.restart_state(h, W.half_filled_rho(h), t, order, n_start, nt, device="cuda")
    ctx = kbe.Context(M, nt)
    ctx.set_grid(t, order)
    win = kbe.Window(ctx, L, R, F, n_start, nt, h, v, pulse, P=2)
    Ut = torch.tensor(U, dtype=torch.float64, requires_grad=True)
    Et = torch.tensor(pulse["E0"], dtype=torch.float64, requires_grad=True)
    kbe.window_final_block(Ut, Et, win)  # warm-up
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    blk = kbe.window_final_block(Ut, Et, win)
    e1.record(stream)
    (2.0 * blk[0, 0].imag).backward()
    e2.record(stream)
    torch.cuda.synchronize()
    ctx.sync_status()
    fwd, bwd = e0.elapsed_time(e1), e1.elapsed_time(e2)
    gU, gE = float(Ut.grad.sum()), float(Et.grad)
    hh = 1e-5
    dens = lambda u, e: 2.0 * float(win.forward(u, e)[0, 0].imag.cpu())
    fdU = (dens(U + hh, pulse["E0"]) - dens(U - hh, pulse["E0"])) / (2 * hh)
    fdE = (dens(U, pulse["E0"] + hh) - dens(U, pulse["E0"] - hh)) / (2 * hh)
    # the same window with the double-float contraction (forward and recompute)
    win_d = kbe.Window(ctx, L, R, F, n_start, nt, h, v, pulse, P=2, precision="df64")
    Ud = torch.tensor(U, dtype=torch.float64, requires_grad=True)
    Ed = torch.tensor(pulse["E0"], dtype=torch.float64, requires_grad=True)
    kbe.window_final_block(Ud, Ed, win_d)  # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    blk_d = kbe.window_final_block(Ud, Ed, win_d)
    e1.record(stream)
    (2.0 * blk_d[0, 0].imag).backward()
    e2.record(stream)
    torch.cuda.synchronize()
    ctx.sync_status()
    fwd_d, bwd_d = e0.elapsed_time(e1), e1.elapsed_time(e2)
    gUd, gEd = float(Ud.grad.sum()), float(Ed.grad)
    ctx.close()
    # FP64 work: the forward window is 2 slices per step; the reverse sweep recomputes them and
    # runs 2 adjoint slices per step (Sigma-row cotangent, 24 M^3 (n+1)^2 flops each; the
    # cotangents of the window rows add 64 M^3 (n - n_start + 1)(n+1))
    fwd_flops = sum(2 * slice_flops(M, n) for n in range(n_start, nt))
    bwd_flops = sum(2 * slice_flops(M, n) + 2 * (24.0 * M ** 3 * (n + 1) ** 2 +
                                                  64.0 * M ** 3 * (n - n_start + 1) * (n + 1))
                    for n in range(n_start, nt))
    return {"workload": "chain_m16_n512_w32: M=16, N_t=512, gradient through the last %d steps (P=2), "
                        "pulse centred 0.35 before the final time" % Wn,
            "forward_ms": round(fwd, 2), "backward_ms": round(bwd, 2),
            "forward_tflops": round(fwd_flops / (fwd * 1e-3) / 1e12, 4),
            "backward_tflops": round(bwd_flops / (bwd * 1e-3) / 1e12, 4),
            "backward_frac_of_fp64_peak": round(bwd_flops / (bwd * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
            "dF_dU": gU, "dF_dU_fd": fdU, "rel_err_U": abs(gU - fdU) / abs(fdU),
            "dF_dE0": gE, "dF_dE0_fd": fdE, "rel_err_E0": abs(gE - fdE) / abs(fdE),
            "df64": {"forward_ms": round(fwd_d, 2), "backward_ms": round(bwd_d, 2),
                     "rel_diff_from_fp64_gradient_U": abs(gUd - gU) / abs(gU),
                     "rel_diff_from_fp64_gradient_E0": abs(gEd - gE) / abs(gE)}}


def precision_m32_bench(kbe, seed, stream, steps):
    """The precision form on its own workload: the 32-orbital GOE model
    (U = 1.5, N_t = 1024, orders 1..5), one KBE step of row n = 1023 (P = 2)
    restarted from the non-interacting history, FP64 and split paths.
    Reports ms per step, the split contraction against HBM (its digit planes
    are streamed once per 8-orbital part) and the deviation of the split
    step's new row and last slice from the FP64 step's (max-norm relative;
    the FP64 path matches the oracle to 1e-12)."""
    import torch
    cfg, t, order, h, U, v, pulse, ctx, run, n = setup_workload(kbe, seed, name="goe_m32_n1024")
    M, P = cfg["M"], 2
    ms, launches, _, _ = time_steps(ctx, run, n, P, 1, 1, stream)
    ref = step_rows(run, n)
    ms_s, launches_s, kc_s, kms_s = time_steps(ctx, run, n, P, steps, 2, stream, "split")
    got = step_rows(run, n)
    ms_d, _, _, _ = time_steps(ctx, run, n, P, 1, 1, stream, "df64")
    got_d = step_rows(run, n)
    ctx.sync_status()
    ctx.close()
    del run
    torch.cuda.empty_cache()
    dev = {}
    for name, a, b in (("new_row", np.concatenate([got[0], got[1]]), np.concatenate([ref[0], ref[1]])),
                       ("slice", got[2], ref[2])):
        dev[name] = float(np.abs(a - b).max() / np.abs(b).max())
    dev_d = {}
    for name, a, b in (("new_row", np.concatenate([got_d[0], got_d[1]]), np.concatenate([ref[0], ref[1]])),
                       ("slice", got_d[2], ref[2])):
        dev_d[name] = float(np.abs(a - b).max() / np.abs(b).max())
    k_avg = kms_s / max(kc_s, 1)
    flops = P * slice_flops(M, n)
    return {"workload": "goe_m32_n1024: GOE one-body h (M=32), local U=1.5, N_t=1024 nonuniform, orders 1..5; "
                        "KBE step of row n=%d with P=%d" % (n, P),
            "fp64_ms_per_step": round(ms, 3), "fp64_tflops": round(flops / (ms * 1e-3) / 1e12, 4),
            "split_ms_per_step": round(ms_s / steps, 3),
            "split_tflops_fp64_equivalent": round(flops / (ms_s / steps * 1e-3) / 1e12, 4),
            "speedup_vs_fp64_step": round(ms / (ms_s / steps), 3),
            "split_contraction": split_roofline(M, n, k_avg),
            "split_deviation_from_fp64_step": dev, "stated_error_bound": 1e-8,
            "df64_ms_per_step": round(ms_d, 3), "df64_speedup_vs_fp64_step": round(ms / ms_d, 3),
            "df64_deviation_from_fp64_step": dev_d,
            "gpu_launches": {"fp64": launches, "split": launches_s}}


def whole_runs(kbe, seed, P, stream, oracle_rows=64):
    """Whole second-Born runs from the uncorrelated state: every KBE step of
    the dimer (N_t = 64) and of the 8-orbital chain (N_t = 1024, with its
    pulse), in FP64, split and double-float precision.  Per run: the time of
    all steps (CUDA events around one kbe_run_steps call, host launches
    included; for the dimer also one kbe_step call per step from Python),
    the final site densities n_a(T_f) = Im G^<_aa(T_f, T_f) and their
    deviation from the FP64 run's, and the FP64 and split runs' first rows
    against the oracle's run of the same grid."""
    import torch
    import oracle
    import workloads as W
    out = {}
    for name in ("dimer_m2_n64", "chain_m8_n1024"):
        cfg = W.CONFIGS[name]
        M, n_t = cfg["M"], cfg["n_t"]
        t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], seed)
        h, U, v, pulse = W.build_model(cfg, seed)
        rho0 = W.half_filled_rho(h)
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        res = {"workload": "%s: all %d KBE steps from the uncorrelated state, P=%d" % (name, n_t - 1, P),
               "slice_flops_total": sum(P * slice_flops(M, n) for n in range(1, n_t))}
        dens = {}
        head = {}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for prec in ("fp64", "split", "df64"):
            run = kbe.Run(ctx)
            ctx.reset_cache()
            run.init_uncorrelated(rho0, stream=stream)
            torch.cuda.synchronize()
            step_calls_ms = None
            if n_t <= 128:  # small runs: one call per step from Python as well, on a second run
                e0.record(stream)
                for n in range(1, n_t):
                    run.step(n, P=P, precision=prec, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                step_calls_ms = e0.elapsed_time(e1)
                run.init_uncorrelated(rho0, stream=stream)
                ctx.reset_cache()
                torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            run.run_steps(1, n_t - 1, P=P, precision=prec, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            ctx.sync_status()
            ms = e0.elapsed_time(e1)
            last = run.L[W.tri_index(n_t - 1, n_t - 1)].cpu().numpy()
            dens[prec] = np.imag(np.diag(last))
            head[prec] = run.L[: W.tri_size(min(oracle_rows, n_t))].cpu().numpy()
            res[prec] = {"ms_total": round(ms, 2), "host_wall_s": round(wall, 3),
                         "tflops": round(res["slice_flops_total"] / (ms * 1e-3) / 1e12, 4)}
            if step_calls_ms is not None:
                res[prec]["ms_total_one_call_per_step"] = round(step_calls_ms, 2)
            del run
            torch.cuda.empty_cache()
        for prec in ("split", "df64"):
            d = dens[prec] - dens["fp64"]
            res[prec]["final_density_max_abs_dev_from_fp64"] = float(np.abs(d).max())
            res[prec]["final_density_rel_dev_from_fp64"] = float(np.abs(d).max() / np.abs(dens["fp64"]).max())
            res[prec]["speedup_vs_fp64_run"] = round(res["fp64"]["ms_total"] / res[prec]["ms_total"], 3)
        res["fp64"]["final_density"] = [round(float(x), 12) for x in dens["fp64"]]
        # the oracle's run of the first rows of the same grid
        k = min(oracle_rows, n_t)
        L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
        Lo = np.zeros((W.tri_size(k), M, M), np.complex128)
        Ro = np.zeros_like(Lo)
        Lo[0], Ro[0] = L0[0], R0[0]
        Lo, _, _ = oracle.run(t[:k], order[:k], h, U, v, pulse, P, Lo, Ro, {0: F0}, 1, k,
                              nthreads=oracle.threads_available())
        for prec in ("fp64", "split", "df64"):
            res[prec]["rows_0_%d_rel_dev_from_oracle" % (k - 1)] = float(
                np.abs(head[prec] - Lo).max() / np.abs(Lo).max())
        out[name] = res
        ctx.close()
    return out


def seed_spread(kbe, seeds, n_t, P, stream):
    """The main KBE step (FP64 and split) on the inputs of each seed (grid
    and pulse drawn from it): ms per step per seed and their medians."""
    import torch
    out = {"seeds": list(seeds), "fp64_ms_per_step": [], "split_ms_per_step": []}
    for sd in seeds:
        cfg, t, order, h, U, v, pulse, ctx, run, n = setup_workload(kbe, sd, n_t)
        ms, _, _, _ = time_steps(ctx, run, n, P, 4, 3, stream)
        ms_s, _, _, _ = time_steps(ctx, run, n, P, 4, 3, stream, "split")
        ctx.sync_status()
        ctx.close()
        del run
        torch.cuda.empty_cache()
        out["fp64_ms_per_step"].append(round(ms / 4, 4))
        out["split_ms_per_step"].append(round(ms_s / 4, 4))
    out["median_fp64_ms_per_step"] = float(np.median(out["fp64_ms_per_step"]))
    out["median_split_ms_per_step"] = float(np.median(out["split_ms_per_step"]))
    return out


def step_rows(run, n):
    p = W_tri(n)
    return (run.L[p:p + n + 1].cpu().numpy(), run.R[p:p + n + 1].cpu().numpy(),
            run.I[:, : n + 1].cpu().numpy())


def sharded_bench(kbe, args, rank, world):
    """The N-GPU line: ONE system (the chain workload's KBE step of row
    n = N_t - 1) split by row bands of its stored triangles across the ranks
    (parallel.row_bands, about equal stored blocks each); every step is
    parallel.sharded_step: predictor, then P sweeps of {self-energy row and
    the band's partial slice, NCCL all-reduce of the 2 (n+1) M^2 partials,
    Fock matrix, right-hand side and corrector}.  Strong scaling: the work of
    the step is fixed, `value` is its flops over the max-over-ranks time.
    e2e: the same step with each rank's band rows, row n-1 and the
    right-hand-side ring copied in from pinned host memory every step and the
    new row read back."""
    import torch
    from paper_2405_08737_gb300 import parallel
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    kbe.lib()
    cfg, t, order, h, U, v, pulse, ctx, run, n = setup_workload(kbe, args.seed, args.n_t)
    M = cfg["M"]
    stream = torch.cuda.current_stream()
    bands = parallel.row_bands(n + 1, world)
    band = bands[rank]

    launches = [0]

    def step():
        launches[0] = parallel.sharded_step(ctx, n, args.P, band, run.L, run.R, run.Sl, run.Sg, run.I, run.F,
                                            stream=stream)["kernels"]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    ctx.set_profiling(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    k_count, k_ms = ctx.read_profiling()
    ctx.set_profiling(False)
    clk = clocks.stop()
    barrier()
    ms = parallel.max_over_ranks(ms)
    ms_step = ms / args.steps
    flops_step = args.P * slice_flops(M, n)
    lo, hi = band
    band_blocks = parallel.tri(min(hi, n + 1)) - parallel.tri(min(lo, n + 1))
    band_flops = slice_flops(M, n) * band_blocks / parallel.tri(n + 1)
    k_avg = k_ms / max(k_count, 1)
    achieved = band_flops / (k_avg * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
            "kernel": "history_partial over rank 0's row band (kbe_step_sweep_band)", "launches_timed": k_count,
            "avg_ms": round(k_avg, 4), "band_rows": [int(lo), int(hi)],
            "algorithmic_flops_per_launch": band_flops,
            "peak_source": "unit counts x clock: 152 SMs x 2 DFMA/clk x 2 flops x 2070 MHz"}
    # e2e: band rows, row n-1 and the ring from pinned host memory, row n back
    blk = M * M
    L_h = run.L.cpu().pin_memory()
    R_h = run.R.cpu().pin_memory()
    F_h = run.F.cpu().pin_memory()
    out_L = torch.empty((n + 1, M, M), dtype=torch.complex128).pin_memory()
    out_R = torch.empty_like(out_L).pin_memory()
    p0, p1 = parallel.tri(min(lo, n)), parallel.tri(min(hi, n))
    pr0, pr1 = parallel.tri(n - 1), parallel.tri(n)
    extra = 0 if lo <= n - 1 < hi else pr1 - pr0
    h2d = 2 * ((p1 - p0) + extra) * blk * 16 + F_h.numel() * 16
    d2h = 2 * (n + 1) * blk * 16

    def one_host():
        if p1 > p0:
            run.L[p0:p1].copy_(L_h[p0:p1], non_blocking=True)
            run.R[p0:p1].copy_(R_h[p0:p1], non_blocking=True)
        if extra:
            run.L[pr0:pr1].copy_(L_h[pr0:pr1], non_blocking=True)
            run.R[pr0:pr1].copy_(R_h[pr0:pr1], non_blocking=True)
        run.F.copy_(F_h, non_blocking=True)
        step()
        q = parallel.tri(n)
        out_L.copy_(run.L[q:q + n + 1], non_blocking=True)
        out_R.copy_(run.R[q:q + n + 1], non_blocking=True)

    e2e = None
    if not args.no_e2e:
        one_host()
        barrier()
        e0.record(stream)
        reps = max(3, args.steps // 4)
        for _ in range(reps):
            one_host()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1) / reps)
        e2e = {"value": round(flops_step / (e2e_ms * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
               "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    ctx.sync_status()
    line = {"metric": METRIC, "value": round(flops_step / (ms_step * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%s: Hubbard chain M=8, N_t=%d nonuniform, orders 1..5, pulse; KBE step of row "
                                   "n=%d with P=%d (FP64 path), one system split by row bands" % (WORKLOAD, n + 1, n,
                                                                                                args.P),
                       "norb": M, "n_t": n + 1, "n": n, "P": args.P, "precision": "fp64",
                       "l2": "inputs larger than L2 (history %.2f GB per step)"
                             % (2 * (n + 1) * (n + 2) / 2 * M * M * 16 / 1e9),
                       "parallelism": "row bands of one system over %d GPU(s), all-reduce of the slice per sweep"
                                      % world,
                       "bands": [list(b) for b in bands]},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches[0] * args.steps,
            "all_reduces_per_step": args.P}
    if clk:
        line["clocks"] = clk
    ctx.close()
    del run
    torch.cuda.empty_cache()
    if not args.no_batch:
        line["batching_form"] = batch_bench(kbe, args.seed, args.P, stream, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def profile_slice(kbe, args):
    """Three history slices of row n_t - 1 with one contraction (the launch
    a profiler captures), then one JSON line with their mean duration."""
    import torch
    cfg, t, order, h, U, v, pulse, ctx, run, n = setup_workload(kbe, args.seed, args.n_t, args.workload)
    stream = torch.cuda.current_stream()
    prec = "split" if args.profile_slice.startswith("split") else args.profile_slice
    if args.profile_slice == "split-fused":
        ctx.set_split_planes(False)
    ctx.selfenergy_slice(n, run.L, run.R, run.Sl, run.Sg, stream=stream)
    I = torch.empty_like(run.I)
    ctx.set_profiling(True)
    for _ in range(3):
        ctx.history_slice(n, run.L, run.R, run.Sl, run.Sg, I, precision=prec, stream=stream)
    torch.cuda.synchronize()
    k, ms = ctx.read_profiling()
    ctx.set_profiling(False)
    ctx.sync_status()
    print(json.dumps({"profile_slice": args.profile_slice, "workload": args.workload or WORKLOAD, "n": n,
                      "contraction_ms": round(ms / max(k, 1), 4)}))


def profile_run(kbe, args):
    """The FP64 whole run of a small workload (every step in one
    kbe_run_steps call, the cooperative run kernel), twice, then one JSON
    line with the second run's duration."""
    import torch
    import workloads as W
    cfg = W.CONFIGS[args.profile_run]
    M, n_t = cfg["M"], cfg["n_t"]
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], args.seed)
    h, U, v, pulse = W.build_model(cfg, args.seed)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    run = kbe.Run(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        run.init_uncorrelated(W.half_filled_rho(h))
        e0.record()
        run.run_steps(1, n_t - 1, P=args.P)
        launches = ctx.last_launch_count
        e1.record()
        torch.cuda.synchronize()
    ctx.sync_status()
    print(json.dumps({"profile_run": args.profile_run, "steps": n_t - 1, "launches": launches,
                      "ms": round(e0.elapsed_time(e1), 3)}))


def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        return main_reference(args, rank, world)
    if args.profile_run:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_2405_08737_gb300 as kbe
        return profile_run(kbe, args)
    if args.profile_slice:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_2405_08737_gb300 as kbe
        return profile_slice(kbe, args)
    if world > 1 or args.sharded:
        import paper_2405_08737_gb300 as kbe
        return sharded_bench(kbe, args, rank, world)
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_2405_08737_gb300 as kbe
    kbe.lib()
    cfg, t, order, h, U, v, pulse, ctx, run, n = setup_workload(kbe, args.seed + rank, args.n_t)
    M = cfg["M"]
    stream = torch.cuda.current_stream()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ms, launches, k_count, k_ms = time_steps(ctx, run, n, args.P, args.steps, args.warmup, stream)
    rows = {"fp64": step_rows(run, n)}
    # the precision form: the same step with the contraction on the tensor cores
    ms_s, launches_s, kc_s, kms_s = time_steps(ctx, run, n, args.P, args.steps, args.warmup, stream, "split")
    rows["split"] = step_rows(run, n)
    # the double-float contraction on the FP32 pipe (KBE_DF64)
    ms_d, launches_d, kc_d, kms_d = time_steps(ctx, run, n, args.P, args.steps, args.warmup, stream, "df64")
    rows["df64"] = step_rows(run, n)
    clk = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([ms, ms_s, ms_d], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms, ms_s, ms_d = float(tt[0].item()), float(tt[1].item()), float(tt[2].item())
        dist.barrier()
    ms_step = ms / args.steps
    flops_step = args.P * slice_flops(M, n)
    value = world * flops_step / (ms_step * 1e-3) / 1e12
    k_avg = k_ms / max(k_count, 1)
    achieved = slice_flops(M, n) / (k_avg * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
            "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
            "traffic": FP64_SLICE_TRAFFIC if (M, n) == (8, 1023) else None,
            "traffic_source": "ncu dram__bytes_read+write of the launch at n=767, scaled by stored blocks to n=1023",
            "kernel": "history_partial (FP64 DFMA contraction)", "launches_timed": k_count,
            "avg_ms": round(k_avg, 4), "peak_source": "unit counts x clock: 152 SMs x 2 DFMA/clk x 2 flops x 2070 MHz "
                              "(FP64 is not in MEASURED_PEAKS.json)"}
    ms_step_s = ms_s / args.steps
    k_avg_s = kms_s / max(kc_s, 1)
    split_roof = split_roofline(M, n, k_avg_s)
    split_roof["traffic"] = SPLIT_SLICE_TRAFFIC if (M, n) == (8, 1023) else None
    split_roof["traffic_source"] = SPLIT_TRAFFIC_SOURCE
    split = {"precision": "split: 4-digit fixed-point slices (fp16 digits) on tcgen05, exact FP32 chunk sums, "
                          "double-float accumulation (KBE_SPLIT_BF16)", "roofline": split_roof,
             "ms_per_step": round(ms_step_s, 4),
             "value": round(world * flops_step / (ms_step_s * 1e-3) / 1e12, 4), "unit": "TFLOP/s (FP64-equivalent)",
             "speedup_vs_fp64_step": round(ms_step / ms_step_s, 3), "stated_error_bound": 1e-8,
             "contraction_kernel_ms": round(kms_s / max(kc_s, 1), 4), "gpu_launches": launches_s}
    ms_step_d = ms_d / args.steps
    k_avg_d = kms_d / max(kc_d, 1)
    df64 = {"precision": "double-float contraction on the FP32 pipe (KBE_DF64): hi + lo floats, compensated sums",
            "ms_per_step": round(ms_step_d, 4),
            "value": round(world * flops_step / (ms_step_d * 1e-3) / 1e12, 4), "unit": "TFLOP/s (FP64-equivalent)",
            "speedup_vs_fp64_step": round(ms_step / ms_step_d, 3),
            "contraction_kernel_ms": round(k_avg_d, 4),
            "contraction_tflops_fp64_equivalent": round(slice_flops(M, n) / (k_avg_d * 1e-3) / 1e12, 4),
            "contraction_vs_fp64_peak": round(slice_flops(M, n) / (k_avg_d * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 3),
            "gpu_launches": launches_d}
    e2e = None
    if not args.no_e2e:
        e2e_ms, h2d, d2h = e2e_steps(ctx, run, n, args.P, max(3, args.steps // 4), 1, stream)
        e2e = {"value": round(world * flops_step / (e2e_ms * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
               "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    line = {"metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%s: Hubbard chain M=8, N_t=%d nonuniform, orders 1..5, pulse; "
                                   "KBE step of row n=%d with P=%d (FP64 path)" % (WORKLOAD, n + 1, n, args.P),
                       "norb": M, "n_t": n + 1, "n": n, "P": args.P, "precision": "fp64",
                       "l2": "inputs larger than L2 (history %.2f GB per step)" % (2 * (n + 1) * (n + 2) / 2 * M * M * 16 / 1e9),
                       "parallelism": "independent replicas" if world > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "precision_form": split, "df64_form": df64}
    if clk:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tf, threads, sample, errs, _ = cpu_baseline(run, t, order, h, U, v, pulse, n, M, args.P, rows)
        line["cpu_baseline"] = {"value": round(tf, 6), "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": sample}
        line["cpu_thread_scaling"] = cpu_thread_scaling(run, t, order, U)
        line["error_vs_oracle"] = dict(errs["fp64"], where="new row n and last history slice of the timed KBE "
                                                           "step, max-norm relative")
        line["precision_form"]["error_vs_oracle"] = errs["split"]
        line["df64_form"]["error_vs_oracle"] = errs["df64"]
    if rank == 0 and not args.no_selfenergy:
        line["selfenergy"] = sigma_bench(kbe, ctx, run, n + 1, stream)
        line["slice_sweep"] = slice_sweep(kbe, ctx, run, M, stream,
                                          rows=tuple(r for r in (255, 511, 767, 1023) if r <= n))
        line["band_split"] = band_split(kbe, ctx, run, n, stream)
    if rank == 0 and not args.no_window:
        line["differentiation_form"] = window_bench(kbe, args.seed, stream)
    if rank == 0 and not args.no_adaptive:
        line["adaptive_orders"] = adaptive_bench(kbe, args.seed, stream)
    if rank == 0 and not args.no_thermal:
        th = thermal_bench(kbe, ctx, run, n, args.P, stream, t, h, max(3, args.steps // 4))
        th["fp64_step_without_thermal_ms"] = round(ms_step, 4)
        d_ms = th["fp64_ms_per_step"] - ms_step
        th["thermal_terms_tflops_from_step_difference"] = (round(th["thermal_flops_per_step"] / (d_ms * 1e-3) / 1e12, 4)
                                                           if d_ms > 0 else None)
        line["thermal_branch"] = th
    if rank == 0 and not args.no_controller:
        line["adaptive_time_stepping"] = controller_bench(kbe, args.seed, stream)
    if rank == 0 and not args.no_dense:
        import workloads as W
        # the same chain and step with a dense Coulomb tensor in Eq. (SE) and Eq. (eps)
        ctx.set_interaction(W.coulomb_tensor(M, args.seed, U=1.0))
        steps_d = max(3, args.steps // 4)
        ms_d, launches_d, _, _ = time_steps(ctx, run, n, args.P, steps_d, 2, stream)
        ms_ds, _, _, _ = time_steps(ctx, run, n, args.P, steps_d, 2, stream, "split")
        ctx.set_interaction(None)
        dense = dense_bench(kbe, args.seed, stream, n + 1, [int(x) for x in args.dense_norb.split(",") if x])
        dense["step"] = {"workload": "%s with a dense synthetic Coulomb tensor (norb %d), row n=%d, P=%d"
                                     % (WORKLOAD, M, n, args.P),
                         "fp64_ms_per_step": round(ms_d / steps_d, 4), "split_ms_per_step": round(ms_ds / steps_d, 4),
                         "local_fp64_ms_per_step": round(ms_step, 4), "gpu_launches": launches_d}
        line["dense_interaction"] = dense
    ctx.close()
    del run
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_seeds:
        line["seed_spread"] = seed_spread(kbe, sorted({args.seed, 1, 2} | {0}), args.n_t, args.P, stream)
    if rank == 0 and not args.no_runs:
        line["whole_runs"] = whole_runs(kbe, args.seed, args.P, stream)
    if rank == 0 and not args.no_m32:
        line["precision_form_goe_m32"] = precision_m32_bench(kbe, args.seed, stream, 3)
    if not args.no_batch:
        line["batching_form"] = batch_bench(kbe, args.seed, args.P, stream, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main_reference(args, rank, world):
    """The oracle (plain FP64 CPU C++, test infrastructure) on the host cores:
    each step is one full oracle KBE step of row n = N_t - 1 of the same
    workload (P sweeps of self-energy row, history slice and corrector)."""
    if rank != 0:
        return
    import oracle
    import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    M, n_t = cfg["M"], cfg["n_t"]
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], args.seed)
    if args.n_t:
        n_t = int(args.n_t)
        t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, args.seed)
    rho0 = W.half_filled_rho(h)
    n = n_t - 1
    threads = oracle.threads_available()
    Lh, Rh = W.free_triangles(h, rho0, t, n_rows=n)
    L, R, F = oracle_step_inputs(t, order, h, U, v, pulse, Lh, Rh, n, threads)
    for _ in range(args.warmup):
        oracle.run(t, order, h, U, v, pulse, args.P, L, R, F, n, n + 1, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(t, order, h, U, v, pulse, args.P, L, R, F, n, n + 1, nthreads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = args.P * slice_flops(M, n) / dt / 1e12
    sample = "one full oracle KBE step of row n=%d per step (P=%d), %d threads" % (n, args.P, threads)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: Hubbard chain M=8, N_t=%d; KBE step of row n=%d with P=%d (CPU oracle)"
                                   % (WORKLOAD, n_t, n, args.P)},
            "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
