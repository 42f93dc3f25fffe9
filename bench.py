"""Benchmark: energy-solves/s of the per-energy open-boundary solve at block size 512.

Workload (default, "ribbon512"): a 13 nm armchair ribbon (214 atoms per cell) with
256 Bloch waves at Gamma and at Z (block n = 512, G_cut = 30 nm^-1), N = 200 nodes, a
seeded smooth potential <= 0.3 eV and the 1024-point energy grid
[E_64 - 0.1, E_64 + 1.0] eV (~45 open channels per contact); one step solves one
batch of energies of that grid (contact self-energies resident in the cache, built
before timing and reported separately as sigma_cold_s_per_energy).

Default run (mixed precision, the headline `value`): complex64 block sweep on the
tensor cores + refinement with the FP64-accurate slice-product residual, K timed
steps of 32 energies without profiling; then one profiled step (phase and kernel
times for the rooflines); then the FP64 GPU arm on the same box (one step of one
energy per SM, the mixed step's energies among them; `fp64_arm`, with the largest
|T_mixed - T_FP64| over the shared energies); then one step end to end through the
host-buffer C ABI (`e2e`).  Meanwhile the oracle runs full 200-node solves on the
host cores (`cpu_baseline`).  --precision fp64 times the complex128 path alone.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--precision mixed|fp64|auto] [--batch B] [--fp64-batch B] [--clocks-csv PATH]
Under torchrun every rank solves its own batch (weak scaling, no data-path
collective); the timed region is bracketed by a barrier and synchronize and the
max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "energy-solves/s at block 512 (FP64 vs mixed+refine, <=1e-8 in T); p50/p99 latency"
UNIT = "energy-solves/s"
L2_BYTES = 129 * 2 ** 20
# nominal dense rates of GB300 used to scale the measured bf16 peak to other dtypes
NOMINAL_TFLOPS = {"bf16": 2250.0, "tf32": 1100.0, "f64": 1.25}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("bf16_tflops", 1900.0), p.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, device: int, path: str):
        self.path = path
        self.proc = None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU) legs
BLAS_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
# host memory one full-length oracle solve at block 512 holds (banded global matrix,
# its LU and the right-hand sides), with margin
ORACLE_BYTES_PER_WORKER = 14e9
ORACLE_SAMPLE_NODES = 20


def _mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return float(line.split()[1]) * 1024.0
    except OSError:
        pass
    return 16e9


def oracle_workers(reserve=16e9):
    """Processes the oracle legs may run at once: one per host core, bounded by the
    memory of full-length solves (leaving `reserve` bytes for the GPU process)."""
    cores = os.cpu_count() or 1
    return max(1, min(cores, int((_mem_available() - reserve) // ORACLE_BYTES_PER_WORKER)))


def _oracle_energy(task):
    """One oracle energy-solve, timed: the system is assembled and the contact
    self-energies are computed first (untimed, as the GPU leg keeps them resident),
    then the global system is solved `reps` times on a device of `nodes` nodes."""
    wl_name, nodes, E, reps = task
    try:
        from oracle import pwqt_oracle as O
        from paper_1903_00548_gb300 import workloads as W
        wl = getattr(W, wl_name)()
        U = W.random_smooth(nodes) if nodes != wl.n_nodes else wl.U
        s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, U)
        t0 = time.perf_counter()
        contacts = O.contacts_at(s.blk, E, U[0], U[-1])
        t_sigma = time.perf_counter() - t0
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E, contacts=contacts)
            times.append(time.perf_counter() - t0)
        return {"ok": True, "E": E, "times": times, "t_sigma": t_sigma}
    except Exception as e:  # pragma: no cover - reported in the JSON line
        return {"ok": False, "error": repr(e)}


def start_oracle_pool(wl_name, energies, nodes, reps=1, workers=None):
    """Spawned pool (one BLAS thread per process, set in the environment the children
    inherit before numpy starts its threads), one energy per process."""
    workers = workers or oracle_workers()
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in BLAS_THREAD_VARS}
    for k in BLAS_THREAD_VARS:
        os.environ[k] = "1"
    try:
        pool = ctx.Pool(workers)
        tasks = [(wl_name, nodes, float(E), reps) for E in energies[:workers]]
        res = pool.map_async(_oracle_energy, tasks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, res, workers


def finish_oracle_pool(pool, res, timeout=1500):
    try:
        out = res.get(timeout)
    except Exception as e:
        out = [{"ok": False, "error": f"oracle pool: {e!r}"}]
    pool.terminate()
    pool.join()
    return out


# ----------------------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_energies(grid, batch, rank, world):
    """Energies of one rank's step: `batch` points spread over the grid, interleaved
    across ranks so that ranks never share an energy while world * batch <= len(grid)."""
    n = len(grid)
    stride = max(1, n // (batch * world))
    idx = (np.arange(batch) * world * stride + rank * stride) % n
    return np.sort(grid[idx])


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The oracle as it stands, on the host cores: one energy per process, each step
    a banded solve of a shortened device (ORACLE_SAMPLE_NODES nodes; the solve's cost
    is linear in the node count, which the default run's cpu_baseline checks against
    full-length solves), so that the whole run ends within minutes."""
    if rank != 0:
        return 0
    from paper_1903_00548_gb300 import workloads as W
    wl = getattr(W, args.workload)()
    E = shard_energies(wl.energies, 32, 0, 1)
    pool, res, workers = start_oracle_pool(args.workload, E, ORACLE_SAMPLE_NODES, reps=args.warmup + args.steps)
    out = finish_oracle_pool(pool, res)
    ok = [r for r in out if r.get("ok")]
    if not ok:
        print(json.dumps({"impl": "reference", "unavailable": out[0].get("error", "oracle failed")}))
        return 0
    # step k: every process solves its energy once; the step lasts as long as the slowest
    steps = [max(r["times"][k] for r in ok) for k in range(args.warmup, args.warmup + args.steps)]
    t_step = statistics.mean(steps) * wl.n_nodes / ORACLE_SAMPLE_NODES
    value = len(ok) / t_step
    sample = (f"{len(ok)} processes (one BLAS thread each), one energy of {args.workload} (n={wl.n}) per process and "
              f"step, banded solve of {ORACLE_SAMPLE_NODES} of {wl.n_nodes} nodes scaled by {wl.n_nodes}/"
              f"{ORACLE_SAMPLE_NODES}; contact self-energies computed before timing")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n": wl.n, "nodes": wl.n_nodes},
            "cpu_baseline": {"kind": "oracle", "cores": len(ok), "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- our arm
def fp64_energies(grid, E_mixed, total):
    """`total` energies for the FP64 arm (one per SM): the mixed step's own energies
    and the rest spread over the grid between them."""
    extra = [e for e in shard_energies(grid, total, 0, 1) if e not in set(E_mixed.tolist())]
    keep = max(0, total - len(E_mixed))
    idx = np.linspace(0, len(extra) - 1, keep).round().astype(int) if keep and extra else np.array([], int)
    return np.sort(np.concatenate([E_mixed, np.asarray(extra)[idx]]))


def timed_steps(step, stream, steps):
    """CUDA-event time of `steps` calls on `stream` (synchronised on both sides)."""
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    marks = []
    a.record(stream)
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        marks.append((e0, e1))
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), [x.elapsed_time(y) for x, y in marks]


def run_ours(args, world, rank, local):
    import torch
    from paper_1903_00548_gb300 import build as B
    from paper_1903_00548_gb300 import pwqt as pw
    from paper_1903_00548_gb300 import workloads as W

    wl = getattr(W, args.workload)()
    if args.nodes:
        wl.n_nodes = args.nodes
        wl.U = W.random_smooth(args.nodes)
    prec_name = "mixed" if args.precision == "auto" else args.precision
    prec = pw.MIXED if prec_name == "mixed" else pw.FP64
    batch = args.batch
    if not batch and prec == pw.MIXED and not args.nodes:
        from paper_1903_00548_gb300 import autotune
        batch = autotune.lookup(args.workload, 2 * wl.n_bands, wl.n_nodes, "mixed") or 0
    batch = batch or (32 if prec == pw.MIXED else 152)
    n_grid = len(wl.energies)
    E = shard_energies(wl.energies, batch, rank, world)

    # the oracle on the host cores: full-length solves, one energy per process, started
    # first (spawned; it runs while the GPU legs do)
    oracle = None
    if rank == 0 and not args.no_cpu_baseline:
        oracle = start_oracle_pool(args.workload, E, wl.n_nodes, reps=1)

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_batch = args.fp64_batch if args.fp64_batch >= 0 else sms
    E64 = fp64_energies(wl.energies, E, fp64_batch) if (prec == pw.MIXED and fp64_batch > 0) else np.zeros(0)

    ctx = pw.Context(device=local)
    t0 = time.perf_counter()
    n = ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    ctx.set_extrinsic(0, wl.U)
    t_setup = time.perf_counter() - t0
    E_all = np.union1d(E, E64)
    t0 = time.perf_counter()
    ctx.prepare_leads(0, E_all)
    t_leads = time.perf_counter() - t0

    N = wl.n_nodes
    def outs_for(nb):
        return {"T": torch.empty(nb, dtype=torch.float64, device=dev), "R": torch.empty(nb, dtype=torch.float64, device=dev),
                "T_ds": torch.empty(nb, dtype=torch.float64, device=dev),
                "n_open": torch.empty(2 * nb, dtype=torch.int32, device=dev),
                "node_n": torch.empty(nb * N * 2, dtype=torch.float64, device=dev),
                "resid": torch.empty(nb, dtype=torch.float64, device=dev),
                "iters": torch.empty(nb, dtype=torch.int32, device=dev),
                "status": torch.empty(nb, dtype=torch.int32, device=dev)}
    outs = outs_for(batch)
    ptrs = {k: v.data_ptr() for k, v in outs.items()}
    stream = torch.cuda.Stream(device=dev)

    def step():
        ctx.solve_dev(0, E, prec, ptrs, stream.cuda_stream)

    # ---- headline: unprofiled timed steps
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches0 = ctx.kernel_launches()
    clocks = Clocks(local, args.clocks_csv.format(rank=rank))
    barrier(world)
    total_ms, per_step = timed_steps(step, stream, args.steps)
    barrier(world)
    clk_info = clocks.stop()
    launches = (ctx.kernel_launches() - launches0) // max(1, args.steps)
    total_ms = max_over_ranks(world, total_ms)
    value = world * batch * args.steps / (total_ms / 1e3)
    status = outs["status"].cpu().numpy()
    iters = outs["iters"].cpu().numpy()
    resid = outs["resid"].cpu().numpy()
    nopen = outs["n_open"].cpu().numpy().reshape(batch, 2)
    T_step = outs["T"].cpu().numpy()

    # ---- end to end through the host-buffer C ABI (copies inside the timed region)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = ctx.solve(0, E, prec)
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = world * batch / t_e2e
    h2d = 8 * batch
    d2h = batch * (8 * 4 + 4 * 4 + 8 * 2 * N)

    # ---- density-matrix route (reported apart from the energy-solve metric)
    dens = None
    if not args.no_density:
        w = np.full(len(E), (wl.energies[1] - wl.energies[0]) if len(wl.energies) > 1 else 1.0)
        mu = float(np.median(E))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.accumulate_density(0, E, w, mu, mu - 0.1, 0.025852, prec)
        t_acc = time.perf_counter() - t0
        nx, nz = 64, 16
        t0 = time.perf_counter()
        grid = ctx.density_grid(0, nx, nz)
        t_grid = time.perf_counter() - t0
        t_solve = (total_ms / args.steps) / 1e3
        dens = {"accumulate_s_per_energy": max(t_acc - t_solve, 0.0) / len(E),
                "solve_plus_accumulate_s": t_acc, "grid_s": t_grid, "grid": [nx, nz],
                "grid_points": int(grid.size), "n_max": float(grid.max())}

    # ---- one more step with CUDA-event profiling (phases and kernel times for the roofline)
    ctx.profile(True, reset=True)
    prof_ms, _ = timed_steps(step, stream, 1)
    ir_res_ms, ir_cor_ms, ir_iters = ctx.profile_refinement()
    oz_ms, oz_cmacs, oz_mma, oz_launches = ctx.profile_residual()
    cor_ms, cor_cmacs, cor_launches = ctx.profile_correction()
    sweep_ms, sweep_n, sweep_flops = ctx.profile(False)

    # ---- the FP64 GPU arm on the same box: one energy per SM, the mixed step's energies among
    # them (last: its panels of 152 energies take most of the device memory)
    fp64 = None
    if len(E64):
        o64 = outs_for(len(E64))
        p64 = {k: v.data_ptr() for k, v in o64.items()}
        ctx.solve_dev(0, E64[:1], pw.FP64, p64, stream.cuda_stream)          # warm-up (one energy)
        clocks64 = Clocks(local, args.clocks_csv.format(rank=f"{rank}_fp64"))
        ms64, _ = timed_steps(lambda: ctx.solve_dev(0, E64, pw.FP64, p64, stream.cuda_stream), stream, 1)
        clk64 = clocks64.stop()
        T64 = o64["T"].cpu().numpy()
        st64 = o64["status"].cpu().numpy()
        pos = np.searchsorted(E64, E)
        dT = np.abs(T_step - T64[pos])
        fp64 = {"value": world * len(E64) / (ms64 / 1e3), "unit": UNIT, "energies": int(len(E64)),
                "ms": ms64, "clocks": clk64, "status_nonzero": int(np.count_nonzero(st64 & 7)),
                "max_abs_dT_mixed_vs_fp64": float(np.max(dT)), "mean_abs_dT_mixed_vs_fp64": float(np.mean(dT))}

    # ---- a short serving pass (continuous batching; p50/p99 latency), on its own contexts
    serving = None
    if rank == 0 and not args.no_serving:
        ctx.close()
        torch.cuda.empty_cache()
        clk_srv = Clocks(local, args.clocks_csv.format(rank=f"{rank}_serving"))
        serving = serving_pass(local, args.serving_requests, blocks=(64, 128, 256))
        serving["clocks"] = clk_srv.stop()

    # ---- rooflines (algorithmic work; peaks from MEASURED_PEAKS.json)
    bf16, hbm, src = peaks()
    tf32 = bf16 * NOMINAL_TFLOPS["tf32"] / NOMINAL_TFLOPS["bf16"]
    f64_peak = bf16 * NOMINAL_TFLOPS["f64"] / NOMINAL_TFLOPS["bf16"]
    sweep_alg = (56.0 / 3.0) * N * float(n) ** 3 * batch
    roof_sweep = {"bound": "tensor" if prec == pw.MIXED else "fp64",
                  "achieved": sweep_alg / (sweep_ms / 1e3) / 1e12 if sweep_ms else None,
                  "peak": tf32 if prec == pw.MIXED else f64_peak, "unit": "TFLOP/s",
                  "kernel": "block sweep (k_cgemm_tc, k_mx_panel_reg, k_mx_panel_apply, k_mx_trsm_up)" if prec == pw.MIXED else "k_sweep_fp64",
                  "work": "(56/3) N n^3 real flop per energy (complex LU, X_i solve, Schur product)",
                  "peak_source": f"{src} bf16 x nominal {'tf32' if prec == pw.MIXED else 'f64'}/bf16", "traffic": None,
                  "ms_per_step": sweep_ms, "launches": sweep_n}
    if roof_sweep["achieved"]:
        roof_sweep["frac"] = roof_sweep["achieved"] / roof_sweep["peak"]
    roof_res = None
    if oz_ms > 0:
        ach = oz_mma / (oz_ms / 1e3) / 1e12
        roof_res = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                    "kernel": "k_oz_gemm (slice-product residual)",
                    "work": "bf16 MMA flops of the 34 exact slice products per real product (7-bit slices, "
                            "split form E M c - HV c - Sigma c)",
                    "peak_source": f"{src} bf16 (burst)", "traffic": None,
                    "fp64_equivalent": {"achieved": 8 * oz_cmacs / (oz_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                                        "work": "8 real flop per complex MAC of B - A c (3 N n^2 per column)",
                                        "fp64_pipe_peak": f64_peak},
                    "ms_per_step": oz_ms, "launches": oz_launches}
    # the correction solves: FP32 complex multiply-adds on the CUDA cores (4 FMAs each),
    # against the FP32 FMA peak of the device: SMs x 128 lanes x 2 flop x the maximum SM clock
    roof_corr = None
    if prec == pw.MIXED and cor_ms > 0:
        mhz = (clk_info or {}).get("sm_max_mhz") or 2070.0
        fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        ach = 8 * cor_cmacs / (cor_ms / 1e3) / 1e12
        roof_corr = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                     "kernel": "k_mx_correct (correction solve, one launch per refinement step and lane)",
                     "work": "8 real flop per complex MAC, 3 N n^2 MACs per refining column and step "
                             "(products with L_i and X_i, the two triangular solves)",
                     "peak_source": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz", "traffic": None,
                     "ms_per_step": cor_ms, "launches": cor_launches,
                     "note": "event time of the launches in the profiled step, whose two halves run one "
                             "after the other"}
    # the roofline object: the single kernel with the largest event time per step among the
    # refinement kernels; the block sweep (several kernels per panel) is reported beside it
    singles = {"residual": (oz_ms, roof_res), "correction": (cor_ms, roof_corr)}
    cand = [(t, r) for t, r in singles.values() if r]
    roof = max(cand, key=lambda x: x[0])[1] if cand else roof_sweep
    if roof is not roof_sweep and sweep_ms > max(t for t, _ in cand):
        roof = dict(roof)
        roof["note_step"] = (f"the block sweep (k_cgemm_tc, k_mx_panel_reg, k_mx_panel_apply, k_mx_trsm_up: "
                             f"{sweep_ms:.0f} ms per step over its launches) is the largest phase; "
                             "its own object is roofline_sweep")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == pw.FP64 else "c64 (3xTF32 tensor cores) + FP64-accurate residual (bf16 slice products)",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nodes": N, "energies_per_step": batch,
                       "energy_grid": n_grid, "precision": prec_name, "l2": "inputs larger than L2 "
                       f"(factor panels {N * n * n * 8 * batch / 1e9:.0f} GB per step)"},
            "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99)),
                           "unit": f"per step of {batch} energies"},
            "fp64_arm": fp64, "serving": serving,
            "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
            "sigma_cold_s_per_energy": t_leads / max(1, len(E_all)), "setup_s": t_setup,
            "gpu_launches": int(launches), "clocks": clk_info, "roofline": roof, "roofline_sweep": roof_sweep,
            "roofline_residual": roof_res, "roofline_correction": roof_corr, "density": dens,
            "phases_ms_per_step": {"sweep": sweep_ms, "refine_residual": ir_res_ms, "refine_correction": ir_cor_ms,
                                   "refine_iterations": ir_iters, "profiled_step_ms": prof_ms,
                                   "note": "one extra step with CUDA events, after the timed steps; its two halves "
                                           "run one after the other (the timed steps overlap them on two streams), "
                                           "so each kernel's event time is its own; profiled_step_ms is that step"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "results": {"max_resid": float(np.max(resid)), "max_iters": int(np.max(iters)),
                        "status_nonzero": int(np.count_nonzero(status)),
                        "status_bits": {name: int(np.count_nonzero(status & bit)) for name, bit in
                                        (("singular_pivot", 1), ("mode_count", 2), ("ir_no_converge", 4),
                                         ("degenerate", 8), ("near_unit", 16))},
                        "max_resid_unflagged": float(np.max(resid[(status & 7) == 0])) if np.any((status & 7) == 0) else None,
                        "mean_modes": float(nopen.sum(1).mean()),
                        "T_mean": float(np.mean(res.T))}}
    if oracle is not None:
        out = finish_oracle_pool(oracle[0], oracle[1])
        ok = [r for r in out if r.get("ok")]
        if ok:
            t_solve = statistics.mean(r["times"][0] for r in ok)
            line["cpu_baseline"] = {
                "value": len(ok) / t_solve, "unit": UNIT, "cores": len(ok), "kind": "oracle",
                "sample": f"{len(ok)} processes (one BLAS thread each) on {os.cpu_count()} host cores, one full "
                          f"{N}-node energy-solve of {args.workload} each (banded LU of the global system, "
                          f"mean {t_solve:.1f} s); contact self-energies computed first, untimed "
                          f"(mean {statistics.mean(r['t_sigma'] for r in ok):.1f} s per energy)"}
        else:
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                                    "sample": "failed: " + out[0].get("error", "?")}
    if rank == 0:
        print(json.dumps(line))
    if serving is None:
        ctx.close()
    return 0


# ----------------------------------------------------------------------------- batching
def run_batching(args, world, rank, local):
    """Energies x bias points in one batched solve (pwqt_solve_multi): per step, the
    same `batch` energies at every bias point of workloads.bias_points (0..0.35 V),
    every (bias point, energy) pair in the same launches; mixed precision with the
    sliced residual.  Accuracy: the largest |T_mixed - T_FP64| over a subset of the
    pairs, both from the GPU.  Contact self-energies are computed before timing."""
    import torch
    from paper_1903_00548_gb300 import build as B
    from paper_1903_00548_gb300 import pwqt as pw
    from paper_1903_00548_gb300 import workloads as W

    B.build()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    wl = getattr(W, args.batching_workload)()
    Us = W.bias_points(wl, args.bias_points)
    batch = args.batch or 16
    E = shard_energies(wl.energies, batch, 0, 1)
    ctx = pw.Context(device=local)
    n = ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    for q, U in enumerate(Us):
        ctx.set_extrinsic(q, U)
    systems = list(range(len(Us)))
    t0 = time.perf_counter()
    for q in systems:
        ctx.prepare_leads(q, E)
    t_leads = time.perf_counter() - t0
    for _ in range(args.warmup):
        ctx.solve_multi(systems, E, pw.MIXED)
    clocks = Clocks(local, args.clocks_csv.format(rank=f"{rank}_batching"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = ctx.solve_multi(systems, E, pw.MIXED)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    clk = clocks.stop()
    jobs = len(systems) * len(E)
    sub = E[:: max(1, len(E) // 4)]
    ref = ctx.solve_multi(systems, sub, pw.FP64)
    pos = np.searchsorted(E, sub)
    dT = max(float(np.max(np.abs(r.T[pos] - f.T))) for r, f in zip(res, ref))
    st = np.concatenate([r.status for r in res])
    line = {"metric": "energy-solves/s, energies x bias points in one batched solve (mixed + refinement)",
            "value": jobs * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "impl": "ours",
            "dtype": "c64 (3xTF32 tensor cores) + FP64-accurate residual (bf16 slice products)", "data": "synthetic",
            "config": {"workload": args.batching_workload, "n": n, "nodes": wl.n_nodes, "bias_points": len(Us),
                       "bias_V": [round(q * 0.05, 3) for q in systems], "energies_per_step": len(E),
                       "jobs_per_step": jobs},
            "max_abs_dT_vs_fp64": dT, "fp64_check_jobs": int(len(sub) * len(systems)),
            "status_nonzero": int(np.count_nonzero(st & 7)), "max_iters": int(max(int(r.iters.max()) for r in res)),
            "sigma_cold_s": t_leads, "clocks": clk,
            "timing": "host wall clock around the synchronous host-buffer solve_multi calls (copies included)"}
    print(json.dumps(line))
    ctx.close()
    return 0


# ----------------------------------------------------------------------------- serving
def serving_pass(local, n_req, blocks=(64, 128, 256, 512), seed=7):
    """Serving loop: a catalog of bases (the 13 nm ribbon at the given block sizes),
    requests with a random basis, device length, energy count and precision, first
    submitted all at once (capacity), then with Poisson arrivals at 70 % of that rate
    (latency).  Energies come from a fixed 48-point grid per basis whose contact
    self-energies are computed before timing, as a serving deployment keeps them
    resident.  Returns the measurements as a dict."""
    from paper_1903_00548_gb300 import pwqt as pw
    from paper_1903_00548_gb300 import workloads as W

    # one structure (the 13 nm ribbon, whose Bloch basis stays well conditioned); energy
    # windows inside each basis' band range (top Gamma/Z bands: 1.0/1.4 eV at 32 bands,
    # 7.0/3.1 eV at 64, 8.9/9.5 eV at 128)
    wl512 = W.ribbon512()
    cat = {nb: (wl512.cell, wl512.ff, wl512.gcut, nb // 2) for nb in blocks}
    e64 = W.RIBBON13_G30_E64
    grids = {64: np.linspace(0.0, 0.9, 48), 128: np.linspace(1.5, 2.8, 48),
             256: np.linspace(e64 - 0.05, e64 + 0.9, 48), 512: np.linspace(e64 - 0.05, e64 + 0.9, 48)}
    srv = pw.Server(device=local)
    t0 = time.perf_counter()
    for nb in cat:
        srv.add_basis(nb, *cat[nb])
    warm = [srv.submit(nb, np.zeros(4), grids[nb], pw.FP64) for nb in cat]
    for t in warm:
        srv.wait(t)
    t_setup = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    logb = np.log2(np.array(sorted(cat)))

    def make():
        out = []
        for _ in range(n_req):
            nb = int(2 ** rng.integers(int(logb[0]), int(logb[-1]) + 1))   # block size, log-uniform
            N = int(rng.integers(50, 201))
            nE = int(np.exp(rng.uniform(np.log(4), np.log(32))))   # 4..32 energies, log-uniform
            E = np.sort(rng.choice(grids[nb], nE, replace=False))
            prec = pw.FP32 if rng.random() < 0.5 else pw.MIXED
            U = W.random_smooth(N, 0.3, int(rng.integers(1 << 30)))
            out.append((nb, U, E, prec))
        return out

    # capacity: everything submitted at once
    reqs = make()
    srv.stats(reset=True)
    t0 = time.perf_counter()
    tickets = [srv.submit(*r) for r in reqs]
    solves = 0
    for t, r in zip(tickets, reqs):
        srv.wait(t)
        solves += len(r[2])
    t_cap = time.perf_counter() - t0
    cap = solves / t_cap
    req_rate = n_req / t_cap
    # latency: Poisson arrivals at 70 % of the measured request rate
    reqs = make()
    srv.stats(reset=True)
    gaps = rng.exponential(1.0 / (0.7 * req_rate), n_req)
    t0 = time.perf_counter()
    tickets = []
    due = 0.0
    for g, r in zip(gaps, reqs):
        due += g
        d = due - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        tickets.append(srv.submit(*r))
    solves = 0
    bad = 0
    for t, r in zip(tickets, reqs):
        res, _ = srv.wait(t)
        solves += len(r[2])
        bad += int(np.count_nonzero(res.status & ~(pw.ST_NEAR_UNIT | pw.ST_DEGENERATE)))
    t_open = time.perf_counter() - t0
    st = srv.stats()
    nbatch, nreq, largest = srv.batch_stats()
    srv.close()
    return {"solves_per_s": solves / t_open, "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"]},
            "capacity_solves_per_s": cap, "arrival_rate_req_per_s": 0.7 * req_rate, "requests": n_req,
            "bad_status": bad, "setup_s": t_setup,
            "continuous_batching": {"batched_solves": nbatch, "requests": nreq, "largest_batch": largest,
                                    "rule": "queued requests of one basis with the same node count and precision "
                                            "share the next batched solve (up to 8 potentials, within the budget)"},
            "config": {"structure": "13 nm armchair ribbon, G_cut 30 nm^-1", "catalog_block_sizes": sorted(cat),
                       "nodes": "U[50,200]", "energies_per_request": "log-uniform 4..32 from a 48-point grid per basis",
                       "precision_mix": "50% complex64 alone (PWQT_FP32), 50% mixed + refinement",
                       "arrivals": f"Poisson at 70% of the measured closed-loop request rate, seed {seed}"}}


def run_serving(args, world, rank, local):
    """The serving loop's own line (see serving_pass): catalog block sizes 64..512."""
    import torch
    from paper_1903_00548_gb300 import build as B

    B.build()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    r = serving_pass(local, args.requests)
    line = {"metric": "serving: energy-solves/s and p50/p99 request latency (mixed catalog)", "value": r["solves_per_s"],
            "unit": "energy-solves/s", "n_gpus": 1, "higher_is_better": True, "impl": "ours",
            "latency_s": r["latency_s"], "capacity_solves_per_s": r["capacity_solves_per_s"],
            "arrival_rate_req_per_s": r["arrival_rate_req_per_s"], "requests": r["requests"], "bad_status": r["bad_status"],
            "setup_s": r["setup_s"], "continuous_batching": r["continuous_batching"], "data": "synthetic",
            "config": dict(r["config"], workload="serving")}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"])
    ap.add_argument("--workload", default="ribbon512")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--fp64-batch", type=int, default=-1,
                    help="energies of the FP64 arm (default: one per SM; 0 skips it)")
    ap.add_argument("--nodes", type=int, default=0, help="development only: shorter device")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-density", action="store_true", help="skip the density-matrix timing")
    ap.add_argument("--serving", action="store_true", help="measure the serving loop instead of the headline metric")
    ap.add_argument("--batching", action="store_true",
                    help="measure energies x bias points in one batched solve instead of the headline metric")
    ap.add_argument("--batching-workload", default="ribbon256_wide")
    ap.add_argument("--bias-points", type=int, default=8)
    ap.add_argument("--requests", type=int, default=60, help="requests per serving pass (--serving)")
    ap.add_argument("--serving-requests", type=int, default=24, help="requests per pass of the default run's serving leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the default run's serving leg")
    ap.add_argument("--clocks-csv", default="/tmp/pwqt_clocks_{rank}.csv",
                    help="where the nvidia-smi clock samples of the timed region are kept ({rank} is replaced)")
    args = ap.parse_args(argv)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.serving:
        return run_serving(args, world, rank, local)
    if args.batching:
        return run_batching(args, world, rank, local)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
