"""Run-time tuning table of the mixed path: energies per batched solve.

The mixed path's throughput depends on how many energies one call batches: the sweep's
panel kernels run one CTA per energy and the correction solves one CTA per energy and
column group, so small batches leave SMs idle, while large ones lengthen every launch
and hold more device memory.  The autotuner times candidate batch sizes of a workload
through the public API (`Context.solve_dev` on device buffers, CUDA events around the
whole call, after warm-up calls) and writes the best per (workload, n, nodes, precision)
into a JSON table, which `bench.py` reads for its default batch.

    python -m paper_1903_00548_gb300.autotune --workload ribbon512 --candidates 32,64,128

The table lives beside this module (tuning.json); entries of other workloads are kept.
"""
import argparse
import json
import os
import time

import numpy as np

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def key(workload: str, n: int, nodes: int, precision: str) -> str:
    return f"{workload}/n{n}/N{nodes}/{precision}"


def load(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(workload: str, n: int, nodes: int, precision: str, path: str = TABLE):
    """The tuned batch for this configuration, or None."""
    e = load(path).get(key(workload, n, nodes, precision))
    return int(e["best"]) if e and "best" in e else None


def choose(rates: dict, tolerance: float = 0.02) -> int:
    """The candidate with the highest rate; among candidates within `tolerance` of it the
    smallest (less device memory and latency for the same throughput)."""
    if not rates:
        raise ValueError("no measured candidate")
    top = max(rates.values())
    return min(b for b, r in rates.items() if r >= (1.0 - tolerance) * top)


def record(workload: str, n: int, nodes: int, precision: str, rates: dict, meta: dict, path: str = TABLE) -> dict:
    table = load(path)
    entry = {"best": choose(rates), "energy_solves_per_s": {str(b): r for b, r in sorted(rates.items())}}
    entry.update(meta)
    table[key(workload, n, nodes, precision)] = entry
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")
    return entry


def measure(workload: str, candidates, steps: int = 2, warmup: int = 1, device: int = 0):
    """Energy-solves/s of the mixed path per candidate batch size (CUDA events around
    `steps` calls of `solve_dev` after `warmup` calls; contacts prepared beforehand)."""
    import torch

    from . import build as B
    from . import pwqt as pw
    from . import workloads as W

    B.build()
    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    wl = getattr(W, workload)()
    ctx = pw.Context(device=device)
    n = ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    ctx.set_extrinsic(0, wl.U)
    N = wl.n_nodes
    grid = wl.energies
    sets = {b: np.sort(grid[(np.arange(b) * max(1, len(grid) // b)) % len(grid)]) for b in candidates}
    ctx.prepare_leads(0, np.unique(np.concatenate(list(sets.values()))))
    stream = torch.cuda.Stream(device=dev)
    rates = {}
    for b, E in sets.items():
        outs = {"T": torch.empty(b, dtype=torch.float64, device=dev), "R": torch.empty(b, dtype=torch.float64, device=dev),
                "T_ds": torch.empty(b, dtype=torch.float64, device=dev),
                "n_open": torch.empty(2 * b, dtype=torch.int32, device=dev),
                "node_n": torch.empty(b * N * 2, dtype=torch.float64, device=dev),
                "resid": torch.empty(b, dtype=torch.float64, device=dev),
                "iters": torch.empty(b, dtype=torch.int32, device=dev),
                "status": torch.empty(b, dtype=torch.int32, device=dev)}
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        for _ in range(warmup):
            ctx.solve_dev(0, E, pw.MIXED, ptrs, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.solve_dev(0, E, pw.MIXED, ptrs, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        rates[b] = b * steps / (e0.elapsed_time(e1) / 1e3)
        del outs
        torch.cuda.empty_cache()
    ctx.close()
    return n, N, rates


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="ribbon512")
    ap.add_argument("--candidates", default="32,64,128",
                    help="batch sizes; powers of two share their energies (a smaller set is a subset)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--out", default=TABLE)
    a = ap.parse_args(argv)
    cands = [int(x) for x in a.candidates.split(",")]
    t0 = time.time()
    n, N, rates = measure(a.workload, cands, a.steps, a.warmup)
    import torch
    meta = {"device": torch.cuda.get_device_name(0), "steps": a.steps, "warmup": a.warmup,
            "seconds": round(time.time() - t0, 1), "timing": "CUDA events around solve_dev calls after warm-up"}
    entry = record(a.workload, n, N, "mixed", rates, meta, a.out)
    print(json.dumps({key(a.workload, n, N, "mixed"): entry}))


if __name__ == "__main__":
    main()
