"""Writes ribbon512_n200.json, the expected values of tests/test_gpu_fullsize.py.

Test infrastructure: calls only the oracle (oracle/pwqt_oracle.py) and the seeded
input generators.  The system is the block-512 benchmark workload at full length:
13 nm armchair ribbon, G_cut = 30 nm^-1, 256 bands at each of Gamma and Z
(n = 512), 200 nodes, the workload's random smooth potential; the energies are four
of the 32 that one benchmark step solves (entries 0, 10, 21 and 31 of the step's
energy set).  Per energy the oracle solves the assembled global system by banded
LU (Sec. 3.2) with the lead modes of the symmetric pencil (Sec. 3.1), and once more
with the modes of the reciprocal pencil; stored: T, R and T_ds (Eq. transmission),
open-channel counts, node densities n_s, n_d (Sec. 3.3), and the oracle's error bar
(reciprocity defect |T - T_ds| and the spread between the two pencils).

One energy per process (spawned), two BLAS threads each; about 7 minutes per
energy and ~12 GB of memory per process (the banded matrix of the 102400 x 102400
global system).  Run from the repository root:
    python tests/golden/make_ribbon512_full.py [--procs 4]"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "..")
STEP_ENTRIES = (0, 10, 21, 31)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ribbon512_n200.json")


def step_energies():
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1903_00548_gb300 import workloads as W
    wl = W.ribbon512()
    # the energies of one benchmark step: 32 points spread over the 1024-point grid
    # (the same rule as bench.shard_energies with one rank)
    n = len(wl.energies)
    stride = max(1, n // 32)
    E = np.sort(wl.energies[(np.arange(32) * stride) % n])
    return [float(E[i]) for i in STEP_ENTRIES]


def one_energy(E):
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import pwqt_oracle as O
    from paper_1903_00548_gb300 import workloads as W
    wl = W.ribbon512()
    t0 = time.time()
    s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, wl.U)
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
    alt = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E, reciprocal=True)
    return {"E": E, "T": r.T, "R": r.R, "T_ds": r.T_ds, "n_open": [r.n_open_s, r.n_open_d],
            "node_n": np.asarray(r.node_n).tolist(), "defect": abs(r.T - r.T_ds),
            "bar": O.error_bar(r, alt), "T_reciprocal": alt.T, "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=4)
    a = ap.parse_args()
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "2"
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1903_00548_gb300 import workloads as W
    wl = W.ribbon512()
    Es = step_energies()
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(one_energy, Es)
    out = {"workload": "13 nm armchair ribbon, block 512, 200 nodes, random smooth potential (the benchmark workload)",
           "n": 2 * wl.n_bands, "n_nodes": wl.n_nodes, "step_entries": list(STEP_ENTRIES),
           "U": [float(u) for u in wl.U], "energies": res}
    for r in res:
        print(f"E={r['E']:.6f} T={r['T']:.12f} T_ds={r['T_ds']:.12f} bar={r['bar']:.2e} modes={r['n_open']} "
              f"({r['seconds']:.0f} s)", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
