"""Writes block512_n8.json, the expected values of tests/test_gpu_block512.py.

Test infrastructure: calls only the oracle (oracle/pwqt_oracle.py) and the seeded
input generators.  The system is the block-512 workload's basis (13 nm armchair
ribbon, G_cut = 30 nm^-1, 256 bands at each of Gamma and Z, Gaussian form factor)
on an 8-node device with the workload's random smooth potential; the energies are
points 160 and 640 of the workload's 1024-point midpoint grid (two of the energies
a 32-energy bench step solves).  Stored per energy: T, R and T_ds (Eq. transmission
and the reflection of Sec. 3.2-3.3), the open-channel counts, the node densities
n_s, n_d (Sec. 3.3), and the oracle's own reciprocity defect |T - T_ds|.  Also
stored: the gap between the last kept band and the next one at Gamma and Z, so
that a test can assert the band cut is not inside a degenerate subspace (then any
correct eigensolver spans the same basis and these quantities do not depend on it).

Run from the repository root:  python tests/golden/make_block512.py
(about 4 minutes: the lead eigenproblems at block 512 dominate)."""
import json
import math
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import numpy as np  # noqa: E402

from oracle import pwqt_oracle as O  # noqa: E402
from paper_1903_00548_gb300 import workloads as W  # noqa: E402

N_NODES = 8
GRID_POINTS = (160, 640)


def main():
    wl = W.ribbon512(n_nodes=N_NODES)
    grid = W.ribbon512().energies
    s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, wl.U)
    gaps = []
    for k in (0.0, math.pi / wl.cell.Lz):
        eps, _, _, _ = O.epm_bands(wl.cell, wl.ff, k, wl.gcut, wl.n_bands + 1)
        gaps.append(float(eps[wl.n_bands] - eps[wl.n_bands - 1]))
    out = {"workload": "13 nm armchair ribbon, block 512, 8 nodes, random smooth potential",
           "n": int(s.blk["n"]), "n_nodes": N_NODES, "grid_points": list(GRID_POINTS),
           "U": [float(u) for u in wl.U], "band_cut_gaps_eV": gaps, "energies": []}
    cache = {}
    for gi in GRID_POINTS:
        E = float(grid[gi])
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E, cache=cache)
        out["energies"].append({"E": E, "T": r.T, "R": r.R, "T_ds": r.T_ds, "n_open": [r.n_open_s, r.n_open_d],
                                "node_n": np.asarray(r.node_n).tolist(), "defect": abs(r.T - r.T_ds)})
        print(f"E={E:.6f} T={r.T:.12f} R={r.R:.12f} T_ds={r.T_ds:.12f} modes={r.n_open_s},{r.n_open_d}", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "block512_n8.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, "gaps", gaps)


if __name__ == "__main__":
    main()
