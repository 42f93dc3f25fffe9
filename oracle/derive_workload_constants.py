"""Derives the conduction-band-edge constants of the ribbon workloads.

Test infrastructure: run with `python -m oracle.derive_workload_constants`.  It
prints the minimum over Gamma and Z of band index 52 (the 53rd band; 26
carbon-like atoms with 4 electrons fill 52 spin-degenerate bands) of the
1.5 nm armchair ribbon at the two plane-wave cutoffs the ribbon workloads use.
The printed values are the RIBBON15_G*_ECB constants of
paper_1903_00548_gb300/workloads.py (inputs only: they place the energy window).
"""
import math

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W


def main():
    cell = W.armchair_ribbon_cell(W.ribbon_lines_for_width(1.5))
    for gcut in (45.0, 60.0):
        ecb = min(O.epm_bands(cell, W.FormFactor(), k, gcut, 53)[0][52]
                  for k in (0.0, math.pi / cell.Lz))
        print(f"RIBBON15_G{int(gcut)}_ECB = {float(ecb)!r}")


if __name__ == "__main__":
    main()
