"""Derives the conduction-band-edge constants of the ribbon workloads.

Test infrastructure: run with `python -m oracle.derive_workload_constants`.  It
prints the minimum over Gamma and Z of band index 52 (the 53rd band; 26
carbon-like atoms with 4 electrons fill 52 spin-degenerate bands) of the
1.5 nm armchair ribbon at the two plane-wave cutoffs the ribbon workloads use.
It also prints the bottom of band index 64 of the 13 nm ribbon at G_cut = 30 nm^-1.
The printed values are the RIBBON*_ constants of paper_1903_00548_gb300/workloads.py
(inputs only: they place the energy windows).
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
    wide = W.armchair_ribbon_cell(W.ribbon_lines_for_width(13.0))
    e64 = min(O.epm_bands(wide, W.FormFactor(), k, 30.0, 65)[0][64] for k in (0.0, math.pi / wide.Lz))
    print(f"RIBBON13_G30_E64 = {float(e64)!r}")


if __name__ == "__main__":
    main()
