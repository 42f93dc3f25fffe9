"""Shared, cached oracle systems for the tests (test infrastructure)."""
import functools
import math

import numpy as np

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W


@functools.lru_cache(maxsize=None)
def chain_system(n_nodes=20, drop=0.1, v0=-5.0):
    wl = W.chain8(n_nodes=n_nodes)
    U = W.linear_drop(n_nodes, drop)
    return O.build_system(wl.cell, W.FormFactor(v0=v0), wl.gcut, wl.n_bands, U)


@functools.lru_cache(maxsize=None)
def small_ribbon_system(n_bands=12, n_nodes=6, gcut=28.0, width=0.5, amp=0.3, seed=11):
    cell = W.armchair_ribbon_cell(W.ribbon_lines_for_width(width))
    U = W.random_smooth(n_nodes, amp, seed)
    return O.build_system(cell, W.FormFactor(), gcut, n_bands, U)


def with_potential(sys_, U):
    Vd, Vu = O.extrinsic_blocks(sys_.blk, U)
    return O.System(sys_.basis, sys_.elem, sys_.blk, np.asarray(U, float), Vd, Vu)


def open_channels_from_bands(blk, E, nk=4001):
    """Number of right-moving traveling channels at E counted from the PU band
    structure: crossings of E(k') = E with positive slope over one Brillouin zone."""
    L = blk["L"]
    ks = np.linspace(-math.pi / L, math.pi / L, nk)
    bands = np.array([O.pu_bands(blk, k) for k in ks])      # (nk, n)
    cnt = 0
    for b in range(bands.shape[1]):
        e = bands[:, b] - E
        s = np.sign(e)
        cnt += int(np.sum((s[:-1] < 0) & (s[1:] >= 0)))
    return cnt


def symmetric_empty_lattice(U, Lz=0.4, Lx=0.5):
    """A 2D cell without crystal potential and a Bloch basis symmetric under x -> -x:
    plane waves with G_x in {0, +b_x, -b_x} (G_z = 0) at Gamma and at Z, so every +b_x
    channel has a -b_x partner at the same lambda and with the same velocity (degenerate
    traveling modes, Sec. 3.1).  Returns (cell, oracle system with node potentials U)."""
    cell = W.Cell(dim=2, Lz=Lz, Lx=Lx, atoms=np.array([[0.0, 0.0]]), omega0=Lx * Lz)
    bx = 2 * math.pi / Lx
    mx, mz = np.array([0, 1, -1]), np.array([0, 0, 0])
    groups, eps, kz = [], [], []
    for k in (0.0, math.pi / Lz):
        e = O.HB2M * ((mx * bx) ** 2 + k ** 2)
        groups.append(dict(k=k, mx=mx, mz=mz, C=np.eye(3, dtype=complex), eps=e))
        eps.append(e)
        kz.append(np.full(3, k))
    basis = O.basis_from_coefficients(cell, np.concatenate(eps), np.concatenate(kz), groups)
    return cell, O.build_system(cell, W.FormFactor(v0=0.0), 0.0, 3, U, basis=basis)
