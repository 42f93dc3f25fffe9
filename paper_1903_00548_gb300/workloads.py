"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only builds inputs: cell geometry, pseudopotential form-factor
parameters, node potentials and energy grids. It holds none of the method's
arithmetic (no Fourier transforms, no matrix elements, no solves).

The paper's own inputs (Kurokawa C/H pseudopotentials, the 25-aGNR FET
geometry of Sec. 5) are not available; these seeded stand-ins have the same
structure: a periodic supercell along the transport direction z, a local
Gaussian form factor v(q) (Sec. 2.1, Eq. local_epp), N nodes at the supercell
boundaries (Sec. 2.2), a device-scale potential that varies slowly between
nodes, and a grid of injection energies (Sec. 3.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# hbar^2 / (2 m_e) in eV nm^2 (free-electron mass).
HB2M = 0.0380998212


@dataclass(frozen=True)
class Cell:
    """One periodic supercell (Sec. 2.1, Fig. structure).

    dim   : 1 (chain along z) or 2 (ribbon in the x-z plane, periodic
            supercell with vacuum in x).
    Lz    : supercell length along transport (nm); nodes sit at z_i = i*Lz.
    Lx    : transverse supercell width (nm); 1.0 for dim == 1.
    atoms : (n_atoms, 2) array of (x, z) positions in nm.
    omega0: reference volume per atom (nm^dim) of the form-factor
            normalisation V_G = (omega0 / Omega_cell) sum_a v(|G|) e^{-iG.R_a}.
    """
    dim: int
    Lz: float
    Lx: float
    atoms: np.ndarray
    omega0: float

    @property
    def omega_cell(self) -> float:
        return self.Lz * self.Lx


@dataclass(frozen=True)
class FormFactor:
    """Gaussian local pseudopotential v(q) = v0 * exp(-q^2 / (2 sigma^2)) (eV, nm^-1)."""
    v0: float = -5.0
    sigma: float = 8.0


def chain_cell(a: float = 0.4) -> Cell:
    """1D periodic chain, one atom per cell of length a."""
    return Cell(dim=1, Lz=a, Lx=1.0, atoms=np.array([[0.0, 0.0]]), omega0=a)


def armchair_ribbon_cell(n_lines: int, a: float = 0.246, vacuum: float = 1.0) -> Cell:
    """Armchair ribbon with n_lines dimer lines across x (carbon-like, no H).

    The dimer lines run along z (transport); their spacing across the ribbon is
    a/2 and the transport period is sqrt(3)*a (three C-C bonds).  Width
    (n_lines-1)*a/2; vacuum on both sides in x.
    """
    acc = a / math.sqrt(3.0)
    Lz = 3.0 * acc
    dx = 0.5 * a
    width = (n_lines - 1) * dx
    Lx = width + 2.0 * vacuum
    pos = []
    for j in range(n_lines):
        x = vacuum + j * dx
        if j % 2 == 0:
            pos += [(x, 0.0), (x, acc)]
        else:
            pos += [(x, 1.5 * acc), (x, 2.5 * acc)]
    omega0 = math.sqrt(3.0) * a * a / 2.0
    return Cell(dim=2, Lz=Lz, Lx=Lx, atoms=np.array(pos, dtype=np.float64), omega0=omega0)


def ribbon_lines_for_width(width_nm: float, a: float = 0.246) -> int:
    return int(round(width_nm / (0.5 * a))) + 1


# ----------------------------------------------------------------------------
# node potentials (extrinsic potential energy U_i at node i, eV)
# ----------------------------------------------------------------------------

def linear_drop(n_nodes: int, drop_eV: float) -> np.ndarray:
    """U = 0 at node 1, falling linearly to -drop at node N (leads flat beyond)."""
    t = np.linspace(0.0, 1.0, n_nodes)
    return -drop_eV * t


def random_smooth(n_nodes: int, amp_eV: float = 0.3, seed: int = 20190301,
                  n_modes: int = 8) -> np.ndarray:
    """Seeded smooth potential U(z) = amp * s(z) / max|s|, zero at both ends.

    s(z) = sum_{j=1..n_modes} a_j sin(j pi z / L_dev), a_j ~ N(0,1)/j^2.
    The end values are zero, so both leads sit at U = 0.
    """
    rng = np.random.default_rng(seed)
    aj = rng.standard_normal(n_modes) / (np.arange(1, n_modes + 1) ** 2)
    t = np.linspace(0.0, 1.0, n_nodes)
    s = np.zeros(n_nodes)
    for j in range(1, n_modes + 1):
        s += aj[j - 1] * np.sin(j * math.pi * t)
    m = np.max(np.abs(s))
    return amp_eV * s / m if m > 0 else s


def midpoint_grid(e_lo: float, e_hi: float, n: int) -> np.ndarray:
    """E_j = e_lo + (j + 1/2) dE; avoids the band-edge singularities at grid ends."""
    de = (e_hi - e_lo) / n
    return e_lo + (np.arange(n) + 0.5) * de


def seeded_energy_sample(energies: np.ndarray, k: int, seed: int = 7) -> np.ndarray:
    """A seeded subset of k energies, sorted, always including both grid ends."""
    rng = np.random.default_rng(seed)
    n = len(energies)
    if k >= n:
        return energies.copy()
    idx = set([0, n - 1])
    while len(idx) < k:
        idx.add(int(rng.integers(0, n)))
    return energies[np.array(sorted(idx))]


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    cell: Cell
    ff: FormFactor
    gcut: float          # plane-wave cutoff |k + G| <= gcut (nm^-1)
    n_bands: int         # bands kept per enhancement k-point (Gamma and Z): n = 2*n_bands
    n_nodes: int
    energies: np.ndarray
    U: np.ndarray        # potential energy at nodes 1..N (eV); leads flat at U[0], U[-1]
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 2 * self.n_bands


# Conduction-band edge of the 1.5 nm ribbon: the minimum over Gamma and Z of
# band index 52 (the 53rd band; 26 carbon-like atoms x 4 electrons fill 52
# spin-degenerate bands).  Written by oracle/derive_workload_constants.py.
RIBBON15_G45_ECB = 15.4042629215437
RIBBON15_G60_ECB = 15.404261893989412
# Bottom of band index 64 (minimum over Gamma and Z) of the 13 nm armchair ribbon at
# G_cut = 30 nm^-1.  Written by oracle/derive_workload_constants.py.
RIBBON13_G30_E64 = 3.204472869713024


def chain8(n_nodes: int = 20, n_energies: int = 64) -> Workload:
    """Config: 1D chain a=0.4 nm, ~30 plane waves, 8 enhancement functions/node,
    20 nodes, 64 energies over 0..2 eV, linear 0.1 V drop."""
    cell = chain_cell(0.4)
    gcut = 15.25 * 2.0 * math.pi / 0.4
    return Workload("chain8", cell, FormFactor(), gcut, 4, n_nodes,
                    midpoint_grid(0.0, 2.0, n_energies), linear_drop(n_nodes, 0.1),
                    notes="1D chain, linear 0.1 V drop")


def _ribbon(name, gcut, n_bands, n_nodes, n_energies, ecb, width=1.5, seed=20190301):
    cell = armchair_ribbon_cell(ribbon_lines_for_width(width))
    e_lo, e_hi = (ecb - 0.1, ecb + 1.0) if ecb is not None else (0.0, 1.1)
    return Workload(name, cell, FormFactor(), gcut, n_bands, n_nodes,
                    midpoint_grid(e_lo, e_hi, n_energies),
                    random_smooth(n_nodes, 0.3, seed),
                    notes=f"armchair ribbon {width} nm, random smooth U <= 0.3 eV")


def ribbon256(n_nodes: int = 200, n_energies: int = 1024) -> Workload:
    """Config: 1.5 nm ribbon, block 256, 200 nodes, 1024 energies, complex128."""
    return _ribbon("ribbon256", 45.0, 128, n_nodes, n_energies, RIBBON15_G45_ECB)


def ribbon512(n_nodes: int = 200, n_energies: int = 1024) -> Workload:
    """Block-512 workload: 13 nm armchair ribbon (214 atoms per cell), 256 Bloch waves
    at Gamma and at Z (G_cut = 30 nm^-1), 200 nodes, 1024 energies on
    [E_64 - 0.1, E_64 + 1.0] eV (about 45 open channels per contact).

    The PU basis of 256 bands per k-point on the 1.5 nm ribbon (26 atoms) is
    numerically redundant (smallest/largest eigenvalue of M(k) ~ 4e-10, lead pencil
    cond ~ 1e16); on this wider ribbon the same block size keeps ~1.2 bands per atom
    (M(k) ratio ~ 2e-5, lead pencil cond ~ 4e6)."""
    cell = armchair_ribbon_cell(ribbon_lines_for_width(13.0))
    e0 = RIBBON13_G30_E64
    return Workload("ribbon512", cell, FormFactor(), 30.0, 256, n_nodes,
                    midpoint_grid(e0 - 0.1, e0 + 1.0, n_energies),
                    random_smooth(n_nodes, 0.3, 20190301),
                    notes="armchair ribbon 13 nm, block 512, random smooth U <= 0.3 eV")


def ribbon256_wide(n_nodes: int = 200, n_energies: int = 1024) -> Workload:
    """Block 256 on the 13 nm ribbon (128 Bloch waves at Gamma and at Z, G_cut = 30
    nm^-1), 200 nodes, the block-512 workload's energy window and potential.  The
    batching configuration (energies x bias points, mixed precision) runs here: on the
    1.5 nm ribbon the block-256 basis is too redundant for complex64 factors to refine
    (M(k) eigenvalue ratio 4e-7; refinement stalls above 1e-6)."""
    wl = ribbon512(n_nodes, n_energies)
    wl.name, wl.n_bands = "ribbon256_wide", 128
    wl.notes = "armchair ribbon 13 nm, block 256, random smooth U <= 0.3 eV"
    return wl


def ribbon512_narrow(n_nodes: int = 200, n_energies: int = 1024) -> Workload:
    """The 1.5 nm ribbon at G_cut = 60 nm^-1 with 256 bands per k-point (block 512):
    kept to document the numerically redundant basis (not a benchmark workload)."""
    return _ribbon("ribbon512_narrow", 60.0, 256, n_nodes, n_energies, RIBBON15_G60_ECB)


def small_ribbon(n_bands: int = 16, n_nodes: int = 8, n_energies: int = 8,
                 gcut: float = 30.0, width: float = 0.5) -> Workload:
    """A narrow ribbon small enough for dense oracle solves (tests)."""
    cell = armchair_ribbon_cell(ribbon_lines_for_width(width))
    return Workload(f"ribbon_w{width}_n{2*n_bands}", cell, FormFactor(), gcut, n_bands,
                    n_nodes, midpoint_grid(0.0, 1.0, n_energies),
                    random_smooth(n_nodes, 0.3, 11), notes="small ribbon for tests")


def bias_points(wl: Workload, n_bias: int = 8, step_eV: float = 0.05) -> list:
    """Bias points of a workload (the batching configuration: energies x bias points):
    node potentials U_q = U + a linear drop of V_q = q * step_eV (q < n_bias, 0..0.35 V
    by default); the source lead stays at U(0), the drain lead sits at U(N) - V_q, so
    every bias point needs its own drain self-energies at energy E + V_q."""
    return [wl.U + linear_drop(wl.n_nodes, q * step_eV) for q in range(n_bias)]
