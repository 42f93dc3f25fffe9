"""Pins of the oracle's open-boundary treatment (Sec. 3.1-3.4) and band
reconstruction (Sec. 5.1) against invariants the physics fixes."""
import math

import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W
from tests.oracle_fixtures import (chain_system, open_channels_from_bands, small_ribbon_system,
                                   symmetric_empty_lattice, with_potential)


def _reconstruction_error(s):
    blk, basis = s.blk, s.basis
    err = 0.0
    for gi, kp in ((0, 0.0), (1, math.pi / blk["L"])):
        ev = O.pu_bands(blk, kp)
        for e in basis.groups[gi]["eps"]:
            err = max(err, np.min(np.abs(ev - e)) / max(1.0, abs(e)))
    return err


def test_band_reconstruction_exact_at_enhancement_points():
    # The Bloch waves at Gamma (Z) are exactly representable in the PU basis at
    # k' = 0 (pi/L), so their plane-wave energies are eigenvalues of H(k') c = E M(k') c.
    # Exact when the plane-wave basis is converged (the eigenvalue substitution of
    # App. A assumes exact Bloch eigenfunctions of the local Hamiltonian).
    assert _reconstruction_error(chain_system()) < 1e-9
    assert _reconstruction_error(small_ribbon_system(n_bands=8, n_nodes=3, gcut=55.0)) < 1e-9
    # ... and the residual mismatch shrinks with the plane-wave cutoff
    e28 = _reconstruction_error(small_ribbon_system(n_bands=8, n_nodes=3, gcut=28.0))
    e40 = _reconstruction_error(small_ribbon_system(n_bands=8, n_nodes=3, gcut=40.0))
    assert e40 < 1e-2 * e28


def test_band_reconstruction_empty_lattice():
    cell = W.chain_cell(0.4)
    s = O.build_system(cell, W.FormFactor(v0=0.0), 9.25 * 2 * math.pi / 0.4, 3, np.zeros(3))
    # empty lattice at k'=Gamma: the three lowest free-electron levels at k=0
    # (0 and the +-G pair) must be reproduced (the degenerate pair as a pair).
    ev = O.pu_bands(s.blk, 0.0)
    for e in s.basis.groups[0]["eps"]:
        assert np.min(np.abs(ev - e)) < 1e-9 * max(1.0, e)


def test_hellmann_feynman_velocity_matches_band_slope():
    s = chain_system()
    blk = s.blk
    L = blk["L"]
    for E in (0.3, 1.0):
        lm = O.lead_modes(blk, E)
        for j in np.flatnonzero(lm.traveling):
            k = np.angle(lm.lam[j]) / L
            h = 1e-5
            ep = O.pu_bands(blk, k + h)
            em = O.pu_bands(blk, k - h)
            b = np.argmin(np.abs(O.pu_bands(blk, k) - E))
            slope = (ep[b] - em[b]) / (2 * h)
            assert abs(slope - lm.dEdk[j]) < 1e-6 * max(1.0, abs(slope))


@pytest.mark.parametrize("which", ["chain", "ribbon"])
def test_lead_modes_invariants(which):
    s = chain_system() if which == "chain" else small_ribbon_system()
    blk = s.blk
    n, L = blk["n"], blk["L"]
    energies = (0.3, 1.0, 1.5) if which == "chain" else (0.3, 0.9, 2.2)
    for E in energies:
        lm = O.lead_modes(blk, E)
        trav = lm.traveling
        assert np.all(np.abs(np.abs(lm.lam[trav]) - 1.0) < 1e-10)
        # normalisation c^H M(lambda) c = L/2pi for traveling modes
        for j in np.flatnonzero(trav):
            c = lm.C[:, j]
            Ml = O._m_lambda(blk, lm.lam[j])
            assert abs(np.vdot(c, Ml @ c) - L / (2 * math.pi)) < 1e-10
        # pencil residual of every eigenpair
        for j in range(2 * n):
            c, lam = lm.C[:, j], lm.lam[j]
            r = (lm.Km / lam + lm.K0 + lam * lm.Kp) @ c
            assert np.linalg.norm(r) < 1e-8 * max(1.0, abs(lam), 1 / abs(lam)) * np.linalg.norm(lm.K0)
        # Sec. 3.1: exactly n out-flow modes per contact, from the physics alone
        # (decay into the lead or velocity out of the device), and every traveling
        # mode leaves through exactly one contact
        od, os_ = O.out_flow_mask(lm, "d"), O.out_flow_mask(lm, "s")
        assert od.sum() == n and os_.sum() == n
        assert not np.any(od & os_) and np.all(od | os_)
        cd = O.contact(lm, "d")
        cs = O.contact(lm, "s")
        assert not cd.mode_sorted and not cs.mode_sorted
        # X = B Lambda B^-1 solves the matrix quadratic of the semi-infinite lead
        Xd = cd.B @ np.diag(cd.lam_out) @ np.linalg.inv(cd.B)
        Xs = cs.B @ np.diag(cs.lam_out) @ np.linalg.inv(cs.B)
        sc = np.linalg.norm(lm.K0)
        assert np.linalg.norm(lm.Km + lm.K0 @ Xd + lm.Kp @ Xd @ Xd) < 1e-8 * sc * max(1, np.linalg.norm(Xd)) ** 2
        assert np.linalg.norm(lm.Kp + lm.K0 @ Xs + lm.Km @ Xs @ Xs) < 1e-8 * sc * max(1, np.linalg.norm(Xs)) ** 2
        # open channels: in-flow traveling at the source == right-moving band crossings
        assert cs.c_in.shape[1] == cd.c_in.shape[1] == open_channels_from_bands(blk, E, nk=1501)


def test_pristine_chain_plateaus():
    s0 = chain_system()
    s = with_potential(s0, np.zeros(20))
    for E in (0.05, 0.3, 0.9, 1.5):       # inside the lowest band (-0.111 .. 1.596 eV)
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert r.n_open_s == 1
        assert abs(r.T - 1.0) < 1e-9 and abs(r.R) < 1e-9
        nn = r.node_n[:, 0]
        assert np.max(np.abs(nn - nn.mean())) < 1e-6 * nn.mean()
    for E in (1.7, 2.5):                  # inside the gap (1.596 .. 3.049 eV)
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert r.n_open_s == 0 and r.T == 0.0


def test_pristine_ribbon_integer_transmission():
    s0 = small_ribbon_system()
    s = with_potential(s0, np.zeros(6))
    seen = set()
    for E in np.linspace(0.2, 2.6, 9):
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert abs(r.T - r.n_open_s) < 1e-8 * max(1, r.n_open_s)
        assert np.max(np.abs(r.T_modes - 1.0)) < 1e-8 if r.n_open_s else True
        seen.add(r.n_open_s)
    assert len(seen) >= 2


@pytest.mark.parametrize("which", ["chain", "ribbon"])
def test_current_conservation_and_reciprocity(which):
    s = chain_system() if which == "chain" else small_ribbon_system()
    energies = (0.2, 0.7, 1.2, 1.55) if which == "chain" else (0.4, 1.1, 1.9, 2.5)
    for E in energies:
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        if r.n_open_s:
            assert np.max(np.abs(r.T_modes + r.R_modes - 1.0)) < 1e-8
        assert abs(r.T - r.T_ds) < 1e-8 * max(1.0, r.T)


def test_shift_invariance():
    s0 = chain_system()
    U = s0.U
    c = 0.23
    s1 = with_potential(s0, U + c)
    for E in (0.4, 1.1):
        r0 = O.solve_energy(s0.blk, s0.Vd, s0.Vu, s0.U, E)
        r1 = O.solve_energy(s1.blk, s1.Vd, s1.Vu, s1.U, E + c)
        assert abs(r0.T - r1.T) < 1e-9
        assert np.max(np.abs(r0.node_n - r1.node_n)) < 1e-7 * max(1.0, np.max(r0.node_n))


def test_dense_and_banded_global_solves_agree():
    s = small_ribbon_system()
    for E in (0.6, 1.7):
        rd = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E, dense_limit=10 ** 9)
        rb = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E, dense_limit=0)
        assert abs(rd.T - rb.T) < 1e-9
        assert np.max(np.abs(rd.c - rb.c)) < 1e-7 * np.max(np.abs(rd.c))


def test_linear_drop_blocks_transport_above_drain_band():
    # 0.1 V drop: the drain band top is 1.596 - 0.1 eV; no transmission above it.
    s = chain_system()
    for E in (1.52, 1.58):
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert r.n_open_s == 1 and abs(r.T) < 1e-12 and abs(r.R - 1.0) < 1e-8
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.5)
    assert 0.0 < r.T <= 1.0 + 1e-12


def test_density_routes_agree():
    # Eq. density_3d (naive, wavefunctions on the grid) == Eq. density_3d_fast
    # (density matrix in the Bloch basis): an exact algebraic identity.
    for s, Es in ((chain_system(), (0.3, 0.8, 1.2)), (small_ribbon_system(), (0.6, 1.3))):
        res = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E) for E in Es]
        w = np.full(len(Es), 0.05)
        kT = 0.025852
        nx = 6 if s.basis.cell.dim == 2 else 1
        dn = O.density_naive(s.basis, res, w, 1.0, 0.9, kT, nx, 7)
        rd, ru = O.density_matrix(res, w, 1.0, 0.9, kT)
        dm = O.density_from_matrix(s.basis, rd, ru, nx, 7)
        assert np.max(np.abs(dn - dm)) < 1e-11 * np.max(np.abs(dn))


def test_pristine_density_is_cell_periodic():
    s0 = chain_system()
    s = with_potential(s0, np.zeros(20))
    res = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E) for E in (0.3, 0.7)]
    rd, ru = O.density_matrix(res, np.full(2, 0.1), 5.0, 5.0, 0.025852)
    d = O.density_from_matrix(s.basis, rd, ru, 1, 9)[:, 0, :]
    assert np.max(np.abs(d - d[0][None, :])) < 1e-6 * np.max(d)


def test_caroli_transmission_equals_mode_resolved():
    # the Green's-function form (no mode decomposition at the drain) and the
    # wave-function form of Eq. transmission are the same number
    for s, Es in ((chain_system(), (0.3, 0.77, 1.2)), (small_ribbon_system(), (0.6, 1.1))):
        for E in Es:
            r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
            Tc = O.caroli_transmission(s.blk, s.Vd, s.Vu, s.U, E)
            assert abs(Tc - r.T) <= 1e-9 * max(1.0, r.T) + 4 * abs(r.T - r.T_ds), (E, Tc, r.T)


def test_block512_golden_values_are_physical():
    # the stored block-512 expectations (tests/golden/make_block512.py) obey flux
    # conservation and reciprocity, and the band cut of their basis is not degenerate
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "block512_n8.json")))
    assert g["n"] == 512 and min(g["band_cut_gaps_eV"]) > 1e-3
    for e in g["energies"]:
        ms = e["n_open"][0]
        assert ms == e["n_open"][1] and ms > 0
        assert abs(e["T"] + e["R"] - ms) < 1e-8 * ms
        assert abs(e["T"] - e["T_ds"]) < 1e-8 * ms
        nn = np.array(e["node_n"])
        assert nn.shape == (g["n_nodes"], 2) and np.all(nn > 0)


def test_full_size_golden_values_are_physical():
    # the stored 200-node expectations (tests/golden/make_ribbon512_full.py): flux
    # conservation, reciprocity, both pencils agreeing within the stored bar, positive
    # node densities, and the energies are the bench step's own
    import json
    import os

    import bench
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ribbon512_n200.json")))
    wl = W.ribbon512()
    assert g["n"] == 512 and g["n_nodes"] == 200 and np.allclose(g["U"], wl.U, rtol=0, atol=1e-15)
    E = bench.shard_energies(wl.energies, 32, 0, 1)
    for k, e in zip(g["step_entries"], g["energies"]):
        assert abs(E[k] - e["E"]) < 1e-12
        ms = e["n_open"][0]
        assert ms == e["n_open"][1] and ms > 0
        assert abs(e["T"] + e["R"] - ms) < 1e-8 * ms
        assert abs(e["T"] - e["T_ds"]) <= e["bar"] and abs(e["T"] - e["T_reciprocal"]) <= e["bar"] < 1e-8
        nn = np.array(e["node_n"])
        assert nn.shape == (200, 2) and np.all(nn > 0)


def test_reciprocal_pencil_gives_the_same_modes_and_transport():
    # the error-bar route of the oracle: QZ of the pencil for mu = 1/lambda must give the
    # same eigenvalues (to rounding) and, on the pristine chain, the same integer plateau
    s = chain_system()
    for kind in (True, "cayley"):
        for E in (0.3, 1.0):
            a = O.lead_modes(s.blk, E)
            b = O.lead_modes(s.blk, E, reciprocal=kind)
            # every finite eigenvalue has a partner in the other solve (nearest match)
            fa = a.lam[np.isfinite(a.lam) & (np.abs(a.lam) < 1e6)]
            fb = b.lam[np.isfinite(b.lam)]
            d = np.min(np.abs(fa[:, None] - fb[None, :]), axis=1)
            assert np.all(d <= 1e-7 * np.maximum(1.0, np.abs(fa))), (kind, d.max())
            assert a.traveling.sum() == b.traveling.sum()
        sp = with_potential(s, np.zeros(20))
        for E in (0.3, 0.9):
            r = O.solve_energy(sp.blk, sp.Vd, sp.Vu, sp.U, E, reciprocal=kind)
            assert abs(r.T - 1.0) < 1e-9 and abs(r.R) < 1e-9


def test_degenerate_traveling_pairs():
    # mirror-symmetric empty-lattice cell: the +-b_x channels are degenerate pairs with
    # equal velocities (Sec. 3.1).  Pristine: integer plateaus 1 / 3 with every mode fully
    # transmitted; with a potential: flux conservation per injected mode and reciprocity
    cell, s = symmetric_empty_lattice(np.zeros(6))
    for E, n_open in ((1.0, 1), (6.5, 3), (7.5, 3), (9.0, 3)):
        lm = O.lead_modes(s.blk, E)
        assert lm.n_degenerate_sets == (2 if n_open == 3 else 0)
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert r.n_open_s == n_open and abs(r.T - n_open) < 1e-9 and np.all(np.abs(r.T_modes - 1) < 1e-9)
    cell, s = symmetric_empty_lattice(W.random_smooth(8, 0.4, 21))
    for E in (6.4, 7.1, 8.2, 9.3):
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        assert r.n_open_s == 3
        assert np.max(np.abs(r.T_modes + r.R_modes - 1.0)) < 1e-9
        assert abs(r.T - r.T_ds) < 1e-9


def test_perturbation_spread_measures_conditioning():
    # the oracle's conditioning estimate: tiny where T is well determined (pristine chain
    # mid-band; the biased chain at 1.2 eV, where it grows in proportion to the
    # perturbation once that exceeds the solve's own rounding), and ~1e-8 at the chain
    # energy whose weakly evanescent modes make the contact ill-conditioned (there the
    # eigen-solve's rounding dominates whatever the perturbation)
    s0 = chain_system()
    sp = with_potential(s0, np.zeros(20))
    assert O.perturbation_spread(sp.blk, sp.U, 1.0) < 1e-11
    a = O.perturbation_spread(s0.blk, s0.U, 1.2, eps=1e-14)
    b = O.perturbation_spread(s0.blk, s0.U, 1.2, eps=1e-12)
    assert a < 1e-12 and b > 10 * a
    assert O.perturbation_spread(s0.blk, s0.U, 0.390625) > 1e-9
