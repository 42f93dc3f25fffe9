"""Pins of the oracle's Green's-function diagonal blocks (the NEGF form of Sec. 3.2).

For real E and Hermitian H, M, the spectral function of the open device is
i(G - G^H) = G (Gamma_s + Gamma_d) G^H, and each contact's broadening is the sum over
its injected traveling modes of 2 pi b b^H / |dE/dk| (b the injection vector of the
QTBM right-hand side).  So the diagonal blocks of the spectral function equal
pi sum_gamma g_gamma c_{gamma,i} c_{gamma,i}^H over the wave-function solutions of
Eq. qtbm_system with g = 2/|dE/dk| (Sec. 3.3), and their trace is the sum of the
source- and drain-injected node densities.  The wave-function side is the oracle's
banded/dense solve with the mode decomposition, an independent computation."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O
from tests.oracle_fixtures import chain_system, small_ribbon_system


def test_node_spectral_density_equals_injected_node_densities():
    # the chain's self-energies are accurate to ~1e-9 and its basis is redundant,
    # which the device Green's function amplifies to a few 1e-7
    for s, Es, tol in ((chain_system(), (0.3, 0.77, 1.2), 2e-6), (small_ribbon_system(), (0.6, 1.1), 1e-8)):
        for E in Es:
            r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
            _, dos = O.green_diagonal(s.blk, s.Vd, s.Vu, s.U, E)
            ref = r.node_n.sum(1)
            assert np.all(ref > 0)
            assert np.max(np.abs(dos - ref) / ref) < tol, (E, dos, ref)


def test_spectral_blocks_equal_mode_sums():
    # the full n x n blocks, not only their traces: a transposed or conjugated block
    # keeps the trace but fails here
    s = small_ribbon_system()
    for E in (0.6, 1.1):
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
        Gd, _ = O.green_diagonal(s.blk, s.Vd, s.Vu, s.U, E)
        spec = 1j * (Gd - np.conj(np.transpose(Gd, (0, 2, 1))))
        ref = np.pi * np.einsum("g,iag,ibg->iab", r.g, r.c, r.c.conj())
        assert np.max(np.abs(spec - ref)) < 1e-8 * np.max(np.abs(ref)), E


def test_green_diagonal_rejects_large_systems():
    s = small_ribbon_system()
    big = np.zeros((400, s.blk["n"], s.blk["n"]))
    with pytest.raises(ValueError):
        O.green_diagonal(s.blk, big, big[:-1], np.zeros(400), 0.6)


def _green_pins_hold(s, E):
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
    Gd, dos = O.green_diagonal(s.blk, s.Vd, s.Vu, s.U, E)
    ref_n = r.node_n.sum(1)
    spec = 1j * (Gd - np.conj(np.transpose(Gd, (0, 2, 1))))
    ref = np.pi * np.einsum("g,iag,ibg->iab", r.g, r.c, r.c.conj())
    return (np.max(np.abs(dos - ref_n) / ref_n) < 1e-8 and
            np.max(np.abs(spec - ref)) < 1e-8 * np.max(np.abs(ref)))


@pytest.mark.parametrize("kind", ["drain_sigma_dropped", "advanced", "transposed"])
def test_green_mistakes_are_caught(monkeypatch, kind):
    # each plants one mistake in the matrix the Green's function inverts (the
    # wave-function side is solved first, unmutated) and checks that a pin fails
    s = small_ribbon_system()
    E = 0.6
    assert _green_pins_hold(s, E)
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E)
    orig = O.global_matrix

    def bad(blk, Vd, Vu, E_, Sig_s, Sig_d):
        if kind == "drain_sigma_dropped":
            return orig(blk, Vd, Vu, E_, Sig_s, np.zeros_like(Sig_d))
        if kind == "advanced":
            return orig(blk, Vd, Vu, E_, Sig_s.conj().T, Sig_d.conj().T)
        return orig(blk, Vd, Vu, E_, Sig_s, Sig_d).T

    monkeypatch.setattr(O, "solve_energy", lambda *a, **k: r)
    monkeypatch.setattr(O, "global_matrix", bad)
    assert not _green_pins_hold(s, E)
