"""Degenerate traveling modes (Sec. 3.1): a 2D cell without crystal potential whose
Bloch basis is symmetric under x -> -x (plane waves G_x in {0, +b_x, -b_x} at Gamma
and at Z), so every +b_x channel has a -b_x partner at the same lambda and with the
same velocity.  The mode-resolved transmission needs those pairs made flux
orthogonal; a solver that takes one of them for a duplicate loses a channel.

Pristine device: T must equal the number of open channels counted with their
multiplicity (3 above the +-b_x band bottom, 1 below), per-mode T_gamma = 1; with a
potential: T, R, T_ds against the oracle (which flux-orthogonalises by
diagonalising the velocity form) within 1e-9 relative or four times its own error
bar.  The energies with degenerate sets carry PWQT_ST_DEGENERATE."""
import numpy as np
import pytest

from paper_1903_00548_gb300 import workloads as W
from tests.oracle_fixtures import symmetric_empty_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def _ctx(pw, cell, s):
    ctx = pw.Context()
    ctx.set_enhancement(cell, s.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in s.basis.groups])
    ctx.set_extrinsic(0, s.U)
    return ctx


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_pristine_degenerate_channels_all_transmit(pw, prec):
    cell, s = symmetric_empty_lattice(np.zeros(6))
    ctx = _ctx(pw, cell, s)
    E = np.array([1.0, 6.5, 7.5, 9.0])
    r = ctx.solve(0, E, getattr(pw, prec))
    assert np.all(r.status & (pw.ST_MODE_COUNT | pw.ST_SINGULAR_PIVOT | pw.ST_IR_NO_CONVERGE) == 0), r.status
    assert list(r.n_open[:, 0]) == [1, 3, 3, 3]
    assert np.all(np.abs(r.T - r.n_open[:, 0]) < 1e-8), r.T
    assert np.all(np.abs(r.R) < 1e-8)
    assert np.all(r.status[1:] & pw.ST_DEGENERATE), r.status         # the +-b_x pairs were treated as sets


def test_degenerate_channels_with_potential_match_oracle(pw):
    from tests.test_gpu_parity import _oracle_results
    U = W.random_smooth(8, 0.4, 21)
    cell, s = symmetric_empty_lattice(U)
    ctx = _ctx(pw, cell, s)
    E = np.array([6.4, 7.1, 8.2, 9.3])
    ref = _oracle_results(s, E)
    for prec, tol in (("FP64", 1e-9), ("MIXED", 1e-8)):
        r = ctx.solve(0, E, getattr(pw, prec))
        for e, ro in enumerate(ref):
            assert tuple(r.n_open[e]) == (ro.n_open_s, ro.n_open_d)
            t = max(tol * (max(1.0, ro.n_open_s) if prec == "FP64" else 1.0), 4 * ro.bar)
            for key in ("T", "R", "T_ds"):
                assert abs(getattr(r, key)[e] - getattr(ro, key)) <= t, (prec, E[e], key, getattr(r, key)[e], getattr(ro, key))
