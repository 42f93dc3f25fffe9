"""The refinement residual r = B - A c of the Sec. 3.2 system on the tensor cores
(exact products of 7-bit integer slices, FP64 accuracy) against the float-float
residual on the FP32 pipes, and both refinement paths against the oracle.

PWQT_FP32 reports the residual of the complex64 solution without refining it, so
the two residual kinds evaluate ||B - A c|| / ||B|| of the same c (about 1e-6 here):
they must agree far below that level (float-float floor ~4e-10 at block 512, the
sliced residual ~3e-12).  With refinement, either kind must bring T within 1e-8
absolute of the oracle on the chain (several energies per launch, ragged 32-column
tiles of mode columns) and on the n = 72 ribbon (the 128-row tiles padded from 144
real rows)."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def _ctx(pw, sys_):
    ctx = pw.Context()
    ctx.set_enhancement(sys_.basis.cell, sys_.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in sys_.basis.groups])
    ctx.set_extrinsic(0, sys_.U)
    return ctx


def _oracle_T(sys_, Es):
    from tests.test_gpu_parity import _oracle_results
    return _oracle_results(sys_, Es)


@pytest.fixture(scope="module")
def chain():
    wl = W.chain8()
    return wl, O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, wl.U)


def test_sliced_and_float_float_residuals_agree(pw, chain):
    wl, s = chain
    ctx = _ctx(pw, s)
    E = wl.energies[4:60:4]
    ctx.set_residual(pw.RESIDUAL_FLOAT_FLOAT)
    ff = ctx.solve(0, E, pw.FP32)
    ctx.set_residual(pw.RESIDUAL_SLICED)
    sl = ctx.solve(0, E, pw.FP32)
    open_e = ff.n_open.sum(1) > 0                  # energies in the gap have nothing to solve
    assert open_e.sum() >= 10
    assert np.all(ff.resid[open_e] > 0) and np.all(sl.resid[open_e] > 0)
    assert np.all(sl.resid[~open_e] == ff.resid[~open_e])
    # same complex64 solutions (the factorisation does not depend on the residual kind)
    assert np.array_equal(ff.T, sl.T)
    assert np.all(np.abs(ff.resid - sl.resid) <= 1e-8 * ff.resid + 1e-12), (ff.resid, sl.resid)


@pytest.mark.parametrize("kind", ["RESIDUAL_SLICED", "RESIDUAL_FLOAT_FLOAT"])
def test_refinement_with_each_residual_matches_oracle(pw, chain, kind):
    wl, s = chain
    ctx = _ctx(pw, s)
    ctx.set_residual(getattr(pw, kind))
    ctx.set_refinement(1e-11, 0)
    E = wl.energies[1:64:3]
    r = ctx.solve(0, E, pw.MIXED)
    assert np.all(r.status == 0), r.status
    assert np.max(r.resid) <= 1e-11
    for e, ro in enumerate(_oracle_T(s, E)):
        bar = max(1e-8, 4 * ro.bar)
        assert abs(r.T[e] - ro.T) <= bar and abs(r.R[e] - ro.R) <= bar, (kind, E[e], r.T[e], ro.T)


def test_sliced_residual_on_padded_tiles(pw):
    # n = 72: 144 real rows padded to 256 (two 128-row tiles), K padded likewise
    from tests.oracle_fixtures import small_ribbon_system
    s = small_ribbon_system(n_bands=36, n_nodes=24, gcut=30.0)
    ctx = _ctx(pw, s)
    ctx.set_refinement(1e-11, 0)
    Es = np.array([0.4, 1.3, 2.1])
    r = ctx.solve(0, Es, pw.MIXED)
    assert np.all(r.status & ~pw.ST_NEAR_UNIT == 0), r.status
    assert np.max(r.resid) <= 1e-11
    for e, ro in enumerate(_oracle_T(s, Es)):
        bar = max(1e-8, 4 * ro.bar)
        assert abs(r.T[e] - ro.T) <= bar, (Es[e], r.T[e], ro.T)


def test_residual_kind_is_validated(pw, chain):
    wl, s = chain
    ctx = _ctx(pw, s)
    with pytest.raises(pw.PwqtError):
        ctx.set_residual(7)
