"""Density-matrix route of Sec. 3.3 on the GPU (pwqt_accumulate_density,
pwqt_get_density_matrix, pwqt_density_grid) against the oracle.

The density-matrix blocks are compared element by element when both sides use
the same Bloch waves (pwqt_set_enhancement with the oracle's coefficients); they
are sums of conj(c) c over injected modes, so like the node density they carry
the kappa * u_64 rounding of the coefficients along the basis' near-null
directions and are compared at RHO_TOL = 1e-7 of their largest element.  The
real-space density n(r) does not see those directions (a physical quantity) and
is compared at GRID_TOL = 1e-9 of its largest value; it is also basis-invariant,
so the GPU's own Bloch waves (which differ from the oracle's by a phase per
band) must give the same n(r)."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-7
GRID_TOL = 1e-9
MU_S, MU_D, KT = 1.0, 0.9, 0.025852


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def _groups(basis):
    return [(g["mx"], g["mz"], g["C"]) for g in basis.groups]


def _ctx(pw, s, **kw):
    ctx = pw.Context(**kw)
    ctx.set_enhancement(s.basis.cell, s.basis.eps, _groups(s.basis))
    ctx.set_extrinsic(0, s.U)
    return ctx


def _oracle(s, Es, w):
    cache = {}
    res = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, float(E), cache=cache) for E in Es]
    return res, O.density_matrix(res, w, MU_S, MU_D, KT)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module")
def chain():
    from tests.oracle_fixtures import chain_system
    s = chain_system()
    Es = np.array([0.13, 0.41, 0.77, 0.95, 1.18, 1.52])
    w = np.linspace(0.02, 0.07, len(Es))
    res, (rd, ru) = _oracle(s, Es, w)
    return s, Es, w, res, rd, ru


@pytest.fixture(scope="module")
def ribbon():
    from tests.oracle_fixtures import small_ribbon_system
    s = small_ribbon_system()
    Es = np.array([0.6, 1.1, 1.7])
    w = np.array([0.05, 0.04, 0.03])
    res, (rd, ru) = _oracle(s, Es, w)
    return s, Es, w, res, rd, ru


def test_chain_density_matrix_matches_oracle(pw, chain):
    s, Es, w, res, rd, ru = chain
    ctx = _ctx(pw, s)
    st = ctx.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.FP64)
    assert np.all(st & pw.ST_MODE_COUNT == 0)
    grd, gru = ctx.density_matrix(0)
    assert _rel(grd, rd) < RHO_TOL, _rel(grd, rd)
    assert _rel(gru, ru) < RHO_TOL, _rel(gru, ru)
    # the diagonal blocks are Hermitian by construction on both sides
    assert np.max(np.abs(grd - np.conj(np.transpose(grd, (0, 2, 1))))) <= 1e-14 * np.max(np.abs(grd))


def test_chain_density_grid_matches_both_oracle_routes(pw, chain):
    s, Es, w, res, rd, ru = chain
    ctx = _ctx(pw, s)
    ctx.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.FP64)
    g = ctx.density_grid(0, 1, 9)
    fast = O.density_from_matrix(s.basis, rd, ru, 1, 9)
    naive = O.density_naive(s.basis, res, w, MU_S, MU_D, KT, 1, 9)
    assert g.shape == fast.shape
    assert _rel(g, fast) < GRID_TOL, _rel(g, fast)
    assert _rel(g, naive) < GRID_TOL, _rel(g, naive)
    assert np.all(g > 0)


def test_ribbon_density_matrix_and_grid(pw, ribbon):
    s, Es, w, res, rd, ru = ribbon
    ctx = _ctx(pw, s)
    ctx.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.FP64)
    grd, gru = ctx.density_matrix(0)
    assert _rel(grd, rd) < RHO_TOL, _rel(grd, rd)
    assert _rel(gru, ru) < RHO_TOL, _rel(gru, ru)
    # several x tiles and z-plane groups with ragged ends
    for nx, nz in ((6, 7), (37, 5)):
        g = ctx.density_grid(0, nx, nz)
        ref = O.density_from_matrix(s.basis, rd, ru, nx, nz)
        assert g.shape == ref.shape
        assert _rel(g, ref) < GRID_TOL, (nx, nz, _rel(g, ref))


def test_density_is_basis_invariant(pw, ribbon):
    # the GPU's own EPM Bloch waves differ from the oracle's by a phase per band:
    # rho changes, n(r) does not
    s, Es, w, res, rd, ru = ribbon
    ctx = pw.Context()
    cell = s.basis.cell
    ctx.assemble_intrinsic(cell, W.FormFactor(), 28.0, 12)
    ctx.set_extrinsic(0, s.U)
    ctx.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.FP64)
    g = ctx.density_grid(0, 6, 7)
    ref = O.density_from_matrix(s.basis, rd, ru, 6, 7)
    assert _rel(g, ref) < 1e-8, _rel(g, ref)


def test_mixed_precision_density(pw, chain):
    s, Es, w, res, rd, ru = chain
    ctx = _ctx(pw, s)
    st = ctx.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.MIXED)
    assert np.all(st == 0), st
    g = ctx.density_grid(0, 1, 9)
    ref = O.density_from_matrix(s.basis, rd, ru, 1, 9)
    assert _rel(g, ref) < 1e-8, _rel(g, ref)


def test_accumulation_is_linear_and_batch_independent(pw, chain):
    s, Es, w, res, rd, ru = chain
    one = _ctx(pw, s)
    one.accumulate_density(0, Es, w, MU_S, MU_D, KT, pw.FP64)
    rd1, ru1 = one.density_matrix(0)
    # two calls with half the weights, and batches of two energies per launch
    two = _ctx(pw, s, batch=2)
    two.accumulate_density(0, Es, w / 2, MU_S, MU_D, KT, pw.FP64)
    two.accumulate_density(0, Es, w / 2, MU_S, MU_D, KT, pw.FP64)
    rd2, ru2 = two.density_matrix(0)
    assert _rel(rd2, rd1) < 1e-13 and _rel(ru2, ru1) < 1e-13
    # reset zeroes it; a new potential discards it
    two.density_reset(0)
    rd3, _ = two.density_matrix(0)
    assert np.all(rd3 == 0)
    two.set_extrinsic(0, s.U)
    with pytest.raises(pw.PwqtError):
        two.density_matrix(0)


def test_density_argument_errors(pw, chain):
    s, Es, w, res, rd, ru = chain
    ctx = _ctx(pw, s)
    with pytest.raises(pw.PwqtError):
        ctx.density_grid(0, 1, 4)          # nothing accumulated yet
    with pytest.raises(pw.PwqtError):
        ctx.accumulate_density(0, Es, w, MU_S, MU_D, -1.0)
    with pytest.raises(pw.PwqtError):
        ctx.accumulate_density(0, Es, np.full(len(Es), np.nan), MU_S, MU_D, KT)
    with pytest.raises(pw.PwqtError):
        ctx.accumulate_density(5, Es, w, MU_S, MU_D, KT)   # unknown system
    ctx.accumulate_density(0, Es[:1], w[:1], MU_S, MU_D, KT)
    with pytest.raises(pw.PwqtError):
        ctx.density_grid(0, 0, 4)
    # no energies: nothing added
    ctx.accumulate_density(0, Es[:0], w[:0], MU_S, MU_D, KT)
