"""Mixed-path refinement at every width of the correction solve.  The correction kernel
carries 16, 8, 4 or 2 right-hand sides per CTA, picked per refinement step from the
number of columns still refining, and updates one to eight 32 x 32 tiles per step; a
block size that is not a multiple of 32 (n = 72: three panels, the last eight rows
wide) exercises the zero fill of the edge tiles.  Batches of 1 .. 256 energies of the
13 nm ribbon at 36 bands per k (the bench's structure, a smaller basis) pass through all
widths; every energy must converge and agree with the FP64 path within the mixed path's
1e-8 bar on T and R."""
import numpy as np
import pytest

from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    wl = W.ribbon512()
    c = pwqt.Context(batch=256)
    assert c.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, 36) == 72
    c.set_extrinsic(0, W.random_smooth(12, 0.2, 5))
    E = np.sort(np.random.default_rng(3).uniform(wl.energies[0], wl.energies[-1], 256))
    ref = c.solve(0, E, pwqt.FP64)
    return pwqt, c, E, ref


@pytest.mark.parametrize("count", [1, 6, 24, 60, 128, 256])
def test_mixed_matches_fp64_at_every_width(ctx, count):
    pw, c, E, ref = ctx
    idx = np.linspace(0, len(E) - 1, count).astype(int)
    r = c.solve(0, E[idx], pw.MIXED)
    bad = pw.ST_MODE_COUNT | pw.ST_SINGULAR_PIVOT | pw.ST_IR_NO_CONVERGE
    assert np.all(r.status & bad == 0), r.status
    assert np.array_equal(r.n_open, ref.n_open[idx])
    assert np.max(np.abs(r.T - ref.T[idx])) <= 1e-8, np.max(np.abs(r.T - ref.T[idx]))
    assert np.max(np.abs(r.R - ref.R[idx])) <= 1e-8
