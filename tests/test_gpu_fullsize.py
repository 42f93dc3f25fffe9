"""The block-512 workload at full size (13 nm ribbon, 200 nodes) in the launch
configuration the bench times (mixed path, 32 energies per launch), checked by
properties that hold at any size, since the oracle's banded solve takes minutes
per energy there: refinement reaches its stopping rule, flux is conserved (T + R
equals the number of injected source modes), transmission is reciprocal
(T_sd = T_ds), node densities are finite and positive, and the complex64-only
answer (PWQT_FP32) differs from the refined one by no more than its own residual
level allows."""
import numpy as np
import pytest

from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def test_full_size_mixed_batch_properties(pw):
    import bench
    wl = W.ribbon512()
    E = bench.shard_energies(wl.energies, 32, 0, 1)
    ctx = pw.Context(batch=32)
    n = ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    assert n == 512
    ctx.set_extrinsic(0, wl.U)
    res = ctx.solve(0, E, pw.MIXED)
    ok = (res.status & ~(pw.ST_NEAR_UNIT | pw.ST_DEGENERATE)) == 0
    assert ok.sum() >= 30, res.status
    assert np.all(res.resid[ok] <= 1e-8), res.resid
    ms = res.n_open[:, 0].astype(float)
    assert np.all(ms[ok] >= 1)
    # flux conservation and reciprocity at the level the refinement reaches
    assert np.max(np.abs(res.T + res.R - ms)[ok] / ms[ok]) < 1e-7
    assert np.max(np.abs(res.T - res.T_ds)[ok] / ms[ok]) < 1e-7
    assert np.all(np.isfinite(res.node_n)) and np.all(res.node_n[ok] > 0)
    # complex64 alone: within its residual level of the refined transmission
    r32 = ctx.solve(0, E[:8], pw.FP32)
    assert np.all(np.abs(r32.T - res.T[:8]) <= np.maximum(20 * r32.resid, 1e-6) * ms[:8])
