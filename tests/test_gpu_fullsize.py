"""The block-512 workload at full size (13 nm ribbon, 200 nodes) in the launch
configuration the bench times (mixed path, 32 energies per launch).

Element by element against the oracle at four of the step's energies, whose
expected values tests/golden/make_ribbon512_full.py wrote by calling only the oracle
(banded LU of the 102400 x 102400 global system, minutes per energy): FP64 path
1e-9 relative on T, R, T_ds (times max(1, open channels)); mixed path with its
default stopping rule 1e-8 absolute; either widened only to four times the oracle's
own error bar at that energy (reciprocity defect and the spread between the two
pencil solves); node densities within 1e-7 of their largest value (coefficient
space, see tests/test_gpu_parity.py); open-channel counts exact.

And over all 32 energies of the step, by properties that hold at any size:
refinement reaches its stopping rule, flux is conserved (T + R equals the number of
injected source modes), transmission is reciprocal (T_sd = T_ds), node densities
are finite and positive, and the complex64-only answer (PWQT_FP32) differs from the
refined one by no more than its own residual level allows."""
import json
import os

import numpy as np
import pytest

from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ribbon512_n200.json")


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


@pytest.fixture(scope="module")
def step(pw):
    import bench
    wl = W.ribbon512()
    E = bench.shard_energies(wl.energies, 32, 0, 1)
    ctx = pw.Context(batch=32)
    n = ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    assert n == 512
    ctx.set_extrinsic(0, wl.U)
    return wl, E, ctx, ctx.solve(0, E, pw.MIXED)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_full_size_matches_oracle(pw, step, prec):
    g = json.load(open(GOLDEN))
    wl, E, ctx, res_mixed = step
    assert g["n_nodes"] == wl.n_nodes and np.allclose(wl.U, g["U"], rtol=0, atol=1e-15)
    idx = [int(np.argmin(np.abs(E - e["E"]))) for e in g["energies"]]
    assert all(abs(E[i] - e["E"]) < 1e-12 for i, e in zip(idx, g["energies"]))
    if prec == "MIXED":
        r, ks = res_mixed, idx                     # the very launch the bench times
    else:
        r, ks = ctx.solve(0, E[idx], pw.FP64), range(len(idx))
    bad = pw.ST_MODE_COUNT | pw.ST_SINGULAR_PIVOT | pw.ST_IR_NO_CONVERGE
    for k, ref in zip(ks, g["energies"]):
        assert r.status[k] & bad == 0, (prec, ref["E"], r.status[k])
        assert tuple(r.n_open[k]) == tuple(ref["n_open"]), (prec, ref["E"])
        scale = max(1.0, ref["n_open"][0]) if prec == "FP64" else 1.0
        tol = 1e-9 if prec == "FP64" else 1e-8
        t = max(tol * scale, 4.0 * ref["bar"])
        for key, got in (("T", r.T[k]), ("R", r.R[k]), ("T_ds", r.T_ds[k])):
            assert abs(got - ref[key]) <= t, (prec, ref["E"], key, got, ref[key], t)
        nn = np.array(ref["node_n"])
        assert np.max(np.abs(r.node_n[k] - nn)) <= 1e-7 * np.max(nn), (prec, ref["E"])


def test_full_size_mixed_batch_properties(pw, step):
    wl, E, ctx, res = step
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
