"""Block-512 parity against the oracle: the bench's basis (13 nm armchair ribbon,
256 bands at Gamma and Z, n = 512: four 128-row tensor-core tiles and sixteen
32-column panels per block) on an 8-node device, assembled by the library itself
as the bench does, at two energies of the bench's grid.  The expected values were
written by tests/golden/make_block512.py, which calls only the oracle (its lead
eigenproblems take minutes at this block size, too long to run here).

Tolerances as in the transmission parity tests: FP64 path, T, R, T_ds within 1e-9
relative (times max(1, open channels)); mixed path with its default stopping rule,
1e-8 absolute (the bar on T); either widened only to four times the oracle's own
reciprocity defect where that is larger; node densities (coefficient space, see the
parity tests) within 1e-7 of their largest value; open-channel counts exact."""
import json
import os

import numpy as np
import pytest

from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "block512_n8.json")


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


@pytest.fixture(scope="module")
def solved(pw):
    g = json.load(open(GOLDEN))
    wl = W.ribbon512(n_nodes=g["n_nodes"])
    assert np.allclose(wl.U, g["U"], rtol=0, atol=1e-15)
    E = np.array([e["E"] for e in g["energies"]])
    ctx = pw.Context(batch=32)
    assert ctx.assemble_intrinsic(wl.cell, wl.ff, wl.gcut, wl.n_bands) == g["n"]
    ctx.set_extrinsic(0, wl.U)
    return g, {p: ctx.solve(0, E, p) for p in (pw.FP64, pw.MIXED)}


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-9), ("MIXED", 1e-8)])
def test_block512_matches_oracle(pw, solved, prec, tol):
    g, res = solved
    r = res[getattr(pw, prec)]
    bad = pw.ST_MODE_COUNT | pw.ST_SINGULAR_PIVOT | pw.ST_IR_NO_CONVERGE
    assert np.all(r.status & bad == 0), r.status
    for e, ref in enumerate(g["energies"]):
        assert tuple(r.n_open[e]) == tuple(ref["n_open"]), e
        scale = max(1.0, ref["n_open"][0]) if prec == "FP64" else 1.0
        t = max(tol * scale, 4.0 * ref["defect"])
        for key, got in (("T", r.T[e]), ("R", r.R[e]), ("T_ds", r.T_ds[e])):
            assert abs(got - ref[key]) <= t, (prec, ref["E"], key, got, ref[key], t)
        nn = np.array(ref["node_n"])
        assert np.max(np.abs(r.node_n[e] - nn)) <= 1e-7 * np.max(nn), (prec, ref["E"])
