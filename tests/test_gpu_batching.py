"""Energies x bias points in one batched solve (pwqt_solve_multi): every (bias point,
energy) pair runs in the same launches, each job with its own system's node blocks,
and must give what the bias points give solved one by one (the per-energy arithmetic
does not depend on the batch it runs in), and what the oracle gives.

Bias points: the chain with linear drops of 0, 0.05 and 0.1 eV (Sec. 4: the solve
repeated per applied potential), the source lead at 0 and the drain lead at -V, so
the drain self-energies differ per bias point while the source ones are shared."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DROPS = (0.0, 0.05, 0.1)


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


@pytest.fixture(scope="module")
def chain_bias(pw):
    wl = W.chain8()
    basis = O.bloch_basis(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    ctx = pw.Context()
    ctx.set_enhancement(wl.cell, basis.eps, [(g["mx"], g["mz"], g["C"]) for g in basis.groups])
    Us = [W.linear_drop(wl.n_nodes, v) for v in DROPS]
    for q, U in enumerate(Us):
        ctx.set_extrinsic(q, U)
    return wl, basis, ctx, Us


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_batched_bias_points_equal_one_by_one(pw, chain_bias, prec):
    wl, basis, ctx, Us = chain_bias
    p = getattr(pw, prec)
    E = wl.energies[2:60:3]
    multi = ctx.solve_multi(list(range(len(Us))), E, p)
    for q in range(len(Us)):
        one = ctx.solve(q, E, p)
        assert np.array_equal(multi[q].n_open, one.n_open)
        assert np.array_equal(multi[q].status, one.status)
        # the observables reduce with atomics: equal up to summation order
        assert np.allclose(multi[q].T, one.T, rtol=1e-12, atol=1e-13), (prec, q)
        assert np.allclose(multi[q].R, one.R, rtol=1e-12, atol=1e-13), (prec, q)
        assert np.allclose(multi[q].node_n, one.node_n, rtol=1e-11, atol=0), (prec, q)


def test_batched_bias_points_match_oracle(pw, chain_bias):
    from tests.test_gpu_parity import _oracle_results
    wl, basis, ctx, Us = chain_bias
    ctx.set_refinement(1e-11, 0)
    E = wl.energies[5:60:11]
    multi = ctx.solve_multi(list(range(len(Us))), E, pw.MIXED)
    ctx.set_refinement(0, 0)
    for q, U in enumerate(Us):
        s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, U, basis=basis)
        for e, r in enumerate(_oracle_results(s, E)):
            bar = max(1e-8, 4 * r.bar)
            assert abs(multi[q].T[e] - r.T) <= bar and abs(multi[q].R[e] - r.R) <= bar, (q, E[e], multi[q].T[e], r.T)


def test_batched_bias_points_float_float_residual_falls_back(pw, chain_bias):
    # the float-float residual takes one system per launch: solve_multi then goes system
    # by system, with the same results
    wl, basis, ctx, Us = chain_bias
    E = wl.energies[10:20:3]
    ref = ctx.solve_multi([0, 2], E, pw.MIXED)
    ctx.set_residual(pw.RESIDUAL_FLOAT_FLOAT)
    got = ctx.solve_multi([0, 2], E, pw.MIXED)
    ctx.set_residual(pw.RESIDUAL_SLICED)
    for a, b in zip(ref, got):
        assert np.all(np.abs(a.T - b.T) <= 1e-8)
