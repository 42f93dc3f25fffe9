"""Diagonal blocks of the retarded Green's function (recursive Green's function on the
GPU, through the C ABI) against the oracle's dense inverse, element by element, and
against the GPU's own wave-function solve through the spectral identity
-(2/pi) Im Tr G_ii = n_s[i] + n_d[i] (ballistic device, Sec. 3.2-3.3).

Tolerances: G_ii is a coefficient-space quantity, so it carries the near-null
directions of the redundant PU Bloch basis (kappa(A) ~ 4e6 on these systems) like the
node densities of the wave-function solve: blocks are compared at 1e-7 of their
largest element.  The node spectral density -(2/pi) Im Tr G_ii is small against the
elements of G along those directions (max |G| ~ 2e4 against a density ~ 9 on the
chain), and FP64 rounding scales with the elements: each carries up to ~ kappa u_64
max|G| (first-order perturbation of the inverse), and the trace adds n of them, so
the density is compared at (2/pi) n DOS_TOL max|G| with DOS_TOL = 2e-9 ~ 4 kappa u_64
(measured on the chain: 8e-5 against a bound of 1.9e-4); plus the node densities' own
1e-7 where the wave-function route is the other side."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W
from tests.oracle_fixtures import small_ribbon_system

pytestmark = pytest.mark.gpu

TOL = 1e-7
DOS_TOL = 2e-9


def _dos_bound(G):
    return (2 / np.pi) * G.shape[-1] * DOS_TOL * np.max(np.abs(G))


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def _ctx(pw, sys_, **opts):
    ctx = pw.Context(**opts)
    ctx.set_enhancement(sys_.basis.cell, sys_.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in sys_.basis.groups])
    ctx.set_extrinsic(0, sys_.U)
    return ctx


def _check_against_oracle(pw, sys_, Es, **opts):
    ctx = _ctx(pw, sys_, **opts)
    dos, G, st = ctx.green_diagonal(0, Es, blocks=True)
    assert np.all(st & pw.ST_MODE_COUNT == 0) and np.all(st & pw.ST_SINGULAR_PIVOT == 0), st
    assert G.shape == (len(Es), sys_.Vd.shape[0], sys_.blk["n"], sys_.blk["n"])
    for e, E in enumerate(Es):
        Gref, dref = O.green_diagonal(sys_.blk, sys_.Vd, sys_.Vu, sys_.U, float(E))
        assert np.max(np.abs(G[e] - Gref)) <= TOL * np.max(np.abs(Gref)), E
        t = _dos_bound(Gref)
        assert np.max(np.abs(dos[e] - dref)) <= t, (E, np.max(np.abs(dos[e] - dref)), t)
        # the recorded density is the trace of the returned blocks
        assert np.allclose(dos[e], -(2 / np.pi) * np.trace(G[e], axis1=1, axis2=2).imag, rtol=1e-12, atol=0)
    return ctx, dos


def test_chain_green_diagonal_matches_oracle(pw):
    wl = W.chain8()
    s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, wl.U)
    _check_against_oracle(pw, s, wl.energies[3:60:8])


def test_multi_tile_ribbon_green_diagonal_matches_oracle(pw):
    # n = 72: three 32-wide tiles with a ragged tail of 8; 24 nodes; batches of 2 energies
    s = small_ribbon_system(n_bands=36, n_nodes=24, gcut=30.0)
    _check_against_oracle(pw, s, np.array([0.45, 0.8, 1.3]), batch=2)


def test_spectral_density_equals_solved_node_densities(pw):
    # the GPU's two routes: the Green's-function recursion and the wave-function sweep
    for s, Es in ((small_ribbon_system(), np.array([0.6, 1.1, 1.7])),
                  (small_ribbon_system(n_bands=36, n_nodes=24, gcut=30.0), np.array([0.45, 1.3]))):
        ctx = _ctx(pw, s)
        dos, G, _ = ctx.green_diagonal(0, Es, blocks=True)
        d2, none, _ = ctx.green_diagonal(0, Es)
        assert none is None and np.array_equal(d2, dos)
        res = ctx.solve(0, Es, pw.FP64)
        ns = res.node_n.sum(axis=2)
        assert np.all(ns > 0)
        for e in range(len(Es)):
            t = _dos_bound(G[e]) + TOL * np.max(ns[e])
            assert np.max(np.abs(dos[e] - ns[e])) <= t, (Es[e], np.max(np.abs(dos[e] - ns[e])), t)


def test_green_diagonal_edge_cases(pw):
    s = small_ribbon_system()
    ctx = _ctx(pw, s)
    dos, _, st = ctx.green_diagonal(0, np.zeros(0))
    assert dos.shape == (0, s.Vd.shape[0])
    with pytest.raises(RuntimeError):
        ctx.green_diagonal(7, np.array([0.6]))          # unknown system
    with pytest.raises(RuntimeError):
        ctx.green_diagonal(0, np.array([np.nan]))       # non-finite energy
    # the context stays usable after the errors
    d1, _, _ = ctx.green_diagonal(0, np.array([0.6]))
    assert np.all(np.isfinite(d1)) and np.all(d1 > 0)
