"""Adaptive Simpson energy integration on the GPU path (pwqt_integrate) against
the oracle's adaptive_simpson with the same rule, on the same Bloch waves.

Both sides evaluate the same integrand at the same energies as long as their
accept/refine decisions agree, which they do except where an interval's error
estimate sits within the integrand's rounding (1e-9 relative) of its threshold;
the integrals are compared at a few times the tolerance, and the quadrature
points must coincide to within a handful of intervals."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def _ctx(pw, s):
    ctx = pw.Context()
    ctx.set_enhancement(s.basis.cell, s.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in s.basis.groups])
    ctx.set_extrinsic(0, s.U)
    return ctx


def _fermi_antiderivative(E, mu, kT):
    x = (E - mu) / kT
    return (E - mu) - kT * np.logaddexp(0.0, x)


def test_pristine_current_matches_closed_form(pw):
    from tests.oracle_fixtures import chain_system, with_potential
    s = with_potential(chain_system(), np.zeros(20))
    ctx = _ctx(pw, s)
    a, b, mu_s, mu_d, kT = 0.3, 1.2, 0.8, 0.7, 0.025
    I, err, ne, xs, ws = ctx.integrate(0, pw.INTEGRAND_CURRENT, a, b, mu_s, mu_d, kT, 1e-13)
    exact = O.G0_SIEMENS * ((_fermi_antiderivative(b, mu_s, kT) - _fermi_antiderivative(a, mu_s, kT))
                            - (_fermi_antiderivative(b, mu_d, kT) - _fermi_antiderivative(a, mu_d, kT)))
    assert abs(I[0] - exact) < 1e-12, (I[0], exact)
    assert ne == len(xs) and abs(ws.sum() - (b - a)) < 1e-12


def test_current_and_node_density_match_oracle(pw):
    from tests.oracle_fixtures import chain_system
    s = chain_system()
    ctx = _ctx(pw, s)
    mu_s, mu_d, kT = 0.9, 0.8, 0.025
    # current through the resonant chain
    I, err, ne, xs, ws = ctx.integrate(0, pw.INTEGRAND_CURRENT, 0.0, 1.2, mu_s, mu_d, kT, 1e-11)
    Io, erro, xso, wso = O.adaptive_simpson(O.current_integrand(s, mu_s, mu_d, kT, cache={}), 0.0, 1.2, 1e-11)
    assert abs(I[0] - Io[0]) < 5e-11, (I[0], Io[0])
    assert abs(len(xs) - len(xso)) <= 8
    # node density (vector integrand, error on the max over nodes)
    nI, nerr, nne, nxs, nws = ctx.integrate(0, pw.INTEGRAND_NODE_DENSITY, 0.0, 1.0, mu_s, mu_d, kT, 1e-2)
    nIo, nerro, nxso, nwso = O.adaptive_simpson(O.node_density_integrand(s, mu_s, mu_d, kT, cache={}), 0.0, 1.0, 1e-2)
    assert nI.shape == (20,)
    assert np.max(np.abs(nI - nIo)) < 5e-2 + 1e-6 * np.max(np.abs(nIo)), np.max(np.abs(nI - nIo))
    assert abs(len(nxs) - len(nxso)) <= 8
    # the weights reproduce the integral of a quantity from another call at those energies
    res = ctx.solve(0, nxs, pw.FP64)
    fs = 0.5 * (1 - np.tanh(0.5 * (nxs - mu_s) / kT))
    fd = 0.5 * (1 - np.tanh(0.5 * (nxs - mu_d) / kT))
    again = np.einsum("e,ei->i", nws, res.node_n[:, :, 0] * fs[:, None] + res.node_n[:, :, 1] * fd[:, None])
    assert np.max(np.abs(again - nI)) < 1e-9 * np.max(np.abs(nI))


def test_integrate_errors_and_budget(pw):
    from tests.oracle_fixtures import chain_system
    s = chain_system()
    ctx = _ctx(pw, s)
    with pytest.raises(pw.PwqtError):
        ctx.integrate(0, pw.INTEGRAND_CURRENT, 1.0, 0.5, 0.9, 0.8, 0.025, 1e-9)      # empty range
    with pytest.raises(pw.PwqtError):
        ctx.integrate(0, 7, 0.0, 1.0, 0.9, 0.8, 0.025, 1e-9)                          # unknown integrand
    with pytest.raises(pw.PwqtError):
        ctx.integrate(3, pw.INTEGRAND_CURRENT, 0.0, 1.0, 0.9, 0.8, 0.025, 1e-9)       # unknown system
    # a tolerance out of reach stops at the evaluation budget (the round that crosses it
    # is finished: at most four new points per interval then open)
    I, err, ne, xs, ws = ctx.integrate(0, pw.INTEGRAND_NODE_DENSITY, 0.0, 1.0, 0.9, 0.8, 0.025, 1e-12, max_evals=100)
    assert 100 <= ne <= 500 and err > 1e-12 and np.all(np.isfinite(I))
