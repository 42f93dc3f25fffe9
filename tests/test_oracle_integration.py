"""Pins of the oracle's adaptive Simpson integration (Sec. 3.3 density integral,
Eq. current) against closed forms and brute force."""
import math

import numpy as np

from oracle import pwqt_oracle as O
from tests.oracle_fixtures import chain_system, with_potential


def test_closed_forms_and_weights():
    # integrable end-point behaviour like the density of states at a band edge
    I, err, xs, w = O.adaptive_simpson(lambda x: 1.0 / np.sqrt(x + 1e-3), 0.0, 1.0, 1e-9)
    exact = 2.0 * (math.sqrt(1.001) - math.sqrt(0.001))
    assert abs(I[0] - exact) < 1e-8
    assert err < 1e-8
    assert abs(np.sum(w) - 1.0) < 1e-13                    # weights integrate the constant exactly
    assert abs(np.dot(w, 1.0 / np.sqrt(xs + 1e-3)) - I[0]) < 1e-12   # and reproduce the integral
    # the refinement concentrates where the integrand varies
    assert np.sum(xs < 0.05) > np.sum(xs > 0.95)
    # Simpson is exact for cubics: nothing is refined past the initial pieces
    I, err, xs, w = O.adaptive_simpson(lambda x: [x ** 3 - 2 * x, 1.0], -1.0, 2.0, 1e-12, min_pieces=4)
    assert np.allclose(I, [15.0 / 4.0 - 3.0, 3.0], atol=1e-13, rtol=0)
    assert len(xs) == 4 * 4 + 1
    # a vector-valued integrand is refined on the max norm of its components
    I, err, xs, w = O.adaptive_simpson(lambda x: [np.sin(3 * x), np.exp(-x)], 0.0, 3.0, 1e-10)
    assert np.allclose(I, [(1 - math.cos(9.0)) / 3.0, 1 - math.exp(-3.0)], atol=2e-9, rtol=0)


def _fermi_antiderivative(E, mu, kT):
    # F(E) with F' = f_FD(E - mu): (E - mu) - kT ln(1 + e^{(E - mu)/kT})
    x = (E - mu) / kT
    return (E - mu) - kT * np.logaddexp(0.0, x)


def test_pristine_current_is_the_landauer_integral():
    # flat potential: T_sd = T_ds = 1 across the first band of the chain, so
    # I = G0 * integral of (f_s - f_d) dE in closed form
    s = with_potential(chain_system(), np.zeros(20))
    a, b, mu_s, mu_d, kT = 0.3, 1.2, 0.8, 0.7, 0.025
    I, err, xs, w = O.adaptive_simpson(O.current_integrand(s, mu_s, mu_d, kT, cache={}), a, b, 1e-13)
    exact = O.G0_SIEMENS * ((_fermi_antiderivative(b, mu_s, kT) - _fermi_antiderivative(a, mu_s, kT))
                            - (_fermi_antiderivative(b, mu_d, kT) - _fermi_antiderivative(a, mu_d, kT)))
    assert abs(I[0] - exact) < 1e-12, (I[0], exact)
    assert abs(I[0] - O.G0_SIEMENS * 0.1) < 1e-9            # ~ G0 (mu_s - mu_d) at low temperature


def _dense_simpson(f, a, b, npts):
    grid = np.linspace(a, b, npts)
    vals = np.array([f(E) for E in grid])
    cw = np.ones(npts)
    cw[1:-1:2] = 4
    cw[2:-1:2] = 2
    return (grid[1] - grid[0]) / 3.0 * (cw[:, None] * vals).sum(0)


def test_node_density_integral_matches_dense_grid():
    # smooth case: the pristine chain inside its first band
    s = with_potential(chain_system(), np.zeros(20))
    f = O.node_density_integrand(s, 0.9, 0.8, 0.025, cache={})
    I, err, xs, w = O.adaptive_simpson(f, 0.2, 1.0, 2e-4)     # ~1e-6 of the integral (~221)
    brute = _dense_simpson(f, 0.2, 1.0, 801)
    assert np.max(np.abs(I - brute)) < 1e-6 * np.max(np.abs(brute))
    assert len(xs) < 801


def test_node_density_resonances_are_refined():
    # the chain with a 0.1 V drop has sharp quasi-bound resonances near 0.3-0.6 eV
    s = chain_system()
    f = O.node_density_integrand(s, 0.9, 0.8, 0.025, cache={})
    I, err, xs, w = O.adaptive_simpson(f, 0.0, 1.0, 1e-3)
    brute = _dense_simpson(f, 0.0, 1.0, 4001)
    assert np.max(np.abs(I - brute)) < 1e-4 * np.max(np.abs(brute))
    inside = np.sum((xs > 0.2) & (xs < 0.65)) / 0.45
    outside = np.sum(xs > 0.7) / 0.3
    assert inside > 3 * outside
