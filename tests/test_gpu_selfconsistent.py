"""Self-consistent loop (pwqt_self_consistent: 1D finite-element Poisson, Newton with
the semi-classical Jacobian, DIIS) against the oracle's loop on the same chain, Bloch
waves and model: the converged potentials agree to well within the 1e-6 eV stopping
tolerance plus the integrals' own tolerance, and DIIS needs fewer iterations than
plain Newton on both sides."""
import numpy as np
import pytest

from oracle import pwqt_oracle as O

pytestmark = pytest.mark.gpu

MU, KT, E_LO = 0.5, 0.025852, -0.1
E_HI = MU + 12 * KT


@pytest.fixture(scope="module")
def pw():
    from paper_1903_00548_gb300 import build, pwqt
    build.build()
    return pwqt


def test_self_consistent_potential_matches_oracle(pw):
    from tests.oracle_fixtures import chain_system, with_potential
    s = with_potential(chain_system(), np.zeros(20))
    cache = {}
    n0, d0, _ = O.density_and_jacobian(s, MU, MU, KT, E_LO, E_HI, 1e-2, cache)
    z = np.arange(20) * s.blk["L"]
    Ug = 0.15 * np.exp(-((z - z.mean()) / (0.25 * z[-1])) ** 2)
    model = O.Poisson1D(kappa=0.05, gamma=1.0, alpha=2e-4, U_gate=Ug, n_dop=n0)
    Uo, ho, no, do = O.self_consistent(s, model, MU, MU, KT, E_LO, E_HI, 1e-2, cache=cache, diis_window=5)
    ctx = pw.Context()
    ctx.set_enhancement(s.basis.cell, s.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in s.basis.groups])
    ctx.set_extrinsic(0, np.zeros(20))
    Ug_, hg, ng = ctx.self_consistent(0, np.zeros(20), 0.05, 1.0, 2e-4, Ug, n0, MU, MU, KT, E_LO, E_HI, 1e-2)
    assert hg[-1] <= 1e-6
    assert np.max(np.abs(Ug_ - Uo)) < 2e-5, np.max(np.abs(Ug_ - Uo))
    assert abs(len(hg) - len(ho)) <= 2
    assert np.max(np.abs(ng - no)) < 1e-3 * np.max(no)
    # plain Newton on the GPU path takes more iterations to the same point
    ctx.set_extrinsic(0, np.zeros(20))
    Un, hn, _ = ctx.self_consistent(0, np.zeros(20), 0.05, 1.0, 2e-4, Ug, n0, MU, MU, KT, E_LO, E_HI, 1e-2,
                                    diis_window=1)
    assert len(hn) > len(hg)
    assert np.max(np.abs(Un - Ug_)) < 2e-5
    # the contacts hold the ends
    assert Ug_[0] == 0.0 and Ug_[-1] == 0.0


def test_self_consistent_argument_errors(pw):
    from tests.oracle_fixtures import chain_system
    s = chain_system()
    ctx = pw.Context()
    ctx.set_enhancement(s.basis.cell, s.basis.eps, [(g["mx"], g["mz"], g["C"]) for g in s.basis.groups])
    ctx.set_extrinsic(0, s.U)
    with pytest.raises(pw.PwqtError):
        ctx.self_consistent(3, s.U, 0.05, 1.0, 2e-4, np.zeros(20), np.zeros(20), MU, MU, KT, E_LO, E_HI, 1e-2)
    with pytest.raises(pw.PwqtError):   # no convergence in one iteration: reported, U holds the last iterate
        ctx.self_consistent(0, s.U, 0.05, 1.0, 2e-4, np.full(20, 0.1), np.zeros(20), MU, MU, KT, E_LO, E_HI, 1e-2,
                            max_iters=1)
