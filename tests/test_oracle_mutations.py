"""The pins must catch plausible mistakes: each test plants one in the oracle (on the
CPU, through monkeypatching) and checks that a physics pin then fails."""
import math

import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W


def _system():
    wl = W.chain8()
    return O.build_system(wl.cell, W.FormFactor(), wl.gcut, wl.n_bands, np.zeros(12))


def _pins_hold(sys_):
    """The pristine-chain pins: T = 1 with R = 0 inside the band, and exact
    band reconstruction at Gamma and Z."""
    blk = sys_.blk
    for E in (0.3, 1.0):
        try:
            r = O.solve_energy(blk, sys_.Vd, sys_.Vu, sys_.U, E)
        except RuntimeError:          # a broken contact (mode count) also fails the pins
            return False
        if not (abs(r.T - 1.0) < 1e-8 and abs(r.R) < 1e-8):
            return False
    for gi, kp in ((0, 0.0), (1, math.pi / blk["L"])):
        ev = O.pu_bands(blk, kp)
        for e in sys_.basis.groups[gi]["eps"]:
            if np.min(np.abs(ev - e)) > 1e-8:
                return False
    return True


def test_unmutated_pins_hold():
    assert _pins_hold(_system())


def _mutated_contact(kind):
    orig = O.contact

    def bad(modes, side, allow_sort=False):
        c = orig(modes, side, allow_sort)
        if kind == "sigma_sign":
            c.Sigma = -c.Sigma
        elif kind == "bloch_transpose":
            X = c.B.T @ np.diag(c.lam_out) @ np.linalg.inv(c.B.T)
            c.Sigma = c.Kprime @ X
        elif kind == "rhs_without_sigma":
            c.rhs = (c.Kprime @ c.c_in) * c.lam_in[None, :]
        elif kind == "source_lambda_not_inverted" and side == "s":
            X = c.B @ np.diag(1.0 / c.lam_out) @ np.linalg.inv(c.B)
            c.Sigma = c.Kprime @ X
        return c
    return bad


@pytest.mark.parametrize("kind", ["sigma_sign", "bloch_transpose", "rhs_without_sigma",
                                  "source_lambda_not_inverted"])
def test_self_energy_mistakes_are_caught(monkeypatch, kind):
    s = _system()
    monkeypatch.setattr(O, "contact", _mutated_contact(kind))
    assert not _pins_hold(s)


def test_main_text_momentum_factor_is_caught():
    # P = -hbar^2/m int ... + h.c. read without the 1/2 of App. A
    s = _system()
    el = dict(s.elem)
    el["H"] = el["H"] + el["P"]
    blk = O.intrinsic_blocks(el)
    Vd, Vu = O.extrinsic_blocks(blk, s.U)
    assert not _pins_hold(O.System(s.basis, el, blk, s.U, Vd, Vu))


def test_dropped_kinetic_hat_term_is_caught(monkeypatch):
    s = _system()
    el = dict(s.elem)
    n = el["n"]
    # remove the f_a' f_b' phi^* phi part of T (it equals (1/L^2) x overlap-like term)
    L = el["L"]
    bad_T = el["T"].copy()
    sign = np.block([[np.ones((n, n)), -np.ones((n, n))], [-np.ones((n, n)), np.ones((n, n))]])
    # recompute that term by quadrature-free identity: int phi^* phi over the cell
    # equals M_ll + M_lr + M_rl + M_rr with left phases; use the oracle's J1 proxy
    J = el["M"][:n, :n] + el["M"][:n, n:] + el["M"][n:, :n] + el["M"][n:, n:]
    bad_T -= 0.0380998212 / L ** 2 * sign * np.block([[J, J], [J, J]])
    eps2 = np.concatenate([s.basis.eps, s.basis.eps])
    el["H"] = 0.5 * (eps2[:, None] + eps2[None, :]) * el["M"] + bad_T + el["P"]
    blk = O.intrinsic_blocks(el)
    Vd, Vu = O.extrinsic_blocks(blk, s.U)
    assert not _pins_hold(O.System(s.basis, el, blk, s.U, Vd, Vu))


def test_time_reversed_convention_gives_same_transmission(monkeypatch):
    # Flipping every velocity swaps in- and out-flow: the time-reversed problem,
    # whose transmission is the same (not a mistake the pins should flag).
    wl = W.chain8()
    s = O.build_system(wl.cell, W.FormFactor(), wl.gcut, wl.n_bands, wl.U)
    ref = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E).T for E in (0.4, 1.0)]
    orig = O.lead_modes

    def flipped(blk, Ec, reciprocal=False):
        m = orig(blk, Ec, reciprocal)
        m.dEdk = -m.dEdk
        return m
    monkeypatch.setattr(O, "lead_modes", flipped)
    got = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, E).T for E in (0.4, 1.0)]
    assert np.allclose(ref, got, atol=1e-8)


def test_wrong_mode_normalisation_is_caught(monkeypatch):
    # unit 2-norm instead of c^H M(lambda) c = L/2pi (Eq. normalization)
    orig = O.lead_modes

    def bad(blk, Ec, reciprocal=False):
        m = orig(blk, Ec, reciprocal)
        for j in np.flatnonzero(m.traveling):
            m.C[:, j] /= np.linalg.norm(m.C[:, j])
        return m
    wl = W.chain8()
    s = O.build_system(wl.cell, W.FormFactor(), wl.gcut, wl.n_bands, wl.U)
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.4)
    assert abs(r.T + r.R - 1.0) < 1e-8
    monkeypatch.setattr(O, "lead_modes", bad)
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.4)
    assert abs(r.T + r.R - 1.0) > 1e-4


def test_flipped_traveling_velocity_breaks_the_mode_count(monkeypatch):
    # Sec. 3.1: n out-flow and n in-flow modes per contact.  One traveling mode with
    # the wrong flow direction leaves n + 1 (or n - 1) out-flow modes: the oracle
    # must report it, not absorb it.
    wl = W.chain8()
    s = O.build_system(wl.cell, W.FormFactor(), wl.gcut, wl.n_bands, wl.U)
    O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.4)          # unmutated: count is n
    orig = O.lead_modes

    def flipped_one(blk, Ec, reciprocal=False):
        m = orig(blk, Ec, reciprocal)
        j = int(np.flatnonzero(m.traveling)[0])
        m.dEdk = m.dEdk.copy()
        m.dEdk[j] = -m.dEdk[j]
        return m
    monkeypatch.setattr(O, "lead_modes", flipped_one)
    with pytest.raises(O.ModeCountError):
        O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.4)
    # the diagnostic score sort still returns a result, flagged
    r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, 0.4, allow_sort=True)
    assert r.mode_sorted


def test_jacobian_factor_mistake_is_caught(monkeypatch):
    # Eq. density_jacobian: the weight -f' of the Jacobian; a factor-of-two slip must
    # fail the finite-difference pin of tests/test_oracle_selfconsistent.py
    from tests.test_oracle_selfconsistent import jacobian_matches_mu_derivative
    assert jacobian_matches_mu_derivative()
    orig = O.dfermi
    monkeypatch.setattr(O, "dfermi", lambda x, kT: 0.5 * orig(x, kT))
    assert not jacobian_matches_mu_derivative()
