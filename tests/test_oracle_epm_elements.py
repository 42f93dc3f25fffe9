"""Pins of the oracle's plane-wave EPM and element matrices (Sec. 2.2-2.3, App. A)
against closed forms and exact identities."""
import math

import numpy as np
import pytest

from oracle import pwqt_oracle as O
from paper_1903_00548_gb300 import workloads as W
from tests.oracle_fixtures import chain_system, small_ribbon_system

HB2M = 0.0380998212


def test_empty_lattice_epm_closed_form():
    # v == 0: plane waves are exact eigenstates, eps = hbar^2/2m |k+G|^2.
    for cell in (W.chain_cell(0.4), W.armchair_ribbon_cell(5)):
        for k in (0.0, math.pi / cell.Lz, 0.37 * math.pi / cell.Lz):
            mx, mz = O.pw_set(cell, k, 25.0)
            nb = min(12, len(mx))
            eps, C, _, _ = O.epm_bands(cell, W.FormFactor(v0=0.0), k, 25.0, nb)
            bx = 2 * math.pi / cell.Lx if cell.dim == 2 else 0.0
            exact = np.sort(HB2M * ((mx * bx) ** 2 + (mz * 2 * math.pi / cell.Lz + k) ** 2))[:nb]
            assert np.max(np.abs(eps - exact)) < 1e-12
            assert np.allclose(np.sum(np.abs(C) ** 2, axis=0), 1.0, atol=1e-13)


def test_nearly_free_gap_at_zone_edge():
    # Weak potential: the gap at Z between the two lowest bands is 2|V_G1| + O(v^2).
    cell = W.chain_cell(0.4)
    gcut = 6.2 * 2 * math.pi / 0.4
    for v0 in (-0.02, -0.01):
        ff = W.FormFactor(v0=v0)
        eps, _, _, _ = O.epm_bands(cell, ff, math.pi / cell.Lz, gcut, 2)
        vg1 = abs(v0 * math.exp(-(2 * math.pi / 0.4) ** 2 / (2 * ff.sigma ** 2)))
        e0 = HB2M * (math.pi / 0.4) ** 2
        assert abs((eps[1] - eps[0]) - 2 * vg1) < 50 * vg1 ** 2 / e0 + 1e-12


def test_structure_factor_translation_phase():
    # Moving every atom by R multiplies V_G by exp(-iG.R) (Eq. local_epp): a pure
    # phase, so band energies are unchanged.
    cell = W.armchair_ribbon_cell(5)
    shifted = W.Cell(cell.dim, cell.Lz, cell.Lx, cell.atoms + np.array([0.05, 0.11]), cell.omega0)
    e1, _, _, _ = O.epm_bands(cell, W.FormFactor(), 0.3, 22.0, 10)
    e2, _, _, _ = O.epm_bands(shifted, W.FormFactor(), 0.3, 22.0, 10)
    assert np.max(np.abs(e1 - e2)) < 1e-10


def test_basis_too_small():
    with pytest.raises(ValueError):
        O.epm_bands(W.chain_cell(0.4), W.FormFactor(), 0.0, 20.0, 50)


def _int_spow_exp(p, q, L):
    """int_0^L s^p e^{iqs} ds in closed form (integration by parts; series near q=0)."""
    if abs(q) * L < 1e-3:
        tot = 0.0
        term = 1.0
        for j in range(12):
            tot += term * L ** (p + j + 1) / (p + j + 1)
            term *= 1j * q / (j + 1)
        return tot
    val = (np.exp(1j * q * L) - 1.0) / (1j * q)
    for pp in range(1, p + 1):
        val = (L ** pp * np.exp(1j * q * L) - pp * val) / (1j * q)
    return val


def _single_pw_basis(cell, pws):
    """A basis whose enhancement functions are single plane waves (mx, mz, k)."""
    groups, eps, kz = [], [], []
    for k in (0.0, math.pi / cell.Lz):
        sel = [(mx, mz) for (mx, mz, kk) in pws if kk == k]
        C = np.eye(len(sel), dtype=complex)
        groups.append(dict(k=k, mx=np.array([s[0] for s in sel]), mz=np.array([s[1] for s in sel]),
                           C=C, eps=np.zeros(len(sel))))
        kz += [k] * len(sel)
        eps += [0.0] * len(sel)
    return O.basis_from_coefficients(cell, np.array(eps), np.array(kz), groups)


def test_element_quadrature_vs_closed_form():
    cell = W.armchair_ribbon_cell(5)
    L, Lx = cell.Lz, cell.Lx
    kZ = math.pi / L
    pws = [(0, 0, 0.0), (1, 0, 0.0), (0, 1, 0.0), (0, -2, 0.0), (0, 0, kZ), (1, -1, kZ), (0, 3, kZ)]
    basis = _single_pw_basis(cell, pws)
    el = O.element_matrices(basis)
    n = basis.n
    # closed-form integrals of the single-plane-wave basis
    Q = np.array([mz * 2 * math.pi / L + k for (_, mz, k) in pws])
    MX = np.array([mx for (mx, _, _) in pws])
    K = np.array([k for (_, _, k) in pws])
    f = {"l": (lambda p: [1.0, -1.0 / L][p] if p < 2 else 0.0), }
    # polynomial coefficients in s of the hats: f_l = 1 - s/L, f_r = s/L
    hat = {"l": np.array([1.0, -1.0 / L]), "r": np.array([0.0, 1.0 / L])}
    dhat = {"l": -1.0 / L, "r": 1.0 / L}
    off = {"l": 0.0, "r": L}

    def poly_int(coef, q):
        return sum(c * _int_spow_exp(p, q, L) for p, c in enumerate(coef) if c != 0.0)

    M = np.zeros((2 * n, 2 * n), complex)
    T = np.zeros_like(M)
    Pr = np.zeros_like(M)
    Wl = np.zeros_like(M)
    for ia, a in enumerate("lr"):
        for ib, b in enumerate("lr"):
            for al in range(n):
                for be in range(n):
                    if MX[al] != MX[be]:
                        continue
                    q = Q[be] - Q[al]
                    ph = np.exp(1j * (K[al] * off[a] - K[be] * off[b]))
                    fab = np.polynomial.polynomial.polymul(hat[a], hat[b])
                    dfab = np.polynomial.polynomial.polyder(fab)
                    m = Lx * ph * poly_int(fab, q)
                    t = HB2M * Lx * ph * (0.5 * 1j * q * poly_int(dfab, q)
                                          + dhat[a] * dhat[b] * poly_int([1.0], q))
                    pr = -2 * HB2M * Lx * ph * dhat[b] * 1j * Q[be] * poly_int(hat[a], q)
                    wl = Lx * ph * poly_int(np.polynomial.polynomial.polymul(fab, hat["l"]), q)
                    M[ia * n + al, ib * n + be] = m
                    T[ia * n + al, ib * n + be] = t
                    Pr[ia * n + al, ib * n + be] = pr
                    Wl[ia * n + al, ib * n + be] = wl
    for name, ref in (("M", M), ("T", T), ("Pr", Pr), ("Wl", Wl)):
        err = np.max(np.abs(el[name] - ref))
        assert err < 1e-12 * max(1.0, np.max(np.abs(ref))), (name, err)


@pytest.mark.parametrize("which", ["chain", "ribbon"])
def test_hermiticity_and_pu_identity(which):
    s = chain_system() if which == "chain" else small_ribbon_system()
    el, blk = s.elem, s.blk
    for name in ("M", "T", "P", "H", "Wl", "Wr"):
        X = el[name]
        assert np.max(np.abs(X - X.conj().T)) < 1e-13 * max(1.0, np.max(np.abs(X))), name
    # partition of unity: f_l + f_r = 1 on the element
    assert np.max(np.abs(el["Wl"] + el["Wr"] - el["M"])) < 1e-13
    # constant potential => V^e = U M
    N = 5
    Vd, Vu = O.extrinsic_blocks(blk, np.full(N, 0.37))
    assert np.max(np.abs(Vd - 0.37 * blk["M0"][None])) < 1e-13
    assert np.max(np.abs(Vu - 0.37 * blk["M1"][None])) < 1e-13
    # the assembled global H and M (Eq. infinite_system) are Hermitian and M > 0
    n = blk["n"]
    Hg = np.zeros((N * n, N * n), complex)
    Mg = np.zeros_like(Hg)
    for i in range(N):
        Hg[i*n:(i+1)*n, i*n:(i+1)*n] = blk["H0"]
        Mg[i*n:(i+1)*n, i*n:(i+1)*n] = blk["M0"]
        if i + 1 < N:
            Hg[i*n:(i+1)*n, (i+1)*n:(i+2)*n] = blk["H1"]
            Hg[(i+1)*n:(i+2)*n, i*n:(i+1)*n] = blk["H1"].conj().T
            Mg[i*n:(i+1)*n, (i+1)*n:(i+2)*n] = blk["M1"]
            Mg[(i+1)*n:(i+2)*n, i*n:(i+1)*n] = blk["M1"].conj().T
    assert np.max(np.abs(Hg - Hg.conj().T)) < 1e-12
    np.linalg.cholesky(Mg)
