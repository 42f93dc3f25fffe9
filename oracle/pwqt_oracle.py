"""Oracle for the per-energy open-boundary solve of Van de Put, Fischetti and
Vandenberghe, "Scalable atomistic simulations of quantum electron transport
using empirical pseudopotentials" (arXiv:1903.00548).

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64/complex128 CPU code written from
the paper's equations.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / --impl reference legs may import it.  It shares no code with
the CUDA path (the seeded input generators of paper_1903_00548_gb300.workloads
are inputs only).

Structure, in the paper's order:
  Sec. 2.2      plane-wave EPM Bloch waves u_nk at the enhancement k-points
                (Gamma and Z) -> bloch_basis()
  Sec. 2.3, App. A
                element matrices M, T, P, H^c = (eps+eps')/2 M + T + P and the
                extrinsic-potential weights W, by Gauss-Legendre quadrature in z
                and exact plane-wave orthogonality in x -> element_matrices()
  Eq. infinite_system
                block-tridiagonal H, M and V^e blocks -> intrinsic_blocks(),
                extrinsic_blocks()
  Sec. 3.1      complex band structure of the leads from the symmetric
                linearisation (Eq. linearized_eigenvalue_symmetric), flow
                direction from the generalised Hellmann-Feynman velocity
                (Eq. hellmann-feynman), normalisation (Eq. normalization),
                Bloch matrices and self-energies -> lead_modes(), contact()
  Sec. 3.2      QTBM system [E M - H - Sigma] c = B (Eq. qtbm_system) solved by
                dense (or banded) LU of the assembled global matrix
                -> solve_energy()
  Sec. 3.3-3.4  node density, transmission (Eq. transmission) and reflection,
                density by the naive route (Eq. density_3d) and by the
                density-matrix route (Eqs. density_matrices, density_3d_fast)
  Sec. 5.1      band reconstruction H(k') c = E M(k') c -> pu_bands()

Readings of the paper where it is silent or garbled (each is listed with its
reason in the design notes):
  * V_0 (the G = 0 Fourier component of the crystal potential) is dropped.
  * V_G = (omega0/Omega_cell) sum_a v(|G|) exp(-i G.R_a).
  * P = (P^(r) + P^(l))/2 as derived in App. A (Eq. hc_matel_herm); the
    "-hbar^2/m ... + h.c." of Sec. 2.3 is read as that symmetrised sum.
  * lambda is the ratio (outside neighbour)/(edge node); drain lambda_d =
    c_{i+1}/c_i, source lambda_s = c_{i-1}/c_i = 1/lambda_d with the same c.
  * traveling iff ||lambda| - 1| < 1e-4 on the generalised-QZ eigenvalues;
    each traveling mode is then refined on the unit circle (Newton on k with
    the band structure of Sec. 5.1 and the Hellmann-Feynman slope), so that
    |lambda| = 1 holds to rounding as Sec. 3.1 states for exact arithmetic.
  * out-flow modes are classified by the physics of Sec. 3.1: at the drain a mode
    flows out when |lambda| < 1 (decays into the lead) or when it travels with
    dE/dk > 0; at the source the mirror image.  Sec. 3.1 fixes N_b = n out-flow
    and n in-flow modes per contact, so any other count is an error
    (ModeCountError).  Only on request (allow_sort=True, for diagnosing a nearly
    redundant basis whose close-to-singular pencil breaks the lambda <-> 1/lambda*
    pairing) are the 2n modes instead sorted into two sets of n by an out-flow
    score (log|lambda| for evanescent modes, -/+1e-5 for traveling modes with
    dE/dk >/< 0); every result built that way carries mode_sorted=True.  A
    traveling candidate whose unit-circle refinement does not converge is treated
    as evanescent.
  * degenerate traveling modes are made flux-orthogonal by diagonalising the
    velocity form in the M(lambda) metric.
  * V_e(z) = sum_j U_j f_j(z) (hat interpolation of node potentials); leads
    are flat at the end-node values.
  * g_nu = 2 / |dE/dk| (spin 2, delta(k) normalisation).

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, invariants, brute force); none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

HB2M = 0.0380998212          # hbar^2/(2 m_e), eV nm^2
TRAVEL_TOL = 1e-4            # ||lambda| - 1| below which a mode is traveling
DEGEN_TOL = 1e-8             # |lambda_a - lambda_b| below which traveling modes are degenerate


# =============================================================================
# Sec. 2.2 -- plane-wave empirical pseudopotential Bloch waves
# =============================================================================

def pw_set(cell, k: float, gcut: float):
    """Plane waves G = (2 pi mx/Lx, 2 pi mz/Lz) with |G + k z^| <= gcut (Sec. 2.2)."""
    bz = 2.0 * math.pi / cell.Lz
    mzmax = int(math.ceil((gcut + abs(k)) / bz)) + 1
    if cell.dim == 2:
        bx = 2.0 * math.pi / cell.Lx
        mxmax = int(math.ceil(gcut / bx)) + 1
    else:
        bx, mxmax = 0.0, 0
    mx, mz = np.meshgrid(np.arange(-mxmax, mxmax + 1), np.arange(-mzmax, mzmax + 1),
                         indexing="ij")
    mx, mz = mx.ravel(), mz.ravel()
    g2 = (mx * bx) ** 2 + (mz * bz + k) ** 2
    keep = g2 <= gcut * gcut * (1.0 + 1e-14)
    return mx[keep].astype(np.int64), mz[keep].astype(np.int64)


def crystal_potential_fourier(cell, ff, dmx, dmz):
    """V_G of the local pseudopotential sum (Eq. local_epp): for G != 0,
    V_G = (omega0/Omega_cell) v(|G|) sum_a exp(-i G.R_a); V_0 = 0."""
    bz = 2.0 * math.pi / cell.Lz
    bx = 2.0 * math.pi / cell.Lx if cell.dim == 2 else 0.0
    gx = dmx * bx
    gz = dmz * bz
    q2 = gx * gx + gz * gz
    v = ff.v0 * np.exp(-q2 / (2.0 * ff.sigma ** 2))
    s = np.zeros(np.shape(gx), dtype=np.complex128)
    for (x, z) in cell.atoms:
        s += np.exp(-1j * (gx * x + gz * z))
    V = (cell.omega0 / cell.omega_cell) * v * s
    return np.where((dmx == 0) & (dmz == 0), 0.0, V)


def epm_bands(cell, ff, k: float, gcut: float, n_bands: int):
    """Lowest n_bands eigenpairs of the plane-wave Hamiltonian at Bloch vector k z^:
    H_GG' = hbar^2/2m |k+G|^2 delta_GG' + V_{G-G'} (Sec. 2.2).
    Coefficients are normalised to sum_G |c(G)|^2 = 1, i.e. the integral of
    |u|^2 over the cell is the cell volume (Sec. 3.3)."""
    mx, mz = pw_set(cell, k, gcut)
    if len(mx) < n_bands:
        raise ValueError("basis too small: fewer plane waves than requested bands")
    bz = 2.0 * math.pi / cell.Lz
    bx = 2.0 * math.pi / cell.Lx if cell.dim == 2 else 0.0
    kin = HB2M * ((mx * bx) ** 2 + (mz * bz + k) ** 2)
    H = crystal_potential_fourier(cell, ff, mx[:, None] - mx[None, :], mz[:, None] - mz[None, :])
    H = H + np.diag(kin)
    eps, C = np.linalg.eigh(H)
    return eps[:n_bands].copy(), C[:, :n_bands].copy(), mx, mz


@dataclass
class BlochBasis:
    """Enhancement functions phi_{i n k} = u_nk e^{ik(z - z_i)} (Eq. wavef_expansion)
    for k in {Gamma, Z}; basis index alpha = (Gamma bands..., Z bands...)."""
    cell: object
    eps: np.ndarray          # (n,) band energies eps_alpha
    kz: np.ndarray           # (n,) Bloch vector of each enhancement function
    groups: list             # per k: dict(k, mx, mz, C (N_G x n_bands))
    n_bands: int

    @property
    def n(self):
        return len(self.eps)


def bloch_basis(cell, ff, gcut: float, n_bands: int) -> BlochBasis:
    """Bloch waves at the Brillouin-zone centre and edge (Sec. 2.2, Sec. 5.1)."""
    groups = []
    eps_all, k_all = [], []
    for k in (0.0, math.pi / cell.Lz):
        eps, C, mx, mz = epm_bands(cell, ff, k, gcut, n_bands)
        groups.append(dict(k=k, mx=mx, mz=mz, C=C, eps=eps))
        eps_all.append(eps)
        k_all.append(np.full(n_bands, k))
    return BlochBasis(cell, np.concatenate(eps_all), np.concatenate(k_all), groups, n_bands)


def basis_from_coefficients(cell, eps, kz, groups) -> BlochBasis:
    return BlochBasis(cell, np.asarray(eps), np.asarray(kz), groups, len(eps) // 2)


# =============================================================================
# Sec. 2.3 + App. A -- element matrices by quadrature
# =============================================================================

def _partial_fourier(basis: BlochBasis, s: float):
    """x-Fourier components of phi_alpha (left-node phase) and of d/dz phi_alpha
    at z-offset s within an element: A[mx, alpha], dA[mx, alpha]."""
    cell = basis.cell
    allmx = np.unique(np.concatenate([g["mx"] for g in basis.groups]))
    A = np.zeros((len(allmx), basis.n), dtype=np.complex128)
    dA = np.zeros_like(A)
    bz = 2.0 * math.pi / cell.Lz
    col = 0
    for g in basis.groups:
        k = g["k"]
        qz = g["mz"] * bz + k
        ph = np.exp(1j * qz * s)
        rows = np.searchsorted(allmx, g["mx"])
        nb = g["C"].shape[1]
        for j in range(len(qz)):
            A[rows[j], col:col + nb] += g["C"][j] * ph[j]
            dA[rows[j], col:col + nb] += g["C"][j] * ph[j] * (1j * qz[j])
        col += nb
    return A, dA


def quadrature_order(basis: BlochBasis) -> int:
    cell = basis.cell
    bz = 2.0 * math.pi / cell.Lz
    qmax = 0.0
    for g in basis.groups:
        qmax = max(qmax, float(np.max(np.abs(g["mz"] * bz + g["k"]))))
    return int(2.0 * qmax * cell.Lz) + 48


def element_matrices(basis: BlochBasis, nq: int | None = None):
    """Matrix elements on one element (supercell) between the basis functions
    of its left node (l) and right node (r), in the 2x2 node-block layout
    [[ll, lr], [rl, rr]] (each n x n):

      M_ab = int f_a f_b phi_a^* phi_b                                  (Sec. 2.3)
      T_ab = hbar^2/2m int [ 1/2 d(f_a f_b) d(phi_a^* phi_b) + f_a' f_b' phi_a^* phi_b ]
      P    = (P^r + P^l)/2,  P^r_ab = -hbar^2/m int f_a phi_a^* f_b' d phi_b (App. A)
      H_ab = (eps_a + eps_b)/2 M_ab + T_ab + P_ab                 (Eq. hc_matel_herm)
      W^c_ab = int f_c f_a f_b phi_a^* phi_b   (c in {l, r}; for V^e, Sec. 2.3)

    with hats f_l = 1 - s/L, f_r = s/L on s in [0, L], phi_{r,alpha} =
    u_alpha e^{i k_alpha (s - L)}, phi_{l,alpha} = u_alpha e^{i k_alpha s}.
    Integrals over x are exact (plane-wave orthogonality); over z by
    Gauss-Legendre quadrature with nq points.
    """
    cell = basis.cell
    L, Lx, n = cell.Lz, cell.Lx, basis.n
    if nq is None:
        nq = quadrature_order(basis)
    xg, wg = np.polynomial.legendre.leggauss(nq)
    s_pts = 0.5 * L * (xg + 1.0)
    w_pts = 0.5 * L * wg

    f = {"l": lambda s: 1.0 - s / L, "r": lambda s: s / L}
    fp = {"l": -1.0 / L, "r": 1.0 / L}
    nodes = ("l", "r")
    # per-node constant phase: phi_r = phi_l * exp(-i k L)
    ph = {"l": np.ones(n, dtype=np.complex128), "r": np.exp(-1j * basis.kz * L)}

    M = {(a, b): np.zeros((n, n), complex) for a in nodes for b in nodes}
    T = {(a, b): np.zeros((n, n), complex) for a in nodes for b in nodes}
    Pr = {(a, b): np.zeros((n, n), complex) for a in nodes for b in nodes}
    W = {(c, a, b): np.zeros((n, n), complex) for c in nodes for a in nodes for b in nodes}

    for s, w in zip(s_pts, w_pts):
        A, dA = _partial_fourier(basis, s)
        ov = Lx * (A.conj().T @ A)            # sum_x phi_a^* phi_b (left-node phases)
        d_right = Lx * (A.conj().T @ dA)      # phi_a^* d phi_b
        d_left = d_right.conj().T             # (d phi_a)^* phi_b
        for a in nodes:
            for b in nodes:
                pa, pb = ph[a].conj()[:, None], ph[b][None, :]
                o = pa * ov * pb
                dl = pa * d_left * pb
                dr = pa * d_right * pb
                fa, fb = f[a](s), f[b](s)
                dfafb = fp[a] * fb + fa * fp[b]
                M[a, b] += w * fa * fb * o
                T[a, b] += w * HB2M * (0.5 * dfafb * (dl + dr) + fp[a] * fp[b] * o)
                Pr[a, b] += w * (-2.0 * HB2M) * fa * fp[b] * dr
                for c in nodes:
                    W[c, a, b] += w * f[c](s) * fa * fb * o

    def full(X):
        return np.block([[X["l", "l"], X["l", "r"]], [X["r", "l"], X["r", "r"]]])

    Mf, Tf, Prf = full(M), full(T), full(Pr)
    Pf = 0.5 * (Prf + Prf.conj().T)
    eps2 = np.concatenate([basis.eps, basis.eps])
    Hf = 0.5 * (eps2[:, None] + eps2[None, :]) * Mf + Tf + Pf
    Wf = {c: np.block([[W[c, "l", "l"], W[c, "l", "r"]], [W[c, "r", "l"], W[c, "r", "r"]]])
          for c in nodes}
    return dict(M=Mf, T=Tf, P=Pf, Pr=Prf, H=Hf, Wl=Wf["l"], Wr=Wf["r"], n=n, L=L)


# =============================================================================
# Eq. infinite_system -- block-tridiagonal structure
# =============================================================================

def intrinsic_blocks(elem):
    """Node blocks of the periodic system: H_ii = H^rr (left element) + H^ll
    (right element), H_{i,i+1} = H^lr; the same for M (Eq. infinite_system)."""
    n = elem["n"]
    sl, sr = slice(0, n), slice(n, 2 * n)
    out = {}
    for X in ("H", "M"):
        E = elem[X]
        out[X + "0"] = E[sr, sr] + E[sl, sl]
        out[X + "1"] = E[sl, sr]
    for c in ("l", "r"):
        E = elem["W" + c]
        out["W%s_ll" % c] = E[sl, sl]
        out["W%s_lr" % c] = E[sl, sr]
        out["W%s_rr" % c] = E[sr, sr]
    out["L"] = elem["L"]
    out["n"] = n
    return out


def extrinsic_blocks(blk, U):
    """V^e blocks (Sec. 2.3) for V_e(z) = sum_j U_j f_j(z) with nodes 1..N and
    flat leads (U_0 = U_1, U_{N+1} = U_N):
      V_ii     = U_{i-1} W^l_rr + U_i (W^r_rr + W^l_ll) + U_{i+1} W^r_ll
      V_{i,i+1} = U_i W^l_lr + U_{i+1} W^r_lr
    Returns Vd (N, n, n) and Vu (N-1, n, n)."""
    U = np.asarray(U, dtype=np.float64)
    N = len(U)
    Ue = np.concatenate([[U[0]], U, [U[-1]]])
    Vd = np.empty((N, blk["n"], blk["n"]), complex)
    Vu = np.empty((max(N - 1, 0), blk["n"], blk["n"]), complex)
    for i in range(N):
        um, u0, up = Ue[i], Ue[i + 1], Ue[i + 2]
        Vd[i] = um * blk["Wl_rr"] + u0 * (blk["Wr_rr"] + blk["Wl_ll"]) + up * blk["Wr_ll"]
    for i in range(N - 1):
        Vu[i] = Ue[i + 1] * blk["Wl_lr"] + Ue[i + 2] * blk["Wr_lr"]
    return Vd, Vu


# =============================================================================
# Sec. 3.1 -- contact self-energies from the complex band structure
# =============================================================================

@dataclass
class LeadModes:
    lam: np.ndarray          # (2n,) drain-convention lambda = c_{i+1}/c_i
    C: np.ndarray            # (n, 2n) mode vectors c (normalised)
    dEdk: np.ndarray         # (2n,) dE/dk (eV nm) for traveling modes, 0 otherwise
    traveling: np.ndarray    # (2n,) bool
    Kp: np.ndarray           # K_+ = H_{i,i+1} - E_c M_{i,i+1}
    Km: np.ndarray           # K_- = K_+^dagger
    K0: np.ndarray
    Ec: float
    L: float
    n_degenerate_sets: int = 0


def _m_lambda(blk, lam):
    return blk["M1"].conj().T / lam + blk["M0"] + lam * blk["M1"]


def _velocity_form(Kp, Km, lam, L):
    # d/dk [lambda^-1 K_- + K_0 + lambda K_+] at fixed E, lambda = e^{ikL}
    return 1j * L * (lam * Kp - Km / lam)


def refine_traveling(blk, Ec: float, lam, c, iters: int = 8):
    """Put a traveling mode exactly on the unit circle: with lambda = e^{ikL},
    E(k) is an eigenvalue of H(k) c = E M(k) c (Sec. 5.1); Newton on k with the
    slope dE/dk of Eq. hellmann-feynman until E(k) = Ec, the eigenvector of the
    band closest to Ec from scipy's Hermitian-definite eigensolver."""
    L = blk["L"]
    k = float(np.angle(lam)) / L
    best = None
    for _ in range(iters):
        ph = np.exp(1j * k * L)
        Hk = blk["H0"] + blk["H1"] * ph + blk["H1"].conj().T / ph
        Mk = _m_lambda(blk, ph)
        Hk, Mk = 0.5 * (Hk + Hk.conj().T), 0.5 * (Mk + Mk.conj().T)
        w, V = sla.eigh(Hk, Mk)
        # the band whose eigenvector overlaps most with the current mode; when that band
        # is degenerate at k, the mode is projected onto the whole eigenspace (M-orthogonal
        # projection with the M-orthonormal eigenvectors of eigh), so that candidates of one
        # degenerate set stay distinct for the flux orthogonalisation of Sec. 3.1
        ov = np.abs(V.conj().T @ (Mk @ c))
        b = int(np.argmax(ov / np.sqrt(np.abs(np.einsum("ij,ij->j", V.conj(), Mk @ V)))))
        deg = np.flatnonzero(np.abs(w - w[b]) <= 1e-9 * max(1.0, abs(w[b])))
        if len(deg) > 1:
            Vd = V[:, deg]
            c = Vd @ (Vd.conj().T @ (Mk @ c))
        else:
            c = V[:, b] * (np.vdot(V[:, b], c) / abs(np.vdot(V[:, b], c)))
        # dE/dk of that band at k (Eq. hellmann-feynman with E = w[b])
        Kb = blk["H1"] - w[b] * blk["M1"]
        slope = (np.vdot(c, _velocity_form(Kb, Kb.conj().T, ph, L) @ c) / np.vdot(c, Mk @ c)).real
        best = (ph, c / np.linalg.norm(c))
        if abs(w[b] - Ec) < 1e-12 * max(1.0, abs(Ec)):
            return True, best[0], best[1]
        if slope == 0.0:
            break
        k -= (w[b] - Ec) / slope
    return False, best[0], best[1]


def lead_modes(blk, Ec: float, reciprocal=False) -> LeadModes:
    """Complex band structure at energy Ec of the flat lead (Eqs. complex_bs and
    linearized_eigenvalue_symmetric): the 2n x 2n pencil
        [[K0, K-], [K+, 0]] [d; c] = lambda [[-K+, 0], [0, K+]] [d; c],  d = lambda c,
    K(E) = H - E M, solved by generalised QZ.  Traveling modes get their
    Hellmann-Feynman velocity (Eq. hellmann-feynman) and the normalisation
    c^H M(lambda) c = L/2pi (Eq. normalization); evanescent modes unit norm.
    reciprocal=True solves the same pencil for mu = 1/lambda (QZ of (B, A)), and
    reciprocal="cayley" the standard eigenproblem of its Cayley transform
    (A + B)^-1 (A - B), mu = (lambda - 1)/(lambda + 1): the same modes by other
    rounding paths, so that the spread of the results measures how well FP64
    determines them (the oracle's own error bar, see error_bar)."""
    n, L = blk["n"], blk["L"]
    K0 = blk["H0"] - Ec * blk["M0"]
    Kp = blk["H1"] - Ec * blk["M1"]
    Km = Kp.conj().T
    Z = np.zeros((n, n), complex)
    A = np.block([[K0, Km], [Kp, Z]])
    B = np.block([[-Kp, Z], [Z, Kp]])
    if reciprocal == "cayley":
        mu, V = sla.eig(np.linalg.solve(A + B, A - B))
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = np.where(mu == 1, np.inf, (1.0 + mu) / (1.0 - mu))
    elif reciprocal:
        mu, V = sla.eig(B, A)
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = np.where(mu == 0, np.inf, 1.0 / mu)
    else:
        lam, V = sla.eig(A, B)
    C = V[n:, :].copy()
    C /= np.linalg.norm(C, axis=0)[None, :]
    absl = np.abs(lam)
    trav = np.abs(absl - 1.0) < TRAVEL_TOL
    for j in np.flatnonzero(trav):
        ok, lj, cj = refine_traveling(blk, Ec, lam[j], C[:, j])
        if ok:
            lam[j], C[:, j] = lj, cj
        else:
            trav[j] = False
    dEdk = np.zeros(2 * n)
    # degenerate traveling sets: diagonalise the velocity form in the M metric
    idx = np.flatnonzero(trav)
    done = set()
    nsets = 0
    for a in idx:
        if a in done:
            continue
        grp = [b for b in idx if b not in done and abs(lam[b] - lam[a]) < DEGEN_TOL]
        done.update(grp)
        lm = np.mean(lam[grp])
        lm = lm / abs(lm)
        Cg = C[:, grp]
        F = Cg.conj().T @ _velocity_form(Kp, Km, lm, L) @ Cg
        Mg = Cg.conj().T @ _m_lambda(blk, lm) @ Cg
        F = 0.5 * (F + F.conj().T)
        Mg = 0.5 * (Mg + Mg.conj().T)
        if len(grp) == 1:
            v = (F[0, 0] / Mg[0, 0]).real
            C[:, grp[0]] *= math.sqrt(L / (2.0 * math.pi) / Mg[0, 0].real)
            dEdk[grp[0]] = v
        else:
            nsets += 1
            vals, Ug = sla.eigh(F, Mg)
            C[:, grp] = (Cg @ Ug) * math.sqrt(L / (2.0 * math.pi))
            dEdk[grp] = vals
    return LeadModes(lam, C, dEdk, trav, Kp, Km, K0, Ec, L, nsets)


class ModeCountError(RuntimeError):
    """The out-flow modes of a contact, classified by Sec. 3.1's physics (decay into
    the lead, or group velocity pointing out of the device), do not number N_b = n."""


@dataclass
class Contact:
    """Self-energy, Bloch matrix and injection data of one contact (Sec. 3.1-3.2)."""
    Sigma: np.ndarray        # n x n
    B: np.ndarray            # n x n, columns = out-flow modes
    lam_out: np.ndarray      # out-flow phase factors in this contact's convention
    v_out: np.ndarray        # dE/dk of out-flow modes (0 for evanescent)
    trav_out: np.ndarray     # bool mask over B's columns
    c_in: np.ndarray         # n x m, traveling in-flow (injected) modes
    lam_in: np.ndarray       # their phase factors (this contact's convention)
    v_in: np.ndarray         # their dE/dk
    rhs: np.ndarray          # n x m injection vectors B_{i,gamma} (Eq. qtbm_system)
    Kprime: np.ndarray
    mode_sorted: bool = False   # out-flow set chosen by the score sort (allow_sort)


def out_flow_mask(modes: LeadModes, side: str) -> np.ndarray:
    """Sec. 3.1: the modes leaving the device through this contact.  Drain (lambda =
    c_{i+1}/c_i): |lambda| < 1 for evanescent modes, dE/dk > 0 for traveling ones.
    Source (lambda_s = 1/lambda_d): |lambda_d| > 1, or dE/dk < 0."""
    absl = np.abs(modes.lam)
    v, trav = modes.dEdk, modes.traveling
    if side == "d":
        return np.where(trav, v > 0, absl < 1.0)
    if side == "s":
        return np.where(trav, v < 0, absl > 1.0)
    raise ValueError(side)


def contact(modes: LeadModes, side: str, allow_sort: bool = False) -> Contact:
    """Sec. 3.1: Sigma_i = [H'_i - E M'_i] B_i Lambda B_i^-1 from the out-flow modes;
    Sec. 3.2: B_{i,gamma} = [(H'_i - E M'_i) lambda_gamma - Sigma_i] c_gamma for
    each traveling in-flow mode.  Drain: lambda = lambda_d, K' = K_+; out-flow is
    |lambda| < 1 or traveling with dE/dk > 0.  Source: lambda_s = 1/lambda_d,
    K' = K_-; out-flow is |lambda_d| > 1 or traveling with dE/dk < 0."""
    lam, C, v, trav = modes.lam, modes.C, modes.dEdk, modes.traveling
    absl = np.abs(lam)
    n = C.shape[0]
    out = out_flow_mask(modes, side)
    sorted_ = False
    if int(out.sum()) != n:
        if not allow_sort:
            raise ModeCountError(f"{side}: {int(out.sum())} out-flow modes at Ec = {modes.Ec}, expected n = {n}")
        # diagnostic fallback: two sets of n by the out-flow score
        score = np.where(trav, np.where(v > 0, -1e-5, 1e-5), np.log(np.maximum(absl, 1e-300)))
        order = np.argsort(score, kind="stable")
        out = np.zeros(2 * n, bool)
        out[order[:n] if side == "d" else order[n:]] = True
        sorted_ = True
    if side == "d":
        inn = trav & ~out & (v < 0)
        lam_c = lam
        Kprime = modes.Kp
    else:
        inn = trav & ~out & (v > 0)
        lam_c = 1.0 / lam
        Kprime = modes.Km
    B = C[:, out]
    lo = lam_c[out]
    X = np.linalg.solve(B.T, (B * lo[None, :]).T).T      # B Lambda B^-1
    Sigma = Kprime @ X
    cin = C[:, inn]
    lin = lam_c[inn]
    rhs = (Kprime @ cin) * lin[None, :] - Sigma @ cin
    return Contact(Sigma, B, lo, v[out], trav[out], cin, lin, v[inn], rhs, Kprime, sorted_)


# =============================================================================
# Sec. 3.2 -- the QTBM system and its solution
# =============================================================================

def global_matrix(blk, Vd, Vu, E, Sig_s, Sig_d):
    """Dense A = E M - H - V^e - Sigma (Eq. qtbm_system) for nodes 1..N."""
    N, n = Vd.shape[0], blk["n"]
    A = np.zeros((N * n, N * n), complex)
    D0 = E * blk["M0"] - blk["H0"]
    U0 = E * blk["M1"] - blk["H1"]
    for i in range(N):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = D0 - Vd[i]
    for i in range(N - 1):
        Ui = U0 - Vu[i]
        A[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = Ui
        A[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = Ui.conj().T
    A[:n, :n] -= Sig_s
    A[(N - 1) * n:, (N - 1) * n:] -= Sig_d
    return A


def banded_matrix(blk, Vd, Vu, E, Sig_s, Sig_d):
    """The same matrix in LAPACK band storage (kl = ku = 2n - 1)."""
    N, n = Vd.shape[0], blk["n"]
    kl = ku = 2 * n - 1
    ab = np.zeros((kl + ku + 1, N * n), complex)

    def put(r0, c0, blockm):
        for jj in range(blockm.shape[1]):
            col = c0 + jj
            rows = np.arange(r0, r0 + blockm.shape[0])
            ab[ku + rows - col, col] = blockm[:, jj]

    D0 = E * blk["M0"] - blk["H0"]
    U0 = E * blk["M1"] - blk["H1"]
    for i in range(N):
        Di = D0 - Vd[i]
        if i == 0:
            Di = Di - Sig_s
        if i == N - 1:
            Di = Di - Sig_d
        put(i * n, i * n, Di)
    for i in range(N - 1):
        Ui = U0 - Vu[i]
        put(i * n, (i + 1) * n, Ui)
        put((i + 1) * n, i * n, Ui.conj().T)
    return ab, (kl, ku)


@dataclass
class EnergyResult:
    E: float
    T: float
    R: float
    T_modes: np.ndarray
    R_modes: np.ndarray
    T_ds: float
    node_n: np.ndarray       # (N, 2): node density per contact (source, drain)
    c: np.ndarray            # (N, n, m_s + m_d) coefficients
    g: np.ndarray            # (m_s + m_d,) density of states 2/|dE/dk|
    src: np.ndarray          # (m_s + m_d,) bool, injected from the source
    n_open_s: int
    n_open_d: int
    mode_sorted: bool = False   # a contact's modes came from the score-sort fallback


def contacts_at(blk, E, Us, Ud, cache=None, allow_sort=False, reciprocal=False):
    """Source and drain contact data at energy E with flat leads at Us and Ud."""
    def modes(Ec):
        key = (str(reciprocal), Ec) if reciprocal else Ec
        if cache is not None and key in cache:
            return cache[key]
        m = lead_modes(blk, Ec, reciprocal)
        if cache is not None:
            cache[key] = m
        return m
    ms = modes(E - Us)
    md = ms if Ud == Us else modes(E - Ud)
    return contact(ms, "s", allow_sort), contact(md, "d", allow_sort)


def solve_energy(blk, Vd, Vu, U, E, dense_limit=4000, cache=None, contacts=None, allow_sort=False,
                 reciprocal=False) -> EnergyResult:
    """Solve [E M - H - Sigma] c = B (Eq. qtbm_system) for all injected modes at E
    and reduce to T, R (Eq. transmission) and the node density (Sec. 3.3).
    Raises ModeCountError when a contact's physical out-flow count is not n, unless
    allow_sort (then the result carries mode_sorted=True).  reciprocal: lead modes
    from the reciprocal pencil (see lead_modes)."""
    N, n = Vd.shape[0], blk["n"]
    Us, Ud = float(U[0]), float(U[-1])
    cs, cd = contacts if contacts is not None else contacts_at(blk, E, Us, Ud, cache, allow_sort, reciprocal)
    ms, md = cs.c_in.shape[1], cd.c_in.shape[1]
    m = ms + md
    rhs = np.zeros((N * n, m), complex)
    rhs[:n, :ms] = cs.rhs
    rhs[(N - 1) * n:, ms:] = cd.rhs
    if m == 0:
        sol = np.zeros((N * n, 0), complex)
    elif N * n <= dense_limit:
        A = global_matrix(blk, Vd, Vu, E, cs.Sigma, cd.Sigma)
        sol = sla.solve(A, rhs)
    else:
        ab, (kl, ku) = banded_matrix(blk, Vd, Vu, E, cs.Sigma, cd.Sigma)
        sol = sla.solve_banded((kl, ku), ab, rhs)
    c = sol.reshape(N, n, m)
    return observables(E, c, cs, cd, ms, md)


def observables(E, c, cs: Contact, cd: Contact, ms: int, md: int) -> EnergyResult:
    """Eq. transmission: T_gamma = sum_{mu in traveling out-flow at d}
    |[B_d^-1 c_N]_mu|^2 v_mu / v_gamma; reflection with the injected part removed
    at node 1; node density n_E^c[i] = sum_{gamma in c} g_gamma sum_alpha
    |c_{gamma,i alpha}|^2 with g = 2/|dE/dk| (Sec. 3.3)."""
    N = c.shape[0]
    Tm = np.zeros(ms)
    Rm = np.zeros(ms)
    if ms:
        a_d = np.linalg.solve(cd.B, c[N - 1][:, :ms])
        a_s = np.linalg.solve(cs.B, c[0][:, :ms] - cs.c_in)
        vd = np.where(cd.trav_out, np.abs(cd.v_out), 0.0)
        vs = np.where(cs.trav_out, np.abs(cs.v_out), 0.0)
        Tm = (np.abs(a_d) ** 2 * vd[:, None]).sum(0) / np.abs(cs.v_in)
        Rm = (np.abs(a_s) ** 2 * vs[:, None]).sum(0) / np.abs(cs.v_in)
    T_ds = 0.0
    if md:
        a_s2 = np.linalg.solve(cs.B, c[0][:, ms:])
        vs = np.where(cs.trav_out, np.abs(cs.v_out), 0.0)
        T_ds = float(((np.abs(a_s2) ** 2 * vs[:, None]).sum(0) / np.abs(cd.v_in)).sum())
    g = np.concatenate([2.0 / np.abs(cs.v_in), 2.0 / np.abs(cd.v_in)])
    src = np.concatenate([np.ones(ms, bool), np.zeros(md, bool)])
    w = (np.abs(c) ** 2).sum(axis=1)                     # (N, m)
    node_n = np.stack([(w[:, :ms] * g[None, :ms]).sum(1), (w[:, ms:] * g[None, ms:]).sum(1)], 1)
    return EnergyResult(E, float(Tm.sum()), float(Rm.sum()), Tm, Rm, T_ds, node_n, c, g, src,
                        ms, md, bool(cs.mode_sorted or cd.mode_sorted))


# =============================================================================
# whole-system helper
# =============================================================================

@dataclass
class System:
    basis: BlochBasis
    elem: dict
    blk: dict
    U: np.ndarray
    Vd: np.ndarray
    Vu: np.ndarray


def build_system(cell, ff, gcut, n_bands, U, nq=None, basis=None) -> System:
    if basis is None:
        basis = bloch_basis(cell, ff, gcut, n_bands)
    elem = element_matrices(basis, nq)
    blk = intrinsic_blocks(elem)
    Vd, Vu = extrinsic_blocks(blk, U)
    return System(basis, elem, blk, np.asarray(U, float), Vd, Vu)


def error_bar(r: EnergyResult, *alts: EnergyResult) -> float:
    """The oracle's own rounding error at one energy, from what exact arithmetic
    fixes: total transmission is reciprocal (T_sd = T_ds for a real potential), and
    the same modes from equivalent eigen-solves (the reciprocal pencil, the Cayley
    transform; see lead_modes) give the same T, R, T_ds."""
    bar = abs(r.T - r.T_ds)
    for a in alts:
        bar = max(bar, abs(r.T - a.T), abs(r.T_ds - a.T_ds), abs(r.R - a.R))
    return bar


def perturbation_spread(blk, U, E, eps=1e-14, samples=4, seed=0):
    """How well FP64 input data determine T, R, T_ds at one energy: the largest change
    when the node blocks (H0, M0 Hermitian-symmetric; H1, M1 and the extrinsic weights)
    are perturbed by seeded random matrices of relative size eps -- the rounding that
    any FP64 assembly of the same blocks carries -- and the system is solved again
    with fresh contacts.  Part of the oracle's own error bar (see error_bar's callers)."""
    rng = np.random.default_rng(seed)
    ref = solve_energy(blk, *extrinsic_blocks(blk, U), U, E)
    worst = 0.0
    for _ in range(samples):
        b = dict(blk)
        for k in ("H0", "M0", "H1", "M1", "Wl_ll", "Wl_lr", "Wl_rr", "Wr_ll", "Wr_lr", "Wr_rr"):
            X = blk[k]
            P = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
            if k in ("H0", "M0"):
                P = 0.5 * (P + P.conj().T)
            b[k] = X + eps * np.abs(X).max() * P
        r = solve_energy(b, *extrinsic_blocks(b, U), U, E)
        worst = max(worst, abs(r.T - ref.T), abs(r.T_ds - ref.T_ds), abs(r.R - ref.R))
    return worst


def solve_workload(sys_: System, energies, cache=None):
    cache = {} if cache is None else cache
    return [solve_energy(sys_.blk, sys_.Vd, sys_.Vu, sys_.U, float(E), cache=cache)
            for E in energies]


# =============================================================================
# Sec. 5.1 -- band reconstruction
# =============================================================================

def pu_bands(blk, kprime: float):
    """Eigenvalues of H(k') c = E M(k') c with H(k') = H_ii + H_{i,i+1} e^{ik'L}
    + H_{i,i-1} e^{-ik'L} (no extrinsic potential)."""
    L = blk["L"]
    ph = np.exp(1j * kprime * L)
    H = blk["H0"] + blk["H1"] * ph + blk["H1"].conj().T / ph
    M = blk["M0"] + blk["M1"] * ph + blk["M1"].conj().T / ph
    H = 0.5 * (H + H.conj().T)
    M = 0.5 * (M + M.conj().T)
    return sla.eigh(H, M, eigvals_only=True)


# =============================================================================
# Sec. 3.3 -- density: naive route and density-matrix route
# =============================================================================

def fermi(x, kT):
    return 0.5 * (1.0 - np.tanh(0.5 * x / kT))


def basis_on_grid(basis: BlochBasis, nx: int, nz: int):
    """phi_{l,alpha}(x_j, s_q) on the element grid x_j = j Lx/nx, s_q = (q+1/2) L/nz
    (left-node phase).  Returns Phi (nx*nz, n), s (nz,)."""
    cell = basis.cell
    L, Lx = cell.Lz, cell.Lx
    xs = np.arange(nx) * (Lx / nx) if cell.dim == 2 else np.zeros(1)
    ss = (np.arange(nz) + 0.5) * (L / nz)
    bz = 2.0 * math.pi / L
    bx = 2.0 * math.pi / Lx if cell.dim == 2 else 0.0
    X, S = np.meshgrid(xs, ss, indexing="ij")
    cols = []
    for g in basis.groups:
        ex = np.exp(1j * (np.outer(X.ravel(), g["mx"] * bx)
                          + np.outer(S.ravel(), g["mz"] * bz + g["k"])))
        cols.append(ex @ g["C"])
    return np.concatenate(cols, axis=1), ss


def density_naive(basis: BlochBasis, results, weights, mu_s, mu_d, kT, nx, nz):
    """Eq. density_3d: n(r) = sum_E w_E sum_nu g_nu |psi_nu(r)|^2 f_FD(E - mu_nu),
    psi evaluated directly from Eq. wavef_expansion on every device element.
    Returns (N-1, nx_eff, nz)."""
    Phi, ss = basis_on_grid(basis, nx, nz)
    L = basis.cell.Lz
    phr = np.exp(-1j * basis.kz * L)
    nxe = Phi.shape[0] // nz
    fl = np.tile(1.0 - ss / L, nxe)
    fr = np.tile(ss / L, nxe)
    N = results[0].c.shape[0]
    dens = np.zeros((N - 1, Phi.shape[0]))
    for r, w in zip(results, weights):
        occ = np.where(r.src, fermi(r.E - mu_s, kT), fermi(r.E - mu_d, kT))
        wt = w * r.g * occ
        for e in range(N - 1):
            psi = fl[:, None] * (Phi @ r.c[e]) + fr[:, None] * ((Phi * phr[None, :]) @ r.c[e + 1])
            dens[e] += (np.abs(psi) ** 2 * wt[None, :]).sum(1)
    return dens.reshape(N - 1, nxe, nz)


def density_matrix(results, weights, mu_s, mu_d, kT):
    """Eq. density_matrices: rho_{a alpha, b beta} = sum_{E,nu} w g f_FD c^*_{a alpha} c_{b beta}
    for b in {a, a+1}.  Returns rho_d (N, n, n) and rho_u (N-1, n, n)."""
    N, n = results[0].c.shape[:2]
    rd = np.zeros((N, n, n), complex)
    ru = np.zeros((max(N - 1, 0), n, n), complex)
    for r, w in zip(results, weights):
        occ = np.where(r.src, fermi(r.E - mu_s, kT), fermi(r.E - mu_d, kT))
        wt = w * r.g * occ
        for a in range(N):
            rd[a] += (r.c[a].conj() * wt[None, :]) @ r.c[a].T
        for a in range(N - 1):
            ru[a] += (r.c[a].conj() * wt[None, :]) @ r.c[a + 1].T
    return rd, ru


def density_from_matrix(basis: BlochBasis, rd, ru, nx, nz):
    """Eq. density_3d_fast: n(r) = sum_{a,b} f_a f_b sum_{alpha beta}
    rho_{a alpha, b beta} phi^*_{a alpha}(r) phi_{b beta}(r) on each element."""
    Phi, ss = basis_on_grid(basis, nx, nz)
    L = basis.cell.Lz
    phr = np.exp(-1j * basis.kz * L)
    Phr = Phi * phr[None, :]
    nxe = Phi.shape[0] // nz
    fl = np.tile(1.0 - ss / L, nxe)
    fr = np.tile(ss / L, nxe)
    N = rd.shape[0]
    dens = np.zeros((N - 1, Phi.shape[0]))
    for e in range(N - 1):
        t_ll = np.einsum("pa,ab,pb->p", Phi.conj(), rd[e], Phi)
        t_rr = np.einsum("pa,ab,pb->p", Phr.conj(), rd[e + 1], Phr)
        t_lr = np.einsum("pa,ab,pb->p", Phi.conj(), ru[e], Phr)
        dens[e] = (fl * fl * t_ll + fr * fr * t_rr + 2.0 * fl * fr * t_lr).real
    return dens.reshape(N - 1, nxe, nz)


# =============================================================================
# Sec. 3.3 (density integral) and Eq. current -- adaptive Simpson integration
# =============================================================================

# 2e^2/h in A/V: with energies in eV, I [A] = G0 * integral of (T_sd f_s - T_ds f_d) dE [eV]
G0_SIEMENS = 2.0 * 1.602176634e-19 ** 2 / 6.62607015e-34


def adaptive_simpson(f, a, b, tol, min_pieces=8, max_evals=4000):
    """Adaptive Simpson quadrature of a (vector-valued) f over [a, b] (Sec. 3.3: the
    energy integrals are evaluated adaptively to a prescribed tolerance).

    [a, b] starts as min_pieces equal intervals.  An interval of length h with
    midpoint m and quarter points l, r is accepted when the one- and two-panel
    Simpson estimates S1 = h/6 (f_a + 4 f_m + f_b) and S2 = h/12 (f_a + 4 f_l +
    2 f_m + 4 f_r + f_b) differ by at most 15 tol h / (b - a) in the max norm over
    the components; it then contributes S2 + (S2 - S1)/15 (Richardson), otherwise
    each half is treated the same way.  When max_evals evaluations have been spent,
    the intervals still open are accepted as they stand.
    Returns (integral, error estimate sum |S2 - S1| / 15, sorted energies used,
    their quadrature weights)."""
    cache = {}

    def F(x):
        if x not in cache:
            cache[x] = np.atleast_1d(np.asarray(f(x), dtype=float))
        return cache[x]

    total = np.zeros_like(F(a))
    err = 0.0
    weights = {}
    L = b - a

    def accept(x0, x1, S1, S2):
        nonlocal total, err
        total = total + S2 + (S2 - S1) / 15.0
        err += float(np.max(np.abs(S2 - S1))) / 15.0
        h = x1 - x0
        xm = x0 + (x1 - x0) / 2
        for x, w in zip((x0, x0 + (xm - x0) / 2, xm, xm + (x1 - xm) / 2, x1), (7, 32, 12, 32, 7)):
            weights[x] = weights.get(x, 0.0) + w * h / 90.0

    def piece(x0, x1):
        # depth first, left half before right half (an explicit stack instead of recursion)
        stack = [(x0, x1)]
        while stack:
            x0, x1 = stack.pop()
            h = x1 - x0
            # nested midpoints: a half's own midpoint is computed by the same expression
            # as this interval's quarter point, so the halves reuse these energies exactly
            xm = x0 + (x1 - x0) / 2
            xl, xr = x0 + (xm - x0) / 2, xm + (x1 - xm) / 2
            fa, fm, fb = F(x0), F(xm), F(x1)
            fl, fr = F(xl), F(xr)
            S1 = h / 6.0 * (fa + 4 * fm + fb)
            S2 = h / 12.0 * (fa + 4 * fl + 2 * fm + 4 * fr + fb)
            if np.max(np.abs(S2 - S1)) <= 15.0 * tol * h / L or len(cache) >= max_evals or h <= L * 2.0 ** -40:
                accept(x0, x1, S1, S2)
            else:
                stack.append((xm, x1))
                stack.append((x0, xm))

    edges = a + (b - a) * np.arange(min_pieces + 1) / min_pieces
    for k in range(min_pieces):
        piece(float(edges[k]), float(edges[k + 1]))
    xs = np.array(sorted(weights))
    return total, err, xs, np.array([weights[x] for x in xs])


def current_integrand(sys_, mu_s, mu_d, kT, cache=None):
    """Eq. current (reading): G0 (T_sd(E) f(E - mu_s) - T_ds(E) f(E - mu_d)), in A/eV."""
    def f(E):
        r = solve_energy(sys_.blk, sys_.Vd, sys_.Vu, sys_.U, float(E), cache=cache)
        return G0_SIEMENS * (r.T * fermi(E - mu_s, kT) - r.T_ds * fermi(E - mu_d, kT))
    return f


def node_density_integrand(sys_, mu_s, mu_d, kT, cache=None):
    """Node density per energy (Sec. 3.3): n^s[i] f(E - mu_s) + n^d[i] f(E - mu_d)."""
    def f(E):
        r = solve_energy(sys_.blk, sys_.Vd, sys_.Vu, sys_.U, float(E), cache=cache)
        return r.node_n[:, 0] * fermi(E - mu_s, kT) + r.node_n[:, 1] * fermi(E - mu_d, kT)
    return f


# =============================================================================
# Sec. 3.2 (NEGF alternative) -- transmission from the Green's function
# =============================================================================

def caroli_transmission(blk, Vd, Vu, U, E, cache=None, contacts=None):
    """T(E) = Tr[Gamma_d G_{N1} Gamma_s G_{N1}^dagger] with G = [E M - H - Sigma]^{-1}
    (the Green's function of Sec. 3.2) and Gamma_c = i (Sigma_c - Sigma_c^dagger):
    the source-to-drain transmission without any mode decomposition at the drain.
    G_{N1} is the last node's block of the solution with the identity injected at
    the first node."""
    N, n = Vd.shape[0], blk["n"]
    cs, cd = contacts if contacts is not None else contacts_at(blk, E, float(U[0]), float(U[-1]), cache)
    rhs = np.zeros((N * n, n), complex)
    rhs[:n] = np.eye(n)
    if N * n <= 4000:
        G1 = sla.solve(global_matrix(blk, Vd, Vu, E, cs.Sigma, cd.Sigma), rhs)
    else:
        ab, (kl, ku) = banded_matrix(blk, Vd, Vu, E, cs.Sigma, cd.Sigma)
        G1 = sla.solve_banded((kl, ku), ab, rhs)
    X = G1[(N - 1) * n:]
    Gs = 1j * (cs.Sigma - cs.Sigma.conj().T)
    Gd = 1j * (cd.Sigma - cd.Sigma.conj().T)
    return float(np.trace(Gd @ X @ Gs @ X.conj().T).real)



def green_diagonal(blk, Vd, Vu, U, E, cache=None, contacts=None):
    """Diagonal blocks G_ii of the retarded Green's function G = [E M - H - V^e -
    Sigma]^{-1} (the NEGF form of Sec. 3.2) and the node spectral density
    -(2/pi) Im Tr G_ii.  By definition: the inverse of the assembled global matrix
    (dense; N n <= 4000), then its diagonal blocks.  Returns (G_diag (N, n, n),
    node_dos (N,))."""
    N, n = Vd.shape[0], blk["n"]
    if N * n > 4000:
        raise ValueError("green_diagonal takes N n <= 4000 (dense inverse)")
    cs, cd = contacts if contacts is not None else contacts_at(blk, E, float(U[0]), float(U[-1]), cache)
    G = np.linalg.inv(global_matrix(blk, Vd, Vu, E, cs.Sigma, cd.Sigma))
    Gd = np.stack([G[i * n:(i + 1) * n, i * n:(i + 1) * n] for i in range(N)])
    dos = -(2.0 / math.pi) * np.array([np.trace(b).imag for b in Gd])
    return Gd, dos

# =============================================================================
# Sec. 4 (self-consistent loop): non-linear Poisson by Newton with the semi-classical
# Jacobian and DIIS, on a 1D finite-element model along z
# =============================================================================

def dfermi(x, kT):
    """-d f_FD / dE at E - mu = x."""
    t = np.tanh(0.5 * x / kT)
    return 0.25 * (1.0 - t * t) / kT


@dataclass
class Poisson1D:
    """1D model of Eq. nonlin_poisson_fem on the node hats f_i (the same hats as the
    basis): (kappa S + gamma M) U = gamma M U_gate + alpha M (n[U] - n_dop), with
    S_ij = int f_i' f_j' dz, M_ij = int f_i f_j dz; U is the electron potential
    energy (eV) on the nodes, fixed at both ends by the contacts (Dirichlet),
    n the node density per nm (Sec. 3.3) integrated over energy with f_FD."""
    kappa: float                 # stiffness (eV nm)
    gamma: float                 # coupling to the gate (eV / nm)
    alpha: float                 # charge coupling (eV nm per unit of n)
    U_gate: np.ndarray           # (N,) gate potential energy
    n_dop: np.ndarray            # (N,) fixed background in the units of n


def poisson1d_matrices(N, L):
    S = (np.diag(np.full(N, 2.0)) - np.diag(np.ones(N - 1), 1) - np.diag(np.ones(N - 1), -1)) / L
    M = (np.diag(np.full(N, 4.0)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)) * L / 6.0
    S[0, 0] = S[-1, -1] = 1.0 / L
    M[0, 0] = M[-1, -1] = L / 3.0
    return S, M


def density_and_jacobian(sys_, mu_s, mu_d, kT, E_lo, E_hi, tol, cache=None, max_evals=4000):
    """n_i = int [n^s_i f(E - mu_s) + n^d_i f(E - mu_d)] dE / L and the semi-classical
    Jacobian diagonal d_i = int [n^s_i (-f') + n^d_i (-f')] dE / L (Eq. density_jacobian),
    both from one adaptive integration of the stacked integrand."""
    N = sys_.Vd.shape[0]
    L = sys_.blk["L"]

    def f(E):
        r = solve_energy(sys_.blk, sys_.Vd, sys_.Vu, sys_.U, float(E), cache=cache)
        ns, nd = r.node_n[:, 0], r.node_n[:, 1]
        return np.concatenate([ns * fermi(E - mu_s, kT) + nd * fermi(E - mu_d, kT),
                               ns * dfermi(E - mu_s, kT) + nd * dfermi(E - mu_d, kT)])

    I, err, xs, w = adaptive_simpson(f, E_lo, E_hi, tol, max_evals=max_evals)
    return I[:N] / L, I[N:] / L, len(xs)


def self_consistent(sys_, model: Poisson1D, mu_s, mu_d, kT, E_lo, E_hi, tol_int, tol_sc=1e-6,
                    max_iters=60, diis_window=5, cache=None):
    """Newton-Raphson on F(U) = (kappa S + gamma M) U - gamma M U_gate - alpha M (n[U] - n_dop)
    (Eq. newton_poisson) over the interior nodes, with the Jacobian kappa S + gamma M +
    alpha M diag(d) (n decreases where U rises: dn_i/dU_i ~ -d_i, Eq. density_jacobian);
    the Newton output and its step R = U_new - U enter a DIIS subspace of the last
    diis_window iterates (Sec. 4: least squares by SVD) whose extrapolation is the next
    U (diis_window <= 1: plain Newton).  Stops when ||R||_2 <= tol_sc (eV).
    Returns (U, history of ||R||_2, n, d)."""
    N = sys_.Vd.shape[0]
    L = sys_.blk["L"]
    S, M = poisson1d_matrices(N, L)
    K = model.kappa * S + model.gamma * M
    U = np.array(sys_.U, dtype=float)
    inner = slice(1, N - 1)
    hist, Us, Rs = [], [], []
    n = d = None
    for _ in range(max_iters):
        s = System(sys_.basis, sys_.elem, sys_.blk, U, *extrinsic_blocks(sys_.blk, U))
        n, d, _ = density_and_jacobian(s, mu_s, mu_d, kT, E_lo, E_hi, tol_int, cache)
        F = K @ U - model.gamma * M @ model.U_gate - model.alpha * M @ (n - model.n_dop)
        J = K + model.alpha * M @ np.diag(d)
        step = np.zeros(N)
        step[inner] = -np.linalg.solve(J[inner, inner], F[inner])
        U_new = U + step
        hist.append(float(np.linalg.norm(step)))
        if hist[-1] <= tol_sc:
            return U_new, hist, n, d
        if diis_window > 1:
            Us.append(U_new.copy())
            Rs.append(step.copy())
            Us, Rs = Us[-diis_window:], Rs[-diis_window:]
            if len(Us) > 1:
                # min || R_m + sum_k c_k (R_k - R_m) ||, coefficients of the older iterates
                A = np.stack([Rs[k] - Rs[-1] for k in range(len(Rs) - 1)], axis=1)
                c, *_ = np.linalg.lstsq(A, -Rs[-1], rcond=1e-10)
                U_new = Us[-1] + sum(c[k] * (Us[k] - Us[-1]) for k in range(len(c)))
        U = U_new
    return U, hist, n, d
