"""Thin ctypes binding of libpwqt (include/pwqt.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  The library must have been built (paper_1903_00548_gb300.build);
loading fails loudly when it is missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpwqt.so")

PWQT_OK = 0
ERR_NAMES = {-1: "INVALID_ARG", -2: "BASIS_TOO_SMALL", -3: "OOM", -4: "CUDA", -5: "STATE", -6: "NO_DEVICE",
             -7: "TIMEOUT", -8: "BUSY"}
ERR_TIMEOUT = -7
INTEGRAND_CURRENT, INTEGRAND_NODE_DENSITY, INTEGRAND_NODE_DENSITY_JACOBIAN = 0, 1, 2
FP64, MIXED, FP32 = 0, 1, 2
ST_SINGULAR_PIVOT, ST_MODE_COUNT, ST_IR_NO_CONVERGE, ST_DEGENERATE, ST_NEAR_UNIT = 1, 2, 4, 8, 16
RESIDUAL_SLICED, RESIDUAL_FLOAT_FLOAT = 0, 1

EXPORTS = ["pwqt_create", "pwqt_destroy", "pwqt_last_error", "pwqt_assemble_intrinsic", "pwqt_set_enhancement",
           "pwqt_get_blocks", "pwqt_set_extrinsic", "pwqt_solve", "pwqt_solve_dev", "pwqt_prepare_leads",
           "pwqt_cache_info", "pwqt_bands", "pwqt_kernel_launches", "pwqt_profile", "pwqt_solve_noalloc", "pwqt_cgemm_c64",
           "pwqt_density_reset", "pwqt_accumulate_density", "pwqt_get_density_matrix", "pwqt_density_grid",
           "pwqt_profile_refinement", "pwqt_set_refinement", "pwqt_set_residual", "pwqt_profile_residual", "pwqt_profile_correction", "pwqt_solve_multi",
           "pwqt_server_create", "pwqt_server_add_basis", "pwqt_server_submit", "pwqt_server_wait",
           "pwqt_server_stats", "pwqt_server_batch_stats", "pwqt_server_last_error", "pwqt_server_destroy", "pwqt_integrate",
           "pwqt_transmission_caroli", "pwqt_self_consistent", "pwqt_green_diagonal"]


class PwqtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pwqt error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("ir_tol", C.c_double),
                ("ir_max_iters", C.c_int), ("batch", C.c_int)]


class ServerOpts(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("queue_capacity", C.c_int),
                ("ir_tol", C.c_double), ("batch", C.c_int)]


class RequestC(C.Structure):
    _fields_ = [("basis", C.c_int), ("n_nodes", C.c_int), ("U", C.POINTER(C.c_double)), ("n_E", C.c_int),
                ("E", C.POINTER(C.c_double)), ("precision", C.c_int),
                ("T", C.POINTER(C.c_double)), ("R", C.POINTER(C.c_double)), ("T_ds", C.POINTER(C.c_double)),
                ("n_open", C.POINTER(C.c_int)), ("node_n", C.POINTER(C.c_double)), ("resid", C.POINTER(C.c_double)),
                ("iters", C.POINTER(C.c_int)), ("status", C.POINTER(C.c_int))]


class Poisson1DC(C.Structure):
    _fields_ = [("kappa", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
                ("U_gate", C.POINTER(C.c_double)), ("n_dop", C.POINTER(C.c_double))]


class CellC(C.Structure):
    _fields_ = [("dim", C.c_int), ("Lz", C.c_double), ("Lx", C.c_double), ("n_atoms", C.c_int),
                ("atoms", C.POINTER(C.c_double)), ("omega0", C.c_double)]


class FormFactorC(C.Structure):
    _fields_ = [("v0", C.c_double), ("sigma", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libpwqt.so (no fallback: raises if the library is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpwqt not built: {path} missing (run python -m paper_1903_00548_gb300.build)")
    lib = C.CDLL(path)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.pwqt_create.argtypes = [C.POINTER(P), C.POINTER(Opts)]
    lib.pwqt_destroy.argtypes = [P]
    lib.pwqt_last_error.argtypes = [P]
    lib.pwqt_last_error.restype = C.c_char_p
    lib.pwqt_assemble_intrinsic.argtypes = [P, C.POINTER(CellC), C.POINTER(FormFactorC), D, I, ip]
    lib.pwqt_set_enhancement.argtypes = [P, C.POINTER(CellC), I, dp, ip, ip, ip, dp, ip]
    lib.pwqt_get_blocks.argtypes = [P, dp, dp, dp, dp, dp]
    lib.pwqt_set_extrinsic.argtypes = [P, I, I, dp]
    lib.pwqt_solve.argtypes = [P, I, I, dp, I, dp, dp, dp, ip, dp, dp, ip, ip]
    lib.pwqt_solve_dev.argtypes = [P, I, I, dp, I, P, P, P, P, P, P, P, P, P]
    lib.pwqt_prepare_leads.argtypes = [P, I, I, dp]
    lib.pwqt_cache_info.argtypes = [P, ip, C.POINTER(S)]
    lib.pwqt_bands.argtypes = [P, I, dp, dp]
    lib.pwqt_kernel_launches.argtypes = [P, C.POINTER(C.c_longlong), I]
    lib.pwqt_profile.argtypes = [P, I, dp, C.POINTER(C.c_longlong), dp, I]
    lib.pwqt_solve_noalloc.argtypes = [P, I, I, dp, P, P, P, P, P, P]
    lib.pwqt_density_reset.argtypes = [P, I]
    lib.pwqt_profile_refinement.argtypes = [P, dp, dp, C.POINTER(C.c_longlong)]
    lib.pwqt_set_refinement.argtypes = [P, D, I]
    lib.pwqt_set_residual.argtypes = [P, I]
    lib.pwqt_profile_residual.argtypes = [P, dp, dp, dp, C.POINTER(C.c_longlong)]
    lib.pwqt_profile_correction.argtypes = [P, dp, dp, C.POINTER(C.c_longlong)]
    lib.pwqt_solve_multi.argtypes = [P, I, ip, I, dp, I, dp, dp, dp, ip, dp, dp, ip, ip]
    lib.pwqt_server_create.argtypes = [C.POINTER(P), C.POINTER(ServerOpts)]
    lib.pwqt_server_add_basis.argtypes = [P, I, C.POINTER(CellC), C.POINTER(FormFactorC), D, I, ip]
    lib.pwqt_server_submit.argtypes = [P, C.POINTER(RequestC), C.POINTER(C.c_longlong)]
    lib.pwqt_server_wait.argtypes = [P, C.c_longlong, D, ip, dp]
    lib.pwqt_server_stats.argtypes = [P, C.POINTER(C.c_longlong), dp, dp, C.POINTER(S), I]
    lib.pwqt_server_batch_stats.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.pwqt_server_last_error.argtypes = [P]
    lib.pwqt_server_last_error.restype = C.c_char_p
    lib.pwqt_server_destroy.argtypes = [P]
    lib.pwqt_integrate.argtypes = [P, I, I, D, D, D, D, D, D, I, I, I, dp, dp, ip, dp, dp, ip, I]
    lib.pwqt_transmission_caroli.argtypes = [P, I, I, dp, dp, ip]
    lib.pwqt_green_diagonal.argtypes = [P, I, I, dp, dp, dp, ip]
    lib.pwqt_self_consistent.argtypes = [P, I, C.POINTER(Poisson1DC), D, D, D, D, D, D, D, I, I, I, dp, dp, ip, dp]
    lib.pwqt_accumulate_density.argtypes = [P, I, I, dp, dp, D, D, D, I, ip]
    lib.pwqt_get_density_matrix.argtypes = [P, I, dp, dp]
    lib.pwqt_density_grid.argtypes = [P, I, I, I, dp]
    fp = C.POINTER(C.c_float)
    lib.pwqt_cgemm_c64.argtypes = [I, I, I, I, fp, I, fp, I, fp, I]
    for f in EXPORTS:
        if f not in ("pwqt_last_error", "pwqt_server_last_error"):
            getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def _cell(cell):
    atoms = np.ascontiguousarray(cell.atoms, dtype=np.float64).ravel()
    c = CellC(cell.dim, cell.Lz, cell.Lx, len(cell.atoms), _dptr(atoms), cell.omega0)
    return c, atoms


@dataclass
class SolveResult:
    T: np.ndarray
    R: np.ndarray
    T_ds: np.ndarray
    n_open: np.ndarray      # (n_E, 2)
    node_n: np.ndarray      # (n_E, N, 2)
    resid: np.ndarray
    iters: np.ndarray
    status: np.ndarray


def cgemm_c64(a, b, c):
    """c -= a @ b on the tensor cores for batched complex64 arrays (batch, M, K), (batch, K, N),
    (batch, M, N); returns the updated copy of c."""
    lib = load()
    a = np.ascontiguousarray(a, dtype=np.complex64)
    b = np.ascontiguousarray(b, dtype=np.complex64)
    out = np.array(c, dtype=np.complex64, order="C", copy=True)
    nb, M, K = a.shape
    N = b.shape[2]
    fp = lambda x: x.ctypes.data_as(C.POINTER(C.c_float))
    r = lib.pwqt_cgemm_c64(nb, M, N, K, fp(a), K, fp(b), N, fp(out), N)
    if r != PWQT_OK:
        raise PwqtError(r, "pwqt_cgemm_c64 failed")
    return out


class Context:
    """One libpwqt context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, ir_tol: float = 0.0, ir_max_iters: int = 0,
                 batch: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        o = Opts(device, hbm_budget_bytes, ir_tol, ir_max_iters, batch)
        r = self.lib.pwqt_create(C.byref(self.h), C.byref(o))
        if r != PWQT_OK:
            raise PwqtError(r, "pwqt_create failed")
        self.n = 0
        self.n_nodes = {}

    def close(self):
        if self.h:
            self.lib.pwqt_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, r):
        if r != PWQT_OK:
            raise PwqtError(r, self.lib.pwqt_last_error(self.h).decode())

    def assemble_intrinsic(self, cell, ff, gcut: float, n_bands: int) -> int:
        cc, keep = _cell(cell)
        f = FormFactorC(ff.v0, ff.sigma)
        n = C.c_int()
        self._check(self.lib.pwqt_assemble_intrinsic(self.h, C.byref(cc), C.byref(f), gcut, n_bands, C.byref(n)))
        self.n = n.value
        self.dim = cell.dim
        self.n_nodes = {}
        return self.n

    def set_enhancement(self, cell, eps, groups) -> int:
        """groups: [(mx, mz, C (n_pw x n_bands complex)), ...] for k = 0 and k = pi/Lz."""
        cc, keep = _cell(cell)
        nb = groups[0][2].shape[1]
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        n_pw = np.array([len(g[0]) for g in groups], dtype=np.int32)
        mx = np.ascontiguousarray(np.concatenate([g[0] for g in groups]), dtype=np.int32)
        mz = np.ascontiguousarray(np.concatenate([g[1] for g in groups]), dtype=np.int32)
        coef = np.ascontiguousarray(np.concatenate([g[2] for g in groups], axis=0), dtype=np.complex128)
        n = C.c_int()
        self._check(self.lib.pwqt_set_enhancement(self.h, C.byref(cc), nb, _dptr(eps), _iptr(n_pw), _iptr(mx), _iptr(mz),
                                                  coef.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n)))
        self.n = n.value
        self.dim = cell.dim
        self.n_nodes = {}
        return self.n

    def get_blocks(self):
        n = self.n
        H0, H1, M0, M1 = (np.zeros((n, n), np.complex128) for _ in range(4))
        W = np.zeros((6, n, n), np.complex128)
        ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self.lib.pwqt_get_blocks(self.h, ptr(H0), ptr(H1), ptr(M0), ptr(M1), ptr(W)))
        return dict(H0=H0, H1=H1, M0=M0, M1=M1, W=W)

    def set_extrinsic(self, sys: int, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        self._check(self.lib.pwqt_set_extrinsic(self.h, sys, len(U), _dptr(U)))
        self.n_nodes[sys] = len(U)

    def prepare_leads(self, sys: int, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        self._check(self.lib.pwqt_prepare_leads(self.h, sys, len(E), _dptr(E)))

    def solve(self, sys: int, E, precision: int = FP64) -> SolveResult:
        E = np.ascontiguousarray(E, dtype=np.float64)
        nE, N = len(E), self.n_nodes.get(sys, 0)
        T, R, Tds, resid = (np.zeros(nE) for _ in range(4))
        nopen = np.zeros((nE, 2), np.int32)
        node_n = np.zeros((nE, N, 2))
        iters = np.zeros(nE, np.int32)
        status = np.zeros(nE, np.int32)
        self._check(self.lib.pwqt_solve(self.h, sys, nE, _dptr(E), precision, _dptr(T), _dptr(R), _dptr(Tds), _iptr(nopen),
                                        _dptr(node_n), _dptr(resid), _iptr(iters), _iptr(status)))
        return SolveResult(T, R, Tds, nopen, node_n, resid, iters, status)

    def solve_multi(self, systems, E, precision: int = FP64):
        """pwqt_solve_multi: one SolveResult per system (node_n shaped by each system's node count)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        ids = np.ascontiguousarray(systems, dtype=np.int32)
        nS, nE = len(ids), len(E)
        Ns = [self.n_nodes.get(int(q), 0) for q in ids]
        T, R, Tds, resid = (np.zeros(nS * nE) for _ in range(4))
        nopen = np.zeros((nS * nE, 2), np.int32)
        node_n = np.zeros(sum(nE * N * 2 for N in Ns))
        iters = np.zeros(nS * nE, np.int32)
        status = np.zeros(nS * nE, np.int32)
        self._check(self.lib.pwqt_solve_multi(self.h, nS, _iptr(ids), nE, _dptr(E), precision, _dptr(T), _dptr(R), _dptr(Tds),
                                              _iptr(nopen), _dptr(node_n), _dptr(resid), _iptr(iters), _iptr(status)))
        out, off = [], 0
        for q, N in enumerate(Ns):
            sl = slice(q * nE, (q + 1) * nE)
            nn = node_n[off: off + nE * N * 2].reshape(nE, N, 2)
            off += nE * N * 2
            out.append(SolveResult(T[sl], R[sl], Tds[sl], nopen[sl], nn, resid[sl], iters[sl], status[sl]))
        return out

    def solve_dev(self, sys: int, E, precision: int, out: dict, stream_ptr: int = 0):
        """Device-buffer variant: `out` maps output names to device pointers (int) or None."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        g = lambda k: C.c_void_p(out.get(k)) if out.get(k) else None
        self._check(self.lib.pwqt_solve_dev(self.h, sys, len(E), _dptr(E), precision, g("T"), g("R"), g("T_ds"),
                                            g("n_open"), g("node_n"), g("resid"), g("iters"), g("status"),
                                            C.c_void_p(stream_ptr) if stream_ptr else None))

    def solve_noalloc(self, sys: int, E, out: dict, stream_ptr: int = 0):
        """Allocation-free FP64 solve into caller-owned device buffers; `out` maps
        T, R, T_ds, node_n (required) and status (optional) to device pointers."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        g = lambda k: C.c_void_p(out.get(k)) if out.get(k) else None
        self._check(self.lib.pwqt_solve_noalloc(self.h, sys, len(E), _dptr(E), g("T"), g("R"), g("T_ds"), g("node_n"),
                                                g("status"), C.c_void_p(stream_ptr) if stream_ptr else None))

    def integrate(self, sys: int, integrand: int, E_lo: float, E_hi: float, mu_s: float, mu_d: float, kT: float,
                  tol: float, min_pieces: int = 8, max_evals: int = 4000, precision: int = FP64, max_points: int = 20000):
        """Adaptive Simpson integral: (result, error estimate, energies solved, quadrature energies, weights)."""
        N = self.n_nodes.get(sys, 1)   # an unknown system is reported by the library
        dim = {INTEGRAND_CURRENT: 1, INTEGRAND_NODE_DENSITY: N}.get(integrand, 2 * N)
        res = np.zeros(dim)
        err = C.c_double()
        ne, npts = C.c_int(), C.c_int()
        xs = np.zeros(max_points)
        ws = np.zeros(max_points)
        self._check(self.lib.pwqt_integrate(self.h, sys, integrand, E_lo, E_hi, mu_s, mu_d, kT, tol, min_pieces, max_evals,
                                            precision, _dptr(res), C.byref(err), C.byref(ne), _dptr(xs), _dptr(ws),
                                            C.byref(npts), max_points))
        k = min(npts.value, max_points)
        return res, err.value, ne.value, xs[:k].copy(), ws[:k].copy()

    def self_consistent(self, sys: int, U0, kappa: float, gamma: float, alpha: float, U_gate, n_dop, mu_s: float,
                        mu_d: float, kT: float, E_lo: float, E_hi: float, tol_int: float, tol_sc: float = 1e-6,
                        max_iters: int = 60, diis_window: int = 5, precision: int = FP64):
        """(U, history of Newton-step norms, n) of the self-consistent loop; raises if not converged."""
        U = np.ascontiguousarray(U0, dtype=np.float64).copy()
        Ug = np.ascontiguousarray(U_gate, dtype=np.float64)
        nd = np.ascontiguousarray(n_dop, dtype=np.float64)
        model = Poisson1DC(kappa, gamma, alpha, _dptr(Ug), _dptr(nd))
        hist = np.zeros(max_iters)
        it = C.c_int()
        n = np.zeros(len(U))
        self._check(self.lib.pwqt_self_consistent(self.h, sys, C.byref(model), mu_s, mu_d, kT, E_lo, E_hi, tol_int, tol_sc,
                                                  max_iters, diis_window, precision, _dptr(U), _dptr(hist), C.byref(it),
                                                  _dptr(n)))
        self.n_nodes[sys] = len(U)
        return U, hist[:it.value].copy(), n

    def transmission_caroli(self, sys: int, E):
        """(T, status) from the Green's function, per energy."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        T = np.zeros(len(E))
        st = np.zeros(len(E), np.int32)
        self._check(self.lib.pwqt_transmission_caroli(self.h, sys, len(E), _dptr(E), _dptr(T), _iptr(st)))
        return T, st

    def green_diagonal(self, sys: int, E, blocks: bool = False):
        """(node_dos [n_E, N], G_diag [n_E, N, n, n] complex or None, status) from the
        recursive Green's function."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        N = self.n_nodes.get(sys, 1)   # an unknown system is reported by the library
        dos = np.zeros((len(E), N))
        G = np.zeros((len(E), N, self.n, self.n), np.complex128) if blocks else None
        st = np.zeros(len(E), np.int32)
        gp = G.ctypes.data_as(C.POINTER(C.c_double)) if blocks else None
        self._check(self.lib.pwqt_green_diagonal(self.h, sys, len(E), _dptr(E), _dptr(dos), gp, _iptr(st)))
        return dos, G, st

    def density_reset(self, sys: int):
        self._check(self.lib.pwqt_density_reset(self.h, sys))

    def accumulate_density(self, sys: int, E, w, mu_s: float, mu_d: float, kT: float, precision: int = FP64):
        """Solve at E and add w-weighted contributions to the density matrix; returns the statuses."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        w = np.ascontiguousarray(np.broadcast_to(w, E.shape), dtype=np.float64)
        status = np.zeros(len(E), np.int32)
        self._check(self.lib.pwqt_accumulate_density(self.h, sys, len(E), _dptr(E), _dptr(w), mu_s, mu_d, kT, precision,
                                                     _iptr(status)))
        return status

    def density_matrix(self, sys: int):
        """(rho_d (N, n, n), rho_u (N-1, n, n)) complex128."""
        N, n = self.n_nodes[sys], self.n
        rd = np.zeros((N, n, n), np.complex128)
        ru = np.zeros((max(N - 1, 0), n, n), np.complex128)
        ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self.lib.pwqt_get_density_matrix(self.h, sys, ptr(rd), ptr(ru)))
        return rd, ru

    def density_grid(self, sys: int, nx: int, nz: int):
        """n(r) per element: array (N-1, nx or 1, nz)."""
        N = self.n_nodes[sys]
        nxe = nx if getattr(self, "dim", 1) == 2 else 1
        out = np.zeros((max(N - 1, 0), nxe, nz))
        self._check(self.lib.pwqt_density_grid(self.h, sys, nx, nz, _dptr(out)))
        return out

    def cache_info(self):
        e, b = C.c_int(), C.c_size_t()
        self._check(self.lib.pwqt_cache_info(self.h, C.byref(e), C.byref(b)))
        return e.value, b.value

    def bands(self, k):
        k = np.ascontiguousarray(k, dtype=np.float64)
        out = np.zeros((len(k), self.n))
        self._check(self.lib.pwqt_bands(self.h, len(k), _dptr(k), _dptr(out)))
        return out

    def profile(self, enable: bool = True, reset: bool = False):
        ms, cnt, fl = C.c_double(), C.c_longlong(), C.c_double()
        self._check(self.lib.pwqt_profile(self.h, 1 if enable else 0, C.byref(ms), C.byref(cnt), C.byref(fl),
                                          1 if reset else 0))
        return ms.value, cnt.value, fl.value

    def set_refinement(self, ir_tol: float = 0.0, ir_max_iters: int = 0):
        self._check(self.lib.pwqt_set_refinement(self.h, ir_tol, ir_max_iters))

    def set_residual(self, kind: int):
        """Refinement residual of the mixed path: RESIDUAL_SLICED (tensor cores, FP64
        accuracy; default) or RESIDUAL_FLOAT_FLOAT (FP32 pipes)."""
        self._check(self.lib.pwqt_set_residual(self.h, kind))

    def profile_residual(self):
        """(ms, complex MACs, bf16 MMA flops, launches) of the slice-product residual
        launches recorded while profiling was on."""
        ms, cm, fl = C.c_double(), C.c_double(), C.c_double()
        n = C.c_longlong()
        self._check(self.lib.pwqt_profile_residual(self.h, C.byref(ms), C.byref(cm), C.byref(fl), C.byref(n)))
        return ms.value, cm.value, fl.value, n.value

    def profile_correction(self):
        """(ms, complex MACs, launches) of the correction solves recorded while profiling."""
        ms, cm = C.c_double(), C.c_double()
        n = C.c_longlong()
        self._check(self.lib.pwqt_profile_correction(self.h, C.byref(ms), C.byref(cm), C.byref(n)))
        return ms.value, cm.value, n.value

    def profile_refinement(self):
        """(residual ms, correction ms, refinement iterations) recorded while profiling."""
        r, c, it = C.c_double(), C.c_double(), C.c_longlong()
        self._check(self.lib.pwqt_profile_refinement(self.h, C.byref(r), C.byref(c), C.byref(it)))
        return r.value, c.value, it.value

    def kernel_launches(self, reset: bool = False) -> int:
        v = C.c_longlong()
        self._check(self.lib.pwqt_kernel_launches(self.h, C.byref(v), 1 if reset else 0))
        return v.value


class Server:
    """pwqt_server: a catalog of bases, requests queued and collected by ticket."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, queue_capacity: int = 0, ir_tol: float = 0.0,
                 batch: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        o = ServerOpts(device, hbm_budget_bytes, queue_capacity, ir_tol, batch)
        r = self.lib.pwqt_server_create(C.byref(self.h), C.byref(o))
        if r != PWQT_OK:
            raise PwqtError(r, "pwqt_server_create failed")
        self.pending = {}

    def _check(self, r):
        if r != PWQT_OK:
            raise PwqtError(r, self.lib.pwqt_server_last_error(self.h).decode())

    def add_basis(self, basis: int, cell, ff, gcut: float, n_bands: int) -> int:
        cc, keep = _cell(cell)
        f = FormFactorC(ff.v0, ff.sigma)
        n = C.c_int()
        self._check(self.lib.pwqt_server_add_basis(self.h, basis, C.byref(cc), C.byref(f), gcut, n_bands, C.byref(n)))
        return n.value

    def submit(self, basis: int, U, E, precision: int = FP64) -> int:
        """Queue a request; returns its ticket.  Outputs are held until collected."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.float64)
        nE, N = len(E), len(U)
        out = SolveResult(np.zeros(nE), np.zeros(nE), np.zeros(nE), np.zeros((nE, 2), np.int32), np.zeros((nE, N, 2)),
                          np.zeros(nE), np.zeros(nE, np.int32), np.zeros(nE, np.int32))
        req = RequestC(basis, N, _dptr(U), nE, _dptr(E), precision, _dptr(out.T), _dptr(out.R), _dptr(out.T_ds),
                       _iptr(out.n_open), _dptr(out.node_n), _dptr(out.resid), _iptr(out.iters), _iptr(out.status))
        t = C.c_longlong()
        self._check(self.lib.pwqt_server_submit(self.h, C.byref(req), C.byref(t)))
        self.pending[t.value] = (out, U, E)   # keep the buffers alive until collected
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """(SolveResult, latency seconds); raises PwqtError on a failed request or timeout."""
        rc, lat = C.c_int(), C.c_double()
        r = self.lib.pwqt_server_wait(self.h, ticket, timeout_s, C.byref(rc), C.byref(lat))
        if r != PWQT_OK:
            raise PwqtError(r, self.lib.pwqt_server_last_error(self.h).decode())
        out = self.pending.pop(ticket)[0]
        if rc.value != PWQT_OK:
            raise PwqtError(rc.value, self.lib.pwqt_server_last_error(self.h).decode())
        return out, lat.value

    def stats(self, reset: bool = False):
        done, p50, p99, peak = C.c_longlong(), C.c_double(), C.c_double(), C.c_size_t()
        self._check(self.lib.pwqt_server_stats(self.h, C.byref(done), C.byref(p50), C.byref(p99), C.byref(peak),
                                               1 if reset else 0))
        return dict(completed=done.value, p50_s=p50.value, p99_s=p99.value, peak_admitted_bytes=peak.value)

    def batch_stats(self):
        """(batched solves, requests they held, largest batch) since the last stats reset."""
        b, r, m = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self._check(self.lib.pwqt_server_batch_stats(self.h, C.byref(b), C.byref(r), C.byref(m)))
        return b.value, r.value, m.value

    def close(self):
        if self.h:
            self.lib.pwqt_server_destroy(self.h)
            self.h = C.c_void_p()
            self.pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
