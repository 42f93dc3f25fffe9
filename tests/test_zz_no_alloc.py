"""pwqt_solve_noalloc: the FP64 solve for callers that cannot allocate device memory
during a call (their memory comes from a budget the host program owns, or their
request path must not allocate).  Its scratch is one static device array; this
test checks it against pwqt_solve, the allocating entry point, on two calls in a
row (the array keeps the previous call's contents), plus its limits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def setup():
    import torch

    from oracle import pwqt_oracle as O
    from paper_1903_00548_gb300 import build, pwqt
    from paper_1903_00548_gb300 import workloads as W
    build.build()
    wl = W.chain8()
    basis = O.bloch_basis(wl.cell, wl.ff, wl.gcut, wl.n_bands)
    ctx = pwqt.Context()
    ctx.set_enhancement(wl.cell, basis.eps, [(g["mx"], g["mz"], g["C"]) for g in basis.groups])
    ctx.set_extrinsic(0, wl.U)
    return torch, pwqt, wl, ctx


def _run_noalloc(torch, ctx, E, N):
    dev = torch.device("cuda", 0)
    out = {k: torch.full((len(E),), -1.0, dtype=torch.float64, device=dev) for k in ("T", "R", "T_ds")}
    out["node_n"] = torch.full((len(E) * N * 2,), -1.0, dtype=torch.float64, device=dev)
    out["status"] = torch.full((len(E),), -1, dtype=torch.int32, device=dev)
    ctx.solve_noalloc(0, E, {k: v.data_ptr() for k, v in out.items()})
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_allocating_solve_twice(setup):
    torch, pwqt, wl, ctx = setup
    N = wl.n_nodes
    for E in (wl.energies[5:21], wl.energies[30:38]):        # two calls in a row, different sizes
        ref = ctx.solve(0, E, pwqt.FP64)                        # also fills the self-energy cache
        got = _run_noalloc(torch, ctx, E, N)
        for k in ("T", "R", "T_ds"):
            assert np.max(np.abs(got[k] - getattr(ref, k))) <= TOL * max(1.0, np.max(np.abs(getattr(ref, k))))
        nn = got["node_n"].reshape(len(E), N, 2)
        assert np.max(np.abs(nn - ref.node_n)) <= TOL * max(1.0, np.max(ref.node_n))
        assert np.array_equal(got["status"], ref.status)


def test_noalloc_matches_oracle(setup):
    # the same energies through the oracle: 1e-9 relative (times the open channels),
    # or four times the oracle's own error bar where that is larger
    from oracle import pwqt_oracle as O
    torch, pwqt, wl, ctx = setup
    E = wl.energies[40:48]
    ctx.solve(0, E, pwqt.FP64)                                  # fills the self-energy cache
    got = _run_noalloc(torch, ctx, E, wl.n_nodes)
    s = O.build_system(wl.cell, wl.ff, wl.gcut, wl.n_bands, wl.U)
    cache = {}
    for e, En in enumerate(E):
        r = O.solve_energy(s.blk, s.Vd, s.Vu, s.U, float(En), cache=cache)
        alts = [O.solve_energy(s.blk, s.Vd, s.Vu, s.U, float(En), cache=cache, reciprocal=k) for k in (True, "cayley")]
        bar = max(O.error_bar(r, *alts), O.perturbation_spread(s.blk, s.U, float(En)))
        t = max(TOL * max(1.0, r.n_open_s), 4.0 * bar)
        assert abs(got["T"][e] - r.T) <= t and abs(got["R"][e] - r.R) <= t, (En, got["T"][e], r.T)


def test_noalloc_empty_call_and_device_restore(setup):
    # an empty call does the one-time set-up; the caller's current device is kept
    torch, pwqt, wl, ctx = setup
    before = torch.cuda.current_device()
    ctx.solve_noalloc(0, np.zeros(0), {})
    assert torch.cuda.current_device() == before


def test_noalloc_rejects_what_it_cannot_do(setup):
    torch, pwqt, wl, ctx = setup
    # energies whose self-energies are not cached: it would have to allocate
    with pytest.raises(pwqt.PwqtError) as ei:
        _run_noalloc(torch, ctx, np.array([0.123456789]), wl.n_nodes)
    assert ei.value.code == -5
    # more energies than the entry point takes
    E = np.linspace(0.1, 1.5, 65)
    with pytest.raises(pwqt.PwqtError) as ei:
        _run_noalloc(torch, ctx, E, wl.n_nodes)
    assert ei.value.code == -1
