// Diagonal blocks of the retarded Green's function G = [E M - H - V^e - Sigma]^{-1}
// (the NEGF side of Sec. 3.2) by the recursive Green's-function recursion over the
// nodes, run by the complex128 sweep kernel in its Green's-function form, and the node
// spectral density -(2/pi) Im Tr G_ii.  In a ballistic device the spectral function is
// i(G - G^H) = G (Gamma_s + Gamma_d) G^H, so this density equals the sum of the source-
// and drain-injected node densities of the wave-function solve (Sec. 3.3): a check of
// the QTBM node densities that needs no mode decomposition in the device.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

using namespace pwqt;

extern "C" int pwqt_green_diagonal(pwqt_ctx* c, int sys, int n_E, const double* E, double* node_dos, double* G_diag,
                                   int* status) {
    if (!c) return PWQT_ERR_INVALID_ARG;
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis: call pwqt_assemble_intrinsic first");
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (n_E < 0 || (n_E > 0 && (!E || !node_dos))) return fail(c, PWQT_ERR_INVALID_ARG, "energies and node_dos are required");
    for (int e = 0; e < n_E; ++e)
        if (!std::isfinite(E[e])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite energy");
    if (n_E == 0) return PWQT_OK;
    PWQT_CUDA(c, cudaSetDevice(c->dev));
    System& s = it->second;
    const int n = c->n, N = s.N;
    const size_t nn = (size_t)n * n, sXY = (size_t)N * n * 2 * n;
    cudaStream_t st = c->stream;
    std::vector<double> keys;
    for (int e = 0; e < n_E; ++e) { keys.push_back(E[e] - s.Us); keys.push_back(E[e] - s.Ud); }
    PWQT_TRY(fill_leads(c, keys));
    std::vector<LeadEntry*> ls(n_E), ld(n_E);
    for (int e = 0; e < n_E; ++e) {
        PWQT_TRY(lead_entry(c, E[e] - s.Us, &ls[e]));
        PWQT_TRY(lead_entry(c, E[e] - s.Ud, &ld[e]));
    }
    if (c->zero_nn.bytes < sizeof(double2) * nn) {
        PWQT_TRY(alloc(c, c->zero_nn, sizeof(double2) * nn));
        PWQT_CUDA(c, cudaMemsetAsync(c->zero_nn.p, 0, c->zero_nn.bytes, st));
    }
    const double2* zero = c->zero_nn.as<double2>();
    // per energy: the forward panels N n (2n), the n x n scratch, N densities, a status word
    const size_t per = sizeof(double2) * (sXY + nn) + sizeof(double) * N + sizeof(int) + 64;
    size_t free_b = 0, total_b = 0;
    PWQT_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = c->opts.hbm_budget_bytes ? c->opts.hbm_budget_bytes : (size_t)(0.85 * (double)free_b);
    if (per > budget) return fail(c, PWQT_ERR_OOM, "one energy needs " + std::to_string(per) + " bytes");
    int cap = (int)std::max<size_t>(1, budget / per);
    if (c->opts.batch > 0) cap = std::min(cap, c->opts.batch);
    std::vector<int> sth(n_E);
    DBuf work, jobs_d;
    for (int e0 = 0; e0 < n_E; e0 += cap) {
        const int nb = std::min(cap, n_E - e0);
        PWQT_TRY(ensure(c, work, sizeof(double2) * (sXY + nn) * nb + sizeof(double) * (size_t)N * nb + sizeof(int) * nb + 256));
        double2* XY = work.as<double2>();
        double2* Sb = XY + sXY * nb;
        double* dos = reinterpret_cast<double*>(Sb + nn * nb);
        int* stat = reinterpret_cast<int*>(dos + (size_t)N * nb);
        std::vector<SweepJob> jobs(nb);
        for (int b = 0; b < nb; ++b) {
            const int e = e0 + b;
            sth[e] = ls[e]->status | ld[e]->status;
            const bool bad = (sth[e] & PWQT_ST_MODE_COUNT) != 0;
            SweepJob& J = jobs[b];
            J.E = E[e];
            J.ms = n;
            J.md = 0;
            J.sig_s = bad ? zero : ls[e]->sigma_s.as<double2>();
            J.sig_d = bad ? zero : ld[e]->sigma_d.as<double2>();
            J.XY = XY + sXY * b;
            J.S = Sb + nn * b;
            J.status = stat + b;
            J.dos = dos + (size_t)N * b;
        }
        PWQT_CUDA(c, cudaMemsetAsync(stat, 0, sizeof(int) * nb, st));
        PWQT_TRY(ensure(c, jobs_d, sizeof(SweepJob) * nb));
        PWQT_CUDA(c, cudaMemcpyAsync(jobs_d.p, jobs.data(), sizeof(SweepJob) * nb, cudaMemcpyHostToDevice, st));
        SweepSys sy{n, N, c->M0.as<double2>(), c->M1.as<double2>(), s.HV0.as<double2>(), s.HV1.as<double2>()};
        launch_green_fp64(sy, jobs_d.as<SweepJob>(), nb, st);
        c->launches++;
        PWQT_CUDA(c, cudaGetLastError());
        std::vector<int> sk(nb);
        PWQT_CUDA(c, cudaMemcpyAsync(node_dos + (size_t)e0 * N, dos, sizeof(double) * N * nb, cudaMemcpyDeviceToHost, st));
        PWQT_CUDA(c, cudaMemcpyAsync(sk.data(), stat, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        // G_ii sits in columns n..2n-1 of each node's panel: one strided copy per energy
        if (G_diag)
            for (int b = 0; b < nb; ++b)
                PWQT_CUDA(c, cudaMemcpy2DAsync(G_diag + 2 * (size_t)(e0 + b) * N * nn, sizeof(double2) * n, XY + sXY * b + n,
                                               sizeof(double2) * 2 * n, sizeof(double2) * n, (size_t)N * n,
                                               cudaMemcpyDeviceToHost, st));
        PWQT_CUDA(c, cudaStreamSynchronize(st));
        for (int b = 0; b < nb; ++b) sth[e0 + b] |= sk[b];
    }
    if (status) std::copy(sth.begin(), sth.end(), status);
    return PWQT_OK;
}
