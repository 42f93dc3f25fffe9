// Transmission from the Green's function (the NEGF alternative of Sec. 3.2,
// G = [E M - H - Sigma]^{-1}): T(E) = Tr[Gamma_d G_{N1} Gamma_s G_{N1}^H] with
// Gamma_c = i (Sigma_c - Sigma_c^H).  G_{N1} is the last node's block of the block
// sweep (FP64 kernel) with the n x n identity injected at the first node; the two
// n x n products run as strided-batched ZGEMMs over the energies of a batch and a
// reduction kernel takes the trace.  It needs no mode decomposition at the drain, so
// it cross-checks the mode-resolved transmission of Eq. transmission.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

namespace pwqt {
namespace {

__global__ void k_identity_c128(int n, double2* I) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < (size_t)n * n) I[t] = make_double2((t / n) == (t % n) ? 1.0 : 0.0, 0.0);
}

// Gamma = i (Sigma - Sigma^H), one n x n block per energy (row-major)
__global__ void k_broadening(int n, const double2* const* __restrict__ sig, double2* __restrict__ gam) {
    const int e = blockIdx.y;
    const double2* S = sig[e];
    double2* G = gam + (size_t)e * n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / n, c = t % n;
        const double2 a = S[r * n + c], b = S[c * n + r];
        const double2 d = make_double2(a.x - b.x, a.y + b.y);   // Sigma_rc - conj(Sigma_cr)
        G[t] = make_double2(-d.y, d.x);                          // times i
    }
}

// T[e] = Re sum_ij Y[i][j] Z[j][i]
__global__ void k_trace_product(int n, const double2* __restrict__ Y, const double2* __restrict__ Z, double* __restrict__ T) {
    const int e = blockIdx.x;
    const double2* y = Y + (size_t)e * n * n;
    const double2* z = Z + (size_t)e * n * n;
    double acc = 0.0;
    for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {
        const size_t i = t / n, j = t % n;
        const double2 a = y[t], b = z[j * n + i];
        acc += a.x * b.x - a.y * b.y;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) T[e] = red[0];
}

}  // namespace
}  // namespace pwqt

using namespace pwqt;

extern "C" int pwqt_transmission_caroli(pwqt_ctx* c, int sys, int n_E, const double* E, double* T, int* status) {
    if (!c) return PWQT_ERR_INVALID_ARG;
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis: call pwqt_assemble_intrinsic first");
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (n_E < 0 || (n_E > 0 && (!E || !T))) return fail(c, PWQT_ERR_INVALID_ARG, "energies and T are required");
    for (int e = 0; e < n_E; ++e)
        if (!std::isfinite(E[e])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite energy");
    if (n_E == 0) return PWQT_OK;
    PWQT_CUDA(c, cudaSetDevice(c->dev));
    System& s = it->second;
    const int n = c->n, N = s.N;
    const size_t nn = (size_t)n * n;
    cudaStream_t st = c->stream;
    // contact self-energies from the cache (computed on a miss)
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
    // per energy: the sweep panels N n (2n), one n x n scratch, Gamma_s, Gamma_d, Y, Z
    const size_t per = sizeof(double2) * ((size_t)N * n * 2 * n + 5 * nn) + 64;
    size_t free_b = 0, total_b = 0;
    PWQT_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = c->opts.hbm_budget_bytes ? c->opts.hbm_budget_bytes : (size_t)(0.85 * (double)free_b);
    int cap = (int)std::max<size_t>(1, budget / per);
    if (c->opts.batch > 0) cap = std::min(cap, c->opts.batch);
    if (per > budget) return fail(c, PWQT_ERR_OOM, "one energy needs " + std::to_string(per) + " bytes");
    DBuf ident, work, jobs_d, sig_d;
    PWQT_TRY(alloc(c, ident, sizeof(double2) * nn));
    k_identity_c128<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, ident.as<double2>());
    c->launches++;
    PWQT_BLAS(c, cublasSetStream(c->blas, st));
    std::vector<double> Th(n_E);
    std::vector<int> sth(n_E);
    for (int e0 = 0; e0 < n_E; e0 += cap) {
        const int nb = std::min(cap, n_E - e0);
        const size_t sXY = (size_t)N * n * 2 * n;
        PWQT_TRY(ensure(c, work, sizeof(double2) * (sXY + 5 * nn) * nb + sizeof(int) * nb + 256));
        double2* XY = work.as<double2>();
        double2* Sb = XY + sXY * nb;
        double2* Gs = Sb + nn * nb;
        double2* Gd = Gs + nn * nb;
        double2* Yb = Gd + nn * nb;
        double2* Zb = Yb + nn * nb;
        int* stat = reinterpret_cast<int*>(Zb + nn * nb);
        std::vector<SweepJob> jobs(nb);
        std::vector<const double2*> sig(2 * nb);
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
            J.rhs_s = ident.as<double2>();
            J.rhs_d = zero;
            J.XY = XY + sXY * b;
            J.S = Sb + nn * b;
            J.status = stat + b;
            sig[b] = J.sig_s;
            sig[nb + b] = J.sig_d;
        }
        PWQT_CUDA(c, cudaMemsetAsync(stat, 0, sizeof(int) * nb, st));
        PWQT_TRY(ensure(c, jobs_d, sizeof(SweepJob) * nb));
        PWQT_TRY(ensure(c, sig_d, sizeof(double2*) * 2 * nb));
        PWQT_CUDA(c, cudaMemcpyAsync(jobs_d.p, jobs.data(), sizeof(SweepJob) * nb, cudaMemcpyHostToDevice, st));
        PWQT_CUDA(c, cudaMemcpyAsync(sig_d.p, sig.data(), sizeof(double2*) * 2 * nb, cudaMemcpyHostToDevice, st));
        SweepSys sy{n, N, c->M0.as<double2>(), c->M1.as<double2>(), s.HV0.as<double2>(), s.HV1.as<double2>()};
        launch_sweep_fp64(sy, jobs_d.as<SweepJob>(), nb, st);
        const int gblocks = (int)std::min<size_t>((nn + 255) / 256, 1024);
        k_broadening<<<dim3(gblocks, nb), 256, 0, st>>>(n, sig_d.as<const double2*>(), Gs);
        k_broadening<<<dim3(gblocks, nb), 256, 0, st>>>(n, sig_d.as<const double2*>() + nb, Gd);
        c->launches += 3;
        PWQT_CUDA(c, cudaGetLastError());
        // G_{N1}: the solution columns of the last node, row-major with leading dimension 2n.
        // cuBLAS is column-major: a row-major matrix read in place is its transpose, so
        // Y = Gamma_d X is C = X^T Gamma_d^T and Z = Gamma_s X^H is C = conj(X) Gamma_s^T.
        const double2* X = XY + (size_t)(N - 1) * n * 2 * n + n;
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), nil = make_cuDoubleComplex(0.0, 0.0);
        PWQT_BLAS(c, cublasZgemmStridedBatched(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one,
                                               reinterpret_cast<const cuDoubleComplex*>(X), 2 * n, (long long)sXY,
                                               reinterpret_cast<const cuDoubleComplex*>(Gd), n, (long long)nn, &nil,
                                               reinterpret_cast<cuDoubleComplex*>(Yb), n, (long long)nn, nb));
        PWQT_BLAS(c, cublasZgemmStridedBatched(c->blas, CUBLAS_OP_C, CUBLAS_OP_N, n, n, n, &one,
                                               reinterpret_cast<const cuDoubleComplex*>(X), 2 * n, (long long)sXY,
                                               reinterpret_cast<const cuDoubleComplex*>(Gs), n, (long long)nn, &nil,
                                               reinterpret_cast<cuDoubleComplex*>(Zb), n, (long long)nn, nb));
        DBuf Td;
        PWQT_TRY(alloc(c, Td, sizeof(double) * nb));
        k_trace_product<<<nb, 256, 0, st>>>(n, Yb, Zb, Td.as<double>());
        c->launches++;
        PWQT_CUDA(c, cudaGetLastError());
        std::vector<int> sk(nb);
        PWQT_CUDA(c, cudaMemcpyAsync(Th.data() + e0, Td.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        PWQT_CUDA(c, cudaMemcpyAsync(sk.data(), stat, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        PWQT_CUDA(c, cudaStreamSynchronize(st));
        for (int b = 0; b < nb; ++b) sth[e0 + b] |= sk[b];
    }
    std::copy(Th.begin(), Th.end(), T);
    if (status) std::copy(sth.begin(), sth.end(), status);
    return PWQT_OK;
}
