// Self-consistent potential (Sec. 4): the non-linear Poisson equation of a 1D
// finite-element model along z solved by Newton-Raphson with the semi-classical
// Jacobian (Eq. newton_poisson, Eq. density_jacobian) and DIIS acceleration over the
// last iterates (least squares by SVD).  Host code: every iteration rebuilds the
// system's extrinsic blocks and integrates the node density and its Jacobian with one
// adaptive Simpson pass of batched GPU solves (pwqt_integrate); the Poisson algebra
// (tridiagonal, N unknowns) and the DIIS extrapolation run on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pwqt_internal.cuh"

namespace {

// x = argmin ||A x - b|| by a one-sided Jacobi SVD of A (m x k, k small, column-major),
// singular values below rcond * max dropped
std::vector<double> lstsq_svd(std::vector<double> A, int m, int k, const std::vector<double>& b, double rcond) {
    std::vector<double> V((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) V[(size_t)j * k + j] = 1.0;
    auto col = [&](int j) { return A.data() + (size_t)j * m; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                double a = 0, bb = 0, g = 0;
                const double *ap = col(p), *aq = col(q);
                for (int i = 0; i < m; ++i) { a += ap[i] * ap[i]; bb += aq[i] * aq[i]; g += ap[i] * aq[i]; }
                if (std::fabs(g) <= 1e-15 * std::sqrt(a * bb) || g == 0.0) continue;
                off = std::max(off, std::fabs(g) / std::sqrt(a * bb));
                const double zeta = (bb - a) / (2 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
                const double c = 1 / std::sqrt(1 + t * t), s = c * t;
                double *xp = col(p), *xq = col(q);
                for (int i = 0; i < m; ++i) {
                    const double u = xp[i], v = xq[i];
                    xp[i] = c * u - s * v;
                    xq[i] = s * u + c * v;
                }
                for (int i = 0; i < k; ++i) {
                    const double u = V[(size_t)p * k + i], v = V[(size_t)q * k + i];
                    V[(size_t)p * k + i] = c * u - s * v;
                    V[(size_t)q * k + i] = s * u + c * v;
                }
            }
        if (off < 1e-15) break;
    }
    std::vector<double> sig(k);
    double smax = 0;
    for (int j = 0; j < k; ++j) {
        double s2 = 0;
        for (int i = 0; i < m; ++i) s2 += col(j)[i] * col(j)[i];
        sig[j] = std::sqrt(s2);
        smax = std::max(smax, sig[j]);
    }
    std::vector<double> x(k, 0.0);
    for (int j = 0; j < k; ++j) {
        if (sig[j] <= rcond * smax || sig[j] == 0.0) continue;
        double ub = 0;   // u_j . b with u_j = A_j / sig_j
        for (int i = 0; i < m; ++i) ub += col(j)[i] * b[i];
        ub /= sig[j] * sig[j];
        for (int i = 0; i < k; ++i) x[i] += V[(size_t)j * k + i] * ub;
    }
    return x;
}

}  // namespace

extern "C" int pwqt_self_consistent(pwqt_ctx* c, int sys, const pwqt_poisson1d* model, double mu_s, double mu_d, double kT,
                                    double E_lo, double E_hi, double tol_int, double tol_sc, int max_iters, int diis_window,
                                    int precision, double* U, double* history, int* iters, double* n_out) {
    using namespace pwqt;
    if (!c) return PWQT_ERR_INVALID_ARG;
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (!model || !model->U_gate || !model->n_dop || !U || max_iters < 1 || !(tol_sc > 0) || !(tol_int > 0))
        return fail(c, PWQT_ERR_INVALID_ARG, "model, U, max_iters >= 1, tol_sc > 0 and tol_int > 0 are required");
    const int N = it->second.N;
    if (N < 3) return fail(c, PWQT_ERR_INVALID_ARG, "the self-consistent loop needs an interior node (N >= 3)");
    const double L = c->Lz, ka = model->kappa, ga = model->gamma, al = model->alpha;
    // tridiagonal stiffness and mass of the node hats (interior rows)
    const double s_d = 2.0 / L, s_o = -1.0 / L, m_d = 4.0 * L / 6.0, m_o = L / 6.0;
    std::vector<double> u(U, U + N), res(2 * N), n(N), d(N), F(N), step(N);
    std::vector<std::vector<double>> Us, Rs;
    for (int p = 0; p < max_iters; ++p) {
        PWQT_TRY(pwqt_set_extrinsic(c, sys, N, u.data()));
        PWQT_TRY(pwqt_integrate(c, sys, PWQT_INTEGRAND_NODE_DENSITY_JACOBIAN, E_lo, E_hi, mu_s, mu_d, kT, tol_int, 8, 4000,
                                precision, res.data(), nullptr, nullptr, nullptr, nullptr, nullptr, 0));
        for (int i = 0; i < N; ++i) { n[i] = res[i] / L; d[i] = res[N + i] / L; }
        // F = (kappa S + gamma M) U - gamma M U_gate - alpha M (n - n_dop), interior rows
        auto Mv = [&](const double* v, int i) { return m_o * v[i - 1] + m_d * v[i] + m_o * v[i + 1]; };
        std::vector<double> q(N);
        for (int i = 0; i < N; ++i) q[i] = n[i] - model->n_dop[i];
        for (int i = 1; i < N - 1; ++i)
            F[i] = ka * (s_o * u[i - 1] + s_d * u[i] + s_o * u[i + 1]) + ga * Mv(u.data(), i) - ga * Mv(model->U_gate, i) -
                   al * Mv(q.data(), i);
        // Jacobian kappa S + gamma M + alpha M diag(d): tridiagonal, Thomas algorithm
        const int m = N - 2;
        std::vector<double> lo(m), di(m), up(m), rhs(m);
        for (int r = 0; r < m; ++r) {
            const int i = r + 1;
            di[r] = ka * s_d + ga * m_d + al * m_d * d[i];
            lo[r] = ka * s_o + ga * m_o + al * m_o * d[i - 1];
            up[r] = ka * s_o + ga * m_o + al * m_o * d[i + 1];
            rhs[r] = -F[i];
        }
        for (int r = 1; r < m; ++r) {
            const double w = lo[r] / di[r - 1];
            di[r] -= w * up[r - 1];
            rhs[r] -= w * rhs[r - 1];
        }
        std::fill(step.begin(), step.end(), 0.0);
        step[m] = rhs[m - 1] / di[m - 1];
        for (int r = m - 2; r >= 0; --r) step[r + 1] = (rhs[r] - up[r] * step[r + 2]) / di[r];
        double norm = 0;
        for (double v : step) norm += v * v;
        norm = std::sqrt(norm);
        if (history) history[p] = norm;
        std::vector<double> un(N);
        for (int i = 0; i < N; ++i) un[i] = u[i] + step[i];
        if (norm <= tol_sc) {
            std::copy(un.begin(), un.end(), U);
            if (iters) *iters = p + 1;
            if (n_out) std::copy(n.begin(), n.end(), n_out);
            return PWQT_OK;
        }
        if (diis_window > 1) {
            Us.push_back(un);
            Rs.push_back(step);
            if ((int)Us.size() > diis_window) { Us.erase(Us.begin()); Rs.erase(Rs.begin()); }
            const int k = (int)Us.size() - 1;
            if (k >= 1) {
                // min || R_last + sum_j c_j (R_j - R_last) ||
                std::vector<double> A((size_t)N * k), b(N);
                for (int j = 0; j < k; ++j)
                    for (int i = 0; i < N; ++i) A[(size_t)j * N + i] = Rs[j][i] - Rs[k][i];
                for (int i = 0; i < N; ++i) b[i] = -Rs[k][i];
                const std::vector<double> cj = lstsq_svd(A, N, k, b, 1e-10);
                for (int i = 0; i < N; ++i) {
                    double v = Us[k][i];
                    for (int j = 0; j < k; ++j) v += cj[j] * (Us[j][i] - Us[k][i]);
                    un[i] = v;
                }
            }
        }
        u = un;
    }
    std::copy(u.begin(), u.end(), U);
    if (iters) *iters = max_iters;
    if (n_out) std::copy(n.begin(), n.end(), n_out);
    return fail(c, PWQT_ERR_STATE, "self-consistent loop did not converge within max_iters");
}
