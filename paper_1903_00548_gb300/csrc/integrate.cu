// Energy integrals by adaptive Simpson quadrature (Sec. 3.3: the density integral is
// evaluated adaptively to a prescribed tolerance; Eq. current: the ballistic current
// with the same method).  Host code around the batched solve: every refinement round
// collects the energies that its open intervals still need and solves them in one
// pwqt_solve call, so the GPU sees batches of energies, not single points.
//
// Rule (the same as the interval-by-interval definition): [E_lo, E_hi] starts as
// min_pieces equal intervals; an interval of length h is accepted when the one- and
// two-panel Simpson estimates S1, S2 differ by at most 15 tol h / (E_hi - E_lo) in the
// max norm over the integrand's components, and then contributes S2 + (S2 - S1)/15
// (Boole weights 7, 32, 12, 32, 7 times h/90 on its five points); otherwise its halves
// are examined in the next round.  Once max_evals energies have been solved, or an
// interval is 2^-40 of the range long, open intervals are accepted as they stand.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "pwqt_internal.cuh"

namespace {

constexpr double G0_SIEMENS = 2.0 * 1.602176634e-19 * 1.602176634e-19 / 6.62607015e-34;   // 2 e^2 / h

double fermi_fd(double x, double kT) {
    if (kT <= 0) return x < 0 ? 1.0 : (x == 0 ? 0.5 : 0.0);
    return 0.5 * (1.0 - std::tanh(0.5 * x / kT));
}

// -d f_FD / dE at E - mu = x (zero for kT = 0: the step's derivative is not sampled)
double dfermi_fd(double x, double kT) {
    if (kT <= 0) return 0.0;
    const double t = std::tanh(0.5 * x / kT);
    return 0.25 * (1.0 - t * t) / kT;
}

struct Piece { double x0, x1; };

}  // namespace

extern "C" int pwqt_integrate(pwqt_ctx* c, int sys, int integrand, double E_lo, double E_hi, double mu_s, double mu_d, double kT,
                              double tol, int min_pieces, int max_evals, int precision, double* result, double* err_est,
                              int* n_evals, double* energies, double* weights, int* n_points, int max_points) {
    using namespace pwqt;
    if (!c) return PWQT_ERR_INVALID_ARG;
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (integrand != PWQT_INTEGRAND_CURRENT && integrand != PWQT_INTEGRAND_NODE_DENSITY &&
        integrand != PWQT_INTEGRAND_NODE_DENSITY_JACOBIAN)
        return fail(c, PWQT_ERR_INVALID_ARG, "unknown integrand");
    if (!(E_hi > E_lo) || !std::isfinite(E_lo) || !std::isfinite(E_hi) || !(tol > 0) || !std::isfinite(mu_s) ||
        !std::isfinite(mu_d) || !(kT >= 0) || min_pieces < 1 || max_evals < 1 || !result)
        return fail(c, PWQT_ERR_INVALID_ARG, "need E_lo < E_hi, tol > 0, kT >= 0, min_pieces >= 1, max_evals >= 1, result");
    const int N = it->second.N;
    const int dim = integrand == PWQT_INTEGRAND_CURRENT ? 1 : (integrand == PWQT_INTEGRAND_NODE_DENSITY ? N : 2 * N);
    const double L = E_hi - E_lo;
    std::map<double, std::vector<double>> cache;   // integrand value per solved energy

    auto evaluate = [&](std::vector<double>& xs) -> int {
        if (xs.empty()) return PWQT_OK;
        const int nE = (int)xs.size();
        std::vector<double> T(nE), Tds(nE), nn((size_t)nE * N * 2);
        int rc = pwqt_solve(c, sys, nE, xs.data(), precision, T.data(), nullptr, Tds.data(), nullptr,
                            integrand != PWQT_INTEGRAND_CURRENT ? nn.data() : nullptr, nullptr, nullptr, nullptr);
        if (rc != PWQT_OK) return rc;
        for (int e = 0; e < nE; ++e) {
            const double fs = fermi_fd(xs[e] - mu_s, kT), fd = fermi_fd(xs[e] - mu_d, kT);
            std::vector<double> v(dim);
            if (integrand == PWQT_INTEGRAND_CURRENT) v[0] = G0_SIEMENS * (T[e] * fs - Tds[e] * fd);
            else
                for (int i = 0; i < N; ++i) v[i] = nn[((size_t)e * N + i) * 2] * fs + nn[((size_t)e * N + i) * 2 + 1] * fd;
            if (integrand == PWQT_INTEGRAND_NODE_DENSITY_JACOBIAN) {   // second block: -df/dE weights
                const double gs = dfermi_fd(xs[e] - mu_s, kT), gd = dfermi_fd(xs[e] - mu_d, kT);
                for (int i = 0; i < N; ++i) v[N + i] = nn[((size_t)e * N + i) * 2] * gs + nn[((size_t)e * N + i) * 2 + 1] * gd;
            }
            cache[xs[e]] = std::move(v);
        }
        return PWQT_OK;
    };

    std::vector<double> total(dim, 0.0);
    double err = 0.0;
    std::map<double, double> wmap;
    std::vector<Piece> open;
    for (int k = 0; k < min_pieces; ++k)
        open.push_back({E_lo + (E_hi - E_lo) * k / min_pieces, E_lo + (E_hi - E_lo) * (k + 1) / min_pieces});
    while (!open.empty()) {
        std::vector<double> need;
        // nested midpoints: a half's midpoint is the same expression as this interval's
        // quarter point, so the halves reuse these energies exactly
        auto points = [](const Piece& p, double* x) {
            x[0] = p.x0;
            x[2] = p.x0 + (p.x1 - p.x0) / 2;
            x[1] = p.x0 + (x[2] - p.x0) / 2;
            x[3] = x[2] + (p.x1 - x[2]) / 2;
            x[4] = p.x1;
        };
        for (const Piece& p : open) {
            double x[5];
            points(p, x);
            for (double v : x)
                if (!cache.count(v)) need.push_back(v);
        }
        std::sort(need.begin(), need.end());
        need.erase(std::unique(need.begin(), need.end()), need.end());
        PWQT_TRY(evaluate(need));
        const bool spent = (int)cache.size() >= max_evals;
        std::vector<Piece> next;
        for (const Piece& p : open) {
            const double h = p.x1 - p.x0;
            double xs[5];
            points(p, xs);
            const double xm = xs[2];
            const std::vector<double>&fa = cache[xs[0]], &fl = cache[xs[1]], &fm = cache[xs[2]], &fr = cache[xs[3]],
                                       &fb = cache[xs[4]];
            double d = 0.0;
            std::vector<double> S1(dim), S2(dim);
            for (int q = 0; q < dim; ++q) {
                S1[q] = h / 6.0 * (fa[q] + 4 * fm[q] + fb[q]);
                S2[q] = h / 12.0 * (fa[q] + 4 * fl[q] + 2 * fm[q] + 4 * fr[q] + fb[q]);
                d = std::max(d, std::fabs(S2[q] - S1[q]));
            }
            if (d <= 15.0 * tol * h / L || spent || h <= L * std::ldexp(1.0, -40)) {
                for (int q = 0; q < dim; ++q) total[q] += S2[q] + (S2[q] - S1[q]) / 15.0;
                err += d / 15.0;
                const double ws[5] = {7, 32, 12, 32, 7};
                for (int k = 0; k < 5; ++k) wmap[xs[k]] += ws[k] * h / 90.0;
            } else {
                next.push_back({p.x0, xm});
                next.push_back({xm, p.x1});
            }
        }
        open.swap(next);
    }
    std::copy(total.begin(), total.end(), result);
    if (err_est) *err_est = err;
    if (n_evals) *n_evals = (int)cache.size();
    if (n_points) *n_points = (int)wmap.size();
    int k = 0;
    for (const auto& kv : wmap) {
        if (k >= max_points) break;
        if (energies) energies[k] = kv.first;
        if (weights) weights[k] = kv.second;
        ++k;
    }
    return PWQT_OK;
}
