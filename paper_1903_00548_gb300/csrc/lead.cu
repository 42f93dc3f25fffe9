// Contact self-energies from the complex band structure of the flat leads
// (Sec. 3.1-3.2 of arXiv:1903.00548), FP64 on the GPU.
//
//  1. The symmetric linearisation (Eq. linearized_eigenvalue_symmetric)
//        A x = lambda B x,  A = [[K0, K-], [K+, 0]],  B = [[-K+, 0], [0, K+]],
//     K(E) = H - E M, is brought to standard form by the Cayley transform
//        C = (A + B)^-1 (A - B),  C x = mu x  <=>  A x = lambda B x with
//        lambda = (1 + mu)/(1 - mu),
//     which keeps the transformed spectrum bounded when lambda spans many decades,
//     and C is diagonalised by cuSOLVER's non-Hermitian eigensolver.
//  2. Modes with ||lambda| - 1| < 1e-4 are traveling; each is refined onto the unit
//     circle: with lambda = e^{ikL}, Ec is an eigenvalue of H(k) c = E M(k) c, so
//     Newton on k with the Hellmann-Feynman slope (Eq. hellmann-feynman) and shifted
//     inverse iteration for c converge to |lambda| = 1 exactly.
//  3. Traveling modes are normalised to c^H M(lambda) c = L/2pi (Eq. normalization).
//  4. Out-flow modes form the Bloch matrices B_d (|lambda| < 1 or dE/dk > 0) and
//     B_s (|lambda_d| > 1 or dE/dk < 0, lambda_s = 1/lambda_d), n columns each (any
//     other count: PWQT_ST_MODE_COUNT, energy not solved); Sigma = K' B Lambda B^-1
//     with K'_d = K+, K'_s = K-; injection vectors B_gamma = (K' lambda_gamma - Sigma) c_gamma.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "pwqt_internal.cuh"

namespace pwqt {

size_t LeadEntry::bytes() const {
    return sigma_d.bytes + sigma_s.bytes + P_d.bytes + P_s.bytes + v_out_d.bytes + v_out_s.bytes + rhs_d.bytes +
           rhs_s.bytes + cin_s.bytes + v_in_d.bytes + v_in_s.bytes + sigma_d32.bytes + sigma_s32.bytes + rhs_d32.bytes +
           rhs_s32.bytes;
}

// K0 = H0 - Ec M0, Kp = H1 - Ec M1, written column-major (inputs row-major).
__global__ void k_lead_K(int n, double Ec, const double2* H0, const double2* H1, const double2* M0, const double2* M1,
                         double2* K0cm, double2* Kpcm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= n) return;
    size_t rm = (size_t)r * n + c, cm = (size_t)c * n + r;
    K0cm[cm] = csub(H0[rm], cscale(M0[rm], Ec));
    Kpcm[cm] = csub(H1[rm], cscale(M1[rm], Ec));
}

// A + B and A - B of the symmetric pencil, column-major 2n x 2n.
__global__ void k_lead_cayley(int n, const double2* K0, const double2* Kp, double2* ApB, double2* AmB) {
    int r = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;   // r, c in [0, 2n)
    int n2 = 2 * n;
    if (r >= n2) return;
    int br = r >= n, bc = c >= n, rr = r - br * n, cc = c - bc * n;
    double2 k0 = K0[(size_t)cc * n + rr];
    double2 kp = Kp[(size_t)cc * n + rr];
    double2 km = cconj(Kp[(size_t)rr * n + cc]);   // K- = K+^H
    double2 a, b;
    if (!br && !bc) { a = k0; b = cscale(kp, -1.0); }
    else if (!br && bc) { a = km; b = make_double2(0, 0); }
    else if (br && !bc) { a = kp; b = make_double2(0, 0); }
    else { a = make_double2(0, 0); b = kp; }
    ApB[(size_t)c * n2 + r] = cadd(a, b);
    AmB[(size_t)c * n2 + r] = csub(a, b);
}

// lambda_j from mu_j, unit-norm mode vectors c_j = lower half of the eigenvectors.
__global__ void k_lead_modes(int n, const double2* __restrict__ mu, const double2* __restrict__ VR, double2* lam, double2* Cm) {
    int j = blockIdx.x;
    int n2 = 2 * n;
    __shared__ double red[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += cnorm2(VR[(size_t)j * n2 + n + r]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double inv = red[0] > 0 ? 1.0 / sqrt(red[0]) : 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) Cm[(size_t)j * n + r] = cscale(VR[(size_t)j * n2 + n + r], inv);
    if (threadIdx.x == 0) {
        // C = (A + B)^-1 (A - B): (A - B) x = mu (A + B) x  =>  A x = (1 + mu)/(1 - mu) B x
        double2 m = mu[j];
        lam[j] = cdiv(make_double2(1.0 + m.x, m.y), make_double2(1.0 - m.x, -m.y));
    }
}

// Q = H(k) - Ec M(k) and M(k), column-major, H(k) = H0 + H1 ph + H1^H / ph.
__global__ void k_lead_hk(int n, double2 ph, double Ec, const double2* H0, const double2* H1, const double2* M0,
                          const double2* M1, double2* Qcm, double2* Mkcm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= n) return;
    size_t rm = (size_t)r * n + c, tm = (size_t)c * n + r;
    double2 iph = cconj(ph);   // |ph| = 1
    double2 hk = cadd(H0[rm], cadd(cmul(H1[rm], ph), cmul(cconj(H1[tm]), iph)));
    double2 mk = cadd(M0[rm], cadd(cmul(M1[rm], ph), cmul(cconj(M1[tm]), iph)));
    Qcm[(size_t)c * n + r] = csub(hk, cscale(mk, Ec));
    Mkcm[(size_t)c * n + r] = mk;
}

// y = Mk x (Mk column-major)
__global__ void k_matvec_cm(int n, const double2* __restrict__ A, const double2* __restrict__ x, double2* y) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 s = make_double2(0, 0);
    for (int k = 0; k < n; ++k) cfma(s, A[(size_t)k * n + r], x[k]);
    y[r] = s;
}

// One block: normalise x, and evaluate the forms needed for the Newton step at energy w:
// out[0] = x^H H(k) x / x^H M(k) x (Rayleigh quotient w), out[1] = x^H M(k) x,
// out[2] = x^H [iL(ph K+(w) - K+(w)^H / ph)] x / x^H M(k) x  (dE/dk of that band at k).
__global__ void k_lead_forms(int n, double2 ph, double L, const double2* H0, const double2* H1, const double2* M0,
                             const double2* M1, double2* x, double* out) {
    __shared__ double red[3][256];
    __shared__ double scale;
    double s = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += cnorm2(x[r]);
    red[0][threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[0][threadIdx.x] += red[0][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scale = 1.0 / sqrt(red[0][0]);
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) x[r] = cscale(x[r], scale);
    __syncthreads();
    double2 iph = cconj(ph);
    // per row r: (H(k) x)_r, (M(k) x)_r, (H1 x)_r ph - (H1^H x)_r / ph, same with M1
    double hq = 0, mq = 0, dh = 0, dm = 0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double2 h0 = {0, 0}, h1 = {0, 0}, h1h = {0, 0}, m0 = {0, 0}, m1 = {0, 0}, m1h = {0, 0};
        for (int k = 0; k < n; ++k) {
            double2 xk = x[k];
            cfma(h0, H0[(size_t)r * n + k], xk);
            cfma(h1, H1[(size_t)r * n + k], xk);
            cfma_cj(h1h, H1[(size_t)k * n + r], xk);
            cfma(m0, M0[(size_t)r * n + k], xk);
            cfma(m1, M1[(size_t)r * n + k], xk);
            cfma_cj(m1h, M1[(size_t)k * n + r], xk);
        }
        double2 hx = cadd(h0, cadd(cmul(h1, ph), cmul(h1h, iph)));
        double2 mx = cadd(m0, cadd(cmul(m1, ph), cmul(m1h, iph)));
        double2 dhx = csub(cmul(h1, ph), cmul(h1h, iph));
        double2 dmx = csub(cmul(m1, ph), cmul(m1h, iph));
        double2 xr = cconj(x[r]);
        hq += cmul(xr, hx).x;
        mq += cmul(xr, mx).x;
        // x^H (i L D) x = -L Im(x^H D x)... computed as real part of i L x^H D x
        double2 t = cmul(xr, dhx);
        dh += -L * t.y;
        t = cmul(xr, dmx);
        dm += -L * t.y;
    }
    red[0][threadIdx.x] = hq;
    red[1][threadIdx.x] = mq;
    red[2][threadIdx.x] = 0;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) { red[0][threadIdx.x] += red[0][threadIdx.x + w]; red[1][threadIdx.x] += red[1][threadIdx.x + w]; }
        __syncthreads();
    }
    double H = red[0][0], M = red[1][0];
    __syncthreads();
    red[0][threadIdx.x] = dh;
    red[1][threadIdx.x] = dm;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) { red[0][threadIdx.x] += red[0][threadIdx.x + w]; red[1][threadIdx.x] += red[1][threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double wq = H / M;
        out[0] = wq;
        out[1] = M;
        out[2] = (red[0][0] - wq * red[1][0]) / M;
    }
}

// gather columns idx[j] of Cm (n x 2n col-major) scaled by s[j] into out (n x m col-major)
__global__ void k_gather_cols(int n, const double2* __restrict__ Cm, const int* __restrict__ idx, const double2* __restrict__ s,
                              double2* out) {
    int j = blockIdx.y, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    out[(size_t)j * n + r] = s ? cmul(Cm[(size_t)idx[j] * n + r], s[j]) : Cm[(size_t)idx[j] * n + r];
}
__global__ void k_identity(int n, double2* I) {
    int r = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (r < n) I[(size_t)c * n + r] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}
// rows idx[q] of the col-major n x n matrix A -> row-major out (m x n)
__global__ void k_gather_rows(int n, const double2* __restrict__ A, const int* __restrict__ rows, double2* out) {
    int q = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[(size_t)q * n + c] = A[(size_t)c * n + rows[q]];
}
__global__ void k_scale_col(double2* C, int n, int j, double s) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) C[(size_t)j * n + r] = cscale(C[(size_t)j * n + r], s);
}
__global__ void k_copy_col(double2* dst, const double2* src, int n) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = src[r];
}

// Metric and flux forms of a set of traveling modes at one lambda = ph (|ph| = 1):
// Gm[a][b] = c_a^H M(ph) c_b and F[a][b] = c_a^H V(ph) c_b with M(ph) = M1^H / ph + M0 +
// ph M1 and the velocity form V(ph) = iL (ph K+ - K+^H / ph), K+ = H1 - Ec M1
// (Eqs. hellmann-feynman, normalization).  Grid (g, g), one block per pair.
__global__ void k_group_forms(int n, int g, const int* __restrict__ idx, double2 ph, double Ec, double L,
                              const double2* __restrict__ H1, const double2* __restrict__ M0, const double2* __restrict__ M1,
                              const double2* __restrict__ Cm, double2* Gm, double2* F) {
    const int a = blockIdx.x, b = blockIdx.y;
    const double2* ca = Cm + (size_t)idx[a] * n;
    const double2* cb = Cm + (size_t)idx[b] * n;
    const double2 iph = cconj(ph);
    double2 sm = make_double2(0, 0), sf = make_double2(0, 0);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double2 mv = make_double2(0, 0), kv = make_double2(0, 0);   // (M(ph) c_b)_r, (ph K+ - K+^H/ph) c_b)_r
        for (int k = 0; k < n; ++k) {
            const double2 x = cb[k];
            const size_t rk = (size_t)r * n + k, kr = (size_t)k * n + r;
            const double2 m = cadd(M0[rk], cadd(cmul(ph, M1[rk]), cmul(iph, cconj(M1[kr]))));
            const double2 kp = csub(H1[rk], cscale(M1[rk], Ec));
            const double2 km = cconj(csub(H1[kr], cscale(M1[kr], Ec)));
            cfma(mv, m, x);
            cfma(kv, csub(cmul(ph, kp), cmul(iph, km)), x);
        }
        const double2 cr = cconj(ca[r]);
        sm = cadd(sm, cmul(cr, mv));
        sf = cadd(sf, cmul(cr, kv));
    }
    __shared__ double red[4][256];
    red[0][threadIdx.x] = sm.x; red[1][threadIdx.x] = sm.y; red[2][threadIdx.x] = sf.x; red[3][threadIdx.x] = sf.y;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Gm[a * g + b] = make_double2(red[0][0], red[1][0]);
        // i L (c_a^H K c_b) with K = ph K+ - K+^H / ph
        F[a * g + b] = make_double2(-L * red[3][0], L * red[2][0]);
    }
}

// Generalised Hermitian eigenproblem F u = v Gm u of a small set (g <= 16, one
// thread): Cholesky Gm = L L^H, Jacobi rotations on L^-1 F L^-H, U = L^-H W, so
// that U^H Gm U = I and U^H F U = diag(v).  ok[0] = 0 when Gm is not positive definite.
constexpr int GMAX = 16;
__global__ void k_small_geig(int g, const double2* __restrict__ Gm_in, const double2* __restrict__ F_in, double2* U, double* vals,
                             int* ok) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 Lc[GMAX][GMAX], A[GMAX][GMAX], W[GMAX][GMAX];
    for (int i = 0; i < g; ++i)
        for (int j = 0; j < g; ++j) { Lc[i][j] = make_double2(0, 0); A[i][j] = F_in[i * g + j]; W[i][j] = make_double2(i == j, 0); }
    // Hermitian parts (the forms are Hermitian up to rounding)
    for (int i = 0; i < g; ++i)
        for (int j = i; j < g; ++j) {
            const double2 x = cscale(cadd(A[i][j], cconj(A[j][i])), 0.5);
            A[i][j] = x;
            A[j][i] = cconj(x);
        }
    ok[0] = 1;
    for (int j = 0; j < g; ++j) {
        double d = 0.5 * (Gm_in[j * g + j].x + Gm_in[j * g + j].x);
        for (int k = 0; k < j; ++k) d -= cnorm2(Lc[j][k]);
        if (!(d > 0)) { ok[0] = 0; return; }
        Lc[j][j] = make_double2(sqrt(d), 0);
        for (int i = j + 1; i < g; ++i) {
            double2 x = cscale(cadd(Gm_in[i * g + j], cconj(Gm_in[j * g + i])), 0.5);
            for (int k = 0; k < j; ++k) x = csub(x, cmul(Lc[i][k], cconj(Lc[j][k])));
            Lc[i][j] = cscale(x, 1.0 / Lc[j][j].x);
        }
    }
    // A <- L^-1 A L^-H: forward substitution on the columns, then on the rows
    for (int c = 0; c < g; ++c)
        for (int i = 0; i < g; ++i) {
            double2 x = A[i][c];
            for (int k = 0; k < i; ++k) x = csub(x, cmul(Lc[i][k], A[k][c]));
            A[i][c] = cscale(x, 1.0 / Lc[i][i].x);
        }
    for (int r = 0; r < g; ++r)
        for (int j = 0; j < g; ++j) {
            double2 x = A[r][j];
            for (int k = 0; k < j; ++k) x = csub(x, cmul(A[r][k], cconj(Lc[j][k])));
            A[r][j] = cscale(x, 1.0 / Lc[j][j].x);
        }
    // cyclic Jacobi: the rotation R = diag(1, e^{-i phi}) [[c, s], [-s, c]] zeroes A[p][q]
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0, tot = 0;
        for (int p = 0; p < g; ++p)
            for (int q = 0; q < g; ++q) { tot += cnorm2(A[p][q]); if (p != q) off += cnorm2(A[p][q]); }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < g; ++p)
            for (int q = p + 1; q < g; ++q) {
                const double b = sqrt(cnorm2(A[p][q]));
                if (b == 0) continue;
                const double2 e = cscale(A[p][q], 1.0 / b);         // e^{i phi}
                const double2 ec = cconj(e);
                const double tau = (A[q][q].x - A[p][p].x) / (2 * b);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1 + tau * tau));
                const double cs = 1 / sqrt(1 + t * t), sn = t * cs;
                // columns: X[:,p] = A[:,p] c - A[:,q] s e^{-i phi};  X[:,q] = A[:,p] s + A[:,q] c e^{-i phi}
                for (int k = 0; k < g; ++k) {
                    const double2 ap = A[k][p], aq = A[k][q];
                    A[k][p] = csub(cscale(ap, cs), cscale(cmul(aq, ec), sn));
                    A[k][q] = cadd(cscale(ap, sn), cscale(cmul(aq, ec), cs));
                    const double2 wp = W[k][p], wq = W[k][q];
                    W[k][p] = csub(cscale(wp, cs), cscale(cmul(wq, ec), sn));
                    W[k][q] = cadd(cscale(wp, sn), cscale(cmul(wq, ec), cs));
                }
                // rows (R^H X): Y[p,:] = c X[p,:] - s e^{i phi} X[q,:];  Y[q,:] = s X[p,:] + c e^{i phi} X[q,:]
                for (int k = 0; k < g; ++k) {
                    const double2 xp = A[p][k], xq = A[q][k];
                    A[p][k] = csub(cscale(xp, cs), cscale(cmul(xq, e), sn));
                    A[q][k] = cadd(cscale(xp, sn), cscale(cmul(xq, e), cs));
                }
            }
    }
    // U = L^-H W (back substitution with L^H)
    for (int c = 0; c < g; ++c)
        for (int i = g - 1; i >= 0; --i) {
            double2 x = W[i][c];
            for (int k = i + 1; k < g; ++k) x = csub(x, cmul(cconj(Lc[k][i]), W[k][c]));
            W[i][c] = cscale(x, 1.0 / Lc[i][i].x);
        }
    for (int i = 0; i < g; ++i) {
        vals[i] = A[i][i].x;
        for (int j = 0; j < g; ++j) U[i * g + j] = W[i][j];
    }
}

// columns idx[0..g) of Cm <- scale * (those columns) U
__global__ void k_apply_group(int n, int g, const int* __restrict__ idx, const double2* __restrict__ U, double scale, double2* Cm) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 x[GMAX], y[GMAX];
    for (int a = 0; a < g; ++a) x[a] = Cm[(size_t)idx[a] * n + r];
    for (int j = 0; j < g; ++j) {
        double2 acc = make_double2(0, 0);
        for (int a = 0; a < g; ++a) cfma(acc, x[a], U[a * g + j]);
        y[j] = cscale(acc, scale);
    }
    for (int j = 0; j < g; ++j) Cm[(size_t)idx[j] * n + r] = y[j];
}

namespace {
struct LinSolve {
    DBuf ipiv, info, work;
    std::vector<char> hwork;
};

int lu_solve(pwqt_ctx* c, const LeadWorker& wk, LinSolve& ls, int n, double2* A, double2* B, int nrhs) {
    size_t wd = 0, wh = 0;
    PWQT_SOLVER(c, cusolverDnXgetrf_bufferSize(wk.sol, wk.prm, n, n, CUDA_C_64F, A, n, CUDA_C_64F, &wd, &wh));
    if (ls.work.bytes < wd) PWQT_TRY(alloc(c, ls.work, wd));
    if (ls.ipiv.bytes < sizeof(int64_t) * n) PWQT_TRY(alloc(c, ls.ipiv, sizeof(int64_t) * n));
    if (!ls.info.p) PWQT_TRY(alloc(c, ls.info, sizeof(int)));
    if (ls.hwork.size() < wh + 16) ls.hwork.resize(wh + 16);
    PWQT_SOLVER(c, cusolverDnXgetrf(wk.sol, wk.prm, n, n, CUDA_C_64F, A, n, ls.ipiv.as<int64_t>(), CUDA_C_64F, ls.work.p,
                                    wd, ls.hwork.data(), wh, ls.info.as<int>()));
    PWQT_SOLVER(c, cusolverDnXgetrs(wk.sol, wk.prm, CUBLAS_OP_N, n, nrhs, CUDA_C_64F, A, n, ls.ipiv.as<int64_t>(),
                                    CUDA_C_64F, B, n, ls.info.as<int>()));
    return PWQT_OK;
}
}  // namespace

// bz: the context that owns the basis (read only); c: a private context for errors.
int compute_lead_shared(const pwqt_ctx* bz, pwqt_ctx* c, const LeadWorker& wk, double Ec,
                        std::unique_ptr<LeadEntry>& result) {
    const int n = bz->n, n2 = 2 * n;
    const double L = bz->Lz;
    cudaStream_t st = wk.stream;
    const dim3 b128(128);
    long long launches = 0;
    DBuf K0, Kp, ApB, AmB, Wmu, VR, lam, Cm, Q, Mk, x, y, forms;
    PWQT_TRY(alloc(c, K0, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, Kp, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, ApB, sizeof(double2) * (size_t)n2 * n2));
    PWQT_TRY(alloc(c, AmB, sizeof(double2) * (size_t)n2 * n2));
    k_lead_K<<<dim3((n + 127) / 128, n), b128, 0, st>>>(n, Ec, bz->H0.as<double2>(), bz->H1.as<double2>(), bz->M0.as<double2>(),
                                                      bz->M1.as<double2>(), K0.as<double2>(), Kp.as<double2>());
    k_lead_cayley<<<dim3((n2 + 127) / 128, n2), b128, 0, st>>>(n, K0.as<double2>(), Kp.as<double2>(), ApB.as<double2>(),
                                                             AmB.as<double2>());
    launches += 2;
    PWQT_CUDA(c, cudaGetLastError());
    LinSolve ls;
    PWQT_TRY(lu_solve(c, wk, ls, n2, ApB.as<double2>(), AmB.as<double2>(), n2));   // AmB <- (A+B)^-1 (A-B)
    // eigen-decomposition of the Cayley-transformed pencil
    PWQT_TRY(alloc(c, Wmu, sizeof(double2) * n2));
    PWQT_TRY(alloc(c, VR, sizeof(double2) * (size_t)n2 * n2));
    size_t wd = 0, wh = 0;
    PWQT_SOLVER(c, cusolverDnXgeev_bufferSize(wk.sol, wk.prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n2, CUDA_C_64F,
                                              AmB.p, n2, CUDA_C_64F, Wmu.p, CUDA_C_64F, nullptr, n2, CUDA_C_64F, VR.p, n2,
                                              CUDA_C_64F, &wd, &wh));
    DBuf gw;
    PWQT_TRY(alloc(c, gw, std::max<size_t>(wd, 16)));
    std::vector<char> gh(wh + 16);
    PWQT_SOLVER(c, cusolverDnXgeev(wk.sol, wk.prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n2, CUDA_C_64F, AmB.p, n2,
                                   CUDA_C_64F, Wmu.p, CUDA_C_64F, nullptr, n2, CUDA_C_64F, VR.p, n2, CUDA_C_64F, gw.p, wd,
                                   gh.data(), wh, ls.info.as<int>()));
    int hinfo = 0;
    PWQT_CUDA(c, cudaMemcpyAsync(&hinfo, ls.info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ApB.release(); gw.release();
    PWQT_TRY(alloc(c, lam, sizeof(double2) * n2));
    PWQT_TRY(alloc(c, Cm, sizeof(double2) * (size_t)n * n2));
    k_lead_modes<<<n2, 256, 0, st>>>(n, Wmu.as<double2>(), VR.as<double2>(), lam.as<double2>(), Cm.as<double2>());
    launches++;
    PWQT_CUDA(c, cudaGetLastError());
    std::vector<double2> hlam(n2);
    PWQT_CUDA(c, cudaMemcpyAsync(hlam.data(), lam.p, sizeof(double2) * n2, cudaMemcpyDeviceToHost, st));
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    if (hinfo != 0) return fail(c, PWQT_ERR_CUDA, "non-Hermitian eigensolver info " + std::to_string(hinfo));
    VR.release(); AmB.release(); Wmu.release();

    // ---- traveling modes: refine onto the unit circle
    const std::vector<double2> raw_lam = hlam;
    std::vector<char> trav(n2, 0);
    std::vector<double> dEdk(n2, 0.0);
    int status = 0;
    PWQT_TRY(alloc(c, Q, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, Mk, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, x, sizeof(double2) * n));
    PWQT_TRY(alloc(c, y, sizeof(double2) * n));
    PWQT_TRY(alloc(c, forms, sizeof(double) * 4));
    const double tol_E = 1e-12 * std::max(1.0, std::fabs(Ec));
    // candidates near the unit circle
    for (int j = 0; j < n2; ++j) {
        double al = std::hypot(hlam[j].x, hlam[j].y);
        if (std::fabs(al - 1.0) < 1e-4) trav[j] = 1;
        else if (std::fabs(al - 1.0) < 1e-3) status |= PWQT_ST_NEAR_UNIT;
    }
    for (int j = 0; j < n2; ++j) {
        if (!trav[j]) continue;
        double k = std::atan2(hlam[j].y, hlam[j].x) / L;
        PWQT_CUDA(c, cudaMemcpyAsync(x.p, Cm.as<double2>() + (size_t)j * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
        double hf[4] = {0, 0, 0, 0};
        double2 ph = make_double2(std::cos(k * L), std::sin(k * L));
        bool converged = false;
        for (int iter = 0; iter < 8; ++iter) {
            ph = make_double2(std::cos(k * L), std::sin(k * L));
            k_lead_hk<<<dim3((n + 127) / 128, n), b128, 0, st>>>(n, ph, Ec, bz->H0.as<double2>(), bz->H1.as<double2>(),
                                                               bz->M0.as<double2>(), bz->M1.as<double2>(), Q.as<double2>(),
                                                               Mk.as<double2>());
            k_matvec_cm<<<(n + 127) / 128, b128, 0, st>>>(n, Mk.as<double2>(), x.as<double2>(), y.as<double2>());
            launches += 2;
            PWQT_TRY(lu_solve(c, wk, ls, n, Q.as<double2>(), y.as<double2>(), 1));   // y <- (H(k) - Ec M(k))^-1 M(k) x
            PWQT_CUDA(c, cudaMemcpyAsync(x.p, y.p, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
            k_lead_forms<<<1, 256, 0, st>>>(n, ph, L, bz->H0.as<double2>(), bz->H1.as<double2>(), bz->M0.as<double2>(),
                                            bz->M1.as<double2>(), x.as<double2>(), forms.as<double>());
            launches++;
            PWQT_CUDA(c, cudaMemcpyAsync(hf, forms.p, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
            PWQT_CUDA(c, cudaStreamSynchronize(st));
            double w = hf[0], slope = hf[2];
            if (std::fabs(w - Ec) < tol_E) { converged = true; break; }
            if (slope == 0.0 || !std::isfinite(slope)) break;
            k -= (w - Ec) / slope;
        }
        if (!converged) {   // no traveling wave at this energy along this branch
            trav[j] = 0;
            status |= PWQT_ST_NEAR_UNIT;
            continue;
        }
        hlam[j] = ph;
        dEdk[j] = hf[2];
        // normalise to c^H M(lambda) c = L / 2pi and store back
        double scale = std::sqrt(L / (2.0 * M_PI) / hf[1]);
        PWQT_CUDA(c, cudaMemcpyAsync(Cm.as<double2>() + (size_t)j * n, x.p, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
        k_scale_col<<<(n + 127) / 128, b128, 0, st>>>(Cm.as<double2>(), n, j, scale);
        launches++;
    }
    // ---- traveling modes at one lambda (Sec. 3.1: degenerate modes must be made flux
    // orthogonal, or the mode-resolved transmission picks up cross terms).  Within each
    // set: the metric and flux forms Gm = C^H M(lambda) C, F = C^H V(lambda) C; two
    // candidates whose normalised M-overlap is 1 are one mode found twice (the second is
    // reclassified by its raw lambda); the rest are rotated by the generalised
    // eigenvectors of (F, Gm) and normalised to c^H M c = L/2pi, their velocities the
    // eigenvalues.  PWQT_ST_DEGENERATE marks an energy with such a set.
    {
        std::vector<char> seen(n2, 0);
        for (int a = 0; a < n2; ++a) {
            if (!trav[a] || seen[a]) continue;
            std::vector<int> grp{a};
            seen[a] = 1;
            for (int b = a + 1; b < n2; ++b)
                if (trav[b] && !seen[b] && std::hypot(hlam[a].x - hlam[b].x, hlam[a].y - hlam[b].y) < 1e-8) {
                    grp.push_back(b);
                    seen[b] = 1;
                }
            if (grp.size() < 2) continue;
            if ((int)grp.size() > GMAX) { status |= PWQT_ST_DEGENERATE | PWQT_ST_NEAR_UNIT; continue; }
            double2 lm = make_double2(0, 0);
            for (int j : grp) lm = cadd(lm, hlam[j]);
            lm = cscale(lm, 1.0 / std::hypot(lm.x, lm.y));
            int g = (int)grp.size();
            DBuf didx, dG, dF, dU, dv, dok;
            PWQT_TRY(alloc(c, didx, sizeof(int) * g));
            PWQT_TRY(alloc(c, dG, sizeof(double2) * g * g));
            PWQT_TRY(alloc(c, dF, sizeof(double2) * g * g));
            PWQT_CUDA(c, cudaMemcpyAsync(didx.p, grp.data(), sizeof(int) * g, cudaMemcpyHostToDevice, st));
            k_group_forms<<<dim3(g, g), 256, 0, st>>>(n, g, didx.as<int>(), lm, Ec, L, bz->H1.as<double2>(), bz->M0.as<double2>(),
                                                     bz->M1.as<double2>(), Cm.as<double2>(), dG.as<double2>(), dF.as<double2>());
            launches++;
            std::vector<double2> hG(g * g);
            PWQT_CUDA(c, cudaMemcpyAsync(hG.data(), dG.p, sizeof(double2) * g * g, cudaMemcpyDeviceToHost, st));
            PWQT_CUDA(c, cudaStreamSynchronize(st));
            // one mode found twice: |c_a^H M c_b| = sqrt(c_a^H M c_a c_b^H M c_b)
            std::vector<int> keep;
            for (int q = 0; q < g; ++q) {
                bool dup = false;
                for (int p : keep) {
                    const double2 x = hG[p * g + q];
                    if (std::hypot(x.x, x.y) > (1.0 - 1e-6) * std::sqrt(hG[p * g + p].x * hG[q * g + q].x)) dup = true;
                }
                if (dup) {
                    trav[grp[q]] = 0;
                    hlam[grp[q]] = raw_lam[grp[q]];
                    status |= PWQT_ST_NEAR_UNIT;
                } else {
                    keep.push_back(q);
                }
            }
            if (keep.size() < 2) continue;
            std::vector<int> sub;
            for (int q : keep) sub.push_back(grp[q]);
            g = (int)sub.size();
            PWQT_CUDA(c, cudaMemcpyAsync(didx.p, sub.data(), sizeof(int) * g, cudaMemcpyHostToDevice, st));
            k_group_forms<<<dim3(g, g), 256, 0, st>>>(n, g, didx.as<int>(), lm, Ec, L, bz->H1.as<double2>(), bz->M0.as<double2>(),
                                                     bz->M1.as<double2>(), Cm.as<double2>(), dG.as<double2>(), dF.as<double2>());
            PWQT_TRY(alloc(c, dU, sizeof(double2) * g * g));
            PWQT_TRY(alloc(c, dv, sizeof(double) * g));
            PWQT_TRY(alloc(c, dok, sizeof(int)));
            k_small_geig<<<1, 32, 0, st>>>(g, dG.as<double2>(), dF.as<double2>(), dU.as<double2>(), dv.as<double>(), dok.as<int>());
            k_apply_group<<<(n + 127) / 128, 128, 0, st>>>(n, g, didx.as<int>(), dU.as<double2>(), std::sqrt(L / (2.0 * M_PI)),
                                                          Cm.as<double2>());
            launches += 3;
            std::vector<double> hv(g);
            int hok = 0;
            PWQT_CUDA(c, cudaMemcpyAsync(hv.data(), dv.p, sizeof(double) * g, cudaMemcpyDeviceToHost, st));
            PWQT_CUDA(c, cudaMemcpyAsync(&hok, dok.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            PWQT_CUDA(c, cudaStreamSynchronize(st));
            PWQT_CUDA(c, cudaGetLastError());
            if (!hok) { status |= PWQT_ST_DEGENERATE | PWQT_ST_NEAR_UNIT; continue; }   // not resolved: flagged
            for (int q = 0; q < g; ++q) {
                hlam[sub[q]] = lm;
                dEdk[sub[q]] = hv[q];
            }
            status |= PWQT_ST_DEGENERATE;
        }
    }

    // ---- classification (Sec. 3.1, drain convention lambda = c_{i+1}/c_i): a mode leaves
    // through the drain when it decays into it (|lambda| < 1) or travels with dE/dk > 0,
    // through the source when |lambda| > 1 or dE/dk < 0.  The section fixes n out-flow
    // modes per contact; any other count marks the energy PWQT_ST_MODE_COUNT and it is
    // not solved.
    std::vector<int> out_d, in_d, out_s, in_s;
    for (int j = 0; j < n2; ++j) {
        const double al = std::hypot(hlam[j].x, hlam[j].y);
        const bool od = trav[j] ? dEdk[j] > 0 : al < 1.0;
        const bool os = trav[j] ? dEdk[j] < 0 : al > 1.0;
        if (od) out_d.push_back(j);
        if (os) out_s.push_back(j);
        if (trav[j] && dEdk[j] < 0) in_d.push_back(j);
        if (trav[j] && dEdk[j] > 0) in_s.push_back(j);
    }
    auto E = std::make_unique<LeadEntry>();
    E->Ec = Ec;
    if ((int)out_d.size() != n || (int)out_s.size() != n) {
        E->status = status | PWQT_ST_MODE_COUNT;
        E->launches = launches;
        result = std::move(E);
        return PWQT_OK;
    }
    // ---- self-energies, projections and injection vectors for both contacts
    auto build = [&](bool drain, DBuf& sigma, DBuf& P, DBuf& vout, DBuf& rhs, DBuf& vin, DBuf* cin, int& ntrav,
                     int& min) -> int {
        const std::vector<int>& outl = drain ? out_d : out_s;
        const std::vector<int>& inl = drain ? in_d : in_s;
        std::vector<double2> lo(n), li(inl.size());
        std::vector<int> trows;
        std::vector<double> tv;
        for (int q = 0; q < n; ++q) {
            double2 l = hlam[outl[q]];
            if (!drain) { double a2 = l.x * l.x + l.y * l.y; l = make_double2(l.x / a2, -l.y / a2); }
            lo[q] = l;
            if (trav[outl[q]]) { trows.push_back(q); tv.push_back(std::fabs(dEdk[outl[q]])); }
        }
        for (size_t q = 0; q < inl.size(); ++q) {
            double2 l = hlam[inl[q]];
            if (!drain) { double a2 = l.x * l.x + l.y * l.y; l = make_double2(l.x / a2, -l.y / a2); }
            li[q] = l;
        }
        ntrav = (int)trows.size();
        min = (int)inl.size();
        DBuf didx, dlam, B, BL, Binv, T1, S, Cin, dli, dtr, R1;
        PWQT_TRY(alloc(c, didx, sizeof(int) * n));
        PWQT_TRY(alloc(c, dlam, sizeof(double2) * n));
        PWQT_CUDA(c, cudaMemcpyAsync(didx.p, outl.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        PWQT_CUDA(c, cudaMemcpyAsync(dlam.p, lo.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st));
        PWQT_TRY(alloc(c, B, sizeof(double2) * n * n));
        PWQT_TRY(alloc(c, BL, sizeof(double2) * n * n));
        PWQT_TRY(alloc(c, Binv, sizeof(double2) * n * n));
        PWQT_TRY(alloc(c, T1, sizeof(double2) * n * n));
        PWQT_TRY(alloc(c, S, sizeof(double2) * n * n));
        k_gather_cols<<<dim3((n + 127) / 128, n), b128, 0, st>>>(n, Cm.as<double2>(), didx.as<int>(), nullptr, B.as<double2>());
        k_gather_cols<<<dim3((n + 127) / 128, n), b128, 0, st>>>(n, Cm.as<double2>(), didx.as<int>(), dlam.as<double2>(), BL.as<double2>());
        k_identity<<<dim3((n + 127) / 128, n), b128, 0, st>>>(n, Binv.as<double2>());
        launches += 3;
        PWQT_TRY(lu_solve(c, wk, ls, n, B.as<double2>(), Binv.as<double2>(), n));   // Binv = B^-1
        cuDoubleComplex one = {1, 0}, zero = {0, 0}, mone = {-1, 0};
        // T1 = (B Lambda) B^-1 ; Sigma = K' T1   (K'_d = K+, K'_s = K- = K+^H), column-major
        PWQT_BLAS(c, cublasZgemm(wk.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, BL.as<cuDoubleComplex>(), n,
                                 Binv.as<cuDoubleComplex>(), n, &zero, T1.as<cuDoubleComplex>(), n));
        PWQT_BLAS(c, cublasZgemm(wk.blas, drain ? CUBLAS_OP_N : CUBLAS_OP_C, CUBLAS_OP_N, n, n, n, &one, Kp.as<cuDoubleComplex>(), n,
                                 T1.as<cuDoubleComplex>(), n, &zero, S.as<cuDoubleComplex>(), n));
        PWQT_TRY(alloc(c, sigma, sizeof(double2) * n * n));
        transpose_c128(S.as<double2>(), sigma.as<double2>(), n, n, st);   // column-major -> row-major
        launches++;
        // rows of B^-1 for traveling out-flow modes
        PWQT_TRY(alloc(c, P, sizeof(double2) * (size_t)std::max(ntrav, 1) * n));
        PWQT_TRY(alloc(c, vout, sizeof(double) * std::max(ntrav, 1)));
        if (ntrav) {
            PWQT_TRY(alloc(c, dtr, sizeof(int) * ntrav));
            PWQT_CUDA(c, cudaMemcpyAsync(dtr.p, trows.data(), sizeof(int) * ntrav, cudaMemcpyHostToDevice, st));
            k_gather_rows<<<dim3((n + 127) / 128, ntrav), b128, 0, st>>>(n, Binv.as<double2>(), dtr.as<int>(), P.as<double2>());
            launches++;
            PWQT_CUDA(c, cudaMemcpyAsync(vout.p, tv.data(), sizeof(double) * ntrav, cudaMemcpyHostToDevice, st));
        }
        // injection vectors rhs = K' C_in Lambda_in - Sigma C_in  (n x m), stored row-major
        int m = min;
        PWQT_TRY(alloc(c, rhs, sizeof(double2) * (size_t)n * std::max(m, 1)));
        PWQT_TRY(alloc(c, vin, sizeof(double) * std::max(m, 1)));
        if (cin) PWQT_TRY(alloc(c, *cin, sizeof(double2) * (size_t)n * std::max(m, 1)));
        if (m) {
            std::vector<double> hv(m);
            for (int q = 0; q < m; ++q) hv[q] = std::fabs(dEdk[inl[q]]);
            PWQT_CUDA(c, cudaMemcpyAsync(vin.p, hv.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
            PWQT_TRY(alloc(c, Cin, sizeof(double2) * (size_t)n * m));
            PWQT_TRY(alloc(c, R1, sizeof(double2) * (size_t)n * m));
            PWQT_TRY(alloc(c, dli, sizeof(double2) * m));
            DBuf didx2;
            PWQT_TRY(alloc(c, didx2, sizeof(int) * m));
            PWQT_CUDA(c, cudaMemcpyAsync(didx2.p, inl.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
            PWQT_CUDA(c, cudaMemcpyAsync(dli.p, li.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, st));
            DBuf CinL;
            PWQT_TRY(alloc(c, CinL, sizeof(double2) * (size_t)n * m));
            k_gather_cols<<<dim3((n + 127) / 128, m), b128, 0, st>>>(n, Cm.as<double2>(), didx2.as<int>(), nullptr, Cin.as<double2>());
            k_gather_cols<<<dim3((n + 127) / 128, m), b128, 0, st>>>(n, Cm.as<double2>(), didx2.as<int>(), dli.as<double2>(), CinL.as<double2>());
            launches += 2;
            // R1 = K' (C_in Lambda) - Sigma C_in
            PWQT_BLAS(c, cublasZgemm(wk.blas, drain ? CUBLAS_OP_N : CUBLAS_OP_C, CUBLAS_OP_N, n, m, n, &one,
                                     Kp.as<cuDoubleComplex>(), n, CinL.as<cuDoubleComplex>(), n, &zero, R1.as<cuDoubleComplex>(), n));
            PWQT_BLAS(c, cublasZgemm(wk.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &mone, S.as<cuDoubleComplex>(), n,
                                     Cin.as<cuDoubleComplex>(), n, &one, R1.as<cuDoubleComplex>(), n));
            transpose_c128(R1.as<double2>(), rhs.as<double2>(), m, n, st);   // (n x m col-major) -> row-major n x m
            if (cin) transpose_c128(Cin.as<double2>(), cin->as<double2>(), m, n, st);
            launches += 2;
        }
        PWQT_CUDA(c, cudaStreamSynchronize(st));
        return PWQT_OK;
    };
    
    PWQT_TRY(build(true, E->sigma_d, E->P_d, E->v_out_d, E->rhs_d, E->v_in_d, nullptr, E->n_trav_out_d, E->m_in_d));
    PWQT_TRY(build(false, E->sigma_s, E->P_s, E->v_out_s, E->rhs_s, E->v_in_s, &E->cin_s, E->n_trav_out_s, E->m_in_s));
    size_t nn = (size_t)n * n;
    PWQT_TRY(alloc(c, E->sigma_d32, sizeof(float2) * nn));
    PWQT_TRY(alloc(c, E->sigma_s32, sizeof(float2) * nn));
    PWQT_TRY(alloc(c, E->rhs_d32, sizeof(float2) * (size_t)n * std::max(E->m_in_d, 1)));
    PWQT_TRY(alloc(c, E->rhs_s32, sizeof(float2) * (size_t)n * std::max(E->m_in_s, 1)));
    c128_to_c64(E->sigma_d.as<double2>(), E->sigma_d32.as<float2>(), nn, st);
    c128_to_c64(E->sigma_s.as<double2>(), E->sigma_s32.as<float2>(), nn, st);
    c128_to_c64(E->rhs_d.as<double2>(), E->rhs_d32.as<float2>(), (size_t)n * E->m_in_d, st);
    c128_to_c64(E->rhs_s.as<double2>(), E->rhs_s32.as<float2>(), (size_t)n * E->m_in_s, st);
    launches += 4;
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    E->status = status;
    E->launches = launches;
    result = std::move(E);
    return PWQT_OK;
}

int LeadWorker::init() {
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return PWQT_ERR_CUDA;
    if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS || cusolverDnCreateParams(&prm) != CUSOLVER_STATUS_SUCCESS ||
        cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS)
        return PWQT_ERR_CUDA;
    cusolverDnSetStream(sol, stream);
    cublasSetStream(blas, stream);
    return PWQT_OK;
}
void LeadWorker::destroy() {
    if (prm) cusolverDnDestroyParams(prm);
    if (sol) cusolverDnDestroy(sol);
    if (blas) cublasDestroy(blas);
    if (stream) cudaStreamDestroy(stream);
    prm = nullptr; sol = nullptr; blas = nullptr; stream = nullptr;
}

// Fill the cache for every key in `keys` that is missing, with up to
// opts-independent min(#missing, 8) host threads, each driving its own stream and
// solver handles (the eigensolver is latency-bound; concurrent energies overlap).
int fill_leads(pwqt_ctx* c, const std::vector<double>& keys) {
    std::vector<double> miss;
    for (double k : keys)
        if (!c->cache.count(k) && std::find(miss.begin(), miss.end(), k) == miss.end()) miss.push_back(k);
    if (miss.empty()) return PWQT_OK;
    int nthreads = (int)std::min<size_t>(miss.size(), (size_t)std::max(1, c->lead_threads));
    while ((int)c->workers.size() < nthreads) {
        c->workers.emplace_back(new LeadWorker());
        int r = c->workers.back()->init();
        if (r != PWQT_OK) { c->workers.back()->destroy(); c->workers.pop_back(); if (c->workers.empty()) return fail(c, r, "lead worker init"); break; }
    }
    nthreads = std::min<int>(nthreads, (int)c->workers.size());
    std::vector<std::unique_ptr<LeadEntry>> res(miss.size());
    std::vector<int> rc(nthreads, PWQT_OK);
    std::vector<std::string> errs(nthreads);
    std::atomic<size_t> next{0};
    auto work = [&](int t) {
        cudaSetDevice(c->dev);
        pwqt_ctx local;      // private error slot; the worker owns stream and handles
        local.dev = c->dev;
        local.n = c->n; local.Lz = c->Lz;
        for (;;) {
            size_t i = next.fetch_add(1);
            if (i >= miss.size()) break;
            int r = compute_lead_shared(c, &local, *c->workers[t], miss[i], res[i]);
            if (r != PWQT_OK) { rc[t] = r; errs[t] = local.err; break; }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    for (int t = 0; t < nthreads; ++t)
        if (rc[t] != PWQT_OK) return fail(c, rc[t], errs[t]);
    for (size_t i = 0; i < miss.size(); ++i) {
        c->launches += res[i]->launches;
        c->cache[miss[i]] = std::move(res[i]);
    }
    return PWQT_OK;
}

int lead_entry(pwqt_ctx* c, double Ec, LeadEntry** out) {
    auto it = c->cache.find(Ec);
    if (it == c->cache.end()) {
        PWQT_TRY(fill_leads(c, std::vector<double>{Ec}));
        it = c->cache.find(Ec);
    }
    *out = it->second.get();
    return PWQT_OK;
}

}  // namespace pwqt
