// Intrinsic and extrinsic blocks of the partition-of-unity Bloch-wave basis
// (Sec. 2.2-2.3, App. A of arXiv:1903.00548), computed on the GPU.
//
// Element integrals are evaluated in closed form: the enhancement functions are
// plane-wave sums, the hats are polynomials in the element coordinate s, so every
// integral reduces to J_p(q) = int_0^L s^p e^{iqs} ds (p <= 3) with q L a multiple
// of pi.  The kinetic + momentum-coupling part is used in the compact Hermitian form
//   (T + P)_ab = hbar^2/2m int [ f_a' f_b' phi_a^* phi_b
//                               + 1/2 (f_a f_b' - f_a' f_b)(d phi_a^* phi_b - phi_a^* d phi_b) ],
// which follows from T = (T^r + T^l)/2 and P = (P^r + P^l)/2 of App. A after
// integration by parts; with linear hats (f_a f_b' - f_a' f_b) is a constant.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "pwqt_internal.cuh"
#include "sweep_mixed.cuh"

namespace pwqt {

int fail(pwqt_ctx* c, int code, const std::string& msg) {
    if (c) {
        std::lock_guard<std::mutex> g(c->err_m);
        c->err = msg;
    }
    return code;
}

int Lane::init(int dev) {
    if (st) return PWQT_OK;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return PWQT_ERR_CUDA;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return PWQT_ERR_CUDA;
    for (auto& e : oz_ev)
        if (cudaEventCreate(&e) != cudaSuccess) return PWQT_ERR_CUDA;
    return PWQT_OK;
}

void Lane::destroy() {
    if (st) cudaStreamSynchronize(st);
    ws_mixed.release(); ws_jobs.release(); ws_obs.release(); ws_res.release(); ws_norms.release();
    oz_sig.release(); oz_sig_rexp.release(); oz_sig_tab.release(); oz_B.release(); oz_fexp.release(); oz_act.release();
    for (auto& e : ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    for (auto& e : oz_ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (st) cudaStreamDestroy(st);
    st = nullptr;
}
int cuda_fail(pwqt_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? PWQT_ERR_OOM : PWQT_ERR_CUDA,
                std::string(cudaGetErrorString(e)) + " in " + what);
}
int alloc(pwqt_ctx* c, DBuf& b, size_t bytes) {
    b.release();
    if (bytes == 0) return PWQT_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(c, PWQT_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    b.bytes = bytes;
    return PWQT_OK;
}

int ensure(pwqt_ctx* c, DBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return PWQT_OK;
    return alloc(c, b, bytes + bytes / 8);
}

// ---------------------------------------------------------------- small utilities
__global__ void k_transpose_c128(const double2* __restrict__ in, double2* __restrict__ out, int rows, int cols) {
    __shared__ double2 t[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int r = by + j, cc = bx + threadIdx.x;
        if (r < rows && cc < cols) t[j][threadIdx.x] = in[(size_t)r * cols + cc];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int r = bx + j, cc = by + threadIdx.x;   // out is cols x rows
        if (r < cols && cc < rows) out[(size_t)r * rows + cc] = t[threadIdx.x][j];
    }
}
void transpose_c128(const double2* in, double2* out, int rows, int cols, cudaStream_t st) {
    dim3 g((cols + 31) / 32, (rows + 31) / 32), b(32, 8);
    k_transpose_c128<<<g, b, 0, st>>>(in, out, rows, cols);
}
__global__ void k_c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
void c128_to_c64(const double2* in, float2* out, size_t count, cudaStream_t st) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
    if (blocks > 0) k_c128_to_c64<<<blocks, 256, 0, st>>>(in, out, count);
}

// ---------------------------------------------------------------- EPM Hamiltonian
struct Atoms { int n; const double* xz; };

// H (column-major, ng x ng): hbar^2/2m |k+G|^2 delta_GG' + V_{G-G'}, with
// V_G = (omega0/Omega) v0 exp(-|G|^2/(2 sigma^2)) sum_a exp(-i G.R_a), V_0 = 0.
__global__ void k_epm_hamiltonian(double2* H, int ng, const int* __restrict__ mx, const int* __restrict__ mz,
                                  double bx, double bz, double k, double pref, double inv2s2,
                                  const double* __restrict__ xz, int n_atoms) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;   // row
    int j = blockIdx.y;                                // column
    if (i >= ng) return;
    double2 h = make_double2(0.0, 0.0);
    int dmx = mx[i] - mx[j], dmz = mz[i] - mz[j];
    if (dmx != 0 || dmz != 0) {
        double gx = dmx * bx, gz = dmz * bz;
        double v = pref * exp(-(gx * gx + gz * gz) * inv2s2);
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < n_atoms; ++a) {
            double ph = -(gx * xz[2 * a] + gz * xz[2 * a + 1]);
            double s, cph;
            sincos(ph, &s, &cph);
            sr += cph; si += s;
        }
        h = make_double2(v * sr, v * si);
    }
    if (i == j) {
        double gx = mx[i] * bx, gz = mz[i] * bz + k;
        h.x += HB2M * (gx * gx + gz * gz);
    }
    H[(size_t)j * ng + i] = h;
}

// first nb eigenvectors (columns of V, column-major ng x ng) -> C (ng x nb row-major)
__global__ void k_gather_vectors(const double2* __restrict__ V, double2* __restrict__ C, int ng, int nb) {
    int g = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (g < ng && b < nb) C[(size_t)g * nb + b] = V[(size_t)b * ng + g];
}

static void pw_set(const pwqt_cell* cell, double k, double gcut, std::vector<int>& mx, std::vector<int>& mz) {
    double bz = 2.0 * M_PI / cell->Lz;
    double bx = cell->dim == 2 ? 2.0 * M_PI / cell->Lx : 0.0;
    int mzmax = (int)std::ceil((gcut + std::fabs(k)) / bz) + 1;
    int mxmax = cell->dim == 2 ? (int)std::ceil(gcut / bx) + 1 : 0;
    mx.clear(); mz.clear();
    for (int a = -mxmax; a <= mxmax; ++a)
        for (int b = -mzmax; b <= mzmax; ++b) {
            double gx = a * bx, gz = b * bz + k;
            if (gx * gx + gz * gz <= gcut * gcut * (1.0 + 1e-14)) { mx.push_back(a); mz.push_back(b); }
        }
}

int epm_basis(pwqt_ctx* c, const pwqt_cell* cell, const pwqt_formfactor* ff, double gcut, int n_bands) {
    double ks[2] = {0.0, M_PI / cell->Lz};
    std::vector<int> mxs[2], mzs[2];
    for (int g = 0; g < 2; ++g) {
        pw_set(cell, ks[g], gcut, mxs[g], mzs[g]);
        if ((int)mxs[g].size() < n_bands)
            return fail(c, PWQT_ERR_BASIS_TOO_SMALL, "fewer plane waves (" + std::to_string(mxs[g].size()) +
                                                         ") than requested bands (" + std::to_string(n_bands) + ")");
    }
    double omega = cell->Lz * cell->Lx;
    double pref = cell->omega0 / omega * ff->v0;
    double bz = 2.0 * M_PI / cell->Lz, bx = cell->dim == 2 ? 2.0 * M_PI / cell->Lx : 0.0;
    DBuf d_xz;
    PWQT_TRY(alloc(c, d_xz, sizeof(double) * 2 * std::max(cell->n_atoms, 1)));
    PWQT_CUDA(c, cudaMemcpyAsync(d_xz.p, cell->atoms, sizeof(double) * 2 * cell->n_atoms, cudaMemcpyHostToDevice, c->stream));
    std::vector<double> eps(2 * n_bands);
    int n_pw[2] = {(int)mxs[0].size(), (int)mxs[1].size()};
    DBuf coef;
    PWQT_TRY(alloc(c, coef, sizeof(double2) * (size_t)(n_pw[0] + n_pw[1]) * n_bands));
    size_t off = 0;
    for (int g = 0; g < 2; ++g) {
        int ng = n_pw[g];
        DBuf d_mx, d_mz, H, W;
        PWQT_TRY(alloc(c, d_mx, sizeof(int) * ng));
        PWQT_TRY(alloc(c, d_mz, sizeof(int) * ng));
        PWQT_TRY(alloc(c, H, sizeof(double2) * (size_t)ng * ng));
        PWQT_TRY(alloc(c, W, sizeof(double) * ng));
        PWQT_CUDA(c, cudaMemcpyAsync(d_mx.p, mxs[g].data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c->stream));
        PWQT_CUDA(c, cudaMemcpyAsync(d_mz.p, mzs[g].data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c->stream));
        dim3 grid((ng + 127) / 128, ng);
        k_epm_hamiltonian<<<grid, 128, 0, c->stream>>>(H.as<double2>(), ng, d_mx.as<int>(), d_mz.as<int>(), bx, bz, ks[g],
                                                       pref, 1.0 / (2.0 * ff->sigma * ff->sigma), d_xz.as<double>(), cell->n_atoms);
        c->launches++;
        PWQT_CUDA(c, cudaGetLastError());
        size_t wd = 0, wh = 0;
        PWQT_SOLVER(c, cusolverDnXsyevd_bufferSize(c->sol, c->prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ng,
                                                    CUDA_C_64F, H.p, ng, CUDA_R_64F, W.p, CUDA_C_64F, &wd, &wh));
        DBuf bd, info;
        PWQT_TRY(alloc(c, bd, std::max<size_t>(wd, 16)));
        PWQT_TRY(alloc(c, info, sizeof(int)));
        std::vector<char> bh(wh + 16);
        PWQT_SOLVER(c, cusolverDnXsyevd(c->sol, c->prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ng, CUDA_C_64F, H.p,
                                         ng, CUDA_R_64F, W.p, CUDA_C_64F, bd.p, wd, bh.data(), wh, info.as<int>()));
        int hinfo = 0;
        PWQT_CUDA(c, cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PWQT_CUDA(c, cudaMemcpyAsync(eps.data() + g * n_bands, W.p, sizeof(double) * n_bands, cudaMemcpyDeviceToHost, c->stream));
        dim3 gg((ng + 127) / 128, n_bands);
        k_gather_vectors<<<gg, 128, 0, c->stream>>>(H.as<double2>(), coef.as<double2>() + off, ng, n_bands);
        c->launches++;
        PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
        if (hinfo != 0) return fail(c, PWQT_ERR_CUDA, "Hermitian eigensolver info " + std::to_string(hinfo));
        off += (size_t)ng * n_bands;
    }
    std::vector<int> mx_all, mz_all;
    for (int g = 0; g < 2; ++g) {
        mx_all.insert(mx_all.end(), mxs[g].begin(), mxs[g].end());
        mz_all.insert(mz_all.end(), mzs[g].begin(), mzs[g].end());
    }
    return assemble_from_basis(c, cell, n_bands, eps.data(), n_pw, mx_all.data(), mz_all.data(), coef.as<double2>());
}

// ---------------------------------------------------------------- element integrals
// J_p(q) = int_0^L s^p e^{iqs} ds, p = 0..3, for q L = nu pi (nu integer).
__device__ inline void j_moments(int nu, double L, double2 J[4]) {
    if (nu == 0) {
        J[0] = make_double2(L, 0); J[1] = make_double2(L * L / 2, 0);
        J[2] = make_double2(L * L * L / 3, 0); J[3] = make_double2(L * L * L * L / 4, 0);
        return;
    }
    double q = nu * M_PI / L;
    double e = (nu & 1) ? -1.0 : 1.0;                 // e^{iqL}
    // 1/(iq) = -i/q
    double iq = 1.0 / q;
    // J0 = (e - 1)/(iq)
    J[0] = make_double2(0.0, -(e - 1.0) * iq);
    double Lp = 1.0;
    for (int p = 1; p < 4; ++p) {
        Lp *= L;
        // J_p = (L^p e - p J_{p-1}) / (iq)
        double2 num = make_double2(Lp * e - p * J[p - 1].x, -p * J[p - 1].y);
        J[p] = make_double2(num.y * iq, -num.x * iq);
    }
}

struct PwGroup {
    int ng;
    const int* mx;      // sorted by (mx, mz)
    const int* mz;
    const double2* C;   // ng x nb row-major
    const int* lo;      // per PW of this group: range [lo, hi) in the *other* group with equal mx
    const int* hi;
};

// base sums for one (alpha, beta): S_p (p=0..3) and R0 (with Qsum weight), left-node phases.
// out: 5 n x n row-major planes.
__global__ void k_element_sums(int nb, double Lz, double bz, PwGroup g0, PwGroup g1, const int* __restrict__ lo00,
                               const int* __restrict__ hi00, const int* __restrict__ lo01, const int* __restrict__ hi01,
                               const int* __restrict__ lo10, const int* __restrict__ hi10, const int* __restrict__ lo11,
                               const int* __restrict__ hi11, double Lx, double2* __restrict__ out) {
    int n = 2 * nb;
    int beta = blockIdx.x * blockDim.x + threadIdx.x;
    int alpha = blockIdx.y;
    if (beta >= n) return;
    int ga = alpha >= nb, gb = beta >= nb;
    int ia = alpha - ga * nb, ib = beta - gb * nb;
    const PwGroup& A = ga ? g1 : g0;
    const PwGroup& B = gb ? g1 : g0;
    const int* lo = ga ? (gb ? lo11 : lo10) : (gb ? lo01 : lo00);
    const int* hi = ga ? (gb ? hi11 : hi10) : (gb ? hi01 : hi00);
    double ka = ga ? M_PI / Lz : 0.0, kb = gb ? M_PI / Lz : 0.0;
    int dnu = gb - ga;   // (k_b - k_a) L / pi
    double2 S[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}}, R0 = {0, 0};
    for (int j = 0; j < A.ng; ++j) {
        double2 ca = A.C[(size_t)j * nb + ia];
        if (ca.x == 0.0 && ca.y == 0.0) continue;
        double Qa = A.mz[j] * bz + ka;
        for (int t = lo[j]; t < hi[j]; ++t) {
            double2 w = cmul(cconj(ca), B.C[(size_t)t * nb + ib]);
            int nu = 2 * (B.mz[t] - A.mz[j]) + dnu;
            double2 J[4];
            j_moments(nu, Lz, J);
            for (int p = 0; p < 4; ++p) cfma(S[p], w, J[p]);
            double Qs = Qa + B.mz[t] * bz + kb;
            cfma(R0, cscale(w, Qs), J[0]);
        }
    }
    size_t nn = (size_t)n * n, idx = (size_t)alpha * n + beta;
    for (int p = 0; p < 4; ++p) out[p * nn + idx] = cscale(S[p], Lx);
    out[4 * nn + idx] = cscale(R0, Lx);
}

// Node blocks from the base sums: M0, M1, H0, H1 and the six W blocks.
__global__ void k_element_blocks(int n, int nb, double L, const double* __restrict__ eps, const double2* __restrict__ sums,
                                 double2* M0, double2* M1, double2* H0, double2* H1, double2* W) {
    int beta = blockIdx.x * blockDim.x + threadIdx.x, alpha = blockIdx.y;
    if (beta >= n) return;
    size_t nn = (size_t)n * n, idx = (size_t)alpha * n + beta;
    double2 S0 = sums[idx], S1 = sums[nn + idx], S2 = sums[2 * nn + idx], S3 = sums[3 * nn + idx], R0 = sums[4 * nn + idx];
    double iL = 1.0 / L, iL2 = iL * iL, iL3 = iL2 * iL;
    // phases of the right-node functions: e^{-i k L} = +1 (Gamma) or -1 (Z)
    double pa = alpha >= nb ? -1.0 : 1.0, pb = beta >= nb ? -1.0 : 1.0;
    auto lin = [](double2 a, double ca, double2 b, double cb, double2 c2, double cc, double2 d, double cd) {
        return make_double2(a.x * ca + b.x * cb + c2.x * cc + d.x * cd, a.y * ca + b.y * cb + c2.y * cc + d.y * cd);
    };
    double2 z = make_double2(0, 0);
    double2 Mll = lin(S0, 1.0, S1, -2.0 * iL, S2, iL2, z, 0);
    double2 Mlr = lin(S1, iL, S2, -iL2, z, 0, z, 0);
    double2 Mrr = cscale(S2, iL2);
    double2 Wlll = lin(S0, 1.0, S1, -3.0 * iL, S2, 3.0 * iL2, S3, -iL3);
    double2 Wllr = lin(S1, iL, S2, -2.0 * iL2, S3, iL3, z, 0);
    double2 Wlrr = lin(S2, iL2, S3, -iL3, z, 0, z, 0);
    double2 Wrrr = cscale(S3, iL3);
    double2 Kd = cscale(S0, HB2M * iL2);                                       // ll and rr
    double2 Klr = make_double2(HB2M * (-S0.x * iL2 + R0.y * 0.5 * iL),       // -S0/L^2 - i R0/(2L)
                               HB2M * (-S0.y * iL2 - R0.x * 0.5 * iL));
    double ee = 0.5 * (eps[alpha] + eps[beta]);
    double prr = pa * pb, plr = pb;          // conj(ph_a) ph_b for (r,r) and (l,r)
    double2 mrr = cscale(Mrr, prr), mll = Mll, mlr = cscale(Mlr, plr);
    M0[idx] = cadd(mrr, mll);
    M1[idx] = mlr;
    double2 hll = cadd(cscale(Mll, ee), Kd);
    double2 hrr = cscale(cadd(cscale(Mrr, ee), Kd), prr);
    double2 hlr = cscale(cadd(cscale(Mlr, ee), Klr), plr);
    H0[idx] = cadd(hrr, hll);
    H1[idx] = hlr;
    // W^l_ll = f_l^3, W^l_lr = f_l^2 f_r, W^l_rr = f_l f_r^2, W^r_ll = f_l^2 f_r, W^r_lr = f_l f_r^2, W^r_rr = f_r^3
    W[0 * nn + idx] = Wlll;
    W[1 * nn + idx] = cscale(Wllr, plr);
    W[2 * nn + idx] = cscale(Wlrr, prr);
    W[3 * nn + idx] = Wllr;
    W[4 * nn + idx] = cscale(Wlrr, plr);
    W[5 * nn + idx] = cscale(Wrrr, prr);
}

int assemble_from_basis(pwqt_ctx* c, const pwqt_cell* cell, int n_bands, const double* eps_host, const int* n_pw,
                        const int* mx_in, const int* mz_in, const double2* coef_dev) {
    int nb = n_bands, n = 2 * nb;
    // sort each group's plane waves by (mx, mz) and build equal-mx ranges
    std::vector<int> order[2], mx[2], mz[2];
    size_t off[2] = {0, (size_t)n_pw[0]};
    for (int g = 0; g < 2; ++g) {
        order[g].resize(n_pw[g]);
        std::iota(order[g].begin(), order[g].end(), 0);
        const int* gx = mx_in + off[g];
        const int* gz = mz_in + off[g];
        std::stable_sort(order[g].begin(), order[g].end(), [&](int a, int b) {
            return gx[a] != gx[b] ? gx[a] < gx[b] : gz[a] < gz[b];
        });
        for (int j : order[g]) { mx[g].push_back(gx[j]); mz[g].push_back(gz[j]); }
    }
    std::vector<int> lo[2][2], hi[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            lo[a][b].resize(n_pw[a]); hi[a][b].resize(n_pw[a]);
            for (int j = 0; j < n_pw[a]; ++j) {
                auto r = std::equal_range(mx[b].begin(), mx[b].end(), mx[a][j]);
                lo[a][b][j] = (int)(r.first - mx[b].begin());
                hi[a][b][j] = (int)(r.second - mx[b].begin());
            }
        }
    // permute coefficient rows to the sorted order
    DBuf Cs[2], dmx[2], dmz[2], dlo[2][2], dhi[2][2];
    std::vector<double2> hc;
    for (int g = 0; g < 2; ++g) {
        size_t rows = n_pw[g];
        std::vector<double2> tmp(rows * nb);
        PWQT_CUDA(c, copy_sync(c, tmp.data(), coef_dev + off[g] * nb, sizeof(double2) * rows * nb, cudaMemcpyDeviceToHost));
        hc.assign(rows * nb, make_double2(0, 0));
        for (size_t r = 0; r < rows; ++r)
            for (int b = 0; b < nb; ++b) hc[r * nb + b] = tmp[(size_t)order[g][r] * nb + b];
        PWQT_TRY(alloc(c, Cs[g], sizeof(double2) * rows * nb));
        PWQT_CUDA(c, copy_sync(c, Cs[g].p, hc.data(), sizeof(double2) * rows * nb, cudaMemcpyHostToDevice));
        PWQT_TRY(alloc(c, dmx[g], sizeof(int) * rows));
        PWQT_TRY(alloc(c, dmz[g], sizeof(int) * rows));
        PWQT_CUDA(c, copy_sync(c, dmx[g].p, mx[g].data(), sizeof(int) * rows, cudaMemcpyHostToDevice));
        PWQT_CUDA(c, copy_sync(c, dmz[g].p, mz[g].data(), sizeof(int) * rows, cudaMemcpyHostToDevice));
        for (int b = 0; b < 2; ++b) {
            PWQT_TRY(alloc(c, dlo[g][b], sizeof(int) * rows));
            PWQT_TRY(alloc(c, dhi[g][b], sizeof(int) * rows));
            PWQT_CUDA(c, copy_sync(c, dlo[g][b].p, lo[g][b].data(), sizeof(int) * rows, cudaMemcpyHostToDevice));
            PWQT_CUDA(c, copy_sync(c, dhi[g][b].p, hi[g][b].data(), sizeof(int) * rows, cudaMemcpyHostToDevice));
        }
    }
    PwGroup g0{n_pw[0], dmx[0].as<int>(), dmz[0].as<int>(), Cs[0].as<double2>(), nullptr, nullptr};
    PwGroup g1{n_pw[1], dmx[1].as<int>(), dmz[1].as<int>(), Cs[1].as<double2>(), nullptr, nullptr};
    size_t nn = (size_t)n * n;
    DBuf sums, d_eps;
    PWQT_TRY(alloc(c, sums, sizeof(double2) * nn * 5));
    PWQT_TRY(alloc(c, d_eps, sizeof(double) * n));
    PWQT_CUDA(c, copy_sync(c, d_eps.p, eps_host, sizeof(double) * n, cudaMemcpyHostToDevice));
    double bz = 2.0 * M_PI / cell->Lz;
    dim3 grid((n + 127) / 128, n);
    k_element_sums<<<grid, 128, 0, c->stream>>>(nb, cell->Lz, bz, g0, g1, dlo[0][0].as<int>(), dhi[0][0].as<int>(),
                                                dlo[0][1].as<int>(), dhi[0][1].as<int>(), dlo[1][0].as<int>(),
                                                dhi[1][0].as<int>(), dlo[1][1].as<int>(), dhi[1][1].as<int>(), cell->Lx,
                                                sums.as<double2>());
    c->launches++;
    PWQT_CUDA(c, cudaGetLastError());
    PWQT_TRY(alloc(c, c->H0, sizeof(double2) * nn));
    PWQT_TRY(alloc(c, c->H1, sizeof(double2) * nn));
    c->ozM.release();          // slice panels of the previous basis
    c->ozM_rexp.release();
    PWQT_TRY(alloc(c, c->M0, sizeof(double2) * nn));
    PWQT_TRY(alloc(c, c->M1, sizeof(double2) * nn));
    PWQT_TRY(alloc(c, c->W, sizeof(double2) * nn * 6));
    k_element_blocks<<<grid, 128, 0, c->stream>>>(n, nb, cell->Lz, d_eps.as<double>(), sums.as<double2>(), c->M0.as<double2>(),
                                                  c->M1.as<double2>(), c->H0.as<double2>(), c->H1.as<double2>(), c->W.as<double2>());
    c->launches++;
    PWQT_CUDA(c, cudaGetLastError());
    PWQT_TRY(alloc(c, c->M0f, sizeof(float2) * nn));
    PWQT_TRY(alloc(c, c->M1f, sizeof(float2) * nn));
    PWQT_TRY(alloc(c, c->H0f, sizeof(float2) * nn));
    PWQT_TRY(alloc(c, c->H1f, sizeof(float2) * nn));
    c128_to_c64(c->M0.as<double2>(), c->M0f.as<float2>(), nn, c->stream);
    c128_to_c64(c->M1.as<double2>(), c->M1f.as<float2>(), nn, c->stream);
    c128_to_c64(c->H0.as<double2>(), c->H0f.as<float2>(), nn, c->stream);
    c128_to_c64(c->H1.as<double2>(), c->H1f.as<float2>(), nn, c->stream);
    c->launches += 4;
    PWQT_TRY(alloc(c, c->M0ff, sizeof(float4) * nn));
    PWQT_TRY(alloc(c, c->M1ff, sizeof(float4) * nn));
    split_ff(c->M0.as<double2>(), c->M0ff.as<float4>(), nn, c->stream);
    split_ff(c->M1.as<double2>(), c->M1ff.as<float4>(), nn, c->stream);
    c->launches += 2;
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->n = n;
    c->n_bands = nb;
    c->Lz = cell->Lz;
    c->Lx = cell->Lx;
    c->dim = cell->dim;
    for (int g = 0; g < 2; ++g) {   // kept for evaluating the basis on a real-space grid
        c->pw_n[g] = n_pw[g];
        c->pw_mx[g] = std::move(dmx[g]);
        c->pw_mz[g] = std::move(dmz[g]);
        c->pw_C[g] = std::move(Cs[g]);
    }
    c->eps.assign(eps_host, eps_host + n);
    c->systems.clear();
    c->cache.clear();
    return PWQT_OK;
}

// ---------------------------------------------------------------- extrinsic blocks
// V_ii = U_{i-1} W^l_rr + U_i (W^r_rr + W^l_ll) + U_{i+1} W^r_ll ; V_{i,i+1} = U_i W^l_lr + U_{i+1} W^r_lr
// (nodes 0..N-1 here; U_{-1} = U_0, U_N = U_{N-1}: flat leads).  Writes H0 + V_ii and H1 + V_{i,i+1}.
__global__ void k_system_blocks(int n, int N, const double* __restrict__ U, const double2* __restrict__ H0,
                                const double2* __restrict__ H1, const double2* __restrict__ W, double2* HV0, double2* HV1) {
    size_t nn = (size_t)n * n;
    int i = blockIdx.y;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        double um = U[i > 0 ? i - 1 : 0], u0 = U[i], up = U[i + 1 < N ? i + 1 : N - 1];
        double2 v = cscale(W[2 * nn + e], um);
        v = cadd(v, cscale(cadd(W[5 * nn + e], W[0 * nn + e]), u0));
        v = cadd(v, cscale(W[3 * nn + e], up));
        HV0[(size_t)i * nn + e] = cadd(H0[e], v);
        if (i + 1 < N) {
            double2 w = cadd(cscale(W[1 * nn + e], u0), cscale(W[4 * nn + e], up));
            HV1[(size_t)i * nn + e] = cadd(H1[e], w);
        }
    }
}

int build_system_blocks(pwqt_ctx* c, System& s) {
    s.ozH.release();           // slice panels of the previous potential
    s.ozH_rexp.release();
    int n = c->n, N = s.N;
    size_t nn = (size_t)n * n;
    DBuf dU;
    PWQT_TRY(alloc(c, dU, sizeof(double) * N));
    PWQT_CUDA(c, copy_sync(c, dU.p, s.U.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    PWQT_TRY(alloc(c, s.HV0, sizeof(double2) * nn * N));
    PWQT_TRY(alloc(c, s.HV1, sizeof(double2) * nn * std::max(N - 1, 1)));
    dim3 grid((unsigned)std::min<size_t>((nn + 255) / 256, 1024), N);
    k_system_blocks<<<grid, 256, 0, c->stream>>>(n, N, dU.as<double>(), c->H0.as<double2>(), c->H1.as<double2>(),
                                                 c->W.as<double2>(), s.HV0.as<double2>(), s.HV1.as<double2>());
    c->launches++;
    PWQT_CUDA(c, cudaGetLastError());
    PWQT_TRY(alloc(c, s.HV0f, sizeof(float2) * nn * N));
    PWQT_TRY(alloc(c, s.HV1f, sizeof(float2) * nn * std::max(N - 1, 1)));
    c128_to_c64(s.HV0.as<double2>(), s.HV0f.as<float2>(), nn * N, c->stream);
    c128_to_c64(s.HV1.as<double2>(), s.HV1f.as<float2>(), nn * (N - 1), c->stream);
    c->launches += 2;
    PWQT_TRY(alloc(c, s.HV0ff, sizeof(float4) * nn * N));
    PWQT_TRY(alloc(c, s.HV1ff, sizeof(float4) * nn * std::max(N - 1, 1)));
    split_ff(s.HV0.as<double2>(), s.HV0ff.as<float4>(), nn * N, c->stream);
    split_ff(s.HV1.as<double2>(), s.HV1ff.as<float4>(), nn * (N - 1), c->stream);
    c->launches += 2;
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    return PWQT_OK;
}

}  // namespace pwqt
