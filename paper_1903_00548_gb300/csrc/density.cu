// Electron density by the density-matrix route of Sec. 3.3.
//
// Accumulation (Eq. density_matrices): for every solved energy E with quadrature
// weight w_E and every injected mode gamma (density of states g = 2/|dE/dk|,
// occupation f_FD(E - mu) of the contact that injects it)
//     rho_d[a]_{alpha beta} += w_E g f conj(c_{a alpha}) c_{a beta}
//     rho_u[a]_{alpha beta} += w_E g f conj(c_{a alpha}) c_{a+1 beta}
// on the diagonal node blocks and the blocks coupling node a to a+1 (the only ones
// the density needs, since the hats of nodes further apart do not overlap).
//
// Real-space density (Eq. density_3d_fast): on the element between nodes e and e+1,
// with local coordinate s in [0, L], hats f_l = 1 - s/L and f_r = s/L, and phi the
// enhancement functions with the left node's phase,
//     n(r) = f_l^2 phi^H rho_d[e] phi + f_r^2 phi_r^H rho_d[e+1] phi_r
//          + 2 f_l f_r Re(phi^H rho_u[e] phi_r),     phi_r = phi e^{-ik L}.
// All FP64 on the CUDA cores.
#include <algorithm>
#include <cmath>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

namespace pwqt {

namespace {

// ---------------------------------------------------------------- accumulation
constexpr int DT = 32;   // output tile (rows and columns)
constexpr int DK = 16;   // injected modes per shared-memory chunk

__global__ void __launch_bounds__(256) k_density_accum(const DensJob* __restrict__ jobs, int nb, int n, int N, int tiles,
                                                       double2* __restrict__ rho_d, double2* __restrict__ rho_u) {
    const int a = blockIdx.y, up = blockIdx.z;
    if (up && a >= N - 1) return;
    int ti, tj;
    if (up) {
        ti = blockIdx.x / tiles;
        tj = blockIdx.x % tiles;
    } else {
        // rho_d[a] is Hermitian: tiles on and above the diagonal, mirrored below
        if ((int)blockIdx.x >= tiles * (tiles + 1) / 2) return;
        int k = blockIdx.x;
        ti = 0;
        while (k >= tiles - ti) { k -= tiles - ti; ++ti; }
        tj = ti + k;
    }
    const int a0 = ti * DT, b0 = tj * DT;
    __shared__ double2 As[DK][DT + 1];
    __shared__ double2 Bs[DK][DT + 1];
    const int t = threadIdx.x, tx = t % 32, ty = t / 32;
    double2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_double2(0, 0);
    for (int b = 0; b < nb; ++b) {
        const DensJob J = jobs[b];
        const int K = J.ms + J.md;
        if (K == 0 || !J.C) continue;
        const double2* ca = J.C + (size_t)a * J.node_stride;
        const double2* cb = J.C + (size_t)(a + up) * J.node_stride;
        for (int g0 = 0; g0 < K; g0 += DK) {
            for (int e = t; e < DT * DK; e += 256) {
                const int i = e / DK, k = e % DK, g = g0 + k;
                double2 va = make_double2(0, 0), vb = make_double2(0, 0);
                if (g < K) {
                    const double wt = g < J.ms ? J.scale_s * 2.0 / J.v_in_s[g] : J.scale_d * 2.0 / J.v_in_d[g - J.ms];
                    if (a0 + i < n) {
                        const double2 x = ca[(size_t)(a0 + i) * J.row_stride + g];
                        va = make_double2(wt * x.x, -wt * x.y);
                    }
                    if (b0 + i < n) vb = cb[(size_t)(b0 + i) * J.row_stride + g];
                }
                As[k][i] = va;
                Bs[k][i] = vb;
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < DK; ++k) {
                const double2 y = Bs[k][tx];
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[j], As[k][ty + 8 * j], y);
            }
            __syncthreads();
        }
    }
    double2* R = (up ? rho_u : rho_d) + (size_t)a * n * n;
    const int col = b0 + tx;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int row = a0 + ty + 8 * j;
        if (row >= n || col >= n) continue;
        double2& r = R[(size_t)row * n + col];
        r = cadd(r, acc[j]);
        if (!up && ti != tj) {
            double2& q = R[(size_t)col * n + row];
            q = cadd(q, cconj(acc[j]));
        }
    }
}

// ---------------------------------------------------------------- basis on the grid
// Phi[(q * nxe + j) * n + alpha] = phi_alpha(x_j, s_q), x_j = j Lx/nx, s_q = (q + 1/2) L/nz,
// phi_alpha = sum_G C_{G alpha} e^{i (G_x x + (G_z + k_alpha) s)} (Eq. wavef_expansion with the
// left node's phase).
struct GridGroup {
    int ng;
    const int* mx;
    const int* mz;
    const double2* C;   // ng x nb row-major
    double k;
};

__global__ void k_basis_grid(int nb, int nxe, int nz, double dx, double ds, double bx, double bz, GridGroup g0, GridGroup g1,
                             double2* __restrict__ Phi) {
    const int n = 2 * nb;
    const size_t total = (size_t)nz * nxe * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int alpha = (int)(t % n);
        const size_t p = t / n;
        const int j = (int)(p % nxe), q = (int)(p / nxe);
        const GridGroup& g = alpha < nb ? g0 : g1;
        const int col = alpha < nb ? alpha : alpha - nb;
        const double x = j * dx, s = (q + 0.5) * ds;
        double2 acc = make_double2(0, 0);
        for (int G = 0; G < g.ng; ++G) {
            double sn, cs;
            sincos(g.mx[G] * bx * x + (g.mz[G] * bz + g.k) * s, &sn, &cs);
            cfma(acc, g.C[(size_t)G * nb + col], make_double2(cs, sn));
        }
        Phi[t] = acc;
    }
}

// ---------------------------------------------------------------- n(r) per element
constexpr int QG = 4;    // z-planes per CTA
constexpr int XT = 32;   // x points per CTA
constexpr int GT = 32;   // basis chunk

struct GridArgs {
    int n, N, nxe, nz;
    double L;
    const double2* rho_d;
    const double2* rho_u;
    const double2* Phi;   // nz x nxe x n
    const double2* ph;    // n: e^{-i k_alpha L}
    double* out;          // (N-1) x nxe x nz
};

__global__ void __launch_bounds__(256) k_density_grid(GridArgs A) {
    extern __shared__ double2 sm[];
    double2* Ad = sm;                          // [GT][GT+1]  rho_d[e]
    double2* Bd = Ad + GT * (GT + 1);          // [GT][GT+1]  phase-rotated rho_d[e+1]
    double2* Cd = Bd + GT * (GT + 1);          // [GT][GT+1]  Hermitian part of rho_u[e] phi_r
    double2* Ps = Cd + GT * (GT + 1);          // [QG][XT][GT+1] basis values
    double* dsum = reinterpret_cast<double*>(Ps + QG * XT * (GT + 1));   // [QG][XT]
    const int e = blockIdx.x, q0 = blockIdx.y * QG, x0 = blockIdx.z * XT;
    const int n = A.n, t = threadIdx.x, ar = t / 8, xg = t % 8;
    const double2* Rd0 = A.rho_d + (size_t)e * n * n;
    const double2* Rd1 = A.rho_d + (size_t)(e + 1) * n * n;
    const double2* Ru = A.rho_u + (size_t)e * n * n;
    double fl[QG], fr[QG];
#pragma unroll
    for (int q = 0; q < QG; ++q) {
        const double s = (q0 + q + 0.5) / A.nz;
        fl[q] = 1.0 - s;
        fr[q] = s;
    }
    for (int i = t; i < QG * XT; i += 256) dsum[i] = 0.0;
    for (int ac = 0; ac < n; ac += GT) {
        double2 acc[QG][4];
#pragma unroll
        for (int q = 0; q < QG; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q][u] = make_double2(0, 0);
        for (int bc = 0; bc < n; bc += GT) {
            for (int i = t; i < GT * GT; i += 256) {
                const int r = i / GT, k = i % GT, ga = ac + r, gb = bc + k;
                double2 va = make_double2(0, 0), vb = va, vc = va;
                if (ga < n && gb < n) {
                    const size_t ab = (size_t)ga * n + gb, ba = (size_t)gb * n + ga;
                    const double2 pa = A.ph[ga], pb = A.ph[gb];
                    va = Rd0[ab];
                    vb = cmul(cmul(cconj(pa), Rd1[ab]), pb);
                    vc = cadd(cmul(Ru[ab], pb), cconj(cmul(Ru[ba], pa)));
                }
                Ad[r * (GT + 1) + k] = va;
                Bd[r * (GT + 1) + k] = vb;
                Cd[r * (GT + 1) + k] = vc;
            }
            for (int i = t; i < QG * XT * GT; i += 256) {
                const int k = i % GT, x = (i / GT) % XT, q = i / (GT * XT);
                const int gq = q0 + q, gx = x0 + x, gb = bc + k;
                double2 v = make_double2(0, 0);
                if (gq < A.nz && gx < A.nxe && gb < n) v = A.Phi[((size_t)gq * A.nxe + gx) * n + gb];
                Ps[(q * XT + x) * (GT + 1) + k] = v;
            }
            __syncthreads();
            for (int k = 0; k < GT; ++k) {
                const double2 va = Ad[ar * (GT + 1) + k], vb = Bd[ar * (GT + 1) + k], vc = Cd[ar * (GT + 1) + k];
#pragma unroll
                for (int q = 0; q < QG; ++q) {
                    const double wl = fl[q] * fl[q], wr = fr[q] * fr[q], wc = fl[q] * fr[q];
                    const double2 G = make_double2(wl * va.x + wr * vb.x + wc * vc.x, wl * va.y + wr * vb.y + wc * vc.y);
#pragma unroll
                    for (int u = 0; u < 4; ++u) cfma(acc[q][u], G, Ps[(q * XT + xg + 8 * u) * (GT + 1) + k]);
                }
            }
            __syncthreads();
        }
        // n += Re(conj(phi_a) (G phi)_a) over this chunk of rows a
        for (int i = t; i < QG * XT * GT; i += 256) {
            const int k = i % GT, x = (i / GT) % XT, q = i / (GT * XT);
            const int gq = q0 + q, gx = x0 + x, ga = ac + k;
            double2 v = make_double2(0, 0);
            if (gq < A.nz && gx < A.nxe && ga < n) v = A.Phi[((size_t)gq * A.nxe + gx) * n + ga];
            Ps[(q * XT + x) * (GT + 1) + k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < QG; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double2 p = Ps[(q * XT + xg + 8 * u) * (GT + 1) + ar];
                atomicAdd(&dsum[q * XT + xg + 8 * u], p.x * acc[q][u].x + p.y * acc[q][u].y);
            }
        __syncthreads();
    }
    for (int i = t; i < QG * XT; i += 256) {
        const int q = i / XT, x = i % XT, gq = q0 + q, gx = x0 + x;
        if (gq < A.nz && gx < A.nxe) A.out[((size_t)e * A.nxe + gx) * A.nz + gq] = dsum[i];
    }
}

__global__ void k_phases(int nb, double L, double kz1, double2* ph) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= 2 * nb) return;
    const double k = a < nb ? 0.0 : kz1;
    double sn, cs;
    sincos(-k * L, &sn, &cs);
    ph[a] = make_double2(cs, sn);
}

double fermi(double x, double kT) {
    if (kT <= 0) return x < 0 ? 1.0 : (x == 0 ? 0.5 : 0.0);
    return 0.5 * (1.0 - std::tanh(0.5 * x / kT));
}

}  // namespace

int density_alloc(pwqt_ctx* c, System& s) {
    const size_t nn = (size_t)c->n * c->n;
    if (!s.rho_d.p) PWQT_TRY(alloc(c, s.rho_d, sizeof(double2) * nn * s.N));
    if (!s.rho_u.p) PWQT_TRY(alloc(c, s.rho_u, sizeof(double2) * nn * std::max(s.N - 1, 1)));
    return PWQT_OK;
}

int density_reset(pwqt_ctx* c, System& s, cudaStream_t st) {
    PWQT_TRY(density_alloc(c, s));
    PWQT_CUDA(c, cudaMemsetAsync(s.rho_d.p, 0, s.rho_d.bytes, st));
    PWQT_CUDA(c, cudaMemsetAsync(s.rho_u.p, 0, s.rho_u.bytes, st));
    s.rho_energies = 0;
    return PWQT_OK;
}

int density_accumulate_batch(pwqt_ctx* c, System& s, const std::vector<ObsJob>& obs, const double* E, const DensityAcc& d, int nb,
                             cudaStream_t st) {
    PWQT_TRY(density_alloc(c, s));
    std::vector<DensJob> jobs(nb);
    for (int b = 0; b < nb; ++b) {
        const ObsJob& O = obs[b];
        DensJob& J = jobs[b];
        J.C = O.C;
        J.node_stride = O.node_stride;
        J.row_stride = O.row_stride;
        J.ms = O.C ? O.ms : 0;
        J.md = O.C ? O.md : 0;
        J.v_in_s = O.v_in_s;
        J.v_in_d = O.v_in_d;
        if (!O.v_in_s) J.ms = 0;
        if (!O.v_in_d) J.md = 0;
        J.scale_s = d.w[b] * fermi(E[b] - d.mu_s, d.kT);
        J.scale_d = d.w[b] * fermi(E[b] - d.mu_d, d.kT);
    }
    PWQT_TRY(ensure(c, c->ws_dens, sizeof(DensJob) * nb));
    PWQT_CUDA(c, cudaMemcpyAsync(c->ws_dens.p, jobs.data(), sizeof(DensJob) * nb, cudaMemcpyHostToDevice, st));
    const int n = c->n, N = s.N, tiles = (n + DT - 1) / DT;
    dim3 grid(tiles * tiles, N, N > 1 ? 2 : 1);
    k_density_accum<<<grid, 256, 0, st>>>(c->ws_dens.as<DensJob>(), nb, n, N, tiles, s.rho_d.as<double2>(), s.rho_u.as<double2>());
    c->launches++;
    PWQT_CUDA(c, cudaGetLastError());
    // the job table is overwritten by the next batch: finish this one first
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    s.rho_energies += nb;
    return PWQT_OK;
}

int density_grid(pwqt_ctx* c, System& s, int nx, int nz, double* out_dev, cudaStream_t st) {
    const int n = c->n, nb = c->n_bands, N = s.N;
    const int nxe = c->dim == 2 ? nx : 1;
    const size_t P = (size_t)nz * nxe;
    DBuf Phi, ph;
    PWQT_TRY(alloc(c, Phi, sizeof(double2) * P * n));
    PWQT_TRY(alloc(c, ph, sizeof(double2) * n));
    const double bz = 2.0 * M_PI / c->Lz, bx = c->dim == 2 ? 2.0 * M_PI / c->Lx : 0.0;
    const double dx = c->dim == 2 ? c->Lx / nx : 0.0, ds = c->Lz / nz;
    GridGroup g0{c->pw_n[0], c->pw_mx[0].as<int>(), c->pw_mz[0].as<int>(), c->pw_C[0].as<double2>(), 0.0};
    GridGroup g1{c->pw_n[1], c->pw_mx[1].as<int>(), c->pw_mz[1].as<int>(), c->pw_C[1].as<double2>(), M_PI / c->Lz};
    const int blocks = (int)std::min<size_t>((P * n + 255) / 256, 8192);
    k_basis_grid<<<blocks, 256, 0, st>>>(nb, nxe, nz, dx, ds, bx, bz, g0, g1, Phi.as<double2>());
    k_phases<<<(n + 127) / 128, 128, 0, st>>>(nb, c->Lz, M_PI / c->Lz, ph.as<double2>());
    c->launches += 2;
    if (N >= 2) {
        const size_t smem = sizeof(double2) * (3 * GT * (GT + 1) + QG * XT * (GT + 1)) + sizeof(double) * QG * XT;
        PWQT_CUDA(c, cudaFuncSetAttribute(k_density_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GridArgs A{n, N, nxe, nz, c->Lz, s.rho_d.as<double2>(), s.rho_u.as<double2>(), Phi.as<double2>(), ph.as<double2>(), out_dev};
        dim3 grid(N - 1, (nz + QG - 1) / QG, (nxe + XT - 1) / XT);
        k_density_grid<<<grid, 256, smem, st>>>(A);
        c->launches++;
    }
    PWQT_CUDA(c, cudaGetLastError());
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    return PWQT_OK;
}

}  // namespace pwqt
