// extern "C" entry points of libpwqt (declared and documented in include/pwqt.h).
#include <cmath>
#include <cstring>

#include "pwqt_internal.cuh"

using namespace pwqt;

namespace {
int check_ctx(pwqt_ctx* c) { return c ? PWQT_OK : PWQT_ERR_INVALID_ARG; }

// H(k') and M(k') (column-major) for the band reconstruction of Sec. 5.1.
__global__ void k_bands_hk(int n, double2 ph, const double2* H0, const double2* H1, const double2* M0, const double2* M1,
                           double2* Hk, double2* Mk) {
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= n) return;
    size_t rm = (size_t)r * n + c, tm = (size_t)c * n + r;
    double2 iph = cconj(ph);
    Hk[(size_t)c * n + r] = cadd(H0[rm], cadd(cmul(H1[rm], ph), cmul(cconj(H1[tm]), iph)));
    Mk[(size_t)c * n + r] = cadd(M0[rm], cadd(cmul(M1[rm], ph), cmul(cconj(M1[tm]), iph)));
}

int check_solve_args(pwqt_ctx* c, int n_E, const double* E, int precision) {
    if (precision != PWQT_FP64 && precision != PWQT_MIXED && precision != PWQT_FP32)
        return fail(c, PWQT_ERR_INVALID_ARG, "bad precision");
    if (n_E < 0 || (n_E > 0 && !E)) return fail(c, PWQT_ERR_INVALID_ARG, "bad energies");
    if (c->n > 1024) return fail(c, PWQT_ERR_INVALID_ARG, "block size above 1024");
    for (int e = 0; e < n_E; ++e)
        if (!std::isfinite(E[e])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite energy");
    return PWQT_OK;
}

// host output buffers of a solve (any may be NULL)
struct HostOut {
    double *T, *R, *T_ds;
    int* n_open;
    double *node_n, *resid;
    int *iters, *status;
};

// device outputs for n_E results of N nodes, the solve `run` into them, copies to h
template <class F>
int solve_to_host(pwqt_ctx* c, int n_E, int N, const HostOut& h, F run) {
    DBuf dT, dR, dTds, dno, dnn, dres, dit, dst;
    size_t ne = (size_t)std::max(n_E, 1);
    PWQT_TRY(alloc(c, dT, sizeof(double) * ne));
    PWQT_TRY(alloc(c, dR, sizeof(double) * ne));
    PWQT_TRY(alloc(c, dTds, sizeof(double) * ne));
    PWQT_TRY(alloc(c, dno, sizeof(int) * 2 * ne));
    PWQT_TRY(alloc(c, dnn, sizeof(double) * 2 * ne * std::max(N, 1)));
    PWQT_TRY(alloc(c, dres, sizeof(double) * ne));
    PWQT_TRY(alloc(c, dit, sizeof(int) * ne));
    PWQT_TRY(alloc(c, dst, sizeof(int) * ne));
    SolveOut o{dT.as<double>(), dR.as<double>(), dTds.as<double>(), dnn.as<double>(), dres.as<double>(),
               dno.as<int>(), dit.as<int>(), dst.as<int>()};
    PWQT_TRY(run(o));
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h.T) PWQT_CUDA(c, copy_sync(c, h.T, dT.p, sizeof(double) * n_E, cudaMemcpyDeviceToHost));
    if (h.R) PWQT_CUDA(c, copy_sync(c, h.R, dR.p, sizeof(double) * n_E, cudaMemcpyDeviceToHost));
    if (h.T_ds) PWQT_CUDA(c, copy_sync(c, h.T_ds, dTds.p, sizeof(double) * n_E, cudaMemcpyDeviceToHost));
    if (h.n_open) PWQT_CUDA(c, copy_sync(c, h.n_open, dno.p, sizeof(int) * 2 * n_E, cudaMemcpyDeviceToHost));
    if (h.node_n) PWQT_CUDA(c, copy_sync(c, h.node_n, dnn.p, sizeof(double) * 2 * n_E * N, cudaMemcpyDeviceToHost));
    if (h.resid) PWQT_CUDA(c, copy_sync(c, h.resid, dres.p, sizeof(double) * n_E, cudaMemcpyDeviceToHost));
    if (h.iters) PWQT_CUDA(c, copy_sync(c, h.iters, dit.p, sizeof(int) * n_E, cudaMemcpyDeviceToHost));
    if (h.status) PWQT_CUDA(c, copy_sync(c, h.status, dst.p, sizeof(int) * n_E, cudaMemcpyDeviceToHost));
    return PWQT_OK;
}

int solve_common(pwqt_ctx* c, int sys, int n_E, const double* E, int precision, SolveOut& dev, cudaStream_t st,
                 const DensityAcc* dens = nullptr) {
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis: call pwqt_assemble_intrinsic first");
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    PWQT_TRY(check_solve_args(c, n_E, E, precision));
    return solve_batch(c, it->second, n_E, E, precision, dev, st, dens);
}
}  // namespace

extern "C" {

int pwqt_create(pwqt_ctx** out, const pwqt_opts* opts) {
    if (!out) return PWQT_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { cudaGetLastError(); return PWQT_ERR_NO_DEVICE; }
    auto* c = new pwqt_ctx();
    if (opts) c->opts = *opts;
    if (c->opts.ir_tol <= 0) c->opts.ir_tol = 1e-10;
    if (c->opts.ir_max_iters <= 0) c->opts.ir_max_iters = 40;
    c->dev = c->opts.device;
    if (c->dev < 0 || c->dev >= ndev) { delete c; return PWQT_ERR_INVALID_ARG; }
    if (cudaSetDevice(c->dev) != cudaSuccess) { delete c; return PWQT_ERR_CUDA; }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&c->sol) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnCreateParams(&c->prm) != CUSOLVER_STATUS_SUCCESS) {
        pwqt_destroy(c);
        return PWQT_ERR_CUDA;
    }
    cublasSetStream(c->blas, c->stream);
    cusolverDnSetStream(c->sol, c->stream);
    *out = c;
    return PWQT_OK;
}

int pwqt_destroy(pwqt_ctx* c) {
    if (!c) return PWQT_OK;
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->cache.clear();
    c->systems.clear();
    for (auto& w : c->workers) w->destroy();
    c->workers.clear();
    if (c->prm) cusolverDnDestroyParams(c->prm);
    if (c->sol) cusolverDnDestroy(c->sol);
    if (c->blas) cublasDestroy(c->blas);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev2) cudaEventDestroy(c->ev2);
    if (c->ev3) cudaEventDestroy(c->ev3);
    for (auto& l : c->lanes) l.destroy();
    delete c;
    return PWQT_OK;
}

const char* pwqt_last_error(const pwqt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pwqt_assemble_intrinsic(pwqt_ctx* c, const pwqt_cell* cell, const pwqt_formfactor* ff, double gcut, int n_bands,
                            int* n_out) {
    PWQT_TRY(check_ctx(c));
    if (!cell || !ff || !cell->atoms || cell->n_atoms <= 0 || n_bands <= 0 || gcut <= 0 || cell->Lz <= 0 || cell->Lx <= 0 ||
        (cell->dim != 1 && cell->dim != 2))
        return fail(c, PWQT_ERR_INVALID_ARG, "invalid cell / form factor / cutoff");
    if (2 * n_bands > 1024) return fail(c, PWQT_ERR_INVALID_ARG, "block size 2*n_bands above 1024");
    cudaSetDevice(c->dev);
    PWQT_TRY(epm_basis(c, cell, ff, gcut, n_bands));
    if (n_out) *n_out = c->n;
    return PWQT_OK;
}

int pwqt_set_enhancement(pwqt_ctx* c, const pwqt_cell* cell, int n_bands, const double* eps, const int* n_pw,
                         const int* mx, const int* mz, const double* coef, int* n_out) {
    PWQT_TRY(check_ctx(c));
    if (!cell || !eps || !n_pw || !mx || !mz || !coef || n_bands <= 0 || n_pw[0] < n_bands || n_pw[1] < n_bands ||
        2 * n_bands > 1024 || cell->Lz <= 0 || cell->Lx <= 0)
        return fail(c, PWQT_ERR_INVALID_ARG, "invalid enhancement-function input");
    cudaSetDevice(c->dev);
    size_t rows = (size_t)n_pw[0] + n_pw[1];
    DBuf d;
    PWQT_TRY(alloc(c, d, sizeof(double2) * rows * n_bands));
    PWQT_CUDA(c, copy_sync(c, d.p, coef, sizeof(double2) * rows * n_bands, cudaMemcpyHostToDevice));
    PWQT_TRY(assemble_from_basis(c, cell, n_bands, eps, n_pw, mx, mz, d.as<double2>()));
    if (n_out) *n_out = c->n;
    return PWQT_OK;
}

int pwqt_get_blocks(pwqt_ctx* c, double* H0, double* H1, double* M0, double* M1, double* W) {
    PWQT_TRY(check_ctx(c));
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis");
    size_t nn = (size_t)c->n * c->n * sizeof(double2);
    if (H0) PWQT_CUDA(c, copy_sync(c, H0, c->H0.p, nn, cudaMemcpyDeviceToHost));
    if (H1) PWQT_CUDA(c, copy_sync(c, H1, c->H1.p, nn, cudaMemcpyDeviceToHost));
    if (M0) PWQT_CUDA(c, copy_sync(c, M0, c->M0.p, nn, cudaMemcpyDeviceToHost));
    if (M1) PWQT_CUDA(c, copy_sync(c, M1, c->M1.p, nn, cudaMemcpyDeviceToHost));
    if (W) PWQT_CUDA(c, copy_sync(c, W, c->W.p, 6 * nn, cudaMemcpyDeviceToHost));
    return PWQT_OK;
}

int pwqt_set_extrinsic(pwqt_ctx* c, int sys, int n_nodes, const double* U) {
    PWQT_TRY(check_ctx(c));
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis");
    if (sys < 0 || sys >= 64 || n_nodes < 2 || !U) return fail(c, PWQT_ERR_INVALID_ARG, "invalid system / nodes / potential");
    for (int i = 0; i < n_nodes; ++i)
        if (!std::isfinite(U[i])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite potential");
    cudaSetDevice(c->dev);
    System& s = c->systems[sys];
    s.N = n_nodes;
    s.U.assign(U, U + n_nodes);
    s.Us = U[0];
    s.Ud = U[n_nodes - 1];
    s.rho_d.release();   // a new potential starts a new density
    s.rho_u.release();
    s.rho_energies = 0;
    int r = build_system_blocks(c, s);
    if (r != PWQT_OK) c->systems.erase(sys);
    return r;
}

int pwqt_solve(pwqt_ctx* c, int sys, int n_E, const double* E, int precision, double* T, double* R, double* T_ds,
               int* n_open, double* node_n, double* resid, int* iters, int* status) {
    PWQT_TRY(check_ctx(c));
    cudaSetDevice(c->dev);
    auto it = c->systems.find(sys);
    int N = it == c->systems.end() ? 0 : it->second.N;
    if (n_E == 0) return PWQT_OK;
    HostOut h{T, R, T_ds, n_open, node_n, resid, iters, status};
    return solve_to_host(c, n_E, N, h, [&](SolveOut& o) { return solve_common(c, sys, n_E, E, precision, o, c->stream); });
}
int pwqt_solve_dev(pwqt_ctx* c, int sys, int n_E, const double* E, int precision, double* T, double* R, double* T_ds,
                   int* n_open, double* node_n, double* resid, int* iters, int* status, void* stream) {
    PWQT_TRY(check_ctx(c));
    cudaSetDevice(c->dev);
    auto it = c->systems.find(sys);
    int N = it == c->systems.end() ? 0 : it->second.N;
    if (n_E == 0) return PWQT_OK;
    // outputs the caller did not ask for go to context scratch
    size_t ne = (size_t)n_E;
    size_t need = sizeof(double) * ne * (4 + 2 * std::max(N, 1)) + sizeof(int) * ne * 4 + 1024;
    if (c->work_a.bytes < need) PWQT_TRY(alloc(c, c->work_a, need));
    char* w = c->work_a.as<char>();
    auto take = [&](size_t b) { char* p = w; w += (b + 255) / 256 * 256; return p; };
    SolveOut o;
    o.T = T ? T : (double*)take(sizeof(double) * ne);
    o.R = R ? R : (double*)take(sizeof(double) * ne);
    o.T_ds = T_ds ? T_ds : (double*)take(sizeof(double) * ne);
    o.resid = resid ? resid : (double*)take(sizeof(double) * ne);
    o.node_n = node_n ? node_n : (double*)take(sizeof(double) * ne * 2 * std::max(N, 1));
    o.n_open = n_open ? n_open : (int*)take(sizeof(int) * ne * 2);
    o.iters = iters ? iters : (int*)take(sizeof(int) * ne);
    o.status = status ? status : (int*)take(sizeof(int) * ne);
    cudaStream_t st = stream ? (cudaStream_t)stream : (cudaStream_t)0;
    return solve_common(c, sys, n_E, E, precision, o, st);
}

int pwqt_prepare_leads(pwqt_ctx* c, int sys, int n_E, const double* E) {
    PWQT_TRY(check_ctx(c));
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system");
    if (n_E < 0 || (n_E && !E)) return fail(c, PWQT_ERR_INVALID_ARG, "bad energies");
    cudaSetDevice(c->dev);
    std::vector<double> keys;
    for (int e = 0; e < n_E; ++e) { keys.push_back(E[e] - it->second.Us); keys.push_back(E[e] - it->second.Ud); }
    return fill_leads(c, keys);
}

int pwqt_cache_info(pwqt_ctx* c, int* entries, size_t* bytes) {
    PWQT_TRY(check_ctx(c));
    size_t b = 0;
    for (auto& kv : c->cache) b += kv.second->bytes();
    if (entries) *entries = (int)c->cache.size();
    if (bytes) *bytes = b;
    return PWQT_OK;
}

int pwqt_bands(pwqt_ctx* c, int n_k, const double* k, double* E_out) {
    PWQT_TRY(check_ctx(c));
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis");
    if (n_k < 0 || (n_k && (!k || !E_out))) return fail(c, PWQT_ERR_INVALID_ARG, "bad k list");
    cudaSetDevice(c->dev);
    int n = c->n;
    DBuf Hk, Mk, W, info, work;
    PWQT_TRY(alloc(c, Hk, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, Mk, sizeof(double2) * n * n));
    PWQT_TRY(alloc(c, W, sizeof(double) * n));
    PWQT_TRY(alloc(c, info, sizeof(int)));
    int lwork = 0;
    PWQT_SOLVER(c, cusolverDnZhegvd_bufferSize(c->sol, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                               Hk.as<cuDoubleComplex>(), n, Mk.as<cuDoubleComplex>(), n, W.as<double>(), &lwork));
    PWQT_TRY(alloc(c, work, sizeof(cuDoubleComplex) * std::max(lwork, 1)));
    for (int q = 0; q < n_k; ++q) {
        double2 ph = make_double2(std::cos(k[q] * c->Lz), std::sin(k[q] * c->Lz));
        k_bands_hk<<<dim3((n + 127) / 128, n), 128, 0, c->stream>>>(n, ph, c->H0.as<double2>(), c->H1.as<double2>(),
                                                                 c->M0.as<double2>(), c->M1.as<double2>(), Hk.as<double2>(),
                                                                 Mk.as<double2>());
        c->launches++;
        PWQT_SOLVER(c, cusolverDnZhegvd(c->sol, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                        Hk.as<cuDoubleComplex>(), n, Mk.as<cuDoubleComplex>(), n, W.as<double>(),
                                        work.as<cuDoubleComplex>(), lwork, info.as<int>()));
        PWQT_CUDA(c, cudaMemcpyAsync(E_out + (size_t)q * n, W.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    }
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    return PWQT_OK;
}

int pwqt_profile(pwqt_ctx* c, int enable, double* sweep_ms, long long* sweep_launches, double* sweep_flops, int reset) {
    PWQT_TRY(check_ctx(c));
    cudaSetDevice(c->dev);
    if (enable && !c->ev0) {
        PWQT_CUDA(c, cudaEventCreate(&c->ev0));
        PWQT_CUDA(c, cudaEventCreate(&c->ev1));
        PWQT_CUDA(c, cudaEventCreate(&c->ev2));
        PWQT_CUDA(c, cudaEventCreate(&c->ev3));
    }
    c->profile = enable;
    if (sweep_ms) *sweep_ms = c->prof_ms;
    if (sweep_launches) *sweep_launches = c->prof_launches;
    if (sweep_flops) *sweep_flops = c->prof_flops;
    if (reset) {
        c->prof_ms = 0; c->prof_launches = 0; c->prof_flops = 0;
        c->prof_phase_ms[0] = c->prof_phase_ms[1] = 0; c->prof_ir_iters = 0;
        c->prof_oz_ms = c->prof_oz_cmacs = c->prof_oz_mma_flops = 0; c->prof_oz_launches = 0;
        c->prof_corr_cmacs = 0; c->prof_corr_launches = 0;
    }
    return PWQT_OK;
}

int pwqt_kernel_launches(pwqt_ctx* c, long long* count, int reset) {
    PWQT_TRY(check_ctx(c));
    if (count) *count = c->launches;
    if (reset) c->launches = 0;
    return PWQT_OK;
}


int pwqt_density_reset(pwqt_ctx* c, int sys) {
    PWQT_TRY(check_ctx(c));
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    cudaSetDevice(c->dev);
    PWQT_TRY(density_reset(c, it->second, c->stream));
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    return PWQT_OK;
}

int pwqt_accumulate_density(pwqt_ctx* c, int sys, int n_E, const double* E, const double* w, double mu_s, double mu_d, double kT,
                            int precision, int* status) {
    PWQT_TRY(check_ctx(c));
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (n_E < 0 || (n_E > 0 && (!E || !w))) return fail(c, PWQT_ERR_INVALID_ARG, "energies and weights are required");
    if (!std::isfinite(mu_s) || !std::isfinite(mu_d) || !std::isfinite(kT) || kT < 0)
        return fail(c, PWQT_ERR_INVALID_ARG, "mu_s, mu_d must be finite and kT >= 0");
    for (int e = 0; e < n_E; ++e)
        if (!std::isfinite(w[e])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite weight");
    cudaSetDevice(c->dev);
    System& s = it->second;
    if (!s.rho_d.p) PWQT_TRY(density_reset(c, s, c->stream));
    if (n_E == 0) return PWQT_OK;
    const int N = s.N;
    const size_t ne = (size_t)n_E;
    DBuf out;
    PWQT_TRY(alloc(c, out, sizeof(double) * ne * (4 + 2 * (size_t)N) + sizeof(int) * ne * 4 + 2048));
    char* p = out.as<char>();
    auto take = [&](size_t b) { char* q = p; p += (b + 255) / 256 * 256; return q; };
    SolveOut o;
    o.T = (double*)take(sizeof(double) * ne);
    o.R = (double*)take(sizeof(double) * ne);
    o.T_ds = (double*)take(sizeof(double) * ne);
    o.resid = (double*)take(sizeof(double) * ne);
    o.node_n = (double*)take(sizeof(double) * ne * 2 * N);
    o.n_open = (int*)take(sizeof(int) * ne * 2);
    o.iters = (int*)take(sizeof(int) * ne);
    o.status = (int*)take(sizeof(int) * ne);
    DensityAcc d{w, mu_s, mu_d, kT};
    PWQT_TRY(solve_common(c, sys, n_E, E, precision, o, c->stream, &d));
    PWQT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (status) PWQT_CUDA(c, copy_sync(c, status, o.status, sizeof(int) * ne, cudaMemcpyDeviceToHost));
    return PWQT_OK;
}

int pwqt_get_density_matrix(pwqt_ctx* c, int sys, double* rho_d, double* rho_u) {
    PWQT_TRY(check_ctx(c));
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    System& s = it->second;
    if (!s.rho_d.p) return fail(c, PWQT_ERR_STATE, "no density accumulated: call pwqt_accumulate_density first");
    cudaSetDevice(c->dev);
    const size_t nn = (size_t)c->n * c->n;
    if (rho_d) PWQT_CUDA(c, copy_sync(c, rho_d, s.rho_d.p, sizeof(double2) * nn * s.N, cudaMemcpyDeviceToHost));
    if (rho_u && s.N > 1) PWQT_CUDA(c, copy_sync(c, rho_u, s.rho_u.p, sizeof(double2) * nn * (s.N - 1), cudaMemcpyDeviceToHost));
    return PWQT_OK;
}

int pwqt_density_grid(pwqt_ctx* c, int sys, int nx, int nz, double* n_r) {
    PWQT_TRY(check_ctx(c));
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    System& s = it->second;
    if (!s.rho_d.p) return fail(c, PWQT_ERR_STATE, "no density accumulated: call pwqt_accumulate_density first");
    if (nx < 1 || nz < 1 || nx > 4096 || nz > 4096 || !n_r) return fail(c, PWQT_ERR_INVALID_ARG, "1 <= nx, nz <= 4096 and n_r required");
    cudaSetDevice(c->dev);
    const int nxe = c->dim == 2 ? nx : 1;
    const size_t count = (size_t)std::max(s.N - 1, 0) * nxe * nz;
    if (count == 0) return PWQT_OK;
    DBuf out;
    PWQT_TRY(alloc(c, out, sizeof(double) * count));
    PWQT_TRY(density_grid(c, s, nx, nz, out.as<double>(), c->stream));
    PWQT_CUDA(c, copy_sync(c, n_r, out.p, sizeof(double) * count, cudaMemcpyDeviceToHost));
    return PWQT_OK;
}


int pwqt_profile_refinement(pwqt_ctx* c, double* residual_ms, double* correction_ms, long long* iterations) {
    PWQT_TRY(check_ctx(c));
    if (residual_ms) *residual_ms = c->prof_phase_ms[0];
    if (correction_ms) *correction_ms = c->prof_phase_ms[1];
    if (iterations) *iterations = c->prof_ir_iters;
    return PWQT_OK;
}


int pwqt_set_refinement(pwqt_ctx* c, double ir_tol, int ir_max_iters) {
    PWQT_TRY(check_ctx(c));
    if (!(ir_tol >= 0) || !std::isfinite(ir_tol) || ir_max_iters < 0)
        return fail(c, PWQT_ERR_INVALID_ARG, "ir_tol must be finite and >= 0, ir_max_iters >= 0");
    c->opts.ir_tol = ir_tol > 0 ? ir_tol : 1e-10;
    c->opts.ir_max_iters = ir_max_iters > 0 ? ir_max_iters : 40;
    return PWQT_OK;
}

int pwqt_profile_residual(pwqt_ctx* c, double* ms, double* cmacs, double* mma_flops, long long* launches) {
    PWQT_TRY(check_ctx(c));
    if (ms) *ms = c->prof_oz_ms;
    if (cmacs) *cmacs = c->prof_oz_cmacs;
    if (mma_flops) *mma_flops = c->prof_oz_mma_flops;
    if (launches) *launches = c->prof_oz_launches;
    return PWQT_OK;
}

int pwqt_profile_correction(pwqt_ctx* c, double* ms, double* cmacs, long long* launches) {
    PWQT_TRY(check_ctx(c));
    if (ms) *ms = c->prof_phase_ms[1];
    if (cmacs) *cmacs = c->prof_corr_cmacs;
    if (launches) *launches = c->prof_corr_launches;
    return PWQT_OK;
}

int pwqt_set_residual(pwqt_ctx* c, int kind) {
    PWQT_TRY(check_ctx(c));
    if (kind != PWQT_RESIDUAL_SLICED && kind != PWQT_RESIDUAL_FLOAT_FLOAT)
        return fail(c, PWQT_ERR_INVALID_ARG, "residual kind must be PWQT_RESIDUAL_SLICED or PWQT_RESIDUAL_FLOAT_FLOAT");
    c->residual_kind = kind;
    return PWQT_OK;
}


int pwqt_solve_multi(pwqt_ctx* c, int n_sys, const int* sys_ids, int n_E, const double* E, int precision, double* T, double* R,
                     double* T_ds, int* n_open, double* node_n, double* resid, int* iters, int* status) {
    PWQT_TRY(check_ctx(c));
    if (n_sys < 0 || (n_sys > 0 && !sys_ids)) return fail(c, PWQT_ERR_INVALID_ARG, "bad system list");
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis: call pwqt_assemble_intrinsic first");
    cudaSetDevice(c->dev);
    std::vector<System*> sysq(n_sys);
    bool same_N = true;
    for (int q = 0; q < n_sys; ++q) {
        auto it = c->systems.find(sys_ids[q]);
        if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system in the list");
        sysq[q] = &it->second;
        same_N = same_N && sysq[q]->N == sysq[0]->N;
    }
    if (n_sys == 0 || n_E == 0) return PWQT_OK;
    PWQT_TRY(check_solve_args(c, n_E, E, precision));
    if (same_N && (precision == PWQT_FP64 || c->residual_kind == PWQT_RESIDUAL_SLICED)) {
        // every (system, energy) pair in one batched solve, system-major: the bias points
        // of a device share the launches (each job carries its own system's blocks)
        const int tot = n_sys * n_E;
        std::vector<double> Eall(tot);
        std::vector<System*> of(tot);
        for (int q = 0; q < n_sys; ++q)
            for (int e = 0; e < n_E; ++e) { Eall[(size_t)q * n_E + e] = E[e]; of[(size_t)q * n_E + e] = sysq[q]; }
        HostOut h{T, R, T_ds, n_open, node_n, resid, iters, status};
        return solve_to_host(c, tot, sysq[0]->N, h, [&](SolveOut& o) {
            return solve_batch(c, *sysq[0], tot, Eall.data(), precision, o, c->stream, nullptr, of.data());
        });
    }
    size_t nn_off = 0;
    for (int q = 0; q < n_sys; ++q) {
        const size_t o = (size_t)q * n_E;
        PWQT_TRY(pwqt_solve(c, sys_ids[q], n_E, E, precision, T ? T + o : nullptr, R ? R + o : nullptr, T_ds ? T_ds + o : nullptr,
                            n_open ? n_open + 2 * o : nullptr, node_n ? node_n + nn_off : nullptr, resid ? resid + o : nullptr,
                            iters ? iters + o : nullptr, status ? status + o : nullptr));
        nn_off += (size_t)n_E * sysq[q]->N * 2;
    }
    return PWQT_OK;
}

}  // extern "C"
