// Internal declarations shared by the libpwqt translation units.
#pragma once
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pwqt.h"

namespace pwqt {

constexpr double HB2M = 0.0380998212;   // hbar^2 / 2 m_e  (eV nm^2)

// ---------------------------------------------------------------- complex math
struct cplx { double x, y; };
__host__ __device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a += b * c
__host__ __device__ inline void cfma(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
// a += conj(b) * c
__host__ __device__ inline void cfma_cj(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, fma(b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(-b.y, c.x, a.y));
}
__host__ __device__ inline double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ inline double cnorm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}

// ---------------------------------------------------------------- device buffer
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DBuf& operator=(DBuf&& o) noexcept { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; return *this; }
    ~DBuf() { release(); }
    void release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------- cached contact data
// One entry per lead energy Ec = E - U_lead: drain-side and source-side data of the
// same complex band structure (lambda_s = 1/lambda_d with the same mode vectors).
struct LeadEntry {
    double Ec = 0;
    int n_trav_out_d = 0, n_trav_out_s = 0;   // traveling out-flow modes (rows of P)
    int m_in_d = 0, m_in_s = 0;               // injected (traveling in-flow) modes
    int status = 0;                            // PWQT_ST_* bits
    DBuf sigma_d, sigma_s;                     // n x n row-major complex128
    DBuf P_d, P_s;                             // rows of B^-1 for traveling out-flow modes
    DBuf v_out_d, v_out_s;                     // |dE/dk| of those modes (double)
    DBuf rhs_d, rhs_s;                         // n x m injection vectors (row-major)
    DBuf cin_s;                                // n x m_s injected source modes (for R)
    DBuf v_in_d, v_in_s;                       // |dE/dk| of injected modes
    DBuf sigma_d32, sigma_s32, rhs_d32, rhs_s32;   // complex64 copies (mixed path)
    long long launches = 0;                    // kernels launched to build this entry
    size_t bytes() const;
};

// Stream and library handles of one host thread that fills the contact cache.
struct LeadWorker {
    cudaStream_t stream = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cusolverDnParams_t prm = nullptr;
    cublasHandle_t blas = nullptr;
    int init();
    void destroy();
};

struct System {
    int N = 0;
    double Us = 0, Ud = 0;
    std::vector<double> U;
    DBuf HV0, HV1;        // N and N-1 blocks: H_ii + V_ii, H_{i,i+1} + V_{i,i+1} (complex128)
    DBuf HV0f, HV1f;      // complex64 copies (mixed path)
    DBuf HV0ff, HV1ff;    // float-float splits (refinement residual)
    DBuf ozH, ozH_rexp;   // slice tiles of the per-node [HV1^H | HV0 | HV1] panels (tensor-core residual)
    // density matrix of Sec. 3.3: N diagonal blocks and N-1 blocks (a, a+1), n x n complex128
    DBuf rho_d, rho_u;
    long long rho_energies = 0;   // energies accumulated since the last reset
};

// Density-matrix accumulation requested alongside a solve (Sec. 3.3)
struct DensityAcc {
    const double* w;              // host, quadrature weight per energy of the call
    double mu_s, mu_d, kT;        // contact electrochemical potentials, temperature (eV)
};

// one solved energy as seen by the accumulation kernel
struct DensJob {
    const double2* C;             // c: node i at C + i*node_stride, row r at + r*row_stride
    size_t node_stride;
    int row_stride;
    int ms, md;
    const double* v_in_s;         // |dE/dk| of the injected modes
    const double* v_in_d;
    double scale_s, scale_d;      // w_E f_FD(E - mu_s), w_E f_FD(E - mu_d)
};

}  // namespace pwqt

namespace pwqt {
// One of the two halves of a mixed-precision batch: its own stream, workspaces, profiling
// events and counters, so that the halves run on two host threads and the GPU overlaps
// one half's residual (FP32-issue-bound) with the other's latency-bound sweep/correction.
struct Lane {
    cudaStream_t st = nullptr;
    DBuf ws_mixed, ws_jobs, ws_obs, ws_res, ws_norms;
    // tensor-core residual: self-energy panels of the batch, their pointer table, the
    // solution slices, column exponents and the active-energy list
    DBuf oz_sig, oz_sig_rexp, oz_sig_tab, oz_B, oz_fexp, oz_act;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t oz_ev[2] = {nullptr, nullptr};   // around the slice-product launches of one residual
    double prof_ms = 0, prof_flops = 0, prof_phase_ms[2] = {0, 0};
    long long prof_launches = 0, prof_ir_iters = 0;
    // slice-product residual: event time, the method's complex MACs (3 N n^2 per column),
    // bf16 MMA flops issued for the 34 kept slice pairs, launches
    double prof_oz_ms = 0, prof_oz_cmacs = 0, prof_oz_mma_flops = 0;
    long long prof_oz_launches = 0;
    // correction solves: the method's complex MACs (3 N n^2 per refining column), launches
    double prof_corr_cmacs = 0;
    long long prof_corr_launches = 0;
    int init(int dev);      // stream and events on first use
    void destroy();
};
}  // namespace pwqt

struct pwqt_ctx {
    int dev = 0;
    pwqt_opts opts{};
    cudaStream_t stream = nullptr;
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cusolverDnParams_t prm = nullptr;
    std::string err;
    std::mutex err_m;                       // the mixed path may fail on two host threads at once
    std::atomic<long long> launches{0};
    int sm_count = 0;
    // basis
    int n = 0, n_bands = 0;
    double Lz = 0, Lx = 0;
    int dim = 1;
    // plane-wave expansion of the Bloch waves per k group (0: k = 0, 1: k = pi/Lz),
    // rows sorted by (mx, mz): mx, mz (int) and coefficients (n_pw x n_bands complex128)
    int pw_n[2] = {0, 0};
    pwqt::DBuf pw_mx[2], pw_mz[2], pw_C[2];
    std::vector<double> eps;               // 2 n_bands
    pwqt::DBuf H0, H1, M0, M1, W;          // n x n row-major complex128; W: 6 blocks
    pwqt::DBuf M0f, M1f, H0f, H1f;         // complex64 copies
    pwqt::DBuf M0ff, M1ff;                 // float-float splits
    pwqt::DBuf ozM, ozM_rexp;              // slice tiles of the [M1^H | M0 | M1] panel (tensor-core residual)
    int residual_kind = PWQT_RESIDUAL_SLICED;   // refinement residual of the mixed path
    std::map<int, pwqt::System> systems;
    std::map<double, std::unique_ptr<pwqt::LeadEntry>> cache;
    // scratch reused across calls
    pwqt::DBuf work_a, work_b;
    // grow-only workspaces of the sweep (kept across calls: no allocation in steady state)
    pwqt::DBuf ws_xy, ws_s, ws_norms, ws_jobs, ws_obs, ws_res, ws_mixed, ws_dens;
    pwqt::DBuf zero_nn;   // n x n zeros
    // optional CUDA-event timing of the dominant (block-sweep) kernels
    int profile = 0;
    double prof_ms = 0.0;
    long long prof_launches = 0;
    double prof_flops = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // refinement phases of the mixed path: [0] residuals, [1] corrections; iterations
    double prof_phase_ms[2] = {0.0, 0.0};
    long long prof_ir_iters = 0;
    double prof_oz_ms = 0, prof_oz_cmacs = 0, prof_oz_mma_flops = 0;
    long long prof_oz_launches = 0;
    double prof_corr_cmacs = 0;
    long long prof_corr_launches = 0;
    cudaEvent_t ev2 = nullptr, ev3 = nullptr;
    // host threads that fill the contact cache concurrently
    int lead_threads = 8;
    std::vector<std::unique_ptr<pwqt::LeadWorker>> workers;
    // the two halves of a mixed-precision batch (lane 0 also serves undivided batches)
    pwqt::Lane lanes[2];
    ~pwqt_ctx() {
        for (auto& w : workers) w->destroy();
        for (auto& l : lanes) l.destroy();
    }
};

namespace pwqt {
// Host <-> device copy ordered on the context's stream and complete on return.  A plain
// cudaMemcpy runs on the legacy default stream, which is not ordered with the context's
// non-blocking stream: for a pageable host source it may return before the data reaches
// the device, and a kernel on the context's stream could then read stale memory.
inline cudaError_t copy_sync(pwqt_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}

// error helpers
int fail(pwqt_ctx* c, int code, const std::string& msg);
int cuda_fail(pwqt_ctx* c, cudaError_t e, const char* what);

#define PWQT_CUDA(ctx, x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return ::pwqt::cuda_fail(ctx, e_, #x); } while (0)
#define PWQT_SOLVER(ctx, x) do { cusolverStatus_t e_ = (x); if (e_ != CUSOLVER_STATUS_SUCCESS) return ::pwqt::fail(ctx, PWQT_ERR_CUDA, std::string("cusolver ") + std::to_string((int)e_) + ": " #x); } while (0)
#define PWQT_BLAS(ctx, x) do { cublasStatus_t e_ = (x); if (e_ != CUBLAS_STATUS_SUCCESS) return ::pwqt::fail(ctx, PWQT_ERR_CUDA, std::string("cublas ") + std::to_string((int)e_) + ": " #x); } while (0)
#define PWQT_TRY(x) do { int r_ = (x); if (r_ != PWQT_OK) return r_; } while (0)

int alloc(pwqt_ctx* c, DBuf& b, size_t bytes);
int ensure(pwqt_ctx* c, DBuf& b, size_t bytes);   // grow-only

// assembly (assemble.cu)
int assemble_from_basis(pwqt_ctx* c, const pwqt_cell* cell, int n_bands, const double* eps_host,
                        const int* n_pw, const int* mx, const int* mz, const double2* coef_dev_rowmajor);
int epm_basis(pwqt_ctx* c, const pwqt_cell* cell, const pwqt_formfactor* ff, double gcut, int n_bands);
int build_system_blocks(pwqt_ctx* c, System& s);

// leads (lead.cu)
int lead_entry(pwqt_ctx* c, double Ec, LeadEntry** out);
int fill_leads(pwqt_ctx* c, const std::vector<double>& keys);

// solve (solve.cu)
struct SolveOut {
    double *T, *R, *T_ds, *node_n, *resid;
    int *n_open, *iters, *status;
};
// sys_of[e] (optional): the system of energy e (bias points of one device, all with
// s's node count) -- several systems in one batched launch; NULL: every energy is s's
int solve_batch(pwqt_ctx* c, System& s, int nE, const double* E_host, int precision,
                const SolveOut& dev_out, cudaStream_t st, const DensityAcc* dens = nullptr,
                System* const* sys_of = nullptr);

// density (density.cu)
int density_alloc(pwqt_ctx* c, System& s);
int density_reset(pwqt_ctx* c, System& s, cudaStream_t st);
int density_grid(pwqt_ctx* c, System& s, int nx, int nz, double* out_dev, cudaStream_t st);

// small kernels (util.cu)
void transpose_c128(const double2* in, double2* out, int rows, int cols, cudaStream_t st);
void c128_to_c64(const double2* in, float2* out, size_t count, cudaStream_t st);
}  // namespace pwqt
