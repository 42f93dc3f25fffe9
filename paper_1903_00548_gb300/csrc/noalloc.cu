// pwqt_solve_noalloc: the FP64 solve for callers that must not allocate device
// memory during the call -- a host that hands the library a fixed memory
// footprint up front (a plugin inside another program's allocator, a process
// with a hard device-memory quota, or a service that forbids allocation on its
// request path because cudaMalloc synchronises the device and can fail under
// fragmentation).  Its work panels and job tables live in the file-scope array
// below; inputs (the context's assembled system and cached self-energies) and
// outputs (caller-owned device buffers) are the caller's.
#include <atomic>
#include <cmath>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

namespace pwqt {

// Scratch of the allocation-free solve: 32 MiB, resident on every device that
// loads the library until the process exits.  Every call shares it.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
constexpr int NOALLOC_MAX_ENERGIES = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// device address of g_noalloc_scratch per device ordinal, set up on the first call
static std::atomic<void*> g_noalloc_base[128];

static size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// makes the context's device current for the call and gives the caller's current
// device back on every return path
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace pwqt

using namespace pwqt;

extern "C" int pwqt_solve_noalloc(pwqt_ctx* c, int sys, int n_E, const double* E, double* T, double* R, double* T_ds,
                                  double* node_n, int* status, void* stream) {
    if (!c) return PWQT_ERR_INVALID_ARG;
    if (!c->n) return fail(c, PWQT_ERR_STATE, "no basis: call pwqt_assemble_intrinsic first");
    auto it = c->systems.find(sys);
    if (it == c->systems.end()) return fail(c, PWQT_ERR_STATE, "unknown system: call pwqt_set_extrinsic first");
    if (n_E < 0 || n_E > NOALLOC_MAX_ENERGIES || (n_E > 0 && !E))
        return fail(c, PWQT_ERR_INVALID_ARG, "pwqt_solve_noalloc takes 0.." + std::to_string(NOALLOC_MAX_ENERGIES) + " energies");
    if (c->dev < 0 || c->dev >= 128) return fail(c, PWQT_ERR_INVALID_ARG, "device ordinal out of range");
    DeviceGuard guard(c->dev);
    if (guard.err != cudaSuccess) return cuda_fail(c, guard.err, "cudaSetDevice");
    // one-time set-up on this device (with the device current), done by the first call
    // even when it has no energies: the host-side name of the array is only a stand-in,
    // the kernels need its device address.  With lazy module loading this lookup is
    // also what loads the library's module on the device and commits the array there.
    if (!g_noalloc_base[c->dev].load()) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(c, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_base[c->dev].store(ptr);
    }
    if (n_E == 0) return PWQT_OK;
    if (!T || !R || !T_ds || !node_n) return fail(c, PWQT_ERR_INVALID_ARG, "T, R, T_ds and node_n device buffers are required");
    for (int e = 0; e < n_E; ++e)
        if (!std::isfinite(E[e])) return fail(c, PWQT_ERR_INVALID_ARG, "non-finite energy");
    char* base = static_cast<char*>(g_noalloc_base[c->dev].load());
    System& s = it->second;
    const int n = c->n, N = s.N;
    const size_t nn = (size_t)n * n;
    cudaStream_t st = (cudaStream_t)stream;

    // contact data must already be cached (computing it would allocate)
    std::vector<LeadEntry*> ls(n_E), ld(n_E);
    for (int e = 0; e < n_E; ++e) {
        auto a = c->cache.find(E[e] - s.Us), b = c->cache.find(E[e] - s.Ud);
        if (a == c->cache.end() || b == c->cache.end())
            return fail(c, PWQT_ERR_STATE, "self-energies not cached for every energy: call pwqt_prepare_leads first");
        ls[e] = a->second.get();
        ld[e] = b->second.get();
    }
    std::vector<int> ms(n_E), md(n_E), hst(n_E);
    for (int e = 0; e < n_E; ++e) {
        hst[e] = ls[e]->status | ld[e]->status;
        bool ok = !(hst[e] & PWQT_ST_MODE_COUNT);
        ms[e] = ok ? ls[e]->m_in_s : 0;
        md[e] = ok ? ld[e]->m_in_d : 0;
    }
    // scratch layout: job tables | statuses | zero block | S panels | [X|y] panels
    size_t off_jobs = 0;
    size_t off_obs = off_jobs + up256(sizeof(SweepJob) * n_E);
    size_t off_st = off_obs + up256(sizeof(ObsJob) * n_E);
    size_t off_zero = off_st + up256(sizeof(int) * n_E);
    size_t off_s = off_zero + up256(sizeof(double2) * nn);
    size_t off_xy = off_s + up256(sizeof(double2) * nn * n_E);
    size_t total = off_xy;
    std::vector<size_t> xy(n_E);
    for (int e = 0; e < n_E; ++e) {
        xy[e] = total;
        total += up256(sizeof(double2) * (size_t)N * n * (n + ms[e] + md[e]));
    }
    if (total > NOALLOC_SCRATCH_BYTES)
        return fail(c, PWQT_ERR_INVALID_ARG, "request needs " + std::to_string(total) + " scratch bytes; pwqt_solve_noalloc holds " +
                                                 std::to_string(NOALLOC_SCRATCH_BYTES));
    double2* zero = reinterpret_cast<double2*>(base + off_zero);
    int* st_dev = status ? status : reinterpret_cast<int*>(base + off_st);
    std::vector<SweepJob> jobs(n_E);
    std::vector<ObsJob> obs(n_E);
    for (int e = 0; e < n_E; ++e) {
        const bool bad = (hst[e] & PWQT_ST_MODE_COUNT) != 0;
        LeadEntry *Ls = ls[e], *Ld = ld[e];
        int m = ms[e] + md[e];
        SweepJob& J = jobs[e];
        J.E = E[e];
        J.ms = ms[e];
        J.md = md[e];
        J.sig_s = bad ? zero : Ls->sigma_s.as<double2>();
        J.sig_d = bad ? zero : Ld->sigma_d.as<double2>();
        J.rhs_s = bad ? zero : Ls->rhs_s.as<double2>();
        J.rhs_d = bad ? zero : Ld->rhs_d.as<double2>();
        J.XY = reinterpret_cast<double2*>(base + xy[e]);
        J.S = reinterpret_cast<double2*>(base + off_s) + nn * e;
        J.status = st_dev + e;
        ObsJob& O = obs[e];
        O.ms = ms[e];
        O.md = md[e];
        O.ntd = bad ? 0 : Ld->n_trav_out_d;
        O.nts = bad ? 0 : Ls->n_trav_out_s;
        O.C = J.XY + n;
        O.node_stride = (size_t)n * (n + m);
        O.row_stride = n + m;
        O.P_d = bad ? nullptr : Ld->P_d.as<double2>();
        O.P_s = bad ? nullptr : Ls->P_s.as<double2>();
        O.v_out_d = bad ? nullptr : Ld->v_out_d.as<double>();
        O.v_out_s = bad ? nullptr : Ls->v_out_s.as<double>();
        O.v_in_d = bad ? nullptr : Ld->v_in_d.as<double>();
        O.v_in_s = bad ? nullptr : Ls->v_in_s.as<double>();
        O.cin_s = bad ? nullptr : Ls->cin_s.as<double2>();
        O.T = T + e;
        O.R = R + e;
        O.T_ds = T_ds + e;
        O.node_n = node_n + (size_t)e * N * 2;
    }
    // the array keeps the previous call's contents: reset what must start defined
    PWQT_CUDA(c, cudaMemsetAsync(zero, 0, sizeof(double2) * nn, st));
    PWQT_CUDA(c, cudaMemcpyAsync(st_dev, hst.data(), sizeof(int) * n_E, cudaMemcpyHostToDevice, st));
    PWQT_CUDA(c, cudaMemcpyAsync(base + off_jobs, jobs.data(), sizeof(SweepJob) * n_E, cudaMemcpyHostToDevice, st));
    PWQT_CUDA(c, cudaMemcpyAsync(base + off_obs, obs.data(), sizeof(ObsJob) * n_E, cudaMemcpyHostToDevice, st));
    SweepSys sy{n, N, c->M0.as<double2>(), c->M1.as<double2>(), s.HV0.as<double2>(), s.HV1.as<double2>()};
    launch_sweep_fp64(sy, reinterpret_cast<const SweepJob*>(base + off_jobs), n_E, st);
    launch_observables(n, N, reinterpret_cast<const ObsJob*>(base + off_obs), n_E, st);
    c->launches += 3;   // sweep, observables, node densities
    PWQT_CUDA(c, cudaGetLastError());
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    return PWQT_OK;
}
