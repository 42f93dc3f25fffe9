// Orchestration of one pwqt_solve call: contact self-energies from the cache,
// batched block sweeps, FP64 residuals and the observables of Sec. 3.3-3.4
// (node density, Eq. transmission, reflection) -- all in the library's kernels.
#include <algorithm>
#include <cmath>
#include <thread>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"
#include "sweep_mixed.cuh"

namespace pwqt {

// ---------------------------------------------------------------- observables
// T_gamma = sum_{mu traveling out at d} |(P_d c_N)_{mu gamma}|^2 v_mu / v_gamma  (Eq. transmission)
// R_gamma with the injected part removed at node 1, T_ds for drain-injected modes,
// node density n[i][c] = sum_{gamma in c} (2/|v_gamma|) sum_alpha |c_{i alpha gamma}|^2.
__global__ void k_observables(int n, int N, const ObsJob* __restrict__ jobs) {
    const ObsJob J = jobs[blockIdx.x];
    const int m = J.ms + J.md;
    __shared__ double acc[3];
    if (threadIdx.x < 3) acc[threadIdx.x] = 0.0;
    __syncthreads();
    const double2* cN = J.C + (size_t)(N - 1) * J.node_stride;
    const double2* c1 = J.C;
    double t_loc = 0, r_loc = 0, tds_loc = 0;
    // transmission s -> d
    for (int t = threadIdx.x; t < J.ntd * J.ms; t += blockDim.x) {
        int mu = t / J.ms, g = t % J.ms;
        double2 a = make_double2(0, 0);
        for (int k = 0; k < n; ++k) cfma(a, J.P_d[(size_t)mu * n + k], cN[(size_t)k * J.row_stride + g]);
        t_loc += cnorm2(a) * J.v_out_d[mu] / J.v_in_s[g];
    }
    // reflection at s and transmission d -> s
    for (int t = threadIdx.x; t < J.nts * m; t += blockDim.x) {
        int mu = t / m, g = t % m;
        double2 a = make_double2(0, 0);
        for (int k = 0; k < n; ++k) {
            double2 v = c1[(size_t)k * J.row_stride + g];
            if (g < J.ms) v = csub(v, J.cin_s[(size_t)k * J.ms + g]);
            cfma(a, J.P_s[(size_t)mu * n + k], v);
        }
        if (g < J.ms) r_loc += cnorm2(a) * J.v_out_s[mu] / J.v_in_s[g];
        else tds_loc += cnorm2(a) * J.v_out_s[mu] / J.v_in_d[g - J.ms];
    }
    atomicAdd(&acc[0], t_loc);
    atomicAdd(&acc[1], r_loc);
    atomicAdd(&acc[2], tds_loc);
    __syncthreads();
    if (threadIdx.x == 0) {
        *J.T = acc[0];
        *J.R = acc[1];
        *J.T_ds = acc[2];
    }
}

// node density of node blockIdx.x, energy blockIdx.y: one CTA sums the n x m
// coefficients of the node with the per-mode weights 2/|v| and reduces in the block
constexpr int MAXW = 2048;   // injected modes per energy held in shared memory (m <= 2n <= 2048)
__global__ void __launch_bounds__(256) k_node_density(int n, const ObsJob* __restrict__ jobs) {
    const ObsJob J = jobs[blockIdx.y];
    const int m = J.ms + J.md, i = blockIdx.x;
    __shared__ double wgt[MAXW];
    __shared__ double red[2][8];
    for (int g = threadIdx.x; g < m; g += blockDim.x)
        wgt[g] = g < J.ms ? 2.0 / J.v_in_s[g] : 2.0 / J.v_in_d[g - J.ms];
    __syncthreads();
    double ns = 0, nd = 0;
    if (m > 0) {
        const double2* ci = J.C + (size_t)i * J.node_stride;
        for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
            const int r = t / m, g = t % m;
            const double v = cnorm2(ci[(size_t)r * J.row_stride + g]) * wgt[g];
            if (g < J.ms) ns += v;
            else nd += v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ns += __shfl_down_sync(0xffffffffu, ns, o);
        nd += __shfl_down_sync(0xffffffffu, nd, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ns; red[1][threadIdx.x >> 5] = nd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < 8; ++q) { a += red[0][q]; b += red[1][q]; }
        J.node_n[2 * i] = a;
        J.node_n[2 * i + 1] = b;
    }
}

void launch_observables(int n, int N, const ObsJob* jobs, int nb, cudaStream_t st) {
    k_observables<<<nb, 256, 0, st>>>(n, N, jobs);
    k_node_density<<<dim3(N, nb), 256, 0, st>>>(n, jobs);
}

// ---------------------------------------------------------------- FP64 residual
// r_i = b_i - (L_i c_{i-1} + D_i c_i + U_i c_{i+1}) (FP64), per column sums of |r|^2 and |b|^2.
__global__ void k_residual_fp64(SweepSys sys, const ResJob* __restrict__ jobs) {
    const ResJob J = jobs[blockIdx.y];
    const int n = sys.n, N = sys.N, m = J.ms + J.md;
    const int i = blockIdx.x;
    if (m == 0) return;
    const double E = J.E;
    const double2* ci = J.C + (size_t)i * J.node_stride;
    const double2* cm1 = i > 0 ? J.C + (size_t)(i - 1) * J.node_stride : nullptr;
    const double2* cp1 = i < N - 1 ? J.C + (size_t)(i + 1) * J.node_stride : nullptr;
    const double2* HV0b = J.HV0 ? J.HV0 : sys.HV0;
    const double2* HV1b = J.HV1 ? J.HV1 : sys.HV1;
    const double2* HV0 = HV0b + (size_t)i * n * n;
    const double2* HV1 = HV1b + (size_t)i * n * n;
    const double2* HVm = i > 0 ? HV1b + (size_t)(i - 1) * n * n : nullptr;
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
        int r = t / m, g = t % m;
        double2 acc = make_double2(0, 0);
        for (int k = 0; k < n; ++k) {
            size_t rk = (size_t)r * n + k;
            double2 d = csub(cscale(sys.M0[rk], E), HV0[rk]);
            if (i == 0) d = csub(d, J.sig_s[rk]);
            if (i == N - 1) d = csub(d, J.sig_d[rk]);
            cfma(acc, d, ci[(size_t)k * J.row_stride + g]);
            if (cp1) cfma(acc, csub(cscale(sys.M1[rk], E), HV1[rk]), cp1[(size_t)k * J.row_stride + g]);
            if (cm1) {
                size_t kr = (size_t)k * n + r;
                cfma(acc, cconj(csub(cscale(sys.M1[kr], E), HVm[kr])), cm1[(size_t)k * J.row_stride + g]);
            }
        }
        double2 b = make_double2(0, 0);
        if (i == 0 && g < J.ms) b = J.rhs_s[(size_t)r * J.ms + g];
        if (i == N - 1 && g >= J.ms) b = J.rhs_d[(size_t)r * J.md + (g - J.ms)];
        double2 res = csub(b, acc);
        if (J.Rout) J.Rout[(size_t)i * J.r_node_stride + (size_t)r * J.r_row_stride + g] = res;
        atomicAdd(&J.rn2[g], cnorm2(res));
        atomicAdd(&J.bn2[g], cnorm2(b));
    }
}

__global__ void k_residual_finish(const ResJob* __restrict__ jobs, int nb, const int* __restrict__ active) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || (active && !active[b])) return;
    const ResJob J = jobs[b];
    int m = J.ms + J.md;
    double worst = 0.0;
    for (int g = 0; g < m; ++g) {
        double bb = J.bn2[g];
        double v = bb > 0 ? sqrt(J.rn2[g] / bb) : sqrt(J.rn2[g]);
        worst = (v > worst || isnan(v)) ? v : worst;   // NaN propagates (fmax would drop it)
        if (isnan(worst)) break;
    }
    *J.resid = worst;
}

void launch_residual_finish(const ResJob* jobs, int nb, cudaStream_t st, const int* active) {
    k_residual_finish<<<(nb + 127) / 128, 128, 0, st>>>(jobs, nb, active);
}

void launch_residual_fp64(const SweepSys& sys, const ResJob* jobs, int nb, cudaStream_t st) {
    dim3 grid(sys.N, nb);
    k_residual_fp64<<<grid, 256, 0, st>>>(sys, jobs);
    launch_residual_finish(jobs, nb, st);
}

__global__ void k_fill_int(int* p, int v, int cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) p[i] = v;
}

// ---------------------------------------------------------------- orchestration
int solve_batch(pwqt_ctx* c, System& s, int nE, const double* E, int precision, const SolveOut& o, cudaStream_t st,
                const DensityAcc* dens, System* const* sys_of) {
    const int n = c->n, N = s.N;
    const size_t nn = (size_t)n * n;
    auto sysE = [&](int e) -> System& { return sys_of ? *sys_of[e] : s; };
    if (sys_of) {
        if (dens) return fail(c, PWQT_ERR_INVALID_ARG, "density accumulation takes one system");
        for (int e = 0; e < nE; ++e)
            if (sys_of[e]->N != N) return fail(c, PWQT_ERR_INVALID_ARG, "a batch of several systems needs one node count");
    }
    // 1. contact data (FP64 cache, computed on a miss)
    std::vector<LeadEntry*> ls(nE), ld(nE);
    {
        std::vector<double> keys;
        for (int e = 0; e < nE; ++e) { keys.push_back(E[e] - sysE(e).Us); keys.push_back(E[e] - sysE(e).Ud); }
        PWQT_TRY(fill_leads(c, keys));
    }
    for (int e = 0; e < nE; ++e) {
        PWQT_TRY(lead_entry(c, E[e] - sysE(e).Us, &ls[e]));
        PWQT_TRY(lead_entry(c, E[e] - sysE(e).Ud, &ld[e]));
    }
    std::vector<int> ms(nE), md(nE), hst(nE);
    for (int e = 0; e < nE; ++e) {
        hst[e] = ls[e]->status | ld[e]->status;
        bool ok = !(hst[e] & PWQT_ST_MODE_COUNT);
        ms[e] = ok ? ls[e]->m_in_s : 0;
        md[e] = ok ? ld[e]->m_in_d : 0;
    }
    // 2. batches bounded by the device budget (after the mixed path's per-system slice
    // panels, which stay with the system)
    if (precision != PWQT_FP64) {
        PWQT_TRY(mixed_prepare(c, s, st));
        if (sys_of) {
            if (c->residual_kind != PWQT_RESIDUAL_SLICED)
                return fail(c, PWQT_ERR_INVALID_ARG, "a batch of several systems needs the sliced residual");
            for (int e = 0; e < nE; ++e) PWQT_TRY(mixed_prepare(c, *sys_of[e], st));
        }
    }
    size_t free_b = 0, total_b = 0;
    PWQT_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    size_t budget = c->opts.hbm_budget_bytes ? c->opts.hbm_budget_bytes : (size_t)(0.85 * (double)free_b);
    auto per_energy = [&](int e) {
        int m = ms[e] + md[e];
        if (precision != PWQT_FP64) return mixed_bytes_per_energy(n, N, std::max(m, 1)) + 64 * sizeof(double) * (m + 2);
        return sizeof(double2) * ((size_t)N * n * (n + m) + nn) + 64 * sizeof(double) * (m + 2);
    };
    SweepSys sys{n, N, c->M0.as<double2>(), c->M1.as<double2>(), s.HV0.as<double2>(), s.HV1.as<double2>()};
    // energies whose contacts failed the mode count get zero self-energies and no
    // injected modes (their status carries PWQT_ST_MODE_COUNT)
    if (c->zero_nn.bytes < sizeof(double2) * nn) {
        PWQT_TRY(alloc(c, c->zero_nn, sizeof(double2) * nn));
        // on the stream of the work that reads it (a plain cudaMemset is not ordered with it)
        PWQT_CUDA(c, cudaMemsetAsync(c->zero_nn.p, 0, c->zero_nn.bytes, st));
    }
    const double2* zero = c->zero_nn.as<double2>();
    PWQT_BLAS(c, cublasSetStream(c->blas, st));

    // One group of energies [g0, g0 + gn) of a batch, on stream gs: job tables, the sweep
    // (FP64 kernel, or the mixed path with its refinement on lane L) and the observables.
    // obs receives the group's observable descriptors (solution pointers for the density).
    auto group = [&](int g0, int gn, Lane* L, cudaStream_t gs, std::vector<ObsJob>& obs) -> int {
        std::vector<size_t> off(gn + 1, 0);
        for (int b = 0; b < gn; ++b) off[b + 1] = off[b] + (size_t)N * n * (n + ms[g0 + b] + md[g0 + b]);
        size_t maxm = 1;
        for (int b = 0; b < gn; ++b) maxm = std::max<size_t>(maxm, ms[g0 + b] + md[g0 + b]);
        DBuf &XY = c->ws_xy, &Sb = c->ws_s;
        DBuf &jobs_d = L ? L->ws_jobs : c->ws_jobs, &obs_d = L ? L->ws_obs : c->ws_obs, &res_d = L ? L->ws_res : c->ws_res,
             &norms = L ? L->ws_norms : c->ws_norms;
        if (precision == PWQT_FP64) {
            PWQT_TRY(ensure(c, XY, sizeof(double2) * std::max<size_t>(off[gn], 1)));
            PWQT_TRY(ensure(c, Sb, sizeof(double2) * nn * gn));
        }
        PWQT_TRY(ensure(c, norms, sizeof(double) * 2 * gn * maxm));
        PWQT_CUDA(c, cudaMemsetAsync(norms.p, 0, sizeof(double) * 2 * gn * maxm, gs));
        std::vector<SweepJob> jobs(gn);
        obs.assign(gn, ObsJob{});
        std::vector<ResJob> res(gn);
        for (int b = 0; b < gn; ++b) {
            int e = g0 + b;
            LeadEntry *Ls = ls[e], *Ld = ld[e];
            int m = ms[e] + md[e];
            SweepJob& J = jobs[b];
            J.E = E[e];
            J.ms = ms[e];
            J.md = md[e];
            J.HV0 = sysE(e).HV0.as<double2>();
            J.HV1 = sysE(e).HV1.as<double2>();
            const bool bad = (hst[e] & PWQT_ST_MODE_COUNT) != 0;
            J.sig_s = bad ? zero : Ls->sigma_s.as<double2>();
            J.sig_d = bad ? zero : Ld->sigma_d.as<double2>();
            J.rhs_s = bad ? zero : Ls->rhs_s.as<double2>();
            J.rhs_d = bad ? zero : Ld->rhs_d.as<double2>();
            J.XY = precision != PWQT_FP64 ? nullptr : XY.as<double2>() + off[b];
            J.S = precision != PWQT_FP64 ? nullptr : Sb.as<double2>() + nn * b;
            J.status = o.status + e;
            ObsJob& O = obs[b];
            O.ms = ms[e]; O.md = md[e];
            O.ntd = (hst[e] & PWQT_ST_MODE_COUNT) ? 0 : Ld->n_trav_out_d;
            O.nts = (hst[e] & PWQT_ST_MODE_COUNT) ? 0 : Ls->n_trav_out_s;
            O.C = J.XY ? J.XY + n : nullptr;   // the mixed path points this at its FP64 solution
            O.node_stride = (size_t)n * (n + m);
            O.row_stride = n + m;
            O.P_d = bad ? nullptr : Ld->P_d.as<double2>(); O.P_s = bad ? nullptr : Ls->P_s.as<double2>();
            O.v_out_d = bad ? nullptr : Ld->v_out_d.as<double>(); O.v_out_s = bad ? nullptr : Ls->v_out_s.as<double>();
            O.v_in_d = bad ? nullptr : Ld->v_in_d.as<double>(); O.v_in_s = bad ? nullptr : Ls->v_in_s.as<double>();
            O.cin_s = bad ? nullptr : Ls->cin_s.as<double2>();
            O.T = o.T + e; O.R = o.R + e; O.T_ds = o.T_ds + e; O.node_n = o.node_n + (size_t)e * N * 2;
            ResJob& Rj = res[b];
            Rj.E = E[e]; Rj.ms = ms[e]; Rj.md = md[e];
            Rj.HV0 = J.HV0; Rj.HV1 = J.HV1;
            Rj.sig_s = J.sig_s; Rj.sig_d = J.sig_d; Rj.rhs_s = J.rhs_s; Rj.rhs_d = J.rhs_d;
            Rj.C = O.C; Rj.node_stride = O.node_stride; Rj.row_stride = O.row_stride;
            Rj.Rout = nullptr; Rj.r_node_stride = 0; Rj.r_row_stride = 0;
            Rj.rn2 = norms.as<double>() + 2 * maxm * b;
            Rj.bn2 = Rj.rn2 + maxm;
            Rj.resid = o.resid + e;
        }
        // statuses from the contacts
        PWQT_CUDA(c, cudaMemcpyAsync(o.status + g0, &hst[g0], sizeof(int) * gn, cudaMemcpyHostToDevice, gs));
        PWQT_TRY(ensure(c, jobs_d, sizeof(SweepJob) * gn));
        PWQT_TRY(ensure(c, obs_d, sizeof(ObsJob) * gn));
        PWQT_TRY(ensure(c, res_d, sizeof(ResJob) * gn));
        PWQT_CUDA(c, cudaMemcpyAsync(jobs_d.p, jobs.data(), sizeof(SweepJob) * gn, cudaMemcpyHostToDevice, gs));
        PWQT_CUDA(c, cudaMemcpyAsync(obs_d.p, obs.data(), sizeof(ObsJob) * gn, cudaMemcpyHostToDevice, gs));
        PWQT_CUDA(c, cudaMemcpyAsync(res_d.p, res.data(), sizeof(ResJob) * gn, cudaMemcpyHostToDevice, gs));
        if (precision != PWQT_FP64) {
            PWQT_TRY(solve_mixed(c, s, sys, jobs, jobs_d.as<SweepJob>(), res, res_d.as<ResJob>(), obs, obs_d.as<ObsJob>(), gn,
                                 o.iters + g0, gs, precision == PWQT_MIXED, *L, sys_of ? sys_of + g0 : nullptr));
        } else {
            if (c->profile) PWQT_CUDA(c, cudaEventRecord(c->ev0, gs));
            launch_sweep_fp64(sys, jobs_d.as<SweepJob>(), gn, gs);
            c->launches++;
            if (c->profile) {
                PWQT_CUDA(c, cudaEventRecord(c->ev1, gs));
                PWQT_CUDA(c, cudaEventSynchronize(c->ev1));
                float msec = 0;
                cudaEventElapsedTime(&msec, c->ev0, c->ev1);
                c->prof_ms += msec;
                c->prof_launches += 1;
                c->prof_flops += (56.0 / 3.0) * (double)N * n * n * (double)n * gn;
            }
            PWQT_CUDA(c, cudaGetLastError());
            launch_residual_fp64(sys, res_d.as<ResJob>(), gn, gs);
            c->launches += 2;
            if (o.iters) {
                k_fill_int<<<(gn + 127) / 128, 128, 0, gs>>>(o.iters + g0, 0, gn);
                c->launches++;
            }
        }
        launch_observables(n, N, obs_d.as<ObsJob>(), gn, gs);
        c->launches += 2;
        PWQT_CUDA(c, cudaGetLastError());
        PWQT_CUDA(c, cudaStreamSynchronize(gs));
        return PWQT_OK;
    };

    int e0 = 0;
    while (e0 < nE) {
        int nb = 0;
        size_t need = 0;
        int cap = c->opts.batch > 0 ? c->opts.batch : 1 << 30;
        while (e0 + nb < nE && nb < cap) {
            size_t pe = per_energy(e0 + nb);
            if (nb > 0 && need + pe > budget) break;
            need += pe;
            ++nb;
        }
        if (need > budget) return fail(c, PWQT_ERR_OOM, "one energy needs " + std::to_string(need) + " bytes, budget " + std::to_string(budget));
        std::vector<ObsJob> obs_a, obs_b;
        int split = nb;
        if (precision == PWQT_FP64) {
            PWQT_TRY(group(e0, nb, nullptr, st, obs_a));
        } else {
            PWQT_TRY(c->lanes[0].init(c->dev) == PWQT_OK ? PWQT_OK : fail(c, PWQT_ERR_CUDA, "lane stream"));
            if (nb >= 16) {
                // two halves on two lanes (streams, host threads): the GPU runs one half's
                // residual and correction launches beside the other half's latency-bound sweep
                // kernels.  While profiling, the halves run one after the other, so that each
                // kernel's event time is its own and not the other lane's work on shared SMs.
                PWQT_TRY(c->lanes[1].init(c->dev) == PWQT_OK ? PWQT_OK : fail(c, PWQT_ERR_CUDA, "lane stream"));
                split = nb / 2;
                PWQT_CUDA(c, cudaStreamSynchronize(st));   // work the halves depend on (zero block)
                int rc_b = PWQT_OK;
                auto run_b = [&] {
                    cudaSetDevice(c->dev);
                    rc_b = group(e0 + split, nb - split, &c->lanes[1], c->lanes[1].st, obs_b);
                };
                int rc_a;
                if (c->profile) {
                    rc_a = group(e0, split, &c->lanes[0], c->lanes[0].st, obs_a);
                    if (rc_a == PWQT_OK) run_b();
                } else {
                    std::thread tb(run_b);
                    rc_a = group(e0, split, &c->lanes[0], c->lanes[0].st, obs_a);
                    tb.join();
                }
                PWQT_TRY(rc_a);
                PWQT_TRY(rc_b);
            } else {
                PWQT_TRY(group(e0, nb, &c->lanes[0], st, obs_a));
            }
            // the lanes' profile counters into the context's: times, flops and launches add up
            // (per-lane rates stay per launch); a batch counts the larger of the halves'
            // iteration counts
            long long it_max = 0;
            for (auto& L : c->lanes) {
                c->prof_ms += L.prof_ms; c->prof_flops += L.prof_flops; c->prof_launches += L.prof_launches;
                c->prof_phase_ms[0] += L.prof_phase_ms[0]; c->prof_phase_ms[1] += L.prof_phase_ms[1];
                c->prof_oz_ms += L.prof_oz_ms; c->prof_oz_cmacs += L.prof_oz_cmacs;
                c->prof_oz_mma_flops += L.prof_oz_mma_flops; c->prof_oz_launches += L.prof_oz_launches;
                c->prof_corr_cmacs += L.prof_corr_cmacs; c->prof_corr_launches += L.prof_corr_launches;
                L.prof_corr_cmacs = 0; L.prof_corr_launches = 0;
                it_max = std::max(it_max, L.prof_ir_iters);
                L.prof_ms = L.prof_flops = L.prof_phase_ms[0] = L.prof_phase_ms[1] = 0;
                L.prof_oz_ms = L.prof_oz_cmacs = L.prof_oz_mma_flops = 0;
                L.prof_launches = L.prof_ir_iters = L.prof_oz_launches = 0;
            }
            c->prof_ir_iters += it_max;
        }
        if (dens) {
            DensityAcc d = *dens;
            d.w = dens->w + e0;
            PWQT_TRY(density_accumulate_batch(c, s, obs_a, E + e0, d, split, st));
            if (split < nb) {
                d.w = dens->w + e0 + split;
                PWQT_TRY(density_accumulate_batch(c, s, obs_b, E + e0 + split, d, nb - split, st));
            }
        }
        // n_open (source, drain) per energy
        std::vector<int> nopen(2 * nb);
        for (int b = 0; b < nb; ++b) { nopen[2 * b] = ms[e0 + b]; nopen[2 * b + 1] = md[e0 + b]; }
        if (o.n_open) PWQT_CUDA(c, cudaMemcpyAsync(o.n_open + 2 * e0, nopen.data(), sizeof(int) * 2 * nb, cudaMemcpyHostToDevice, st));
        PWQT_CUDA(c, cudaStreamSynchronize(st));
        e0 += nb;
    }
    return PWQT_OK;
}

}  // namespace pwqt
