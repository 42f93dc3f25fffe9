// Mixed-precision path: complex64 block sweep on the tensor cores + FP64 refinement.
#pragma once
#include <vector>

#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

namespace pwqt {

// FP64 residual r = B - A c of one energy (Sec. 3.2 system), optionally written out.
struct ResJob {
    double E;
    int ms, md;
    const double2* HV0;        // this energy's system blocks; NULL: the launch's SweepSys blocks
    const double2* HV1;
    const double2* sig_s;
    const double2* sig_d;
    const double2* rhs_s;
    const double2* rhs_d;
    const double2* C;          // current solution
    size_t node_stride;
    int row_stride;
    double2* Rout;             // residual output (nullable)
    size_t r_node_stride;
    int r_row_stride;
    double* rn2;               // per column sum |r|^2 (m entries, zeroed by the caller)
    double* bn2;               // per column sum |b|^2
    double* resid;             // max over columns of ||r|| / ||b||
};

void launch_residual_fp64(const SweepSys& sys, const ResJob* jobs, int nb, cudaStream_t st);
// the same residual in float-float arithmetic on the FP32 pipes (~48-bit significand):
// blocks pre-split into (hi, lo) float pairs, stored as float4 (re_hi, re_lo, im_hi, im_lo)
struct ResidualFF {
    int n, N;
    const float4* M0; const float4* M1;      // n x n
    const float4* HV0; const float4* HV1;    // N and N-1 blocks
    float4* Cff; size_t per;                 // float-float copy of the solution, per-energy stride
};
void split_ff(const double2* in, float4* out, size_t count, cudaStream_t st);
// energies with active[b] == 0 (may be NULL: all) are skipped and keep their last residual
void launch_residual_ff(const ResidualFF& R, const ResJob* jobs, int nb, int m_max, const int* active, cudaStream_t st);
void launch_residual_finish(const ResJob* jobs, int nb, cudaStream_t st, const int* active = nullptr);

size_t mixed_bytes_per_energy(int n, int N, int m);
// slice panels of the tensor-core residual for the basis and system (once; kept)
int mixed_prepare(pwqt_ctx* c, System& s, cudaStream_t st);
// sys_of[b]: the system of energy b of the batch (all with the same node count), or
// NULL when every energy belongs to s; several systems need the sliced residual
int solve_mixed(pwqt_ctx* c, System& s, const SweepSys& sys, std::vector<SweepJob>& jobs, SweepJob* jobs_d,
                std::vector<ResJob>& res, ResJob* res_d, std::vector<ObsJob>& obs, ObsJob* obs_d, int nb, int* iters_dev,
                cudaStream_t st, bool refine, Lane& lane, System* const* sys_of = nullptr);

}  // namespace pwqt
