// Work descriptors shared by the sweep, residual and observable kernels.
#pragma once
#include <cuda_runtime.h>

namespace pwqt {

// Per-system data of the block-tridiagonal matrix (complex128, row-major n x n blocks).
struct SweepSys {
    int n, N;
    const double2* M0;    // M_ii
    const double2* M1;    // M_{i,i+1}
    const double2* HV0;   // N blocks H_ii + V_ii
    const double2* HV1;   // N-1 blocks H_{i,i+1} + V_{i,i+1}
};

// One energy of a batch.
struct SweepJob {
    double E;
    int ms, md;                 // injected modes from source / drain (m = ms + md columns)
    const double2* HV0;         // this energy's system blocks (several bias points in one
    const double2* HV1;         // launch); NULL: the launch's SweepSys blocks
    const double2* sig_s;       // n x n
    const double2* sig_d;
    const double2* rhs_s;       // n x ms, row-major
    const double2* rhs_d;       // n x md
    double2* XY;                // N x n x (n + m): [X_i | y_i], y overwritten by c_i
    double2* S;                 // n x n scratch
    int* status;
    double* dos;                // Green's-function recursion only: N node spectral densities
};

// Reduction descriptors of one energy (observables of Eq. transmission and Sec. 3.3).
struct ObsJob {
    int ms, md, ntd, nts;
    const double2* C;           // c: node i at C + i*node_stride, row r at + r*row_stride
    size_t node_stride;
    int row_stride;
    const double2* P_d;         // ntd x n
    const double2* P_s;         // nts x n
    const double* v_out_d;      // ntd
    const double* v_out_s;      // nts
    const double* v_in_d;       // md
    const double* v_in_s;       // ms
    const double2* cin_s;       // n x ms
    double* T; double* R; double* T_ds; double* node_n;   // node_n: N x 2
};

void launch_sweep_fp64(const SweepSys& sys, const SweepJob* jobs, int nb, cudaStream_t st);
// Diagonal blocks of G = [E M - H - Sigma]^{-1} by the recursive Green's-function
// recursion over the nodes (jobs with ms = n, md = 0; XY holds N x n x 2n):
// on return XY_i = [* | G_ii] and dos[i] = -(2/pi) Im Tr G_ii.
void launch_green_fp64(const SweepSys& sys, const SweepJob* jobs, int nb, cudaStream_t st);
void launch_observables(int n, int N, const ObsJob* jobs, int nb, cudaStream_t st);
// rank-m updates of the density matrix from one batch of solved energies (density.cu);
// E and the weights in d.w are this batch's
int density_accumulate_batch(pwqt_ctx* c, System& s, const std::vector<ObsJob>& obs, const double* E, const DensityAcc& d, int nb,
                             cudaStream_t st);

}  // namespace pwqt
