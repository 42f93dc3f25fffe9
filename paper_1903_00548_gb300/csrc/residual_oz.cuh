// FP64-accurate refinement residual on the bf16 tensor cores by exact slice products
// (residual_oz.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sweep_mixed.cuh"

namespace pwqt {
namespace oz {

enum { MODE_M = 0, MODE_HV = 1, MODE_SIGMA = 2 };

// Source of a sliced matrix panel: item `it` has up to three n x n complex128 blocks
// (segments) side by side, row-major.  Segment s of item it is
//   tab[s][it]                                   when tab[s] is set (per-item pointers), else
//   blk[s] + (it + off[s]) * stride[s]           when 0 <= it + off[s] < count[s],
// absent otherwise (zero slices); ct[s] takes the conjugate transpose of the block.
struct PanelSrc {
    int n, nseg;
    const double2* blk[3];
    const double2* const* tab[3];
    long long stride[3];
    int off[3], count[3], ct[3];
    __host__ __device__ const double2* block(int it, int s) const {
        if (s >= nseg) return nullptr;
        if (tab[s]) return tab[s][it];
        const int j = it + off[s];
        return (blk[s] && j >= 0 && j < count[s]) ? blk[s] + (long long)j * stride[s] : nullptr;
    }
    __device__ bool present(int it, int s) const { return block(it, s) != nullptr; }
};

// One slice-product launch.  Columns k m + g: column g of active energy k = act-index.
struct GemmArgs {
    int mode, n, N, m, n_pad, nct, n_act;
    const __nv_bfloat16* A;     // panel tiles
    size_t a_item_bytes;        // bytes per item (0 would share item 0; the M panel has one item)
    const int* rexp;            // panel row exponents [item][2 n_pad] (biased)
    const __nv_bfloat16* B;     // solution slice tiles of every node
    const int* fexp;            // column exponents (biased) [nct * 32]
    const int* act;             // active energy list (indices into jobs)
    const ResJob* jobs;         // energy, injected modes, right-hand sides
    double2* R;                 // residual, per energy stride sC: [node][row][m]
    long long sC;
    int sigma_side;             // MODE_SIGMA: 0 source (node 0), 1 drain (node N-1); item = active energy
    int col_lo, col_hi;         // MODE_M / MODE_HV: the columns this launch writes (one system's energies)
};

int padded(int n);                                  // n rounded up to a multiple of 64
int col_tiles(int ncols);
size_t panel_bytes(int n, int items, int nseg);
size_t panel_item_bytes(int n, int nseg);
size_t rexp_bytes(int n, int items);
size_t b_bytes(int n, int N, int ncols);

int gemm_init();
int error_flag(bool reset, cudaStream_t st);
void build_panel(const PanelSrc& P, int items, int* rexp, __nv_bfloat16* tiles, cudaStream_t st);
// column exponents (fexp, zeroed here) and slice tiles of the active energies' solutions
void slice_solution(const double2* C, long long sC, const int* act, int n_act, int n, int N, int m, int* fexp,
                    __nv_bfloat16* tiles, cudaStream_t st);
void gemm(const GemmArgs& G, int items, cudaStream_t st);
// per-column |r|^2 (all nodes) and |b|^2 (end nodes) into the jobs' rn2 / bn2
void norms(const double2* R, long long sC, const ResJob* jobs, const int* act, int n_act, int n, int N, int m, cudaStream_t st);

}  // namespace oz
}  // namespace pwqt
