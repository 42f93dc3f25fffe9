// Batched complex64 GEMM on the tensor cores: C -= A * B (3xTF32, FP32 accumulation).
#pragma once
#include <cuda_runtime.h>

namespace pwqt {

// A strided batch of products: entry b uses X + b * sX for every operand X.
// Columns c < split of B and C come from (B1, ldb1) and (C1, ldc1); columns
// c >= split from (B2, ldb2) and (C2, ldc2) at column c - split.  All matrices
// row-major complex64 (float2); leading dimensions and strides in elements.
struct CGemmArgs {
    const float2* A; long long sA; int lda;
    const float2* B1; long long sB1; int ldb1;
    const float2* B2; long long sB2; int ldb2;
    float2* C1; long long sC1; int ldc1;
    float2* C2; long long sC2; int ldc2;
    int split;
};

int cgemm_tc_init();
void launch_cgemm_tc(const CGemmArgs& args, int nbatch, int M, int N, int K, cudaStream_t st);
int cgemm_tc_error(bool reset, cudaStream_t st);

}  // namespace pwqt
