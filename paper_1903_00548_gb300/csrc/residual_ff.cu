// Refinement residual r = B - A c of the Sec. 3.2 system in float-float arithmetic
// (each value a sum of two FP32 numbers, ~48-bit significand; products by FMA
// error-free transformation, sums by two-sum).  GB300's FP64 pipe runs at ~1
// TFLOP/s while the FP32 pipes run at ~68 TFLOP/s, so the residual of every
// refinement step is evaluated on the FP32 pipes to near-FP64 accuracy; block
// elements are formed in FP64 and split once per use, the solution is split per
// load, and the result is written back in FP64.
#include <algorithm>

#include "pwqt_internal.cuh"
#include "sweep_mixed.cuh"

namespace pwqt {

namespace {
struct ff { float hi, lo; };

__device__ __forceinline__ ff split(double x) {
    float h = (float)x;
    return ff{h, (float)(x - (double)h)};
}
// acc += a * b (all float-float), accumulation without renormalising every step
__device__ __forceinline__ void ff_fma(ff& acc, ff a, ff b) {
    float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe));
    float s = acc.hi + p;
    float bb = s - acc.hi;
    float e = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += e + pe;
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ double ff_d(ff a) { return (double)a.hi + (double)a.lo; }

constexpr int COLS = 4;    // solution columns per thread

// acc_c += m * x for complex m (split) and complex x (split), COLS columns
struct cff { ff re, im; };
__device__ __forceinline__ void cmac(cff& acc, const cff& m, const cff& x) {
    ff_fma(acc.re, m.re, x.re);
    ff_fma(acc.re, ff_neg(m.im), x.im);
    ff_fma(acc.im, m.re, x.im);
    ff_fma(acc.im, m.im, x.re);
}
__device__ __forceinline__ cff csplit(double2 v) { return cff{split(v.x), split(v.y)}; }
}  // namespace

// complex float-float stored as float4 (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ cff c4(float4 v) { return cff{{v.x, v.y}, {v.z, v.w}}; }
// e = E * m - h in float-float (E split once)
__device__ __forceinline__ cff form(ff E, float4 mm, float4 hh) {
    cff r{{0.f, 0.f}, {0.f, 0.f}};
    ff_fma(r.re, E, ff{mm.x, mm.y});
    ff_fma(r.im, E, ff{mm.z, mm.w});
    r.re.hi -= hh.x; r.re.lo -= hh.y;
    r.im.hi -= hh.z; r.im.lo -= hh.w;
    return r;
}

__global__ void k_split_ff(const double2* __restrict__ in, float4* __restrict__ out, size_t count) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
        double2 v = in[t];
        ff a = split(v.x), b = split(v.y);
        out[t] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

// solution c (FP64, node stride / row stride of the job) -> float-float copy with the same layout
__global__ void k_split_solution(const ResJob* __restrict__ jobs, int N, int n, float4* __restrict__ out, size_t per) {
    const ResJob J = jobs[blockIdx.y];
    const int m = J.ms + J.md;
    const size_t tot = (size_t)N * J.node_stride;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        size_t rem = t % J.node_stride;
        if ((int)(rem % J.row_stride) >= m) continue;
        double2 v = J.C[t];
        ff a = split(v.x), b = split(v.y);
        out[per * blockIdx.y + t] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

constexpr int RCOLS = 8;

__global__ void __launch_bounds__(256) k_residual_ff(ResidualFF R, const ResJob* __restrict__ jobs) {
    const ResJob J = jobs[blockIdx.y];
    const int n = R.n, N = R.N, m = J.ms + J.md;
    const int i = blockIdx.x;
    if (m == 0) return;
    const double2 Ed = make_double2(J.E, 0.0);
    const ff E = split(Ed.x);
    const float4* cs = R.Cff + R.per * blockIdx.y;
    const float4* ci = cs + (size_t)i * J.node_stride;
    const float4* cm1 = i > 0 ? cs + (size_t)(i - 1) * J.node_stride : nullptr;
    const float4* cp1 = i < N - 1 ? cs + (size_t)(i + 1) * J.node_stride : nullptr;
    const float4* HV0 = R.HV0 + (size_t)i * n * n;
    const float4* HV1 = R.HV1 + (size_t)i * n * n;
    const float4* HVm = i > 0 ? R.HV1 + (size_t)(i - 1) * n * n : nullptr;
    const int groups = (m + RCOLS - 1) / RCOLS;
    for (int t = threadIdx.x; t < n * groups; t += blockDim.x) {
        const int r = t / groups, g0 = (t % groups) * RCOLS;
        cff acc[RCOLS];
#pragma unroll
        for (int q = 0; q < RCOLS; ++q) acc[q] = cff{{0.f, 0.f}, {0.f, 0.f}};
        for (int k = 0; k < n; ++k) {
            const size_t rk = (size_t)r * n + k;
            cff D = form(E, R.M0[rk], HV0[rk]);
            if ((i == 0 && J.sig_s) || (i == N - 1 && J.sig_d)) {   // end blocks: subtract Sigma (FP64, two nodes only)
                double2 sg = i == 0 ? J.sig_s[rk] : J.sig_d[rk];
                if (i == 0 && i == N - 1) sg = cadd(J.sig_s[rk], J.sig_d[rk]);
                ff a = split(sg.x), b = split(sg.y);
                D.re.hi -= a.hi; D.re.lo -= a.lo; D.im.hi -= b.hi; D.im.lo -= b.lo;
            }
#pragma unroll
            for (int q = 0; q < RCOLS; ++q)
                if (g0 + q < m) cmac(acc[q], D, c4(ci[(size_t)k * J.row_stride + g0 + q]));
            if (cp1) {
                const cff U = form(E, R.M1[rk], HV1[rk]);
#pragma unroll
                for (int q = 0; q < RCOLS; ++q)
                    if (g0 + q < m) cmac(acc[q], U, c4(cp1[(size_t)k * J.row_stride + g0 + q]));
            }
            if (cm1) {
                const size_t kr = (size_t)k * n + r;
                cff L = form(E, R.M1[kr], HVm[kr]);
                L.im.hi = -L.im.hi; L.im.lo = -L.im.lo;   // conjugate transpose of U_{i-1}
#pragma unroll
                for (int q = 0; q < RCOLS; ++q)
                    if (g0 + q < m) cmac(acc[q], L, c4(cm1[(size_t)k * J.row_stride + g0 + q]));
            }
        }
#pragma unroll
        for (int q = 0; q < RCOLS; ++q) {
            const int g = g0 + q;
            if (g >= m) continue;
            double2 b = make_double2(0, 0);
            if (i == 0 && g < J.ms) b = J.rhs_s[(size_t)r * J.ms + g];
            if (i == N - 1 && g >= J.ms) b = J.rhs_d[(size_t)r * J.md + (g - J.ms)];
            double2 res = make_double2(b.x - ff_d(acc[q].re), b.y - ff_d(acc[q].im));
            if (J.Rout) J.Rout[(size_t)i * J.r_node_stride + (size_t)r * J.r_row_stride + g] = res;
            atomicAdd(&J.rn2[g], cnorm2(res));
            atomicAdd(&J.bn2[g], cnorm2(b));
        }
    }
}

void split_ff(const double2* in, float4* out, size_t count, cudaStream_t st) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
    if (blocks > 0) k_split_ff<<<blocks, 256, 0, st>>>(in, out, count);
}

void launch_residual_ff(const ResidualFF& R, const ResJob* jobs, int nb, cudaStream_t st) {
    k_split_solution<<<dim3(256, nb), 256, 0, st>>>(jobs, R.N, R.n, R.Cff, R.per);
    k_residual_ff<<<dim3(R.N, nb), 256, 0, st>>>(R, jobs);
    launch_residual_finish(jobs, nb, st);
}

}  // namespace pwqt
