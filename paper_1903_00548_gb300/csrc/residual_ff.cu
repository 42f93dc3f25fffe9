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
    // __fmul_rn / __fadd_rn keep the compiler from contracting the product into the
    // two-sum below, which would break its exactness
    float p = __fmul_rn(a.hi, b.hi);
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe));
    float s = __fadd_rn(acc.hi, p);
    float bb = s - acc.hi;
    float e = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += e + pe;
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
// acc -= b, with the rounding error of the leading subtraction kept (two-sum)
__device__ __forceinline__ void ff_sub(ff& acc, float bhi, float blo) {
    float s = acc.hi - bhi;
    float bb = s - acc.hi;
    float e = (acc.hi - (s - bb)) - (bhi + bb);
    acc.hi = s;
    acc.lo += e - blo;
}
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
    ff_sub(r.re, hh.x, hh.y);
    ff_sub(r.im, hh.z, hh.w);
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
__global__ void k_split_solution(const ResJob* __restrict__ jobs, int N, int n, float4* __restrict__ out, size_t per,
                                 const int* __restrict__ active) {
    if (active && !active[blockIdx.y]) return;
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

// Tiled residual: one CTA computes a 64-row x 32-column tile of r_i = b_i - [L_i D_i U_i] [c_{i-1}; c_i; c_{i+1}]
// for one node i of one energy.  The K dimension (3n: the three blocks of the row) runs in chunks of 32: the
// block elements E M - H (and -Sigma at the end nodes) are formed in float-float while they are staged in
// shared memory, the solution chunk is staged beside them, and every thread accumulates a 4 x 2 micro-tile.
constexpr int RT = 64;    // rows per CTA
constexpr int CT = 32;    // columns per CTA
constexpr int KC = 32;    // K chunk

__global__ void __launch_bounds__(256) k_residual_ff(ResidualFF R, const ResJob* __restrict__ jobs, int col_tiles,
                                                     const int* __restrict__ active) {
    if (active && !active[blockIdx.z]) return;
    extern __shared__ float4 rsm[];
    float4 (*As)[KC + 1] = reinterpret_cast<float4 (*)[KC + 1]>(rsm);          // [RT][KC + 1]
    float4 (*Cs)[CT] = reinterpret_cast<float4 (*)[CT]>(rsm + RT * (KC + 1));   // [KC][CT]
    __shared__ double rsum[CT], bsum[CT];
    const ResJob J = jobs[blockIdx.z];
    const int n = R.n, N = R.N, m = J.ms + J.md;
    const int i = blockIdx.y;
    const int r0 = (blockIdx.x / col_tiles) * RT, c0 = (blockIdx.x % col_tiles) * CT;
    if (c0 >= m) return;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const ff E = split(J.E);
    const float4* cs = R.Cff + R.per * blockIdx.z;
    const double2* sig = nullptr;
    if (i == 0 && J.sig_s) sig = J.sig_s;
    if (i == N - 1 && J.sig_d) sig = J.sig_d;
    const bool both = i == 0 && i == N - 1 && J.sig_s && J.sig_d;
    if (t < CT) { rsum[t] = 0.0; bsum[t] = 0.0; }
    cff acc[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = cff{{0.f, 0.f}, {0.f, 0.f}};
    // blk 0: L_i = (E M1 - HV1_{i-1})^H with c_{i-1}; blk 1: D_i with c_i; blk 2: U_i with c_{i+1}
    for (int blk = 0; blk < 3; ++blk) {
        if ((blk == 0 && i == 0) || (blk == 2 && i == N - 1)) continue;
        const float4* cn = cs + (size_t)(i + blk - 1) * J.node_stride;
        const float4* Mb = blk == 1 ? R.M0 : R.M1;
        const float4* Hb = blk == 1 ? R.HV0 + (size_t)i * n * n : R.HV1 + (size_t)(blk == 0 ? i - 1 : i) * n * n;
        for (int k0 = 0; k0 < n; k0 += KC) {
            // stage the formed block elements
            for (int e = t; e < RT * KC; e += 256) {
                int r, k;
                if (blk == 0) { r = e % RT; k = e / RT; }   // transposed source: consecutive threads along r
                else { r = e / KC; k = e % KC; }
                const int gr = r0 + r, gk = k0 + k;
                cff v{{0.f, 0.f}, {0.f, 0.f}};
                if (gr < n && gk < n) {
                    if (blk == 0) {
                        const size_t kr = (size_t)gk * n + gr;
                        v = form(E, Mb[kr], Hb[kr]);
                        v.im.hi = -v.im.hi;
                        v.im.lo = -v.im.lo;
                    } else {
                        const size_t rk = (size_t)gr * n + gk;
                        v = form(E, Mb[rk], Hb[rk]);
                        if (blk == 1 && sig) {
                            double2 sg = sig[rk];
                            if (both) sg = cadd(J.sig_s[rk], J.sig_d[rk]);
                            const ff a = split(sg.x), b = split(sg.y);
                            ff_sub(v.re, a.hi, a.lo);
                            ff_sub(v.im, b.hi, b.lo);
                        }
                    }
                }
                As[r][k] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
            }
            // stage the solution chunk
            for (int e = t; e < KC * CT; e += 256) {
                const int k = e / CT, cc = e % CT, gk = k0 + k, gc = c0 + cc;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gk < n && gc < m) v = cn[(size_t)gk * J.row_stride + gc];
                Cs[k][cc] = v;
            }
            __syncthreads();
#pragma unroll 2
            for (int k = 0; k < KC; ++k) {
                const cff x0 = c4(Cs[k][tx]), x1 = c4(Cs[k][tx + 16]);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const cff d = c4(As[ty + 16 * a][k]);
                    cmac(acc[a][0], d, x0);
                    cmac(acc[a][1], d, x1);
                }
            }
            __syncthreads();
        }
    }
    // epilogue: r = b - A c in FP64, column norms reduced in the CTA first
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gr = r0 + ty + 16 * a, cc = tx + 16 * b, g = c0 + cc;
            if (gr >= n || g >= m) continue;
            double2 bv = make_double2(0, 0);
            if (i == 0 && g < J.ms) bv = J.rhs_s[(size_t)gr * J.ms + g];
            if (i == N - 1 && g >= J.ms) bv = J.rhs_d[(size_t)gr * J.md + (g - J.ms)];
            const double2 res = make_double2(bv.x - ff_d(acc[a][b].re), bv.y - ff_d(acc[a][b].im));
            if (J.Rout) J.Rout[(size_t)i * J.r_node_stride + (size_t)gr * J.r_row_stride + g] = res;
            atomicAdd(&rsum[cc], cnorm2(res));
            if (i == 0 || i == N - 1) atomicAdd(&bsum[cc], cnorm2(bv));
        }
    __syncthreads();
    if (t < CT && c0 + t < m) {
        atomicAdd(&J.rn2[c0 + t], rsum[t]);
        if (i == 0 || i == N - 1) atomicAdd(&J.bn2[c0 + t], bsum[t]);
    }
}

void split_ff(const double2* in, float4* out, size_t count, cudaStream_t st) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
    if (blocks > 0) k_split_ff<<<blocks, 256, 0, st>>>(in, out, count);
}

void launch_residual_ff(const ResidualFF& R, const ResJob* jobs, int nb, int m_max, const int* active, cudaStream_t st) {
    k_split_solution<<<dim3(256, nb), 256, 0, st>>>(jobs, R.N, R.n, R.Cff, R.per, active);
    const int col_tiles = (std::max(m_max, 1) + CT - 1) / CT;
    const int smem = (int)(sizeof(float4) * (RT * (KC + 1) + KC * CT));
    // idempotent attribute set; per call, so that contexts on several host threads need no shared flag
    cudaFuncSetAttribute(k_residual_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_residual_ff<<<dim3(((R.n + RT - 1) / RT) * col_tiles, R.N, nb), 256, smem, st>>>(R, jobs, col_tiles, active);
    launch_residual_finish(jobs, nb, st, active);
}

}  // namespace pwqt
