// Mixed-precision block sweep of [E M - H - Sigma] c = B (Eq. qtbm_system): complex64
// factorisation with the products on the tensor cores (3xTF32 tcgen05 GEMM, FP32
// accumulation), refined to FP64 residuals (Sec. 3.2 system, north of the
// paper's own direct FP64 solve).
//
// Per node i, for every energy of the batch at once:
//   form     F_i = E M0 - HV0_i (- Sigma at the ends),  XY_i = [U_i | b_i],  Lb = L_i
//   Schur    [F_i | y-part of XY_i] -= L_i [X_{i-1} | y_{i-1}]               (tensor cores)
//   LU       right-looking, 32-column panels with partial pivoting (FP32, one CTA
//            per energy: pivot search, row swaps over F_i and XY_i, L-solve of the
//            32-row strip), trailing update on the tensor cores
//   U-solve  32-row blocks from the bottom: diagonal block (FP32) + update above
//            (tensor cores)  ->  XY_i = [X_i | y_i]
// then c_i = y_i - X_i c_{i+1} (tensor cores), FP64 copy, and refinement:
//   r = B - A c (FP64-accurate: exact slice products on the bf16 tensor cores,
//   residual_oz.cu), A d = r with the stored complex64 factors, c += d.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "cgemm_tc.cuh"
#include "residual_oz.cuh"
#include "sweep_mixed.cuh"

namespace pwqt {

namespace {

constexpr int PW = 32;      // panel width
constexpr int NT = 256;
constexpr int MV_INTS = 4 * PW + 4;   // per energy: count, then 2 PW destination and 2 PW source rows
constexpr int APT = 128;              // threads of the column-parallel panel kernels

struct MixSys {
    int n, N, m, w;                       // w = n + m rounded up to even (16-byte rows), uniform over the batch
    const double2* M0; const double2* M1; const double2* HV0; const double2* HV1;   // FP64 blocks
    const float2* M1f; const float2* HV1f;                                         // complex64 copies
    float2* F; long long sF;              // per energy N x n x n factors
    int* piv; long long sP;               // per energy N x n pivot rows
    float2* XY; long long sXY;            // per energy N x n x w
    float2* Lb; long long sL;             // per energy N x n x n couplings L_i = A_{i,i-1} (node 0 unused)
    int* mv;                              // per energy MV_INTS: the row moves of the current panel
    double2* C64; double2* R64; long long sC;   // per energy N x n x m (FP64 solution, residual)
    const SweepJob* jobs;
};

__device__ __forceinline__ void ffma(float2& a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
__device__ __forceinline__ float2 fdiv(float2 a, float2 b) {
    if (fabsf(b.x) >= fabsf(b.y)) {
        float r = b.y / b.x, d = b.x + b.y * r;
        return make_float2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    float r = b.x / b.y, d = b.x * r + b.y;
    return make_float2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ float2 to32(double2 v) { return make_float2((float)v.x, (float)v.y); }

// ---------------------------------------------------------------- form the node blocks
__global__ void k_mx_form(MixSys S, int i) {
    const int e = blockIdx.y;
    const SweepJob& J = S.jobs[e];
    const int n = S.n, N = S.N, w = S.w, ms = J.ms, md = J.md;
    const double E = J.E;
    float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    float2* Lb = S.Lb + e * S.sL + (size_t)i * n * n;   // kept for the correction solves
    const double2* HV0b = J.HV0 ? J.HV0 : S.HV0;
    const double2* HV1b = J.HV1 ? J.HV1 : S.HV1;
    const double2* HV0 = HV0b + (size_t)i * n * n;
    const double2* HV1 = HV1b + (size_t)i * n * n;
    const double2* HVm = HV1b + (size_t)(i > 0 ? i - 1 : 0) * n * n;
    const size_t nn = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t / n), c = (int)(t % n);
        double2 d = csub(cscale(S.M0[t], E), HV0[t]);
        if (i == 0 && J.sig_s) d = csub(d, J.sig_s[t]);
        if (i == N - 1 && J.sig_d) d = csub(d, J.sig_d[t]);
        F[t] = to32(d);
        if (i > 0) {
            size_t tt = (size_t)c * n + r;
            Lb[t] = to32(cconj(csub(cscale(S.M1[tt], E), HVm[tt])));
        }
        XY[(size_t)r * w + c] = i < N - 1 ? to32(csub(cscale(S.M1[t], E), HV1[t])) : make_float2(0.f, 0.f);
    }
    const int wy = w - n;   // y columns: m and, for even rows, a zero padding column
    const size_t nm = (size_t)n * wy;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nm; t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t / wy), g = (int)(t % wy);
        float2 v = make_float2(0.f, 0.f);
        if (i == 0 && g < ms) v = to32(J.rhs_s[(size_t)r * ms + g]);
        if (i == N - 1 && g >= ms && g < ms + md) v = to32(J.rhs_d[(size_t)r * md + (g - ms)]);
        XY[(size_t)r * w + n + g] = v;
    }
}

// ---------------------------------------------------------------- panel factorisation
// Factor F_i[k0:n, k0:k0+wd] with partial pivoting (max |re|+|im|), one CTA per energy;
// the row interchanges, composed into a list of row moves, and the strip solve against
// the unit-lower 32 x 32 block go to the other columns in k_mx_panel_apply.
__global__ void __launch_bounds__(NT) k_mx_panel(MixSys S, int i, int k0, int wd) {
    // the panel, column-major with an odd leading dimension: threads walk rows of one
    // column (consecutive words) in the elimination and columns of one row (odd stride,
    // distinct banks) when it is loaded and stored
    extern __shared__ float2 P[];                     // PW columns x pld rows
    __shared__ int prow[PW];
    __shared__ float bv[NT / 32];
    __shared__ int bi[NT / 32];
    const int e = blockIdx.x;
    const int n = S.n, rows = n - k0, pld = rows | 1;   // panel leading dimension (odd)
    float2* F = S.F + e * S.sF + (size_t)i * n * n;
    int* piv = S.piv + e * S.sP + (size_t)i * n;
    int st = 0;
#pragma unroll 8
    for (int t = threadIdx.x; t < rows * PW; t += NT) {
        int r = t / PW, c = t % PW;
        P[c * pld + r] = c < wd ? F[(size_t)(k0 + r) * n + k0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // pivot candidates of column 0; afterwards each elimination pass also finds the
    // candidates of the next column while it updates the rows
    float best = -1.f;
    int idx = 0;
    for (int r = threadIdx.x; r < rows; r += NT) {
        const float2 v = P[r];
        const float a = fabsf(v.x) + fabsf(v.y);
        if (a > best) { best = a; idx = r; }
    }
    for (int j = 0; j < wd; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_down_sync(0xffffffff, best, o);
            int oi = __shfl_down_sync(0xffffffff, idx, o);
            if (ov > best || (ov == best && oi < idx)) { best = ov; idx = oi; }
        }
        if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = idx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < NT / 32; ++q)
                if (bv[q] > bv[0] || (bv[q] == bv[0] && bi[q] < bi[0])) { bv[0] = bv[q]; bi[0] = bi[q]; }
            const int pr = bv[0] < 0.f ? j : bi[0];   // no candidate rows: keep the diagonal
            prow[j] = pr;
            piv[k0 + j] = k0 + pr;
        }
        __syncthreads();
        const int p = prow[j];
        if (p != j && threadIdx.x < PW) {
            float2 a = P[threadIdx.x * pld + j];
            P[threadIdx.x * pld + j] = P[threadIdx.x * pld + p];
            P[threadIdx.x * pld + p] = a;
        }
        __syncthreads();
        float2 pv = P[j * pld + j];
        if (pv.x == 0.f && pv.y == 0.f) { st |= PWQT_ST_SINGULAR_PIVOT; pv = make_float2(1.f, 0.f); }
        const float2 inv = fdiv(make_float2(1.f, 0.f), pv);
        best = -1.f;
        idx = j + 1;
        for (int r = j + 1 + threadIdx.x; r < rows; r += NT) {
            const float2 x = P[j * pld + r];
            const float2 l = make_float2(x.x * inv.x - x.y * inv.y, x.x * inv.y + x.y * inv.x);
            P[j * pld + r] = l;
            for (int c = j + 1; c < wd; ++c) ffma(P[c * pld + r], make_float2(-l.x, -l.y), P[c * pld + j]);
            if (j + 1 < wd) {
                const float2 v = P[(j + 1) * pld + r];
                const float a = fabsf(v.x) + fabsf(v.y);
                if (a > best) { best = a; idx = r; }
            }
        }
        __syncthreads();
    }
#pragma unroll 8
    for (int t = threadIdx.x; t < rows * wd; t += NT) {
        int r = t / wd, c = t % wd;
        F[(size_t)(k0 + r) * n + k0 + c] = P[c * pld + r];
    }
    // the wd swaps in order, as a map panel row -> original row (in the panel's shared
    // memory, free after the write-back); rows with a new origin (at most 2 wd) become
    // the list of moves (destination row <- source row) for k_mx_panel_apply
    __shared__ int mvc;
    int* orig = reinterpret_cast<int*>(P);
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += NT) orig[r] = r;
    if (threadIdx.x == 0) mvc = 0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < wd; ++j) {
            const int p = prow[j];
            if (p != j) { const int x = orig[j]; orig[j] = orig[p]; orig[p] = x; }
        }
    __syncthreads();
    int* mv = S.mv + (size_t)e * MV_INTS;
    for (int r = threadIdx.x; r < rows; r += NT)
        if (orig[r] != r) {
            const int k = atomicAdd(&mvc, 1);
            mv[1 + k] = r;
            mv[1 + 2 * PW + k] = orig[r];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        mv[0] = mvc;
        if (st) atomicOr(S.jobs[e].status, st);
    }
}

// k_mx_panel for panels of at most 512 rows: the panel in registers (thread t holds panel
// rows t and t + 256, all 32 columns), so the rank-1 updates touch no shared memory; per
// column the pivot (max |re|+|im|, the lower row on ties, as k_mx_panel) is found by warp
// shuffles and one pass over the warps' candidates, and rows j and p are exchanged and
// the pivot row broadcast through shared memory.  Pivots, the factored panel and the list
// of row moves are written as k_mx_panel writes them.
constexpr int PR_NT = 256;
__global__ void __launch_bounds__(PR_NT) k_mx_panel_reg(MixSys S, int i, int k0, int wd) {
    __shared__ float2 prow_s[PW], jrow_s[PW];
    __shared__ float bv[PR_NT / 32];
    __shared__ int bi[PR_NT / 32], prow[PW], sel;
    const int e = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n = S.n, rows = n - k0;
    float2* F = S.F + e * S.sF + (size_t)i * n * n + (size_t)k0 * n + k0;   // panel origin, row stride n
    int* piv = S.piv + e * S.sP + (size_t)i * n;
    float2 a[2][PW];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = t + q * PR_NT;
#pragma unroll
        for (int c = 0; c < PW; ++c) a[q][c] = (r < rows && c < wd) ? F[(size_t)r * n + c] : make_float2(0.f, 0.f);
    }
    int st = 0;
#pragma unroll
    for (int j = 0; j < PW; ++j) {
        if (j >= wd) break;
        float best = -1.f;
        int idx = j;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = t + q * PR_NT;
            if (r >= j && r < rows) {
                const float v = fabsf(a[q][j].x) + fabsf(a[q][j].y);
                if (v > best) { best = v; idx = r; }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, idx, o);
            if (ov > best || (ov == best && oi < idx)) { best = ov; idx = oi; }
        }
        if (lane == 0) { bv[warp] = best; bi[warp] = idx; }
        __syncthreads();
        if (t == 0) {
            float b = bv[0];
            int ii = bi[0];
            for (int q = 1; q < PR_NT / 32; ++q)
                if (bv[q] > b || (bv[q] == b && bi[q] < ii)) { b = bv[q]; ii = bi[q]; }
            const int p = b < 0.f ? j : ii;   // no candidate rows: keep the diagonal
            sel = p;
            prow[j] = p;
            piv[k0 + j] = k0 + p;
        }
        __syncthreads();
        const int p = sel;
        // the owners publish row p (the pivot row) and, if different, row j
        if (t == p % PR_NT) {
            const bool hi = p >= PR_NT;
#pragma unroll
            for (int c = 0; c < PW; ++c) prow_s[c] = hi ? a[1][c] : a[0][c];
        }
        if (p != j && t == j) {
#pragma unroll
            for (int c = 0; c < PW; ++c) jrow_s[c] = a[0][c];
        }
        __syncthreads();
        if (p != j) {
            if (t == j)
#pragma unroll
                for (int c = 0; c < PW; ++c) a[0][c] = prow_s[c];
            if (t == p % PR_NT) {
                if (p >= PR_NT) {
#pragma unroll
                    for (int c = 0; c < PW; ++c) a[1][c] = jrow_s[c];
                } else {
#pragma unroll
                    for (int c = 0; c < PW; ++c) a[0][c] = jrow_s[c];
                }
            }
        }
        float2 pv = prow_s[j];
        if (pv.x == 0.f && pv.y == 0.f) { st |= PWQT_ST_SINGULAR_PIVOT; pv = make_float2(1.f, 0.f); }
        const float2 inv = fdiv(make_float2(1.f, 0.f), pv);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = t + q * PR_NT;
            if (r > j && r < rows) {
                const float2 x = a[q][j];
                const float2 l = make_float2(x.x * inv.x - x.y * inv.y, x.x * inv.y + x.y * inv.x);
                a[q][j] = l;
#pragma unroll
                for (int c = j + 1; c < PW; ++c) {
                    const float2 u = prow_s[c];
                    ffma(a[q][c], make_float2(-l.x, -l.y), u);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = t + q * PR_NT;
        if (r < rows)
#pragma unroll
            for (int c = 0; c < PW; ++c)
                if (c < wd) F[(size_t)r * n + c] = a[q][c];
    }
    // the swaps in order, as a map panel row -> original row; rows with a new origin (at
    // most 2 wd) become the move list
    __shared__ int orig[2 * PR_NT], mvc;
    for (int r = t; r < rows; r += PR_NT) orig[r] = r;
    if (t == 0) mvc = 0;
    __syncthreads();
    if (t == 0)
        for (int j = 0; j < wd; ++j) {
            const int p = prow[j];
            if (p != j) { const int x = orig[j]; orig[j] = orig[p]; orig[p] = x; }
        }
    __syncthreads();
    int* mv = S.mv + (size_t)e * MV_INTS;
    for (int r = t; r < rows; r += PR_NT)
        if (orig[r] != r) {
            const int k = atomicAdd(&mvc, 1);
            mv[1 + k] = r;
            mv[1 + 2 * PW + k] = orig[r];
        }
    __syncthreads();
    if (t == 0) {
        mv[0] = mvc;
        if (st) atomicOr(S.jobs[e].status, st);
    }
}

// The panel's row moves on the other columns of F_i and on XY_i (one column per thread,
// all loads of a column issued before its stores), then the strip rows k0..k0+wd of
// [F right of the panel | XY] <- L11^{-1} strip (unit lower, L11 from the factored panel).
// Grid (column chunks of APT, energies): the columns are independent.
__global__ void __launch_bounds__(APT) k_mx_panel_apply(MixSys S, int i, int k0, int wd) {
    __shared__ float2 L11[PW][PW + 1];
    __shared__ int mv_dst[2 * PW], mv_src[2 * PW], mv_cnt;
    const int e = blockIdx.y;
    const int n = S.n, w = S.w;
    float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    const int* mv = S.mv + (size_t)e * MV_INTS;
    for (int t = threadIdx.x; t < PW * PW; t += APT) {
        const int r = t / PW, c = t % PW;
        L11[r][c] = (r < wd && c < r) ? F[(size_t)(k0 + r) * n + k0 + c] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) mv_cnt = mv[0];
    if (threadIdx.x < 2 * PW) { mv_dst[threadIdx.x] = mv[1 + threadIdx.x]; mv_src[threadIdx.x] = mv[1 + 2 * PW + threadIdx.x]; }
    __syncthreads();
    const int nmv = mv_cnt;
    const int ncolF = n - wd;
    const int c = blockIdx.x * APT + threadIdx.x;
    if (c >= ncolF + w) return;
    float2* base;
    size_t ld;
    bool right;
    if (c < ncolF) { base = F + (c < k0 ? c : c + wd); ld = n; right = c >= k0; }
    else { base = XY + (c - ncolF); ld = w; right = true; }
    base += (size_t)k0 * ld;
    {
        float2 v[2 * PW];
#pragma unroll
        for (int q = 0; q < 2 * PW; ++q)
            if (q < nmv) v[q] = base[(size_t)mv_src[q] * ld];
#pragma unroll
        for (int q = 0; q < 2 * PW; ++q)
            if (q < nmv) base[(size_t)mv_dst[q] * ld] = v[q];
    }
    if (!right) return;
    float2 x[PW];
#pragma unroll
    for (int j = 0; j < PW; ++j) x[j] = j < wd ? base[(size_t)j * ld] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j < PW; ++j) {
        float2 s = x[j];
#pragma unroll
        for (int l = 0; l < PW; ++l)
            if (l < j) {
                const float2 L = L11[j][l];
                ffma(s, make_float2(-L.x, -L.y), x[l]);
            }
        x[j] = s;
    }
#pragma unroll
    for (int j = 0; j < PW; ++j)
        if (j < wd) base[(size_t)j * ld] = x[j];
}

// XY_i[k0:k0+wd, :] <- U11^{-1} XY_i[k0:k0+wd, :]
__global__ void __launch_bounds__(APT) k_mx_trsm_up(MixSys S, int i, int k0, int wd) {
    __shared__ float2 U[PW][PW + 1];
    const int e = blockIdx.y;
    const int n = S.n, w = S.w;
    const float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    for (int t = threadIdx.x; t < PW * PW; t += APT) {
        int r = t / PW, c = t % PW;
        U[r][c] = (r < wd && c < wd) ? F[(size_t)(k0 + r) * n + k0 + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    for (int c = blockIdx.x * APT + threadIdx.x; c < w; c += gridDim.x * APT) {
        float2 x[PW];
        float2* base = XY + (size_t)k0 * w + c;
#pragma unroll
        for (int j = 0; j < PW; ++j) x[j] = j < wd ? base[(size_t)j * w] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = PW - 1; j >= 0; --j) {
            float2 s = x[j];
#pragma unroll
            for (int l = 0; l < PW; ++l)
                if (l > j) ffma(s, make_float2(-U[j][l].x, -U[j][l].y), x[l]);
            float2 d = U[j][j];
            if (d.x == 0.f && d.y == 0.f) d = make_float2(1.f, 0.f);
            x[j] = fdiv(s, d);
        }
#pragma unroll
        for (int j = 0; j < PW; ++j)
            if (j < wd) base[(size_t)j * w] = x[j];
    }
}

// C64 = (double) c (the y columns of XY after the node back substitution)
__global__ void k_mx_to64(MixSys S) {
    const int e = blockIdx.y;
    const int n = S.n, N = S.N, m = S.m, w = S.w;
    const size_t tot = (size_t)N * n * m;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        size_t i = t / ((size_t)n * m), rem = t % ((size_t)n * m);
        int r = (int)(rem / m), g = (int)(rem % m);
        float2 v = S.XY[e * S.sXY + i * n * w + (size_t)r * w + n + g];
        S.C64[e * S.sC + t] = make_double2(v.x, v.y);
    }
}

// ---------------------------------------------------------------- correction solve
// d = A^{-1} r with the stored complex64 factors, one launch per refinement step.  The
// right-hand sides stay independent through the whole block-tridiagonal solve, so one
// CTA carries LC columns of one energy through every node on its own:
//   forward   w_i = U_i^{-1} L_i^{-1} P_i (r_i - L_i w_{i-1}),   i = 0 .. N-1
//   backward  d_{N-1} = w_{N-1},  d_i = w_i - X_i d_{i+1},  c_i += d_i (FP64)
// with L_i the stored coupling A_{i,i-1}, F_i = P_i^T L_i U_i the node's LU factors
// and X_i the y-free columns of XY_i.  The CTA's two n x LC work vectors live in shared
// memory; the matrices stream through the rest of it in 32 x 32 tiles (tensor-map copies
// into a ring of mbarrier-tracked slots); a tile updates 32 rows x LC columns with the
// multiplicand's values in registers.  The 32 x 32 diagonal blocks of the triangular
// factors hold their inverses (k_mx_diag_inv), so they are tile products too.
// LC is picked per refinement step from the columns still refining: 16 while most
// energies refine (fewest tile reads per column), down to 2 for the last few, where
// the length of one CTA's chain through the nodes is the step's time.
constexpr int TS = 32;     // tile edge
constexpr int CT = 256;    // threads of a correction CTA
constexpr int TILE_BYTES = TS * TS * 8;   // two 128-byte-swizzled halves of 32 rows x 16 complex64
constexpr unsigned long long CORR_WAIT_NS = 2000000000ull;   // bounded mbarrier waits: 2 s

__device__ int g_corr_error = 0;

// A CTA of LC columns updates TPS = 16 / LC tiles per step, one per group of 32 LC / 2
// threads (a thread: one tile row, two columns); the ring holds NSTG tiles, two steps' worth
// at least, so that the next step's tiles are in flight while one step computes.
__host__ __device__ constexpr int corr_tps(int lc) { return 16 / lc; }
__host__ __device__ constexpr int corr_nstg(int lc) { return 2 * corr_tps(lc) > 8 ? 2 * corr_tps(lc) : 8; }

// shared memory: the tile ring (1024-byte aligned for the swizzle, hence the slack), its
// mbarriers, the permutation, the two work vectors
size_t correct_smem(int n, int lc) {
    const size_t np = (size_t)((n + TS - 1) / TS) * TS;
    const int nstg = corr_nstg(lc);
    return 1024 + (size_t)nstg * TILE_BYTES + 16 * ((nstg * 8 + 15) / 16) + ((n * sizeof(int) + 15) / 16) * 16 +
           sizeof(float2) * 2 * np * lc;
}

// A ring tile is two halves (columns 0-15, 16-31) of 32 rows of 128 bytes whose 16-byte
// chunks are permuted by the 128-byte swizzle: chunk c of row r sits at chunk c ^ (r % 8).

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ unsigned long long gclock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait on an mbarrier phase; false when it gave up
__device__ __forceinline__ bool corr_wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = gclock();
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 63) == 63 && gclock() - t0 > CORR_WAIT_NS) return false;
    }
}

enum CorrPhase { PH_SCHUR, PH_LOWER, PH_UPPER };

// Steps of a phase, in tile order: SCHUR (and the backward X_i product) per column panel
// kb the row blocks 0 .. nbk-1, TPS at a time; LOWER per panel kb the diagonal block (a
// step of its own), then the blocks below it; UPPER from the last panel, the diagonal
// block, then the blocks above it.  The tiles of one step update distinct row blocks.
struct StepCursor {
    int kb, rb0, cnt;    // cnt == 0: the diagonal block of panel kb
    __device__ void first(int ph, int nbk, int tps) {
        if (ph == PH_SCHUR) { kb = 0; rb0 = 0; cnt = min(tps, nbk); }
        else { kb = ph == PH_LOWER ? 0 : nbk - 1; rb0 = kb; cnt = 0; }
    }
    // advance; false past the phase's last step
    __device__ bool next(int ph, int nbk, int tps) {
        if (ph == PH_SCHUR) {
            rb0 += cnt;
            if (rb0 == nbk) { if (++kb == nbk) return false; rb0 = 0; }
            cnt = min(tps, nbk - rb0);
        } else if (ph == PH_LOWER) {
            rb0 = cnt == 0 ? kb + 1 : rb0 + cnt;
            if (rb0 == nbk) { if (++kb == nbk) return false; rb0 = kb; cnt = 0; }
            else cnt = min(tps, nbk - rb0);
        } else {
            rb0 = cnt == 0 ? 0 : rb0 + cnt;
            if (rb0 == kb) { if (--kb < 0) return false; rb0 = kb; cnt = 0; }
            else cnt = min(tps, kb - rb0);
        }
        return true;
    }
    __device__ int tiles() const { return cnt == 0 ? 1 : cnt; }
};

// The ring of a CTA: tile j (counted over the whole kernel) sits in slot j % NSTG and
// completes phase (j / NSTG) & 1 of that slot's mbarrier.
struct CorrRing {
    unsigned char* buf;
    uint32_t mbar;       // shared address of NSTG consecutive mbarriers
    int* abort;          // shared flag: a wait gave up
};

// One phase over the matrices of tensor map tm (matrix index mat, n x n used): SCHUR
// T -= M V (T and V distinct n x LC vectors), LOWER/UPPER  V <- M^{-1} V with the unit
// lower / upper triangle of the LU factors.  A step updates TPS row blocks at once, one
// tile per group of TG = 256 / TPS threads; a thread of a group takes row rr of its tile
// and columns gq, gq + GW (GW = LC / 2), the multiplicand's 32 rows of those columns in
// registers (reloaded when the column panel changes), so that a tile row costs 16
// shared-memory loads and 256 FMAs whatever LC is.  A diagonal block is a step of its
// own: the factorisation left the inverses of the diagonal blocks of L and U in place
// (k_mx_diag_inv), so the step is one more triangular tile product, with no dependent
// chain.  Lane 0 of each warp fetches in turn: two tensor-map copies per tile (the 16-column halves,
// 128-byte swizzle) completing on the slot's mbarrier; the map's bounds (n columns, n rows
// per matrix) zero-fill the edge tiles.  Tiles base .. of the kernel's count; returns the
// next base, or -1 when a wait gave up (after the copies in flight have landed or timed out).
template <int LC>
__device__ __noinline__ int corr_phase(int ph, const CUtensorMap* tm, int mat, int n, CorrRing R, int base, float2* V, float2* T) {
    constexpr int TPS = corr_tps(LC), NSTG = corr_nstg(LC);
    constexpr int GW = LC / 2, TG = CT / TPS;
    static_assert(TG == TS * GW, "a group: 32 rows x GW column pairs");
    const int t = threadIdx.x;
    const int tw = t / TG, gq = t % GW, rr = (t % TG) / GW;
    const int nbk = (n + TS - 1) / TS;
    const int ntiles = ph == PH_SCHUR ? nbk * nbk : nbk * (nbk + 1) / 2;
    StepCursor fc, cc;      // fetch cursor (tile granularity through fsub), compute cursor
    fc.first(ph, nbk, TPS);
    cc.first(ph, nbk, TPS);
    int fsub = 0, issued = 0;
    // issue the tiles up to (not including) tile `upto` of the phase
    auto fetch_to = [&](int upto) {
        upto = min(upto, ntiles);
        for (int q = 0; issued < upto; ++q) {
            if (t == 32 * (q % (CT / 32))) {   // lane 0 of warp q % 8 issues the call's q-th tile
                const uint32_t j = (uint32_t)(base + issued), slot = j % NSTG;
                const uint32_t dst = su32(R.buf + (size_t)slot * TILE_BYTES), mb = R.mbar + 8 * slot;
                const int rb = fc.cnt == 0 ? fc.kb : fc.rb0 + fsub;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"((uint32_t)TILE_BYTES) : "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                        :: "r"(dst + h * (TILE_BYTES / 2)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(fc.kb * TS + 16 * h),
                           "r"(rb * TS), "r"(mat), "r"(mb)
                        : "memory");
            }
            ++issued;
            if (++fsub == fc.tiles()) { fsub = 0; fc.next(ph, nbk, TPS); }
        }
    };
    fetch_to(NSTG);
    float2 tk[2][TS];
    float2* Tgt = ph == PH_SCHUR ? T : V;
    int done = 0;
    for (bool more = true; more; more = cc.next(ph, nbk, TPS)) {
        const int nt = cc.tiles();
        // this thread's tile of the step (the diagonal block: every thread's)
        const int mine = cc.cnt == 0 ? 0 : min(tw, nt - 1);
        const uint32_t j = (uint32_t)(base + done + mine), slot = j % NSTG;
        if (!corr_wait(R.mbar + 8 * slot, (j / NSTG) & 1)) {
            *R.abort = 1;
            atomicExch(&g_corr_error, 1);
        }
        __syncthreads();          // the step's tiles landed; the previous step's consumed; V, T settled
        if (*R.abort) {
            // wait (bounded again) for the copies still in flight before the CTA stops
            if (t == 0)
                for (int q = done; q < issued; ++q) corr_wait(R.mbar + 8 * ((base + q) % NSTG), ((base + q) / NSTG) & 1);
            return -1;
        }
        fetch_to(done + NSTG);    // refill the slots of the steps consumed so far
        const int kb = cc.kb;
        if (cc.cnt == 0) {
            // diagonal block (rows past n are zero and their zero-filled tile rows keep them so)
            const unsigned char* tile = R.buf + (size_t)((base + done) % NSTG) * TILE_BYTES;
            // the stored block is L_kk^{-1} (strict lower part, unit diagonal implied) over
            // U_kk^{-1} (upper part with the diagonal): group 0 multiplies V rows kb*32 .. +32
            // by the triangle of the phase, all rows read before any is written
            float2 own[2];
            if (tw == 0) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    own[k] = V[(kb * TS + rr) * LC + gq + k * GW];
#pragma unroll
                    for (int l = 0; l < TS; ++l) tk[k][l] = V[(kb * TS + l) * LC + gq + k * GW];
                }
            }
            __syncthreads();
            if (tw == 0) {
                const unsigned char* trow = tile + rr * 128;
                const int sw = rr & 7;
                const bool lower = ph == PH_LOWER;
                float2 a0[2], a1[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    a0[k] = lower ? own[k] : make_float2(0.f, 0.f);
                    a1[k] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int c2 = 0; c2 < TS / 2; ++c2) {
                    float4 x = *reinterpret_cast<const float4*>(trow + (c2 >> 3) * (TILE_BYTES / 2) + (((c2 & 7) ^ sw) << 4));
                    // columns 2 c2, 2 c2 + 1 of row rr: below the diagonal for the lower
                    // triangle, on or above it for the upper one
                    const bool k0 = lower ? 2 * c2 < rr : 2 * c2 >= rr, k1 = lower ? 2 * c2 + 1 < rr : 2 * c2 + 1 >= rr;
                    if (!k0) { x.x = 0.f; x.y = 0.f; }
                    if (!k1) { x.z = 0.f; x.w = 0.f; }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        ffma(a0[k], make_float2(x.x, x.y), tk[k][2 * c2]);
                        ffma(a1[k], make_float2(x.z, x.w), tk[k][2 * c2 + 1]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    V[(kb * TS + rr) * LC + gq + k * GW] = make_float2(a0[k].x + a1[k].x, a0[k].y + a1[k].y);
            }
        } else {
            const bool first = ph == PH_LOWER ? cc.rb0 == kb + 1 : cc.rb0 == 0;
            if (first) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int l = 0; l < TS; ++l) tk[k][l] = V[(kb * TS + l) * LC + gq + k * GW];
            }
            if (tw < nt) {
                const unsigned char* trow = R.buf + (size_t)((base + done + tw) % NSTG) * TILE_BYTES + rr * 128;
                const int sw = rr & 7;
                float2 a0[2], a1[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) a0[k] = a1[k] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c2 = 0; c2 < TS / 2; ++c2) {   // 16-byte chunk c2 of the row: columns 2 c2, 2 c2 + 1
                    const float4 x = *reinterpret_cast<const float4*>(trow + (c2 >> 3) * (TILE_BYTES / 2) + (((c2 & 7) ^ sw) << 4));
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        ffma(a0[k], make_float2(-x.x, -x.y), tk[k][2 * c2]);
                        ffma(a1[k], make_float2(-x.z, -x.w), tk[k][2 * c2 + 1]);
                    }
                }
                float2* out = Tgt + ((cc.rb0 + tw) * TS + rr) * LC + gq;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float2 o0 = out[k * GW];
                    out[k * GW] = make_float2(o0.x + a0[k].x + a1[k].x, o0.y + a0[k].y + a1[k].y);
                }
            }
        }
        done += nt;
    }
    __syncthreads();
    return base + ntiles;
}

template <int LC>
__global__ void __launch_bounds__(CT) k_mx_correct(MixSys S, const int* __restrict__ active, const __grid_constant__ CUtensorMap tmL,
                                                   const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmX) {
    constexpr int NT = CT, NSTG = corr_nstg(LC);
    const int e = blockIdx.x;
    if (!active[e]) return;
    const SweepJob& J = S.jobs[e];
    const int n = S.n, N = S.N, w = S.w, m = S.m;
    const int c0 = blockIdx.y * LC;
    const int ncol = min(LC, J.ms + J.md - c0);
    if (ncol <= 0) return;
    const int np = ((n + TS - 1) / TS) * TS;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int abort_flag;
    unsigned char* ring = sm + ((1024 - (su32(sm) & 1023)) & 1023);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ring + (size_t)NSTG * TILE_BYTES);
    int* perm = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(mbar) + 16 * ((NSTG * 8 + 15) / 16));
    float2* Wv = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(perm) + ((n * sizeof(int) + 15) / 16) * 16);   // w_i / d_{i+1}
    float2* Sv = Wv + (size_t)np * LC;       // scratch: r_i - L_i w_{i-1} (forward), d_i (backward)
    const int t = threadIdx.x;
    if (t == 0) {
        abort_flag = 0;
        for (int s = 0; s < NSTG; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(mbar + s)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int q = t; q < 2 * np * LC; q += NT) Wv[q] = make_float2(0.f, 0.f);   // rows past n stay zero
    __syncthreads();
    const CorrRing R{ring, su32(mbar), &abort_flag};
    int base = 0;
    const int mat0 = e * N;   // tensor-map matrix index of (energy e, node 0)
    float2* XYe = S.XY + e * S.sXY;
    const int* pe = S.piv + e * S.sP;
    const double2* Re = S.R64 + e * S.sC;
    double2* Ce = S.C64 + e * S.sC;
    const size_t nw = (size_t)n * w, nm = (size_t)n * m;
    for (int i = 0; i < N && base >= 0; ++i) {
        for (int j = t; j < n; j += NT) perm[j] = pe[(size_t)i * n + j];
        __syncthreads();
        const double2* Ri = Re + i * nm;
        if (i == 0) {
            for (int q = t; q < n * LC; q += NT) {
                const int r = q / LC, g = q % LC;
                Wv[q] = g < ncol ? to32(Ri[(size_t)perm[r] * m + c0 + g]) : make_float2(0.f, 0.f);
            }
        } else {
            for (int q = t; q < n * LC; q += NT) {
                const int r = q / LC, g = q % LC;
                Sv[q] = g < ncol ? to32(Ri[(size_t)r * m + c0 + g]) : make_float2(0.f, 0.f);
            }
            base = corr_phase<LC>(PH_SCHUR, &tmL, mat0 + i, n, R, base, Wv, Sv);   // Sv -= L_i w_{i-1}
            if (base < 0) break;
            for (int q = t; q < n * LC; q += NT) Wv[q] = Sv[perm[q / LC] * LC + q % LC];
        }
        base = corr_phase<LC>(PH_LOWER, &tmF, mat0 + i, n, R, base, Wv, Sv);
        if (base < 0) break;
        base = corr_phase<LC>(PH_UPPER, &tmF, mat0 + i, n, R, base, Wv, Sv);
        if (base < 0) break;
        float2* Yi = XYe + i * nw + n + c0;
        for (int q = t; q < n * LC; q += NT) {
            const int r = q / LC, g = q % LC;
            if (g < ncol) Yi[(size_t)r * w + g] = Wv[q];
        }
    }
    // backward; each thread reads back only the (row, column) entries it wrote
    for (int i = N - 1; i >= 0 && base >= 0; --i) {
        if (i < N - 1) {
            const float2* Yi = XYe + i * nw + n + c0;
            for (int q = t; q < n * LC; q += NT) {
                const int r = q / LC, g = q % LC;
                Sv[q] = g < ncol ? Yi[(size_t)r * w + g] : make_float2(0.f, 0.f);
            }
            base = corr_phase<LC>(PH_SCHUR, &tmX, mat0 + i, n, R, base, Wv, Sv);   // Sv -= X_i d_{i+1}
            if (base < 0) break;
            float2* x = Wv; Wv = Sv; Sv = x;
        }
        double2* Ci = Ce + i * nm + c0;
        for (int q = t; q < n * LC; q += NT) {
            const int r = q / LC, g = q % LC;
            if (g < ncol) {
                const float2 d = Wv[q];
                double2& c = Ci[(size_t)r * m + g];
                c.x += d.x;
                c.y += d.y;
            }
        }
    }
}

// Once per factorisation: the 32 x 32 diagonal blocks of every node's factors replaced by
// their inverses, L_kk^{-1} over the strict lower part (unit diagonal implied) and
// U_kk^{-1} over the upper part, so that the correction solves apply them as products.
// One warp per block, lane = row; rows of the inverse by substitution against the
// identity (row j final, then broadcast by shuffle to the rows it updates).  Rows and
// columns of an edge block past n are the identity and are not written; a zero pivot
// (flagged by the factorisation) counts as 1.
__global__ void __launch_bounds__(32) k_mx_diag_inv(MixSys S) {
    const int kb = blockIdx.x, i = blockIdx.y, e = blockIdx.z, lane = threadIdx.x;
    const int n = S.n, r0 = kb * TS, wd = min(TS, n - r0);
    float2* B = S.F + e * S.sF + (size_t)i * n * n + (size_t)r0 * n + r0;
    const bool in = lane < wd;
    float2 a[TS], x[TS];
#pragma unroll
    for (int c = 0; c < TS; ++c) a[c] = in && c < wd ? B[(size_t)lane * n + c] : make_float2(0.f, 0.f);
    // L_kk^{-1}
#pragma unroll
    for (int c = 0; c < TS; ++c) x[c] = make_float2(c == lane ? 1.f : 0.f, 0.f);
#pragma unroll
    for (int j = 0; j + 1 < TS; ++j) {
        const float2 l = lane > j ? make_float2(-a[j].x, -a[j].y) : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c <= j; ++c) ffma(x[c], l, shfl2(x[c], j));   // row j has no entries past column j
    }
    if (in)
#pragma unroll
        for (int c = 0; c < TS; ++c)
            if (c < lane && c < wd) B[(size_t)lane * n + c] = x[c];
    // U_kk^{-1}
#pragma unroll
    for (int c = 0; c < TS; ++c) x[c] = make_float2(c == lane ? 1.f : 0.f, 0.f);
#pragma unroll
    for (int j = TS - 1; j >= 0; --j) {
        if (lane == j) {
            float2 d = a[j];
            if (d.x == 0.f && d.y == 0.f) d = make_float2(1.f, 0.f);
            const float2 inv = fdiv(make_float2(1.f, 0.f), d);
#pragma unroll
            for (int c = j; c < TS; ++c) x[c] = make_float2(x[c].x * inv.x - x[c].y * inv.y, x[c].x * inv.y + x[c].y * inv.x);
        }
        const float2 u = lane < j ? make_float2(-a[j].x, -a[j].y) : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = j; c < TS; ++c) ffma(x[c], u, shfl2(x[c], j));   // row j has no entries before column j
    }
    if (in)
#pragma unroll
        for (int c = 0; c < TS; ++c)
            if (c >= lane && c < wd) B[(size_t)lane * n + c] = x[c];
}

// Once per factorisation: the pivot rows of node i (row j exchanged with piv[j], in
// order j = 0..n-1) composed into the row permutation, P w = w[perm[.]], written over
// the pivots, so that the correction solves of every refinement step read it directly.
// Grid (energies, nodes), one warp; the composition is serial in shared memory.
__global__ void k_mx_perm(MixSys S) {
    const int e = blockIdx.x, i = blockIdx.y, n = S.n;
    extern __shared__ int ps[];
    int* pv = ps;          // n pivots
    int* perm = ps + n;    // n
    int* piv = S.piv + e * S.sP + (size_t)i * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) { pv[j] = piv[j]; perm[j] = j; }
    __syncwarp();
    if (threadIdx.x == 0)
        for (int j = 0; j < n; ++j) {
            const int p = pv[j];
            if (p != j) { const int a = perm[j]; perm[j] = perm[p]; perm[p] = a; }
        }
    __syncwarp();
    for (int j = threadIdx.x; j < n; j += blockDim.x) piv[j] = perm[j];
}

__global__ void k_or_status(const SweepJob* __restrict__ jobs, const int* __restrict__ bits, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && bits[b]) atomicOr(jobs[b].status, bits[b]);
}

}  // namespace

namespace {
// 3D tensor map (columns, rows, matrix) over `count` consecutive n x n complex64 matrices of
// row stride ld (elements), boxes of 16 columns x 32 rows, 128-byte swizzle, zero fill
// past the bounds
bool corr_tensor_map(CUtensorMap* tm, const float2* base, int n, int ld, long long count) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q{};
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * 8, (cuuint64_t)n * ld * 8};
    const cuuint32_t box[3] = {16, (cuuint32_t)TS, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float2*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int corr_error_flag(bool reset, cudaStream_t st) {
    int v = 0;
    cudaMemcpyFromSymbolAsync(&v, g_corr_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (reset && v) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_corr_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    return v;
}
}  // namespace

size_t mixed_bytes_per_energy(int n, int N, int m) {
    // F + XY + L_i (complex64) + pivots + FP64 solution and residual
    const size_t w = (size_t)n + m + (m & 1);
    return sizeof(float2) * ((size_t)N * n * n + (size_t)N * n * w + (size_t)N * n * n) + sizeof(int) * ((size_t)N * n + MV_INTS) + 256 +
           3 * sizeof(double2) * (size_t)N * n * m +     // FP64 solution, residual, float-float copy
           2 * oz::panel_item_bytes(n, 1) +               // self-energy slice panels
           oz::b_bytes(n, N, m + 32);                     // solution slices (a column tile of slack)
}

int mixed_prepare(pwqt_ctx* c, System& s, cudaStream_t st) {
    if (c->residual_kind != PWQT_RESIDUAL_SLICED) return PWQT_OK;
    const int n = c->n, N = s.N;
    const size_t nn = (size_t)n * n;
    if (!c->ozM.p) {
        oz::PanelSrc P{};
        P.n = n; P.nseg = 3;
        const double2* M0 = c->M0.as<double2>();
        const double2* M1 = c->M1.as<double2>();
        P.blk[0] = M1; P.ct[0] = 1; P.count[0] = 1;    // M1^H (with c_{i-1})
        P.blk[1] = M0; P.count[1] = 1;                 // M0 (c_i)
        P.blk[2] = M1; P.count[2] = 1;                 // M1 (c_{i+1})
        PWQT_TRY(alloc(c, c->ozM, oz::panel_bytes(n, 1, 3)));
        PWQT_TRY(alloc(c, c->ozM_rexp, oz::rexp_bytes(n, 1)));
        oz::build_panel(P, 1, c->ozM_rexp.as<int>(), c->ozM.as<__nv_bfloat16>(), st);
        c->launches += 2;
    }
    if (!s.ozH.p) {
        oz::PanelSrc P{};
        P.n = n; P.nseg = 3;
        // item i: [HV1_{i-1}^H | HV0_i | HV1_i]; absent blocks at the ends
        P.blk[0] = s.HV1.as<double2>(); P.stride[0] = (long long)nn; P.off[0] = -1; P.count[0] = N - 1; P.ct[0] = 1;
        P.blk[1] = s.HV0.as<double2>(); P.stride[1] = (long long)nn; P.count[1] = N;
        P.blk[2] = s.HV1.as<double2>(); P.stride[2] = (long long)nn; P.count[2] = N - 1;
        PWQT_TRY(alloc(c, s.ozH, oz::panel_bytes(n, N, 3)));
        PWQT_TRY(alloc(c, s.ozH_rexp, oz::rexp_bytes(n, N)));
        oz::build_panel(P, N, s.ozH_rexp.as<int>(), s.ozH.as<__nv_bfloat16>(), st);
        c->launches += 2;
    }
    PWQT_CUDA(c, cudaGetLastError());
    return PWQT_OK;
}

int solve_mixed(pwqt_ctx* c, System& s, const SweepSys& sys, std::vector<SweepJob>& jobs, SweepJob* jobs_d, std::vector<ResJob>& res,
                ResJob* res_d, std::vector<ObsJob>& obs, ObsJob* obs_d, int nb, int* iters_dev, cudaStream_t st, bool refine,
                Lane& L, System* const* sys_of) {
    // idempotent (a function attribute of the device): set per call, no flag shared between host threads
    if (cgemm_tc_init() != 0) return fail(c, PWQT_ERR_CUDA, "tensor-core GEMM set-up failed");
    const int n = sys.n, N = sys.N;
    // the complex64 rows of the factors start on 16-byte boundaries (bulk and cp.async copies)
    if (n % 2) return fail(c, PWQT_ERR_INVALID_ARG, "mixed precision needs an even block size (use PWQT_FP64)");
    int m = 0;
    for (int b = 0; b < nb; ++b) m = std::max(m, jobs[b].ms + jobs[b].md);
    m = std::max(m, 1);
    const int w = n + m + (m & 1);   // even: the rows of XY_i start on 16-byte boundaries (tile copies)
    MixSys S;
    S.n = n; S.N = N; S.m = m; S.w = w;
    S.M0 = sys.M0; S.M1 = sys.M1; S.HV0 = sys.HV0; S.HV1 = sys.HV1;
    S.M1f = c->M1f.as<float2>(); S.HV1f = s.HV1f.as<float2>();
    S.sF = (long long)N * n * n;
    S.sP = (long long)N * n;
    S.sXY = (long long)N * n * w;
    S.sL = (long long)N * n * n;
    S.sC = (long long)N * n * m;
    const size_t bytes = mixed_bytes_per_energy(n, N, m) * nb + 1024 * 4;
    PWQT_TRY(ensure(c, L.ws_mixed, bytes));
    char* base = L.ws_mixed.as<char>();
    auto take = [&](size_t b) { char* p = base; base += (b + 255) / 256 * 256; return p; };
    S.F = (float2*)take(sizeof(float2) * S.sF * nb);
    S.XY = (float2*)take(sizeof(float2) * S.sXY * nb);
    S.Lb = (float2*)take(sizeof(float2) * S.sL * nb);
    S.piv = (int*)take(sizeof(int) * S.sP * nb);
    S.mv = (int*)take(sizeof(int) * MV_INTS * nb);
    S.C64 = (double2*)take(sizeof(double2) * S.sC * nb);
    S.R64 = (double2*)take(sizeof(double2) * S.sC * nb);
    float4* Cff = (float4*)take(sizeof(float4) * S.sC * nb);
    PWQT_CUDA(c, cudaMemsetAsync(S.R64, 0, sizeof(double2) * S.sC * nb, st));
    ResidualFF RF{n, N, c->M0ff.as<float4>(), c->M1ff.as<float4>(), s.HV0ff.as<float4>(), s.HV1ff.as<float4>(), Cff,
                  (size_t)S.sC};
    S.jobs = jobs_d;
    int* active_d = (int*)take(sizeof(int) * nb);
    int* bits_d = (int*)take(sizeof(int) * nb);

    // ---------------- forward sweep over the nodes
    const int fblocks = (int)std::min<size_t>(((size_t)n * n + NT - 1) / NT, 512);
    const size_t panel_smem = sizeof(float2) * (size_t)(n + 1) * PW;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    if (panel_smem > (size_t)smem_optin)
        return fail(c, PWQT_ERR_INVALID_ARG, "the complex64 panel of block size " + std::to_string(n) +
                                                 " exceeds shared memory: use PWQT_FP64 (mixed precision takes n <= " +
                                                 std::to_string(smem_optin / (int)(sizeof(float2) * PW) - 1) + ")");
    // the limit is a property of the kernel, shared by every context in the process (several
    // contexts on several host threads run here at once): always the device maximum, never a
    // per-call value that another thread could lower under a launch in flight
    cudaFuncAttributes fa_panel{};
    PWQT_CUDA(c, cudaFuncGetAttributes(&fa_panel, k_mx_panel));
    // the opt-in maximum counts static and dynamic shared memory together
    const int dyn_panel = smem_optin - (int)fa_panel.sharedSizeBytes;
    if (panel_smem > (size_t)dyn_panel) return fail(c, PWQT_ERR_INVALID_ARG, "panel exceeds shared memory");
    PWQT_CUDA(c, cudaFuncSetAttribute(k_mx_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_panel));
    auto gemm = [&](const float2* A, long long sA, int lda, const float2* B1, long long sB1, int ldb1, const float2* B2, long long sB2,
                    int ldb2, float2* C1, long long sC1, int ldc1, float2* C2, long long sC2, int ldc2, int split, int M, int Nc, int K) {
        CGemmArgs g{A, sA, lda, B1, sB1, ldb1, B2, sB2, ldb2, C1, sC1, ldc1, C2, sC2, ldc2, split};
        launch_cgemm_tc(g, nb, M, Nc, K, st);
        c->launches++;
    };
    if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.ev[0], st));
    for (int i = 0; i < N; ++i) {
        float2* Fi = S.F + (size_t)i * n * n;
        float2* XYi = S.XY + (size_t)i * n * w;
        k_mx_form<<<dim3(fblocks, nb), NT, 0, st>>>(S, i);
        c->launches++;
        if (i > 0) {
            const float2* XYp = S.XY + (size_t)(i - 1) * n * w;
            gemm(S.Lb + (size_t)i * n * n, S.sL, n, XYp, S.sXY, w, XYp + n, S.sXY, w, Fi, S.sF, n, XYi + n, S.sXY, w, n, n, w, n);
        }
        for (int k0 = 0; k0 < n; k0 += PW) {
            const int wd = std::min(PW, n - k0);
            if (n - k0 <= 2 * PR_NT) k_mx_panel_reg<<<nb, PR_NT, 0, st>>>(S, i, k0, wd);
            else k_mx_panel<<<nb, NT, sizeof(float2) * (size_t)((n - k0) | 1) * PW, st>>>(S, i, k0, wd);
            k_mx_panel_apply<<<dim3((n - wd + w + APT - 1) / APT, nb), APT, 0, st>>>(S, i, k0, wd);
            c->launches += 2;
            const int rest = n - k0 - wd;
            if (rest > 0)
                gemm(Fi + (size_t)(k0 + wd) * n + k0, S.sF, n, Fi + (size_t)k0 * n + k0 + wd, S.sF, n, XYi + (size_t)k0 * w, S.sXY, w,
                     Fi + (size_t)(k0 + wd) * n + k0 + wd, S.sF, n, XYi + (size_t)(k0 + wd) * w, S.sXY, w, rest, rest, rest + w, wd);
        }
        for (int k0 = ((n - 1) / PW) * PW; k0 >= 0; k0 -= PW) {
            const int wd = std::min(PW, n - k0);
            k_mx_trsm_up<<<dim3((w + APT - 1) / APT, nb), APT, 0, st>>>(S, i, k0, wd);
            c->launches++;
            if (k0 > 0) gemm(Fi + k0, S.sF, n, XYi + (size_t)k0 * w, S.sXY, w, XYi + (size_t)k0 * w, S.sXY, w, XYi, S.sXY, w, XYi, S.sXY,
                             w, w, k0, w, wd);
        }
    }
    // node back substitution c_i = y_i - X_i c_{i+1}
    for (int i = N - 2; i >= 0; --i) {
        float2* XYi = S.XY + (size_t)i * n * w;
        const float2* XYn = S.XY + (size_t)(i + 1) * n * w;
        gemm(XYi, S.sXY, w, XYn + n, S.sXY, w, XYn + n, S.sXY, w, XYi + n, S.sXY, w, XYi + n, S.sXY, w, m, n, m, n);
    }
    if (c->profile) {
        PWQT_CUDA(c, cudaEventRecord(L.ev[1], st));
        PWQT_CUDA(c, cudaEventSynchronize(L.ev[1]));
        float ms = 0;
        cudaEventElapsedTime(&ms, L.ev[0], L.ev[1]);
        L.prof_ms += ms;
        L.prof_launches += 1;
        L.prof_flops += (56.0 / 3.0) * (double)N * n * n * (double)n * nb;
    }
    PWQT_CUDA(c, cudaGetLastError());
    if (cgemm_tc_error(true, st)) return fail(c, PWQT_ERR_TIMEOUT, "tensor-core GEMM: a bounded mbarrier wait gave up");
    k_mx_to64<<<dim3(256, nb), NT, 0, st>>>(S);
    k_mx_perm<<<dim3(nb, N), 32, 2 * sizeof(int) * n, st>>>(S);
    k_mx_diag_inv<<<dim3((n + TS - 1) / TS, N, nb), 32, 0, st>>>(S);
    c->launches += 3;

    // ---------------- refinement with FP64 residuals
    for (int b = 0; b < nb; ++b) {
        res[b].C = S.C64 + S.sC * b;
        res[b].node_stride = (size_t)n * m;
        res[b].row_stride = m;
        res[b].Rout = S.R64 + S.sC * b;
        res[b].r_node_stride = (size_t)n * m;
        res[b].r_row_stride = m;
    }
    PWQT_CUDA(c, cudaMemcpyAsync(res_d, res.data(), sizeof(ResJob) * nb, cudaMemcpyHostToDevice, st));
    // correction solve: the column counts per CTA whose two n x LC work vectors fit
    const void* corr_fn[4] = {(const void*)k_mx_correct<16>, (const void*)k_mx_correct<8>, (const void*)k_mx_correct<4>,
                              (const void*)k_mx_correct<2>};
    const int corr_lcs[4] = {16, 8, 4, 2};
    bool corr_fits[4];
    for (int k = 0; k < 4; ++k) {
        cudaFuncAttributes fa{};
        PWQT_CUDA(c, cudaFuncGetAttributes(&fa, corr_fn[k]));
        const int dyn = smem_optin - (int)fa.sharedSizeBytes;
        corr_fits[k] = correct_smem(n, corr_lcs[k]) <= (size_t)dyn;
        if (corr_fits[k]) PWQT_CUDA(c, cudaFuncSetAttribute(corr_fn[k], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    }
    if (!corr_fits[3]) return fail(c, PWQT_ERR_INVALID_ARG, "correction solve exceeds shared memory");
    // tensor maps of the stored couplings L_i, factors F_i and X_i (the first n columns of XY_i)
    CUtensorMap tmL, tmF, tmX;
    if (!corr_tensor_map(&tmL, S.Lb, n, n, (long long)nb * N) || !corr_tensor_map(&tmF, S.F, n, n, (long long)nb * N) ||
        !corr_tensor_map(&tmX, S.XY, n, w, (long long)nb * N))
        return fail(c, PWQT_ERR_CUDA, "correction solve: tensor map encoding failed");
    // the widest CTA that still gives half the SMs a CTA of this lane (the other lane
    // takes the rest); with fewer columns left the narrowest that fits
    auto corr_pick = [&](const std::vector<int>& act) {
        for (int k = 0; k < 4; ++k) {
            if (!corr_fits[k]) continue;
            long ctas = 0;
            for (int b = 0; b < nb; ++b)
                if (act[b]) ctas += (jobs[b].ms + jobs[b].md + corr_lcs[k] - 1) / corr_lcs[k];
            if (2 * ctas >= c->sm_count) return k;
        }
        return 3;
    };
    std::vector<double> resid(nb, 1.0), prev(nb, 1e300);
    std::vector<int> iters(nb, 0), active(nb, 1), stall(nb, 0), bits(nb, 0);
    const double tol = c->opts.ir_tol;
    PWQT_CUDA(c, cudaMemcpyAsync(active_d, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));

    // ---------------- the FP64-accurate residual on the tensor cores: self-energy panels
    // of this batch (slice tiles of Sigma_s, Sigma_d per energy), then per evaluation the
    // solution slices of the energies still refining and four slice-product launches
    const bool sliced = c->residual_kind == PWQT_RESIDUAL_SLICED;
    oz::GemmArgs OG{};
    if (sliced) {
        if (oz::gemm_init() != 0) return fail(c, PWQT_ERR_CUDA, "slice-product GEMM set-up failed");
        if (!c->ozM.p || !s.ozH.p) return fail(c, PWQT_ERR_STATE, "slice panels missing (mixed_prepare)");
        std::vector<const double2*> tab(2 * nb);
        for (int b = 0; b < nb; ++b) { tab[2 * b] = jobs[b].sig_s; tab[2 * b + 1] = jobs[b].sig_d; }
        PWQT_TRY(ensure(c, L.oz_sig_tab, sizeof(void*) * 2 * nb));
        PWQT_TRY(ensure(c, L.oz_sig, oz::panel_bytes(n, 2 * nb, 1)));
        PWQT_TRY(ensure(c, L.oz_sig_rexp, oz::rexp_bytes(n, 2 * nb)));
        PWQT_TRY(ensure(c, L.oz_B, oz::b_bytes(n, N, nb * m)));
        PWQT_TRY(ensure(c, L.oz_fexp, sizeof(int) * (size_t)oz::col_tiles(nb * m) * 32));
        PWQT_TRY(ensure(c, L.oz_act, sizeof(int) * nb));
        PWQT_CUDA(c, cudaMemcpyAsync(L.oz_sig_tab.p, tab.data(), sizeof(void*) * 2 * nb, cudaMemcpyHostToDevice, st));
        oz::PanelSrc P{};
        P.n = n; P.nseg = 1;
        P.tab[0] = L.oz_sig_tab.as<const double2*>();
        oz::build_panel(P, 2 * nb, L.oz_sig_rexp.as<int>(), L.oz_sig.as<__nv_bfloat16>(), st);
        c->launches += 2;
        OG.n = n; OG.N = N; OG.m = m; OG.n_pad = oz::padded(n);
        OG.B = L.oz_B.as<__nv_bfloat16>();
        OG.fexp = L.oz_fexp.as<int>();
        OG.act = L.oz_act.as<int>();
        OG.jobs = res_d;
        OG.R = S.R64;
        OG.sC = S.sC;
        OG.col_lo = 0;
        OG.col_hi = 1 << 30;
    } else if (sys_of) {
        for (int b = 1; b < nb; ++b)
            if (sys_of[b] != sys_of[0]) return fail(c, PWQT_ERR_INVALID_ARG, "a batch of several systems needs the sliced residual");
    }
    std::vector<int> act_h;
    auto residual = [&]() -> int {
        if (!sliced) {
            launch_residual_ff(RF, res_d, nb, m, active_d, st);   // energies still refining
            c->launches += 3;
            return PWQT_OK;
        }
        act_h.clear();
        for (int b = 0; b < nb; ++b)
            if (active[b]) act_h.push_back(b);
        const int n_act = (int)act_h.size();
        if (!n_act) return PWQT_OK;
        PWQT_CUDA(c, cudaMemcpyAsync(L.oz_act.p, act_h.data(), sizeof(int) * n_act, cudaMemcpyHostToDevice, st));
        oz::slice_solution(S.C64, S.sC, OG.act, n_act, n, N, m, L.oz_fexp.as<int>(), L.oz_B.as<__nv_bfloat16>(), st);
        OG.n_act = n_act;
        OG.nct = oz::col_tiles(n_act * m);
        if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.oz_ev[0], st));
        // r = b - E (M c): the shared M panel, one item per node
        OG.mode = oz::MODE_M; OG.A = c->ozM.as<__nv_bfloat16>(); OG.a_item_bytes = 0; OG.rexp = c->ozM_rexp.as<int>();
        oz::gemm(OG, N, st);
        // r += Sigma_s c_0 and Sigma_d c_{N-1}: one item per energy and contact
        OG.mode = oz::MODE_SIGMA; OG.A = L.oz_sig.as<__nv_bfloat16>(); OG.a_item_bytes = oz::panel_item_bytes(n, 1);
        OG.rexp = L.oz_sig_rexp.as<int>();
        for (int side = 0; side < 2; ++side) {
            OG.sigma_side = side;
            oz::gemm(OG, n_act, st);
        }
        // r += (HV c): one panel item per node, one launch per system over the columns
        // of its energies (consecutive in the active list)
        OG.mode = oz::MODE_HV; OG.a_item_bytes = oz::panel_item_bytes(n, 3);
        for (int k0 = 0; k0 < n_act;) {
            System& sk = sys_of ? *sys_of[act_h[k0]] : s;
            int k1 = k0 + 1;
            while (k1 < n_act && (sys_of ? sys_of[act_h[k1]] : &s) == &sk) ++k1;
            OG.A = sk.ozH.as<__nv_bfloat16>();
            OG.rexp = sk.ozH_rexp.as<int>();
            OG.col_lo = k0 * m;
            OG.col_hi = k1 * m;
            oz::gemm(OG, N, st);
            k0 = k1;
        }
        OG.col_lo = 0;
        OG.col_hi = 1 << 30;
        if (c->profile) {
            PWQT_CUDA(c, cudaEventRecord(L.oz_ev[1], st));
            // work of these launches: the method's complex MACs (3N - 2 block products and
            // the two self-energies per column) and the bf16 MMA flops of the kept pairs
            // (34 slice products of 128 x 32 x 16 per 16 real K and 32 columns)
            double cols = 0;
            for (int b : act_h) cols += jobs[b].ms + jobs[b].md;
            L.prof_oz_cmacs += (double)(3 * N) * n * (double)n * cols;
            const double kreal_nodes = 2.0 * (3 * N - 2) * 2 * oz::padded(n);   // M and HV launches
            double sig_tiles = 0;
            for (int k = 0; k < n_act; ++k) sig_tiles += (k * m + m - 1) / 32 - (k * m) / 32 + 1;
            const double rt = 2.0 * oz::padded(n) / 128;
            L.prof_oz_mma_flops += (kreal_nodes * OG.nct + 2.0 * sig_tiles * 2 * oz::padded(n)) * rt * 34.0 * 32 * 128 * 2;
            L.prof_oz_launches += 4;
        }
        oz::norms(S.R64, S.sC, res_d, OG.act, n_act, n, N, m, st);
        launch_residual_finish(res_d, nb, st, active_d);
        c->launches += 9;
        return PWQT_OK;
    };
    for (int it = 0;; ++it) {
        if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.ev[0], st));
        PWQT_CUDA(c, cudaMemsetAsync(res[0].rn2, 0, sizeof(double) * 2 * (size_t)nb * m, st));
        PWQT_TRY(residual());
        if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.ev[1], st));
        PWQT_CUDA(c, cudaMemcpyAsync(resid.data(), res[0].resid, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        PWQT_CUDA(c, cudaStreamSynchronize(st));
        if (c->profile) {
            float ms = 0;
            cudaEventElapsedTime(&ms, L.ev[0], L.ev[1]);
            L.prof_phase_ms[0] += ms;
            if (sliced && !act_h.empty()) {
                cudaEventElapsedTime(&ms, L.oz_ev[0], L.oz_ev[1]);
                L.prof_oz_ms += ms;
            }
            if (it > 0) {
                cudaEventElapsedTime(&ms, L.ev[2], L.ev[3]);
                L.prof_phase_ms[1] += ms;
            }
        }
        int any = 0;
        for (int b = 0; b < nb; ++b) {
            if (!active[b]) continue;
            if (!std::isfinite(resid[b])) {   // a non-finite solution is not refined further
                active[b] = 0;
                bits[b] |= PWQT_ST_IR_NO_CONVERGE;
                continue;
            }
            if (!refine || resid[b] <= tol) { active[b] = 0; continue; }   // PWQT_FP32: report, do not refine
            if (resid[b] > 0.5 * prev[b]) stall[b]++;
            else stall[b] = 0;
            // a residual that stops falling above ir_tol (the floor of the residual's own
            // accuracy, or a factorisation too poor to contract) ends refinement, flagged
            if (stall[b] >= 3 || iters[b] >= c->opts.ir_max_iters) {
                active[b] = 0;
                bits[b] |= PWQT_ST_IR_NO_CONVERGE;   // final residual above ir_tol
                continue;
            }
            prev[b] = std::min(prev[b], resid[b]);
            iters[b]++;
            any = 1;
        }
        if (!any) break;
        if (c->profile) {
            PWQT_CUDA(c, cudaEventRecord(L.ev[2], st));
            L.prof_ir_iters++;
        }
        PWQT_CUDA(c, cudaMemcpyAsync(active_d, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
        const int ck = corr_pick(active), lc = corr_lcs[ck];
        if (c->profile) {
            // the method's work: per refining column and node the products with L_i and X_i
            // and the two triangular solves, n^2 complex MACs each of the three
            double cols = 0;
            for (int b = 0; b < nb; ++b)
                if (active[b]) cols += jobs[b].ms + jobs[b].md;
            L.prof_corr_cmacs += 3.0 * N * (double)n * n * cols;
            L.prof_corr_launches += 1;
        }
        const dim3 cgrid(nb, (m + lc - 1) / lc);
        const size_t csm = correct_smem(n, lc);
        if (lc == 16) k_mx_correct<16><<<cgrid, CT, csm, st>>>(S, active_d, tmL, tmF, tmX);
        else if (lc == 8) k_mx_correct<8><<<cgrid, CT, csm, st>>>(S, active_d, tmL, tmF, tmX);
        else if (lc == 4) k_mx_correct<4><<<cgrid, CT, csm, st>>>(S, active_d, tmL, tmF, tmX);
        else k_mx_correct<2><<<cgrid, CT, csm, st>>>(S, active_d, tmL, tmF, tmX);
        c->launches++;
        if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.ev[3], st));
        PWQT_CUDA(c, cudaGetLastError());
    }
    if (sliced && oz::error_flag(true, st)) return fail(c, PWQT_ERR_TIMEOUT, "slice-product residual: a bounded mbarrier wait gave up");
    if (corr_error_flag(true, st)) return fail(c, PWQT_ERR_TIMEOUT, "correction solve: a bounded mbarrier wait gave up");
    PWQT_CUDA(c, cudaMemcpyAsync(iters_dev, iters.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    PWQT_CUDA(c, cudaMemcpyAsync(bits_d, bits.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    k_or_status<<<(nb + 127) / 128, 128, 0, st>>>(jobs_d, bits_d, nb);
    c->launches++;
    // observables read c from the FP64 solution
    for (int b = 0; b < nb; ++b) {
        obs[b].C = S.C64 + S.sC * b;
        obs[b].node_stride = (size_t)n * m;
        obs[b].row_stride = m;
    }
    PWQT_CUDA(c, cudaMemcpyAsync(obs_d, obs.data(), sizeof(ObsJob) * nb, cudaMemcpyHostToDevice, st));
    PWQT_CUDA(c, cudaStreamSynchronize(st));
    return PWQT_OK;
}

}  // namespace pwqt
