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

struct MixSys {
    int n, N, m, w;                       // w = n + m (uniform m over the batch)
    const double2* M0; const double2* M1; const double2* HV0; const double2* HV1;   // FP64 blocks
    const float2* M1f; const float2* HV1f;                                         // complex64 copies
    float2* F; long long sF;              // per energy N x n x n factors
    int* piv; long long sP;               // per energy N x n pivot rows
    float2* XY; long long sXY;            // per energy N x n x w
    float2* Lb; long long sL;             // per energy n x n
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
__global__ void k_mx_form(MixSys S, int i, int only_L) {
    const int e = blockIdx.y;
    const SweepJob& J = S.jobs[e];
    const int n = S.n, N = S.N, w = S.w, ms = J.ms, md = J.md;
    const double E = J.E;
    float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    float2* Lb = S.Lb + e * S.sL;
    const double2* HV0b = J.HV0 ? J.HV0 : S.HV0;
    const double2* HV1b = J.HV1 ? J.HV1 : S.HV1;
    const double2* HV0 = HV0b + (size_t)i * n * n;
    const double2* HV1 = HV1b + (size_t)i * n * n;
    const double2* HVm = HV1b + (size_t)(i > 0 ? i - 1 : 0) * n * n;
    const size_t nn = (size_t)n * n;
    if (only_L) {
        for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
            int r = (int)(t / n), c = (int)(t % n);
            size_t tt = (size_t)c * n + r;
            Lb[t] = to32(cconj(csub(cscale(S.M1[tt], E), HVm[tt])));
        }
        return;
    }
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
    const size_t nm = (size_t)n * S.m;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nm; t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t / S.m), g = (int)(t % S.m);
        float2 v = make_float2(0.f, 0.f);
        if (i == 0 && g < ms) v = to32(J.rhs_s[(size_t)r * ms + g]);
        if (i == N - 1 && g >= ms && g < ms + md) v = to32(J.rhs_d[(size_t)r * md + (g - ms)]);
        XY[(size_t)r * w + n + g] = v;
    }
}

// ---------------------------------------------------------------- panel factorisation
// Factor F_i[k0:n, k0:k0+wd] with partial pivoting (max |re|+|im|), apply the row
// interchanges to the remaining columns of F_i and to XY_i, and solve the unit-lower
// 32 x 32 block against the strip rows k0..k0+wd of [F_i right of the panel | XY_i].
__global__ void __launch_bounds__(NT) k_mx_panel(MixSys S, int i, int k0, int wd) {
    // the panel, column-major with an odd leading dimension: threads walk rows of one
    // column (consecutive words) in the elimination and columns of one row (odd stride,
    // distinct banks) when it is loaded and stored
    extern __shared__ float2 P[];                     // PW columns x pld rows
    __shared__ int prow[PW];
    __shared__ float bv[NT / 32];
    __shared__ int bi[NT / 32];
    const int e = blockIdx.x;
    const int n = S.n, w = S.w, rows = n - k0, pld = rows | 1;   // panel leading dimension (odd)
    float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
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
    // row interchanges on the other columns of F_i and on XY_i: the wd swaps in order
    // compose to a permutation of at most 2 wd panel rows, moved as one gather per
    // column (all loads of a column issued before its stores)
    __shared__ int mv_dst[2 * PW], mv_src[2 * PW], mv_cnt;
    if (threadIdx.x == 0) {
        int pos[2 * PW], cur[2 * PW], cnt = 0;   // panel rows touched and the original row now there
        auto slot = [&](int r) {
            for (int q = 0; q < cnt; ++q)
                if (pos[q] == r) return q;
            pos[cnt] = r;
            cur[cnt] = r;
            return cnt++;
        };
        for (int j = 0; j < wd; ++j) {
            const int p = prow[j];
            if (p == j) continue;
            const int a = slot(j), b = slot(p);
            const int x = cur[a];
            cur[a] = cur[b];
            cur[b] = x;
        }
        int k = 0;
        for (int q = 0; q < cnt; ++q)
            if (cur[q] != pos[q]) { mv_dst[k] = pos[q]; mv_src[k] = cur[q]; ++k; }
        mv_cnt = k;
    }
    __syncthreads();
    const int nmv = mv_cnt;
    const int ncolF = n - wd;
    for (int c = threadIdx.x; c < ncolF + w; c += NT) {
        float2* base;
        size_t ld;
        if (c < ncolF) { base = F + (c < k0 ? c : c + wd); ld = n; }
        else { base = XY + (c - ncolF); ld = w; }
        base += (size_t)k0 * ld;
        float2 v[2 * PW];
#pragma unroll
        for (int q = 0; q < 2 * PW; ++q)
            if (q < nmv) v[q] = base[(size_t)mv_src[q] * ld];
#pragma unroll
        for (int q = 0; q < 2 * PW; ++q)
            if (q < nmv) base[(size_t)mv_dst[q] * ld] = v[q];
    }
    __syncthreads();
    // strip: rows k0..k0+wd of [F cols k0+wd..n | XY] <- L11^{-1} strip (unit lower)
    const int right = n - k0 - wd;
    for (int c = threadIdx.x; c < right + w; c += NT) {
        float2 x[PW];
        float2* base;
        size_t ld;
        if (c < right) { base = F + (size_t)k0 * n + k0 + wd + c; ld = n; }
        else { base = XY + (size_t)k0 * w + (c - right); ld = w; }
#pragma unroll
        for (int j = 0; j < PW; ++j) x[j] = j < wd ? base[(size_t)j * ld] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j < PW; ++j) {
            if (j < wd) {
                float2 s = x[j];
#pragma unroll
                for (int l = 0; l < PW; ++l)
                    if (l < j) {
                        float2 L = P[l * pld + j];
                        ffma(s, make_float2(-L.x, -L.y), x[l]);
                    }
                x[j] = s;
            }
        }
#pragma unroll
        for (int j = 0; j < PW; ++j)
            if (j < wd) base[(size_t)j * ld] = x[j];
    }
    if (threadIdx.x == 0 && st) atomicOr(S.jobs[e].status, st);
}

// XY_i[k0:k0+wd, :] <- U11^{-1} XY_i[k0:k0+wd, :]
__global__ void __launch_bounds__(NT) k_mx_trsm_up(MixSys S, int i, int k0, int wd) {
    __shared__ float2 U[PW][PW + 1];
    const int e = blockIdx.x;
    const int n = S.n, w = S.w;
    const float2* F = S.F + e * S.sF + (size_t)i * n * n;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    for (int t = threadIdx.x; t < PW * PW; t += NT) {
        int r = t / PW, c = t % PW;
        U[r][c] = (r < wd && c < wd) ? F[(size_t)(k0 + r) * n + k0 + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += NT) {
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
// d = A^{-1} r with the stored complex64 factors; the y columns of XY_i hold the work
// vectors.  Per node (all energies at once):  w_i = r_i - L_i w_{i-1}  (tensor cores),
// w_i <- U_i^{-1} L_i^{-1} P_i w_i (k_mx_lusolve); then d_i = w_i - X_i d_{i+1}
// (tensor cores) from the last node back, and c += d in FP64.

// w_i = (complex64) r_i   (active energies)
__global__ void k_mx_load_r(MixSys S, int i, const int* __restrict__ active) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    const int n = S.n, w = S.w, m = S.m;
    float2* XY = S.XY + e * S.sXY + (size_t)i * n * w;
    const double2* R = S.R64 + e * S.sC + (size_t)i * n * m;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * m; t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t / m), g = (int)(t % m);
        XY[(size_t)r * w + n + g] = to32(R[t]);
    }
}

// w <- U^{-1} L^{-1} P w for node i.  The m right-hand sides are independent, so
// every energy gets ceil(m / LC) CTAs of LC columns each; a CTA keeps its columns
// in shared memory (n x LC), solves each 32-row diagonal block with one warp per
// LC / 8 columns (lane = row, the solved value broadcast by shuffle) and applies the
// off-diagonal part of the factors to the rows below (forward) or above
// (backward) in parallel over (row, column).  The solve is latency-bound (a chain
// of 2 n / 32 block steps per CTA), so LC is small: at n = 512 a CTA holds ~59 KB
// of shared memory, three fit on an SM, and a node's launch is one wave of
// ceil(m / 8) CTAs per energy.
constexpr int LC = 8;
constexpr int LCW = LC / (NT / 32);   // columns per warp in the diagonal-block solves
static_assert(LC % (NT / 32) == 0, "every warp takes the same number of columns");

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

constexpr int LR = 64;    // factor rows staged per chunk of the off-diagonal updates
constexpr int LDS = 34;   // padded row of a staged chunk (272 B: 16-byte aligned rows, conflict-free reads)
constexpr int NSTG = 4;   // chunks in flight per CTA

size_t lusolve_smem(int n) {
    return ((n * sizeof(int) + 15) / 16) * 16 + sizeof(float2) * (PW * (PW + 1) + (size_t)NSTG * LR * LDS + (size_t)n * LC);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(d), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// T[r][:] -= F[r][kb .. kb+wd) T[kb .. kb+wd)[:] for rows r in [r_begin, r_end).  One CTA per
// (energy, column group) streams about n^2 / 2 factor elements per triangle through L2, so
// the chunks (LR rows x 32 columns, one 16-byte cp.async per two elements, rows and
// columns past the factor zero-filled) are fetched NSTG - 1 ahead into a shared-memory ring.
__device__ __forceinline__ void lu_offdiag(const float2* __restrict__ F, int n, int kb, int wd, int r_begin, int r_end,
                                           float2* Fs, float2* T) {
    const int t = threadIdx.x;
    const int nch = (r_end - r_begin + LR - 1) / LR;
    auto fetch = [&](int ch) {
        if (ch < nch) {
            float2* dst = Fs + (size_t)(ch % NSTG) * LR * LDS;
            const int rc = r_begin + ch * LR;
            for (int q = t; q < LR * (PW / 2); q += NT) {     // 16-byte pieces: row rr, columns 2l, 2l + 1
                const int rr = q / (PW / 2), l2 = 2 * (q % (PW / 2));
                const bool in = rc + rr < r_end && l2 < wd;
                const float2* src = in ? F + (size_t)(rc + rr) * n + kb + l2 : F;
                cp_async16(dst + rr * LDS + l2, src, in ? (l2 + 1 < wd ? 16 : 8) : 0);
            }
        }
        cp_async_commit();   // an empty group past the end keeps the wait count uniform
    };
    for (int ch = 0; ch < NSTG - 1; ++ch) fetch(ch);
    // thread t updates column g = t % LC of rows r0 and r0 + LR / 2 of every chunk; the
    // solved block rows kb .. kb + wd of its column stay in registers for the whole call
    static_assert(NT / LC * 2 == LR, "two rows per thread and chunk");
    const int g = t % LC, r0 = t / LC;
    float2 tk[PW];
#pragma unroll
    for (int l = 0; l < PW; ++l) tk[l] = l < wd ? T[(kb + l) * LC + g] : make_float2(0.f, 0.f);
    for (int ch = 0; ch < nch; ++ch) {
        cp_async_wait<NSTG - 2>();
        __syncthreads();                    // chunk ch landed for every thread; chunk ch - 1 consumed
        fetch(ch + NSTG - 1);
        const float2* Fc = Fs + (size_t)(ch % NSTG) * LR * LDS;
        const int rc = r_begin + ch * LR, rows = min(LR, r_end - rc);
        const bool in0 = r0 < rows, in1 = r0 + LR / 2 < rows;
        float2 a0 = in0 ? T[(rc + r0) * LC + g] : make_float2(0.f, 0.f);
        float2 a1 = in1 ? T[(rc + r0 + LR / 2) * LC + g] : make_float2(0.f, 0.f);
        const float2* L0 = Fc + r0 * LDS;
        const float2* L1 = Fc + (r0 + LR / 2) * LDS;
#pragma unroll
        for (int l = 0; l < PW; ++l) {      // zero-filled past wd: those terms vanish
            const float2 x0 = L0[l], x1 = L1[l];
            ffma(a0, make_float2(-x0.x, -x0.y), tk[l]);
            ffma(a1, make_float2(-x1.x, -x1.y), tk[l]);
        }
        if (in0) T[(rc + r0) * LC + g] = a0;
        if (in1) T[(rc + r0 + LR / 2) * LC + g] = a1;
    }
    cp_async_wait<0>();
    __syncthreads();
}

__global__ void __launch_bounds__(NT) k_mx_lusolve(MixSys S, int i, const int* __restrict__ active) {
    const int e = blockIdx.x;
    if (!active[e]) return;
    const SweepJob& J = S.jobs[e];
    const int n = S.n, w = S.w, m = J.ms + J.md;
    const int c0 = blockIdx.y * LC;
    if (c0 >= m) return;
    extern __shared__ unsigned char sm[];
    int* perm = reinterpret_cast<int*>(sm);                                              // n
    float2* Ld = reinterpret_cast<float2*>(sm + ((n * sizeof(int) + 15) / 16) * 16);     // PW x (PW+1)
    float2* Fs = Ld + PW * (PW + 1);                                                     // NSTG x LR x LDS
    float2* T = Fs + NSTG * LR * LDS;                                                    // n x LC
    const float2* F = S.F + e * S.sF + (size_t)i * n * n;
    const int* pg = S.piv + e * S.sP + (size_t)i * n;        // row permutation (k_mx_perm)
    float2* W = S.XY + e * S.sXY + (size_t)i * n * w + n;     // row stride w
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int j = t; j < n; j += NT) perm[j] = pg[j];
    __syncthreads();
#pragma unroll 8
    for (int q = t; q < n * LC; q += NT) {
        const int r = q / LC, g = q % LC;
        T[q] = c0 + g < m ? W[(size_t)perm[r] * w + c0 + g] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // forward substitution, unit lower factor
    for (int kb = 0; kb < n; kb += PW) {
        const int wd = min(PW, n - kb);
        {
            float2 v[PW * PW / NT];
#pragma unroll
            for (int u = 0; u < PW * PW / NT; ++u) {
                const int q = t + u * NT, r = q / PW, c = q % PW;
                v[u] = (r < wd && c < wd) ? F[(size_t)(kb + r) * n + kb + c] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < PW * PW / NT; ++u) {
                const int q = t + u * NT;
                Ld[(q / PW) * (PW + 1) + q % PW] = v[u];
            }
        }
        __syncthreads();
        for (int cc = LCW * warp; cc < LCW * (warp + 1); ++cc) {
            float2 v = lane < wd ? T[(kb + lane) * LC + cc] : make_float2(0.f, 0.f);
            for (int j = 0; j + 1 < wd; ++j) {
                const float2 aj = shfl2(v, j);
                if (lane > j) {
                    const float2 L = Ld[lane * (PW + 1) + j];
                    ffma(v, make_float2(-L.x, -L.y), aj);
                }
            }
            if (lane < wd) T[(kb + lane) * LC + cc] = v;
        }
        __syncthreads();
        lu_offdiag(F, n, kb, wd, kb + wd, n, Fs, T);
    }
    // backward substitution, upper factor with its diagonal
    for (int kb = ((n - 1) / PW) * PW; kb >= 0; kb -= PW) {
        const int wd = min(PW, n - kb);
        {
            float2 v[PW * PW / NT];
#pragma unroll
            for (int u = 0; u < PW * PW / NT; ++u) {
                const int q = t + u * NT, r = q / PW, c = q % PW;
                v[u] = (r < wd && c < wd) ? F[(size_t)(kb + r) * n + kb + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < PW * PW / NT; ++u) {
                const int q = t + u * NT;
                Ld[(q / PW) * (PW + 1) + q % PW] = v[u];
            }
        }
        __syncthreads();
        for (int cc = LCW * warp; cc < LCW * (warp + 1); ++cc) {
            float2 v = lane < wd ? T[(kb + lane) * LC + cc] : make_float2(0.f, 0.f);
            for (int j = wd - 1; j >= 0; --j) {
                if (lane == j) {
                    float2 d = Ld[j * (PW + 1) + j];
                    if (d.x == 0.f && d.y == 0.f) d = make_float2(1.f, 0.f);
                    v = fdiv(v, d);
                }
                const float2 aj = shfl2(v, j);
                if (lane < j) {
                    const float2 U = Ld[lane * (PW + 1) + j];
                    ffma(v, make_float2(-U.x, -U.y), aj);
                }
            }
            if (lane < wd) T[(kb + lane) * LC + cc] = v;
        }
        __syncthreads();
        lu_offdiag(F, n, kb, wd, 0, kb, Fs, T);
    }
    for (int q = t; q < n * LC; q += NT) {
        const int r = q / LC, g = q % LC;
        if (c0 + g < m) W[(size_t)r * w + c0 + g] = T[q];
    }
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

// c += d (FP64), active energies
__global__ void k_mx_update(MixSys S, const int* __restrict__ active) {
    const int e = blockIdx.y;
    if (!active[e]) return;
    const int n = S.n, N = S.N, m = S.m, w = S.w;
    const size_t tot = (size_t)N * n * m;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        size_t i = t / ((size_t)n * m), rem = t % ((size_t)n * m);
        int r = (int)(rem / m), g = (int)(rem % m);
        float2 d = S.XY[e * S.sXY + i * n * w + (size_t)r * w + n + g];
        double2& c = S.C64[e * S.sC + t];
        c.x += d.x;
        c.y += d.y;
    }
}

__global__ void k_or_status(const SweepJob* __restrict__ jobs, const int* __restrict__ bits, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && bits[b]) atomicOr(jobs[b].status, bits[b]);
}

}  // namespace

size_t mixed_bytes_per_energy(int n, int N, int m) {
    // F + XY (complex64) + pivots + L scratch + FP64 solution and residual
    return sizeof(float2) * ((size_t)N * n * n + (size_t)N * n * (n + m) + (size_t)n * std::max(n, m)) + sizeof(int) * (size_t)N * n +
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
    int m = 0;
    for (int b = 0; b < nb; ++b) m = std::max(m, jobs[b].ms + jobs[b].md);
    m = std::max(m, 1);
    const int w = n + m;
    MixSys S;
    S.n = n; S.N = N; S.m = m; S.w = w;
    S.M0 = sys.M0; S.M1 = sys.M1; S.HV0 = sys.HV0; S.HV1 = sys.HV1;
    S.M1f = c->M1f.as<float2>(); S.HV1f = s.HV1f.as<float2>();
    S.sF = (long long)N * n * n;
    S.sP = (long long)N * n;
    S.sXY = (long long)N * n * w;
    S.sL = (long long)n * std::max(n, m);   // L_i (n x n), reused as the n x m correction scratch
    S.sC = (long long)N * n * m;
    const size_t bytes = mixed_bytes_per_energy(n, N, m) * nb + 1024 * 4;
    PWQT_TRY(ensure(c, L.ws_mixed, bytes));
    char* base = L.ws_mixed.as<char>();
    auto take = [&](size_t b) { char* p = base; base += (b + 255) / 256 * 256; return p; };
    S.F = (float2*)take(sizeof(float2) * S.sF * nb);
    S.XY = (float2*)take(sizeof(float2) * S.sXY * nb);
    S.Lb = (float2*)take(sizeof(float2) * S.sL * nb);
    S.piv = (int*)take(sizeof(int) * S.sP * nb);
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
    cudaFuncAttributes fa_panel{}, fa_lus{};
    PWQT_CUDA(c, cudaFuncGetAttributes(&fa_panel, k_mx_panel));
    PWQT_CUDA(c, cudaFuncGetAttributes(&fa_lus, k_mx_lusolve));
    // the opt-in maximum counts static and dynamic shared memory together
    const int dyn_panel = smem_optin - (int)fa_panel.sharedSizeBytes, dyn_lus = smem_optin - (int)fa_lus.sharedSizeBytes;
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
        k_mx_form<<<dim3(fblocks, nb), NT, 0, st>>>(S, i, 0);
        c->launches++;
        if (i > 0) {
            const float2* XYp = S.XY + (size_t)(i - 1) * n * w;
            gemm(S.Lb, S.sL, n, XYp, S.sXY, w, XYp + n, S.sXY, w, Fi, S.sF, n, XYi + n, S.sXY, w, n, n, w, n);
        }
        for (int k0 = 0; k0 < n; k0 += PW) {
            const int wd = std::min(PW, n - k0);
            k_mx_panel<<<nb, NT, sizeof(float2) * (size_t)((n - k0) | 1) * PW, st>>>(S, i, k0, wd);
            c->launches++;
            const int rest = n - k0 - wd;
            if (rest > 0)
                gemm(Fi + (size_t)(k0 + wd) * n + k0, S.sF, n, Fi + (size_t)k0 * n + k0 + wd, S.sF, n, XYi + (size_t)k0 * w, S.sXY, w,
                     Fi + (size_t)(k0 + wd) * n + k0 + wd, S.sF, n, XYi + (size_t)(k0 + wd) * w, S.sXY, w, rest, rest, rest + w, wd);
        }
        for (int k0 = ((n - 1) / PW) * PW; k0 >= 0; k0 -= PW) {
            const int wd = std::min(PW, n - k0);
            k_mx_trsm_up<<<nb, NT, 0, st>>>(S, i, k0, wd);
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
    c->launches += 2;

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
    const size_t lus_smem = lusolve_smem(n);
    if (lus_smem > (size_t)dyn_lus) return fail(c, PWQT_ERR_INVALID_ARG, "correction solve exceeds shared memory");
    PWQT_CUDA(c, cudaFuncSetAttribute(k_mx_lusolve, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_lus));
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
        for (int i = 0; i < N; ++i) {
            float2* XYi = S.XY + (size_t)i * n * w;
            k_mx_load_r<<<dim3(64, nb), NT, 0, st>>>(S, i, active_d);
            c->launches++;
            if (i > 0) {
                k_mx_form<<<dim3(fblocks, nb), NT, 0, st>>>(S, i, 1);
                const float2* XYp = S.XY + (size_t)(i - 1) * n * w;
                gemm(S.Lb, S.sL, n, XYp + n, S.sXY, w, XYp + n, S.sXY, w, XYi + n, S.sXY, w, XYi + n, S.sXY, w, m, n, m, n);
                c->launches++;
            }
            k_mx_lusolve<<<dim3(nb, (m + LC - 1) / LC), NT, lus_smem, st>>>(S, i, active_d);
            c->launches++;
        }
        for (int i = N - 2; i >= 0; --i) {
            float2* XYi = S.XY + (size_t)i * n * w;
            const float2* XYn = S.XY + (size_t)(i + 1) * n * w;
            gemm(XYi, S.sXY, w, XYn + n, S.sXY, w, XYn + n, S.sXY, w, XYi + n, S.sXY, w, XYi + n, S.sXY, w, m, n, m, n);
        }
        k_mx_update<<<dim3(256, nb), NT, 0, st>>>(S, active_d);
        c->launches++;
        if (c->profile) PWQT_CUDA(c, cudaEventRecord(L.ev[3], st));
        PWQT_CUDA(c, cudaGetLastError());
    }
    if (sliced && oz::error_flag(true, st)) return fail(c, PWQT_ERR_TIMEOUT, "slice-product residual: a bounded mbarrier wait gave up");
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
