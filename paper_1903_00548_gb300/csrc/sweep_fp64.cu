// Complex128 block sweep of the QTBM system [E M - H - Sigma] c = B (Eq. qtbm_system,
// Sec. 3.2 of arXiv:1903.00548) for a batch of energies, one CTA per energy.
//
// Block forward elimination over the nodes i = 0..N-1 (D_i = E M0 - HV0_i,
// U_i = E M1 - HV1_i, L_{i+1} = U_i^H for real E, Sigma_s / Sigma_d on the end
// blocks):
//     S_i = D_i - L_i X_{i-1},   [X_i | y_i] = S_i^{-1} [U_i | b_i - L_i y_{i-1}]
// by Gaussian elimination with partial pivoting (pivot = max |re| + |im|), then back
// substitution c_{N-1} = y_{N-1}, c_i = y_i - X_i c_{i+1}.  FP64 throughout: on GB300
// the FP64 pipe (~1 TFLOP/s measured) is the bound, so each CTA streams its blocks
// through L2 with 32x32 shared-memory tiles for the products.
#include "pwqt_internal.cuh"
#include "sweep_common.cuh"

namespace pwqt {

constexpr int TS = 32, TK = 16, NT = 256;

// C[r][c] -= sum_k A(r,k) * B[k][c], r < M, c < Nc, k < K.  A is read through a functor,
// B and C are row-major with strides ldb / ldc.  256 threads, 32x32 output tiles, 2x2 per thread.
template <class AF, class CF>
__device__ void cta_gemm_sub(double2* smem, int M, int Nc, int K, AF A, const double2* __restrict__ B, int ldb, CF Cptr) {
    double2 (*As)[TK + 1] = reinterpret_cast<double2 (*)[TK + 1]>(smem);
    double2 (*Bs)[TS + 1] = reinterpret_cast<double2 (*)[TS + 1]>(smem + TS * (TK + 1));
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, each 2x2 outputs
    for (int r0 = 0; r0 < M; r0 += TS)
        for (int c0 = 0; c0 < Nc; c0 += TS) {
            double2 acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
            for (int k0 = 0; k0 < K; k0 += TK) {
                for (int t = threadIdx.x; t < TS * TK; t += NT) {
                    int rr = t / TK, kk = t % TK;
                    As[rr][kk] = (r0 + rr < M && k0 + kk < K) ? A(r0 + rr, k0 + kk) : make_double2(0, 0);
                    int kb = t / TS, cb = t % TS;
                    Bs[kb][cb] = (k0 + kb < K && c0 + cb < Nc) ? B[(size_t)(k0 + kb) * ldb + c0 + cb] : make_double2(0, 0);
                }
                __syncthreads();
#pragma unroll 4
                for (int kk = 0; kk < TK; ++kk) {
                    double2 a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
                    double2 b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
                    cfma(acc[0][0], a0, b0); cfma(acc[0][1], a0, b1);
                    cfma(acc[1][0], a1, b0); cfma(acc[1][1], a1, b1);
                }
                __syncthreads();
            }
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    int r = r0 + ty * 2 + i, cc = c0 + tx * 2 + j;
                    if (r < M && cc < Nc) {
                        double2* p = Cptr(r, cc);
                        *p = csub(*p, acc[i][j]);
                    }
                }
        }
}

// block-wide argmax of |re|+|im| over rows j..n-1 of column j of S (row stride lds)
__device__ int cta_pivot(const double2* S, int lds, int n, int j) {
    __shared__ double bv[NT / 32];
    __shared__ int bi[NT / 32];
    double best = -1.0;
    int idx = j;
    for (int r = j + threadIdx.x; r < n; r += NT) {
        double v = cabs1(S[(size_t)r * lds + j]);
        if (v > best) { best = v; idx = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffff, best, o);
        int oi = __shfl_down_sync(0xffffffff, idx, o);
        if (ov > best || (ov == best && oi < idx)) { best = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) { bv[0] = bv[w]; bi[0] = bi[w]; }
    }
    __syncthreads();
    int p = bi[0];
    __syncthreads();
    return p;
}

// -(2/pi) Im Tr of the n x n block at G (row stride ldg), block-wide; thread 0 gets it
__device__ double cta_dos(const double2* G, int ldg, int n) {
    __shared__ double part[NT / 32];
    double acc = 0.0;
    for (int r = threadIdx.x; r < n; r += NT) acc += G[(size_t)r * ldg + r].y;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffff, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += part[w];
    __syncthreads();
    return -(2.0 / 3.141592653589793) * t;
}

// Backward pass of the Green's-function recursion over the forward panels
// R_i = [X_i | g_i] (row stride 2n).  Per node, with the n x n scratch S:
//   S = -X_i G_{i+1};  X-part of R_i = -L_{i+1} g_i;  g-part of R_i -= (-S)(X-part)
// so that the g-part becomes g_i + (X_i G_{i+1})(L_{i+1} g_i) = G_i.
__device__ void green_backward(const SweepSys& sys, const SweepJob& J, double2* smem, int st) {
    const int n = sys.n, N = sys.N, w = 2 * n;
    const double E = J.E;
    double2* S = J.S;
    double d = cta_dos(J.XY + (size_t)(N - 1) * n * w + n, w, n);
    if (threadIdx.x == 0) J.dos[N - 1] = d;
    for (int i = N - 2; i >= 0; --i) {
        double2* R = J.XY + (size_t)i * n * w;
        const double2* Gn = J.XY + (size_t)(i + 1) * n * w + n;
        for (int t = threadIdx.x; t < n * n; t += NT) S[t] = make_double2(0, 0);
        __syncthreads();
        {
            auto A = [&](int r, int k) { return R[(size_t)r * w + k]; };
            auto C = [&](int r, int cc) -> double2* { return S + (size_t)r * n + cc; };
            cta_gemm_sub(smem, n, n, n, A, Gn, w, C);                 // S = -X_i G_{i+1}
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += NT) R[(size_t)(t / n) * w + t % n] = make_double2(0, 0);
        __syncthreads();
        {
            const double2* HV1 = (J.HV1 ? J.HV1 : sys.HV1) + (size_t)i * n * n;
            const double2* M1 = sys.M1;
            auto A = [&](int r, int k) {                               // L_{i+1}[r][k] = conj(U_i[k][r])
                size_t t = (size_t)k * n + r;
                return cconj(csub(cscale(M1[t], E), HV1[t]));
            };
            auto C = [&](int r, int cc) -> double2* { return R + (size_t)r * w + cc; };
            cta_gemm_sub(smem, n, n, n, A, R + n, w, C);             // X-part = -L_{i+1} g_i
        }
        __syncthreads();
        {
            auto A = [&](int r, int k) { const double2 v = S[(size_t)r * n + k]; return make_double2(-v.x, -v.y); };
            auto C = [&](int r, int cc) -> double2* { return R + (size_t)r * w + n + cc; };
            cta_gemm_sub(smem, n, n, n, A, R, w, C);                 // g-part -= (X_i G_{i+1})(-L_{i+1} g_i)
        }
        __syncthreads();
        d = cta_dos(R + n, w, n);
        if (threadIdx.x == 0) J.dos[i] = d;
    }
    if (threadIdx.x == 0) atomicOr(J.status, st);
}

// GREEN = false: the QTBM solve of the file header.  GREEN = true: the recursive Green's-function
// form of the same elimination (the NEGF side of Sec. 3.2).  The forward pass is the
// sweep with [U_i | I] as every node's right-hand side and no coupling between the
// right-hand sides of neighbouring nodes, so that R_i = [X_i | g_i] with the
// left-connected g_i = S_i^{-1}; the backward pass then forms the diagonal blocks
//     G_{N-1} = g_{N-1},   G_i = g_i + (X_i G_{i+1}) (L_{i+1} g_i)
// in place of g_i, with L_{i+1} = U_i^H, and records -(2/pi) Im Tr G_i.
template <bool GREEN>
__global__ void __launch_bounds__(NT) k_sweep_fp64(SweepSys sys, const SweepJob* __restrict__ jobs) {
    const SweepJob J = jobs[blockIdx.x];
    const int n = sys.n, N = sys.N, m = J.ms + J.md, w = n + m;
    const double E = J.E;
    double2* S = J.S;
    // shared: GEMM tiles, reused as the multiplier column of the elimination (n <= 1024)
    __shared__ double2 smem[TS * (TK + 1) + TK * (TS + 1) > 1024 ? TS * (TK + 1) + TK * (TS + 1) : 1024];
    double2* lcol = smem;
    int st = 0;
    for (int i = 0; i < N; ++i) {
        double2* R = J.XY + (size_t)i * n * w;
        const double2* HV0 = (J.HV0 ? J.HV0 : sys.HV0) + (size_t)i * n * n;
        const double2* HV1 = (J.HV1 ? J.HV1 : sys.HV1) + (size_t)i * n * n;
        for (int t = threadIdx.x; t < n * n; t += NT) {
            double2 v = csub(cscale(sys.M0[t], E), HV0[t]);
            if (i == 0 && J.sig_s) v = csub(v, J.sig_s[t]);
            if (i == N - 1 && J.sig_d) v = csub(v, J.sig_d[t]);
            S[t] = v;
        }
        for (int t = threadIdx.x; t < n * w; t += NT) {
            int r = t / w, cc = t % w;
            double2 v = make_double2(0, 0);
            if (cc < n) {
                if (i < N - 1) v = csub(cscale(sys.M1[(size_t)r * n + cc], E), HV1[(size_t)r * n + cc]);
            } else if (GREEN) {
                if (cc - n == r) v = make_double2(1.0, 0.0);
            } else {
                int col = cc - n;
                if (i == 0 && col < J.ms) v = J.rhs_s[(size_t)r * J.ms + col];
                if (i == N - 1 && col >= J.ms) v = J.rhs_d[(size_t)r * J.md + (col - J.ms)];
            }
            R[t] = v;
        }
        __syncthreads();
        if (i > 0) {
            const double2* P = J.XY + (size_t)(i - 1) * n * w;   // [X_{i-1} | y_{i-1}]
            const double2* HVp = (J.HV1 ? J.HV1 : sys.HV1) + (size_t)(i - 1) * n * n;
            const double2* M1 = sys.M1;
            // L_i[r][k] = conj(U_{i-1}[k][r]), U_{i-1} = E M1 - HV1_{i-1}
            auto A = [&](int r, int k) {
                size_t t = (size_t)k * n + r;
                return cconj(csub(cscale(M1[t], E), HVp[t]));
            };
            auto C = [&](int r, int cc) -> double2* { return cc < n ? S + (size_t)r * n + cc : R + (size_t)r * w + cc; };
            // [S | *, y] -= L_i [X_{i-1} | y_{i-1}]  (cols n..w-1 of R); S alone for GREEN
            cta_gemm_sub(smem, n, GREEN ? n : w, n, A, P, w, C);
            __syncthreads();
        }
        // Gaussian elimination with partial pivoting on S, applied to the rows of R
        for (int j = 0; j < n; ++j) {
            int p = cta_pivot(S, n, n, j);
            if (p != j) {
                for (int cc = threadIdx.x; cc < n; cc += NT) {
                    double2 a = S[(size_t)j * n + cc]; S[(size_t)j * n + cc] = S[(size_t)p * n + cc]; S[(size_t)p * n + cc] = a;
                }
                for (int cc = threadIdx.x; cc < w; cc += NT) {
                    double2 a = R[(size_t)j * w + cc]; R[(size_t)j * w + cc] = R[(size_t)p * w + cc]; R[(size_t)p * w + cc] = a;
                }
            }
            __syncthreads();
            double2 piv = S[(size_t)j * n + j];
            if (piv.x == 0.0 && piv.y == 0.0) { st |= PWQT_ST_SINGULAR_PIVOT; piv = make_double2(1.0, 0.0); }
            for (int r = j + 1 + threadIdx.x; r < n; r += NT) lcol[r] = cdiv(S[(size_t)r * n + j], piv);
            __syncthreads();
            const int rows = n - j - 1, cs = n - j - 1, cols = cs + w;
            for (long t = threadIdx.x; t < (long)rows * cols; t += NT) {
                int r = j + 1 + (int)(t / cols), cc = (int)(t % cols);
                double2 l = lcol[r];
                if (cc < cs) {
                    int col = j + 1 + cc;
                    cfma(S[(size_t)r * n + col], make_double2(-l.x, -l.y), S[(size_t)j * n + col]);
                } else {
                    int col = cc - cs;
                    cfma(R[(size_t)r * w + col], make_double2(-l.x, -l.y), R[(size_t)j * w + col]);
                }
            }
            __syncthreads();
        }
        // back substitution with the upper triangle
        for (int j = n - 1; j >= 0; --j) {
            double2 d = S[(size_t)j * n + j];
            if (d.x == 0.0 && d.y == 0.0) d = make_double2(1.0, 0.0);
            for (int cc = threadIdx.x; cc < w; cc += NT) R[(size_t)j * w + cc] = cdiv(R[(size_t)j * w + cc], d);
            __syncthreads();
            for (long t = threadIdx.x; t < (long)j * w; t += NT) {
                int r = (int)(t / w), cc = (int)(t % w);
                double2 s = S[(size_t)r * n + j];
                cfma(R[(size_t)r * w + cc], make_double2(-s.x, -s.y), R[(size_t)j * w + cc]);
            }
            __syncthreads();
        }
    }
    if constexpr (GREEN) {
        green_backward(sys, J, smem, st);
    } else {
        // back substitution over nodes: c_i = y_i - X_i c_{i+1} (c overwrites y)
        for (int i = N - 2; i >= 0; --i) {
            double2* R = J.XY + (size_t)i * n * w;
            const double2* Cn = J.XY + (size_t)(i + 1) * n * w + n;
            auto A = [&](int r, int k) { return R[(size_t)r * w + k]; };
            auto C = [&](int r, int cc) -> double2* { return R + (size_t)r * w + n + cc; };
            cta_gemm_sub(smem, n, m, n, A, Cn, w, C);
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicOr(J.status, st);
    }
}

void launch_sweep_fp64(const SweepSys& sys, const SweepJob* jobs, int nb, cudaStream_t st) {
    k_sweep_fp64<false><<<nb, NT, 0, st>>>(sys, jobs);
}

void launch_green_fp64(const SweepSys& sys, const SweepJob* jobs, int nb, cudaStream_t st) {
    k_sweep_fp64<true><<<nb, NT, 0, st>>>(sys, jobs);
}

}  // namespace pwqt
