// Batched complex GEMM  C[b] -= A[b] * B[b]  on the 5th-generation tensor cores
// (tcgen05.mma, kind::tf32, FP32 accumulators in tensor memory), sm_103a.
//
// Complex arithmetic by real expansion: with A stored interleaved (re, im) it is
// already the real M x 2K matrix [A_r A_i] (interleaved along K); B is expanded
// while staging into the real 2K x 2N matrix whose 2x2 blocks are
// [[B_r, B_i], [-B_i, B_r]], so the real product lands interleaved as [C_r C_i].
// Each real operand is split x = x_hi + x_lo (x_hi rounded to TF32), and
// A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 ("3xTF32"): the block
// sweep needs FP32-level accuracy, single-pass TF32 does not converge under
// refinement for these ill-conditioned systems.
//
// Tile: 128 rows x 128 complex columns (256 real accumulator columns = 256 TMEM
// columns), K staged 32 complex (64 real) at a time in shared memory, operands
// in the canonical K-major no-swizzle layout (8-row x 16-byte core matrices).
// One thread issues the MMAs and commits them to an mbarrier.  The tensor cores'
// FP32 accumulation truncates, so each 32-complex K stage starts a fresh TMEM
// accumulation and the eight warps add the stage result into FP32 registers
// (round to nearest): truncation then accrues over one stage (24 MMAs), not all
// of K.  Warps w and w + 4 read TMEM lanes 32 (w % 4).. and hold 128 columns each.
#include <cstdint>

#include "cgemm_tc.cuh"
#include "pwqt_internal.cuh"

namespace pwqt {

namespace {
constexpr int BM = 128;            // rows per tile
constexpr int BNC = 128;           // complex columns per tile
constexpr int BKC = 32;            // complex K per stage
constexpr int BNR = 2 * BNC;       // 256 real accumulator columns
constexpr int BKR = 2 * BKC;       // 64 real K per stage
constexpr int THREADS = 256;       // warps w and w+4 share TMEM lanes 32(w%4).. (column halves)
constexpr uint32_t CORE_BYTES = 128;                 // 8 rows x 16 bytes
constexpr uint32_t LBO = CORE_BYTES;                 // next 16-byte chunk along K
constexpr uint32_t SBO = (BKR * 4 / 16) * CORE_BYTES;   // next 8-row group: 16 chunks x 128 B = 2048 B
constexpr uint32_t A_BYTES = BM * BKR * 4;           // 32 KB
constexpr uint32_t B_BYTES = BNR * BKR * 4;          // 64 KB
constexpr uint32_t SMEM_BYTES = 2 * A_BYTES + 2 * B_BYTES + 64;
static_assert(sizeof(float) * BM * (BNR + 1) <= 2 * A_BYTES + 2 * B_BYTES, "epilogue tile fits the stage buffers");
constexpr uint32_t TMEM_COLS = 256;
constexpr long long SPIN_LIMIT = 1ll << 22;   // bounded mbarrier polling (each poll returns within microseconds)

__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of real element (row, k) inside a K-major core-matrix tile
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(k >> 2) * LBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// round-to-nearest TF32 (10 explicit mantissa bits) and the FP32 remainder
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);            // start address
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;        // leading (K) byte offset
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;        // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;                            // descriptor version (sm_100 family)
    // base offset 0, lbo mode 0, layout type 0 = no swizzle
    return d;
}

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BNR >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accum));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (long long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(phase));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__global__ void __launch_bounds__(THREADS, 1)
k_cgemm_tc(const CGemmArgs G, int M, int N, int K) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + A_BYTES;
    unsigned char* b_hi = smem + 2 * A_BYTES;
    unsigned char* b_lo = smem + 2 * A_BYTES + B_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * A_BYTES + 2 * B_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * A_BYTES + 2 * B_BYTES + 16);

    const long long e = blockIdx.z;
    struct {
        const float2 *A, *B1, *B2; float2 *C1, *C2; int lda, ldb1, ldb2, ldc1, ldc2, split;
    } J{G.A + e * G.sA, G.B1 + e * G.sB1, G.B2 + e * G.sB2, G.C1 + e * G.sC1, G.C2 + e * G.sC2,
        G.lda, G.ldb1, G.ldb2, G.ldc1, G.ldc2, G.split};
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BNC;
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    uint32_t phase = 0;
    bool ok = true;
    const int colhalf = (warp >> 2) * 128;     // accumulator columns owned by this warp
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;

    const int nstages = (K + BKC - 1) / BKC;
    for (int s = 0; s < nstages && ok; ++s) {
        const int k0 = s * BKC;
        // ---- stage A: rows row0.., complex k0.. ; real k = 2*kc + {0: re, 1: im}
        for (int t = tid; t < BM * BKC; t += THREADS) {
            int r = t / BKC, kc = t % BKC;
            float2 v = make_float2(0.f, 0.f);
            if (row0 + r < M && k0 + kc < K) v = J.A[(size_t)(row0 + r) * J.lda + k0 + kc];
            float hr = tf32_hi(v.x), hi = tf32_hi(v.y);
            uint32_t o = tile_off(r, 2 * kc);
            *reinterpret_cast<float2*>(a_hi + o) = make_float2(hr, hi);
            *reinterpret_cast<float2*>(a_lo + o) = make_float2(v.x - hr, v.y - hi);
        }
        // ---- stage B as the K-major real expansion: real row 2c = [B_r, -B_i], 2c+1 = [B_i, B_r]
        for (int t = tid; t < BKC * BNC; t += THREADS) {
            int kc = t / BNC, cc = t % BNC;
            float2 v = make_float2(0.f, 0.f);
            const int col = col0 + cc;
            if (k0 + kc < K && col < N)
                v = col < J.split ? J.B1[(size_t)(k0 + kc) * J.ldb1 + col] : J.B2[(size_t)(k0 + kc) * J.ldb2 + (col - J.split)];
            float hr = tf32_hi(v.x), hi = tf32_hi(v.y);
            float lr = v.x - hr, li = v.y - hi;
            uint32_t o0 = tile_off(2 * cc, 2 * kc), o1 = tile_off(2 * cc + 1, 2 * kc);
            *reinterpret_cast<float2*>(b_hi + o0) = make_float2(hr, -hi);
            *reinterpret_cast<float2*>(b_hi + o1) = make_float2(hi, hr);
            *reinterpret_cast<float2*>(b_lo + o0) = make_float2(lr, -li);
            *reinterpret_cast<float2*>(b_lo + o1) = make_float2(li, lr);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
            for (int ks = 0; ks < BKR / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 2 * LBO;   // 8 real K = two 16-byte chunks
                const uint32_t first = ks == 0 ? 0u : 1u;   // every stage restarts the accumulation
                mma_tf32(tmem, make_desc(ah + koff), make_desc(bh + koff), first);
                mma_tf32(tmem, make_desc(ah + koff), make_desc(bl + koff), 1u);
                mma_tf32(tmem, make_desc(al + koff), make_desc(bh + koff), 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(mbar)));
        }
        // the next stage overwrites shared memory: wait until the MMAs have read it; the
        // block agrees on the outcome, so every barrier below is reached by all threads
        ok = mbar_wait(smem_u32(mbar), phase);
        ok = __syncthreads_and(ok) != 0;
        phase ^= 1u;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int c = 0; c < 128; c += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(colhalf + c);
                tmem_ld32(taddr, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[c + j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        __syncthreads();
    }
    bool drained = true;   // no MMA of this CTA can still write its tensor memory
    if (!ok) {
        if (tid == 0) atomicExch(&g_tc_error, 1);
        // bounded second wait for the MMAs in flight (the phase that timed out); the
        // block agrees on the outcome before anyone decides about the dealloc
        drained = __syncthreads_and(mbar_wait(smem_u32(mbar), phase ^ 1u)) != 0;
    } else {
        // ---- epilogue: C -= acc.  A thread holds one tile row ((warp % 4) * 32 + lane) and 128
        // real columns; the tile goes through shared memory (rows padded to an odd stride, so
        // the row-per-lane writes are conflict-free) and C is then read and written along rows,
        // consecutive threads on consecutive columns.
        float* tile = reinterpret_cast<float*>(smem);   // BM x (BNR + 1); the stage buffers are free now
        constexpr int TS = BNR + 1;
        const int lr = (warp & 3) * 32 + (tid & 31);
#pragma unroll
        for (int j = 0; j < 128; ++j) tile[lr * TS + colhalf + j] = acc[j];
        __syncthreads();
        for (int q = tid; q < BM * BNC; q += THREADS) {
            const int rr = q / BNC, cl = q % BNC, r = row0 + rr, cc = col0 + cl;
            if (r < M && cc < N) {
                float2* p = cc < J.split ? J.C1 + (size_t)r * J.ldc1 + cc : J.C2 + (size_t)r * J.ldc2 + (cc - J.split);
                float2 o = *p;
                o.x -= tile[rr * TS + 2 * cl];
                o.y -= tile[rr * TS + 2 * cl + 1];
                *p = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // Tensor memory that an outstanding MMA may still write is not handed back: a
    // later CTA could be given it while the write lands.  The kernel reports error
    // code 2 instead and the host returns PWQT_ERR_TIMEOUT (the device is then not
    // fit for further tensor-core work in this process).
    if (drained) {
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
    } else if (tid == 0) {
        atomicExch(&g_tc_error, 2);
    }
}
}  // namespace

int cgemm_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    return e == cudaSuccess ? 0 : -1;
}

void launch_cgemm_tc(const CGemmArgs& args, int nbatch, int M, int N, int K, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || nbatch <= 0) return;
    dim3 grid((N + BNC - 1) / BNC, (M + BM - 1) / BM, nbatch);
    k_cgemm_tc<<<grid, THREADS, SMEM_BYTES, st>>>(args, M, N, K);
}

int cgemm_tc_error(bool reset, cudaStream_t st) {
    // read on the stream that ran the GEMMs, after them (the flag is shared by all launches)
    int v = 0;
    cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    return v;
}

}  // namespace pwqt

// ---------------------------------------------------------------- test entry point
extern "C" int pwqt_cgemm_c64(int batch, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                              int ldc) {
    using namespace pwqt;
    if (batch <= 0 || M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || lda < K || ldb < N || ldc < N) return PWQT_ERR_INVALID_ARG;
    if (cgemm_tc_init() != 0) return PWQT_ERR_CUDA;
    size_t sa = (size_t)M * lda, sb = (size_t)K * ldb, sc = (size_t)M * ldc;
    float2 *dA = nullptr, *dB = nullptr, *dC = nullptr;
    int rc = PWQT_OK;
    if (cudaMalloc(&dA, sizeof(float2) * sa * batch) != cudaSuccess || cudaMalloc(&dB, sizeof(float2) * sb * batch) != cudaSuccess ||
        cudaMalloc(&dC, sizeof(float2) * sc * batch) != cudaSuccess) {
        rc = PWQT_ERR_OOM;
    } else {
        cudaMemcpy(dA, A, sizeof(float2) * sa * batch, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, sizeof(float2) * sb * batch, cudaMemcpyHostToDevice);
        cudaMemcpy(dC, C, sizeof(float2) * sc * batch, cudaMemcpyHostToDevice);
        CGemmArgs g{dA, (long long)sa, lda, dB, (long long)sb, ldb, dB, (long long)sb, ldb,
                    dC, (long long)sc, ldc, dC, (long long)sc, ldc, N};
        launch_cgemm_tc(g, batch, M, N, K, 0);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = PWQT_ERR_CUDA;
        else if (cgemm_tc_error(true, 0)) rc = PWQT_ERR_CUDA;
        else cudaMemcpy(C, dC, sizeof(float2) * sc * batch, cudaMemcpyDeviceToHost);
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dC);
    return rc;
}
