// Refinement residual r = B - A c of the Sec. 3.2 system (Eq. qtbm_system) to FP64
// accuracy on the bf16 tensor cores, by exact products of integer slices.
//
// Split form.  With A = E M - HV - Sigma at the end nodes,
//     r_i = b_i - E (M c)_i + (HV c)_i + [Sigma_s c_0]_{i=0} + [Sigma_d c_{N-1}]_{i=N-1},
// where (M c)_i = M1^H c_{i-1} + M0 c_i + M1 c_{i+1} and (HV c)_i likewise with the
// node's HV blocks.  M and HV do not depend on the energy, so their slices are made
// once per system; only c is sliced per refinement step, and one product serves every
// energy of a batch (their columns side by side).
//
// Slices.  A real operand row (column) is scaled by a power of two 2^e with
// |x| < 2^e and cut into S = 7 slices of 7 bits: x = 2^e sum_q s_q 2^(-7q) + O(2^(e-49)),
// s_q integers in [-127, 127], exact in bf16.  A slice product sums to an integer;
// pairs (p, q) with p + q = t share an accumulator D_t (t = 2..9, pairs with p + q > 9
// are dropped: 34 pairs, ~2^-53 of the scaled product per term).  FP32 accumulation
// on the tensor cores is exact while |D_t| < 2^24: at most 7 pairs x 128 real K x
// 127^2 < 2^24, so every 128 real K the accumulators are moved to int32 registers
// (exact) and the tensor-core accumulation restarts.  At the end
//     P = 2^(e_row + f_col) sum_t 2^(-7t) D_t   (two int64 partial folds, one FP64 add).
//
// Complex products by real expansion of the matrix: rows interleaved (2r: real part,
// 2r+1: imaginary part), K = [segment][re plane | im plane][k]:
//     A'[2r]   = [ Re a_s(r,:), -Im a_s(r,:) ],   A'[2r+1] = [ Im a_s(r,:), Re a_s(r,:) ],
//     B'[s]    = [ Re c_j ; Im c_j ]  (j = node of segment s),
// so (A'B')[2r] = Re (A c)_r and (A'B')[2r+1] = Im (A c)_r.
//
// Kernel.  One CTA per (item, 128-row tile, 32-column tile); an item is a node (M
// and HV products) or an (energy, contact) pair (Sigma products).  Operand tiles are
// stored pre-packed in the UMMA canonical K-major layout (8 rows x 16 bytes core
// matrices), one contiguous block per 32-K chunk and slice, and moved by 1D bulk
// copies (cp.async.bulk) into a three-stage shared-memory ring guarded by
// mbarriers.  Per 16-K step one tcgen05.mma per A slice p multiplies it by the B
// slices 1..q concatenated along N (the slices are consecutive row groups), writing
// D_(p+1) .. D_(p+q) at once: 7 MMAs with N = 256, 224, ..., 64 (slice 8 of B is a
// fixed zero block so that the first MMA of a stage spans, and clears, all eight
// accumulators).  Accumulators: 8 x 32 columns = 256 TMEM columns, two buffers, so
// that eight warps drain one 128-K stage while the MMAs fill the other.
// Warp 0: bulk-copy producer; warp 1: MMA issuer; warps 2..9: accumulator drain
// and epilogue.  Every mbarrier wait is bounded (globaltimer); on a timeout the CTA
// stops, waits (bounded) for its own copies and MMAs, frees its tensor memory only
// if they drained, and sets an error flag that the host reads.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "pwqt_internal.cuh"
#include "residual_oz.cuh"

namespace pwqt {
namespace oz {

namespace {
constexpr int SL = 7;                    // slices per operand
constexpr int TMAX = 9;                  // largest slice-index sum kept (p + q <= 9)
constexpr int NDIAG = TMAX - 1;          // accumulators D_2 .. D_9
constexpr int TM = 128;                  // real rows per tile
constexpr int TN = 32;                   // columns per tile
constexpr int KCH = 32;                  // real K per chunk (one bulk copy per operand)
constexpr int KSTAGE_CHUNKS = 4;         // chunks per exact accumulation stage (128 real K)
constexpr int NSTAGE = 3;                // shared-memory ring depth
constexpr uint32_t A_SLICE_BYTES = TM * KCH * 2;          // 8 KB
constexpr uint32_t B_SLICE_BYTES = TN * KCH * 2;          // 2 KB
constexpr uint32_t A_CHUNK_BYTES = SL * A_SLICE_BYTES;    // 56 KB
constexpr uint32_t B_CHUNK_BYTES = SL * B_SLICE_BYTES;    // 14 KB
constexpr uint32_t B_STAGE_BYTES = B_CHUNK_BYTES + B_SLICE_BYTES;   // + the zero slice
constexpr uint32_t STAGE_BYTES = A_CHUNK_BYTES + B_STAGE_BYTES;     // 72 KB
constexpr uint32_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 128;
constexpr uint32_t ACC_COLS = NDIAG * TN;                  // 256
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;               // 512: two accumulator buffers
constexpr int THREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr uint32_t LBO = 128;            // next core matrix along K
constexpr uint32_t SBO = 512;            // next 8-row group (4 core matrices of K per chunk)
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded mbarrier waits: 2 s

static_assert(SMEM_BYTES <= 227 * 1024, "shared-memory ring fits");

__device__ int g_oz_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait on an mbarrier phase; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = gtime();
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 63) == 63 && gtime() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;            // descriptor version of the sm_100 family; no swizzle
    return d;
}

// kind::f16 with bf16 A and B, FP32 D, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 2^k as a double (exact; k inside the normal range, else the nearest representable end)
__device__ __forceinline__ double pow2(int k) {
    k = max(-1022, min(1023, k));
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// B slices 1..n_q(p) multiplied by A slice p (slice 8 of B is the zero block)
__device__ __forceinline__ int n_q(int p) { return p == 1 ? 8 : min(SL, TMAX - p); }

// ---------------------------------------------------------------- slicing helpers
// biased binary exponent of |x| (0 for zero), so that |x| < 2^(bexp - 1022)
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// x = sign * X * 2^(f - 49) with X = floor(|x| 2^(49 - f)) < 2^49, f = ebias - 1022;
// slice q (1..7) = sign * ((X >> (49 - 7q)) & 127) as bf16 bits
__device__ __forceinline__ void slice7(double x, int ebias, uint16_t* out) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const uint16_t sign = (uint16_t)((bits >> 48) & 0x8000);
    unsigned long long X = 0;
    if (ex > 0 && ebias > 0) {
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = ebias - ex + 4;             // X = mant * 2^(ex - 1075 + 49 - (ebias - 1022))
        X = sh >= 64 ? 0ull : (mant >> sh);        // sh >= 4 since ex <= ebias
    }
#pragma unroll
    for (int q = 1; q <= SL; ++q) {
        const uint32_t v = (uint32_t)(X >> (49 - 7 * q)) & 127u;
        uint16_t h = 0;
        if (v) {
            const int e = 31 - __clz(v);                        // 0..6
            h = (uint16_t)(sign | ((127 + e) << 7) | ((v << (7 - e)) & 127u));
        }
        out[q - 1] = h;
    }
}

// element (row, k) of a 128 x 32 (A) or 32 x 32 (B) slice tile, in bf16 elements
__device__ __forceinline__ int tile_elem(int row, int k) { return (row >> 3) * 256 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7); }

}  // namespace

// ---------------------------------------------------------------- A panels
// Row exponents of an A panel: for every complex row r of every item the largest
// biased exponent over its segments' real and imaginary parts.  One block per
// (row, item); segment blocks come from the panel source (see PanelSrc).
__device__ __forceinline__ double2 panel_elem(const double2* b, int n, bool ct, int r, int k) {
    if (ct) {
        const double2 v = b[(size_t)k * n + r];
        return make_double2(v.x, -v.y);
    }
    return b[(size_t)r * n + k];
}

__global__ void k_panel_rowexp(PanelSrc P, int* rexp, int n_pad) {
    const int r = blockIdx.x, item = blockIdx.y;
    int mx = 0;
    if (r < P.n)
        for (int s = 0; s < P.nseg; ++s) {
            const double2* b = P.block(item, s);
            if (!b) continue;
            for (int k = threadIdx.x; k < P.n; k += blockDim.x) {
                const double2 v = panel_elem(b, P.n, P.ct[s] != 0, r, k);
                mx = max(mx, max(bexp(v.x), bexp(v.y)));
            }
        }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
        red[0] = max(mx, red[0]);
        rexp[(size_t)item * 2 * n_pad + 2 * r] = red[0];
        rexp[(size_t)item * 2 * n_pad + 2 * r + 1] = red[0];
    }
}

// Slice tiles of an A panel: block per (item, row tile, segment, chunk); 256 threads
// write the 7 slice tiles of 128 rows x 32 K.  Padded rows / K and absent segments
// become zero slices.
__global__ void k_panel_slice(PanelSrc P, const int* rexp, int n_pad, __nv_bfloat16* tiles) {
    const int kc = blockIdx.x, rt = blockIdx.y, item = blockIdx.z / P.nseg, s = blockIdx.z % P.nseg;
    const int RT = 2 * n_pad / TM, KC = 2 * n_pad / KCH;
    uint16_t* out = reinterpret_cast<uint16_t*>(tiles) +
                    ((((size_t)item * RT + rt) * P.nseg + s) * KC + kc) * (size_t)(SL * TM * KCH);
    const double2* blk = P.block(item, s);
    const bool ct = P.ct[s] != 0;
    for (int t = threadIdx.x; t < TM * KCH; t += blockDim.x) {
        const int rr = t / KCH, kk = t % KCH;
        const int rp = rt * TM + rr;                 // real row
        const int kp = kc * KCH + kk;                // real K inside the segment: [re plane | im plane]
        const int r = rp >> 1, part = rp & 1, plane = kp / n_pad, k = kp % n_pad;
        double x = 0.0;
        if (blk && r < P.n && k < P.n) {
            const double2 a = panel_elem(blk, P.n, ct, r, k);
            // row 2r: [Re a, -Im a]; row 2r+1: [Im a, Re a]
            x = part == 0 ? (plane == 0 ? a.x : -a.y) : (plane == 0 ? a.y : a.x);
        }
        uint16_t sl[SL];
        slice7(x, rexp[(size_t)item * 2 * n_pad + rp], sl);
        const int off = tile_elem(rr, kk);
#pragma unroll
        for (int q = 0; q < SL; ++q) out[(size_t)q * TM * KCH + off] = sl[q];
    }
}

// ---------------------------------------------------------------- B (solution) slices
// Column exponents over all nodes of the active energies' solutions: fexp[k m + g].
__global__ void k_c_colexp(const double2* __restrict__ C, long long sC, const int* __restrict__ act, int n, int N, int m,
                           int* fexp) {
    extern __shared__ int cm[];
    const int k = blockIdx.y, j = blockIdx.x;    // active energy, node
    const double2* c = C + act[k] * sC + (size_t)j * n * m;
    for (int g = threadIdx.x; g < m; g += blockDim.x) cm[g] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
        const double2 v = c[t];
        atomicMax(&cm[t % m], max(bexp(v.x), bexp(v.y)));
    }
    __syncthreads();
    for (int g = threadIdx.x; g < m; g += blockDim.x)
        if (cm[g]) atomicMax(&fexp[k * m + g], cm[g]);
}

// B tiles of every node: block per (node, column tile, chunk); columns k m + g of the
// active energies, K = [Re c_j (n_pad) ; Im c_j (n_pad)].
__global__ void k_c_slice(const double2* __restrict__ C, long long sC, const int* __restrict__ act, int n_act, int n, int N,
                          int m, int n_pad, int nct, const int* __restrict__ fexp, __nv_bfloat16* tiles) {
    const int kc = blockIdx.x, ct = blockIdx.y, j = blockIdx.z;
    const int KC = 2 * n_pad / KCH;
    uint16_t* out = reinterpret_cast<uint16_t*>(tiles) + (((size_t)j * nct + ct) * KC + kc) * (size_t)(SL * TN * KCH);
    for (int t = threadIdx.x; t < TN * KCH; t += blockDim.x) {
        const int kk = t / TN, cc = t % TN;          // consecutive threads along columns (one row of c)
        const int col = ct * TN + cc, kp = kc * KCH + kk;
        const int plane = kp / n_pad, r = kp % n_pad;
        const int k = col / m, g = col % m;
        double x = 0.0;
        int fe = 0;
        if (k < n_act && r < n) {
            const double2 v = C[act[k] * sC + ((size_t)j * n + r) * m + g];
            x = plane == 0 ? v.x : v.y;
            fe = fexp[col];
        }
        uint16_t sl[SL];
        slice7(x, fe, sl);
        const int off = tile_elem(cc, kk);
#pragma unroll
        for (int q = 0; q < SL; ++q) out[(size_t)q * TN * KCH + off] = sl[q];
    }
}

// ---------------------------------------------------------------- the slice-product GEMM
__global__ void __launch_bounds__(THREADS, 1) k_oz_gemm(const GemmArgs G) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // column tile: launches over one energy (Sigma) or one system's energies (HV) start at
    // the first tile of their column range
    const int c_first = G.mode == MODE_SIGMA ? (int)blockIdx.z * G.m : G.col_lo;
    const int ct = blockIdx.x + c_first / TN, rt = blockIdx.y, z = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = G.n, N = G.N, m = G.m, n_pad = G.n_pad;
    const int RT = 2 * n_pad / TM, KC = 2 * n_pad / KCH;

    // ---- the item: node and segments (M, HV: node z, segments j = z-1, z, z+1; Sigma:
    // item z = 2 k + side of active energy k, one segment at the contact's edge node)
    // segments present are a contiguous range [s_lo, s_lo + nseg) of the item's
    // segments; segment s reads the solution of node node0 + s
    int node, e_act = -1, aitem, nseg_tot, s_lo, nseg, node0;
    if (G.mode == MODE_SIGMA) {
        e_act = z;
        if (e_act >= G.n_act) return;
        node = G.sigma_side ? N - 1 : 0;
        nseg_tot = 1;
        s_lo = 0;
        nseg = 1;
        node0 = node;
        aitem = 2 * G.act[e_act] + G.sigma_side;
        // columns of that energy only
        const int c_lo = e_act * m, c_hi = c_lo + m;
        if (ct * TN >= c_hi || ct * TN + TN <= c_lo) return;
    } else {
        if (ct >= G.nct || ct * TN >= G.col_hi || ct * TN + TN <= G.col_lo) return;
        node = z;
        nseg_tot = 3;
        s_lo = node == 0 ? 1 : 0;
        const int s_hi = node == N - 1 ? 1 : 2;
        nseg = s_hi - s_lo + 1;
        node0 = node - 1;
        aitem = G.mode == MODE_M ? 0 : z;
    }
    (void)RT;
    const int nchunks = nseg * KC;
    const int nstages = nchunks / KSTAGE_CHUNKS;

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
    // full[3] | empty[3] | accfull[2] | accempty[2] | tmem slot | abort flag
    const uint32_t full0 = smem_u32(bar), empty0 = full0 + 8 * NSTAGE, accf0 = empty0 + 8 * NSTAGE, acce0 = accf0 + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2 * NSTAGE + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    // zero slices (slot 8 of every B stage buffer); never overwritten by the copies
    for (int t = tid; t < NSTAGE * (int)(B_SLICE_BYTES / 16); t += THREADS) {
        const int st = t / (B_SLICE_BYTES / 16), q = t % (B_SLICE_BYTES / 16);
        reinterpret_cast<uint4*>(smem + st * STAGE_BYTES + A_CHUNK_BYTES + B_CHUNK_BYTES)[q] = make_uint4(0, 0, 0, 0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) { mbar_init(full0 + 8 * s, 1); mbar_init(empty0 + 8 * s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(accf0 + 8 * b, 1); mbar_init(acce0 + 8 * b, EPI_WARPS); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem0 = smem_u32(smem);

    int issued = 0;          // producer: chunks whose copies were issued
    int mma_chunks = 0;      // MMA thread: chunks whose MMAs were issued

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            const char* Abase = reinterpret_cast<const char*>(G.A) + (size_t)aitem * G.a_item_bytes;
            for (int c = 0; c < nchunks; ++c) {
                const int st = c % NSTAGE;
                if (c >= NSTAGE && !mbar_wait(empty0 + 8 * st, ((c / NSTAGE) - 1) & 1)) { *abort_flag = 1; break; }
                if (*abort_flag) break;
                const int s = s_lo + c / KC, kc = c % KC, j = node0 + s;
                const char* a = Abase + ((((size_t)rt * nseg_tot + s) * KC + kc) * A_CHUNK_BYTES);
                const char* b = reinterpret_cast<const char*>(G.B) + ((((size_t)j * G.nct + ct) * KC + kc) * B_CHUNK_BYTES);
                const uint32_t dst = smem0 + st * STAGE_BYTES;
                mbar_expect_tx(full0 + 8 * st, A_CHUNK_BYTES + B_CHUNK_BYTES);
                bulk_g2s(dst, a, A_CHUNK_BYTES, full0 + 8 * st);
                bulk_g2s(dst + A_CHUNK_BYTES, b, B_CHUNK_BYTES, full0 + 8 * st);
                issued = c + 1;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            for (int c = 0; c < nchunks; ++c) {
                const int st = c % NSTAGE, ps = c / KSTAGE_CHUNKS, buf = ps & 1;
                if (c % KSTAGE_CHUNKS == 0 && ps >= 2 && !mbar_wait(acce0 + 8 * buf, ((ps >> 1) - 1) & 1)) { *abort_flag = 1; break; }
                if (!mbar_wait(full0 + 8 * st, (c / NSTAGE) & 1)) { *abort_flag = 1; break; }
                if (*abort_flag) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = smem0 + st * STAGE_BYTES, b0 = a0 + A_CHUNK_BYTES;
                const uint32_t d0 = tmem + (uint32_t)buf * ACC_COLS;
#pragma unroll
                for (int h = 0; h < KCH / 16; ++h) {
#pragma unroll
                    for (int p = 1; p <= SL; ++p) {
                        const uint32_t acc = (c % KSTAGE_CHUNKS == 0 && h == 0 && p == 1) ? 0u : 1u;
                        mma_bf16(d0 + (uint32_t)(p - 1) * TN, make_desc(a0 + (p - 1) * A_SLICE_BYTES + h * 256),
                                 make_desc(b0 + h * 256), idesc_bf16((uint32_t)(n_q(p) * TN)), acc);
                    }
                }
                mma_commit(empty0 + 8 * st);
                if (c % KSTAGE_CHUNKS == KSTAGE_CHUNKS - 1) mma_commit(accf0 + 8 * buf);
                mma_chunks = c + 1;
            }
        }
    } else {
        // ---------------- accumulator drain (warps 2..9) and epilogue
        const int quarter = warp & 3, half = (warp - 2) >> 2;   // TMEM lanes 32*quarter.., columns 16*half..
        // running sums of the two diagonal groups, folded per stage:
        //   hi += D2 2^21 + D3 2^14 + D4 2^7 + D5,  lo += D6 2^21 + D7 2^14 + D8 2^7 + D9
        // (|D_t| < 2^24 per stage, so each stage adds < 2^45.1 and 2^51 bounds any K here)
        long long acc[2][16];
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[g][j] = 0;
        bool ok = true;
        for (int ps = 0; ps < nstages; ++ps) {
            const int buf = ps & 1;
            if (!mbar_wait(accf0 + 8 * buf, (ps >> 1) & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                long long tmp[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) tmp[j] = 0;
#pragma unroll
                for (int t = 4 * g; t < 4 * g + 4; ++t) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * ACC_COLS + (uint32_t)t * TN + half * 16, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) tmp[j] = tmp[j] * 128 + __float2int_rz(__uint_as_float(v[j]));
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[g][j] += tmp[j];
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * buf);
        }
        if (!ok) *abort_flag = 1;
        if (ok) {
            // ---- epilogue: P = 2^(e + f) [2^-35 (D2 2^21 + D3 2^14 + D4 2^7 + D5) + 2^-63 (D6 2^21 + ...)]
            const int rp = rt * TM + quarter * 32 + lane;       // real row of this thread
            const int r = rp >> 1, part = rp & 1;
            const int ebias = G.rexp[(size_t)aitem * 2 * n_pad + rp];
            if (r < n) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = ct * TN + half * 16 + j;
                    const int k = col / m, g = col % m;
                    if (k >= G.n_act || (e_act >= 0 && k != e_act) || col < G.col_lo || col >= G.col_hi) continue;
                    const int fe = G.fexp[col];
                    const int e = G.act[k];
                    const ResJob& J = G.jobs[e];
                    if (g >= J.ms + J.md) continue;
                    double P = 0.0;
                    if (fe > 0 && ebias > 0) {
                        const long long hi = acc[0][j], lo = acc[1][j];
                        // scale 2^(e_row + f_col) with e = ebias - 1022, f = fe - 1022
                        const int sc = (ebias - 1022) + (fe - 1022);
                        P = fma((double)lo, pow2(sc - 63), (double)hi * pow2(sc - 35));
                    }
                    double* R = reinterpret_cast<double*>(G.R + e * G.sC + ((size_t)node * n + r) * m + g) + part;
                    if (G.mode == MODE_M) {
                        double b = 0.0;
                        if (node == 0 && g < J.ms) { const double2 bv = J.rhs_s[(size_t)r * J.ms + g]; b = part ? bv.y : bv.x; }
                        if (node == N - 1 && g >= J.ms) { const double2 bv = J.rhs_d[(size_t)r * J.md + (g - J.ms)]; b = part ? bv.y : bv.x; }
                        *R = fma(-J.E, P, b);
                    } else {
                        *R += P;
                    }
                }
            }
        }
    }
    // ---------------- teardown: every copy and MMA of this CTA must have landed
    __syncthreads();
    bool drained = true;
    if (*abort_flag) {
        if (tid == 0) atomicExch(&g_oz_error, 1);
        // each role waits (bounded) for its own outstanding work: the producer for the
        // copies of the last ring's worth of chunks it issued (earlier stages were
        // consumed by the MMAs, so their barriers are past), the MMA thread for its last
        // commit, which tracks all of its MMAs
        if (warp == 0 && lane == 0)
            for (int c = max(issued - NSTAGE, 0); c < issued; ++c)
                if (!mbar_wait(full0 + 8 * (c % NSTAGE), (c / NSTAGE) & 1)) { drained = false; break; }
        if (warp == 1 && lane == 0 && mma_chunks > 0) {
            const int c = mma_chunks - 1;
            if (!mbar_wait(empty0 + 8 * (c % NSTAGE), (c / NSTAGE) & 1)) drained = false;
        }
    }
    drained = __syncthreads_and(drained) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (drained) {
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
    } else if (tid == 0) {
        atomicExch(&g_oz_error, 2);
    }
}

// ---------------------------------------------------------------- residual norms
// Column sums |r|^2 over all nodes and |b|^2 over the end nodes of the active energies.
__global__ void k_oz_norms(const double2* __restrict__ R, long long sC, const ResJob* __restrict__ jobs, const int* __restrict__ act,
                           int n, int N, int m) {
    extern __shared__ double ns[];
    const int k = blockIdx.y, j = blockIdx.x, e = act[k];
    const ResJob& J = jobs[e];
    double* rs = ns;
    double* bs = ns + m;
    for (int g = threadIdx.x; g < m; g += blockDim.x) { rs[g] = 0; bs[g] = 0; }
    __syncthreads();
    const double2* r = R + e * sC + (size_t)j * n * m;
    const int mm = J.ms + J.md;
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
        const int row = t / m, g = t % m;
        if (g >= mm) continue;
        atomicAdd(&rs[g], cnorm2(r[t]));
        double2 bv = make_double2(0, 0);
        if (j == 0 && g < J.ms) bv = J.rhs_s[(size_t)row * J.ms + g];
        if (j == N - 1 && g >= J.ms) bv = J.rhs_d[(size_t)row * J.md + (g - J.ms)];
        if (j == 0 || j == N - 1) atomicAdd(&bs[g], cnorm2(bv));
    }
    __syncthreads();
    for (int g = threadIdx.x; g < mm; g += blockDim.x) {
        atomicAdd(&J.rn2[g], rs[g]);
        if (j == 0 || j == N - 1) atomicAdd(&J.bn2[g], bs[g]);
    }
}

// ---------------------------------------------------------------- host side
int gemm_init() {
    const cudaError_t e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    return e == cudaSuccess ? 0 : -1;
}

int error_flag(bool reset, cudaStream_t st) {
    int v = 0;
    cudaMemcpyFromSymbolAsync(&v, g_oz_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (reset && v) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_oz_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    return v;
}

int padded(int n) { return (n + 63) / 64 * 64; }

size_t panel_bytes(int n, int items, int nseg) {
    const int n_pad = padded(n);
    return (size_t)items * (2 * n_pad / TM) * nseg * (2 * n_pad / KCH) * A_CHUNK_BYTES;
}
size_t panel_item_bytes(int n, int nseg) { return panel_bytes(n, 1, nseg); }
size_t rexp_bytes(int n, int items) { return sizeof(int) * (size_t)items * 2 * padded(n); }
size_t b_bytes(int n, int N, int ncols) {
    const int n_pad = padded(n), nct = (ncols + TN - 1) / TN;
    return (size_t)N * nct * (2 * n_pad / KCH) * B_CHUNK_BYTES;
}
int col_tiles(int ncols) { return (ncols + TN - 1) / TN; }

void build_panel(const PanelSrc& P, int items, int* rexp, __nv_bfloat16* tiles, cudaStream_t st) {
    const int n_pad = padded(P.n);
    k_panel_rowexp<<<dim3(n_pad, items), 256, 0, st>>>(P, rexp, n_pad);
    k_panel_slice<<<dim3(2 * n_pad / KCH, 2 * n_pad / TM, items * P.nseg), 256, 0, st>>>(P, rexp, n_pad, tiles);
}

void slice_solution(const double2* C, long long sC, const int* act, int n_act, int n, int N, int m, int* fexp,
                    __nv_bfloat16* tiles, cudaStream_t st) {
    const int n_pad = padded(n), nct = col_tiles(n_act * m);
    cudaMemsetAsync(fexp, 0, sizeof(int) * (size_t)nct * TN, st);
    k_c_colexp<<<dim3(N, n_act), 256, sizeof(int) * m, st>>>(C, sC, act, n, N, m, fexp);
    k_c_slice<<<dim3(2 * n_pad / KCH, nct, N), 256, 0, st>>>(C, sC, act, n_act, n, N, m, n_pad, nct, fexp, tiles);
}

void gemm(const GemmArgs& G, int items, cudaStream_t st) {
    const int n_pad = G.n_pad;
    int tiles = G.nct;
    if (G.mode == MODE_SIGMA) tiles = std::min(G.nct, (G.m + TN - 1) / TN + 1);     // one energy's columns
    else if (G.col_lo > 0 || G.col_hi < G.nct * TN)                                // one system's columns
        tiles = std::min(G.nct, (std::min(G.col_hi, G.nct * TN) - 1) / TN - G.col_lo / TN + 1);
    if (tiles <= 0 || items <= 0) return;
    dim3 grid(tiles, 2 * n_pad / TM, items);
    k_oz_gemm<<<grid, THREADS, SMEM_BYTES, st>>>(G);
}

void norms(const double2* R, long long sC, const ResJob* jobs, const int* act, int n_act, int n, int N, int m, cudaStream_t st) {
    k_oz_norms<<<dim3(N, n_act), 256, 2 * sizeof(double) * m, st>>>(R, sC, jobs, act, n, N, m);
}

}  // namespace oz
}  // namespace pwqt
