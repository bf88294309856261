// Split-precision tensor-core form of the strided FFT passes on the 5th-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory), for
// lines of N = 64 .. 1024 points.
//
// A line of N = 32 n1 points is transformed in two matrix stages (the
// four-step decomposition n = a + n1 b, k = k2 + 32 k1):
//   stage 1  Y[a, k2] = sum_b x[a + n1 b] w32^{b k2}          (radix 32)
//   twiddle  Y[a, k2] *= wN^{a k2}
//   stage 2  X[k2 + 32 k1] = sum_a Y[a, k2] w_{n1}^{a k1}     (radix n1)
// with w_L = exp(-2 pi i / L).  Each stage is one real matrix product
// D (64 x NC) = A (64 x 64) B (64 x NC) on a whole tile of CX columns:
//   stage 1  A = the 32-point DFT in real form (row 2k + r, column 2b + s),
//            B column a CX + c holds the 32 inputs x[a + n1 b] of (a, c);
//   stage 2  A = 32/n1 copies of the n1-point DFT in real form on the
//            diagonal, B block j holds the inputs Y[a, k2] of the k2 in
//            [j n1, (j+1) n1), column (k2 mod n1) CX + c,
// so NC = n1 CX columns (64 .. 256) and K = 64.  The inverse transform is
// conj(DFT(conj x)): the imaginary parts are negated on the way in and out,
// so only the forward matrices are stored.
//
// Both operands are split into hi + lo parts (float16 or bfloat16, as in
// fft_tc.cuh) and the product is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi,
// accumulated in float32 in tensor memory: 3 x 4 instructions of K = 16
// (kind::f16, M = 64, N = NC), issued by one thread, completion signalled on
// an mbarrier (bounded wait).  The float16 form scales each column by a power
// of two that puts its largest input in [32, 64): stage-1 outputs stay below
// 32 x 64 = 2048, and the stage-2 outputs are read back in float32.
//
// Operands live in shared memory in the K-major layout without swizzle:
// element (row r, k) of a 64-wide operand at byte
//   (r / 8) 1024 + (k / 8) 128 + (r % 8) 16 + (k % 8) 2
// (8 x 8 core matrices; 128 bytes between core matrices along K, 1024 between
// groups of 8 rows).  The accumulator of an M = 64 product occupies 16 lanes
// of each 32-lane quarter of tensor memory: row m in lane 32 (m / 16) + m % 16,
// column n in column n.  A warp reads its quarter's 16 lanes with the
// 16x32bx2 shape: lanes 0..15 of the warp read 8 columns, lanes 16..31 the
// next 8 (probed on the GB300 before use).
#pragma once

#include "fft_tc.cuh"
#include "tma.cuh"

namespace kwgb {

constexpr int TC5_A_BYTES = 64 * 64 * 2;            // one 64 x 64 operand (hi or lo)
constexpr int TC5_A_WORDS = TC5_A_BYTES / 4;        // the same in 32-bit words

__host__ __device__ constexpr int tc5_koff(int r, int k) {
    return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: K-major, no swizzle, 128 bytes between
// core matrices along K (leading), 1024 between 8-row groups (stride).
__device__ __forceinline__ uint64_t tc5_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: float32 accumulator, A and B of the
// same 16-bit type (0 float16, 1 bfloat16), both K-major, N columns, M = 64.
template <int PREC>
__host__ __device__ constexpr uint32_t tc5_idesc(int n) {
    return (1u << 4) | ((PREC == 2 ? 0u : 1u) << 7) | ((PREC == 2 ? 0u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(64 >> 4) << 24);
}

__device__ __forceinline__ void tc5_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc5_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tensor-memory columns a CTA allocates for an accumulator of nc columns
// (a power of two, at least 32).
__host__ __device__ constexpr int tc5_tmem_cols(int nc) { return nc <= 32 ? 32 : (nc <= 64 ? 64 : (nc <= 128 ? 128 : 256)); }

__device__ __forceinline__ void tc5_alloc(uint32_t* slot, int ncols) {      // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc5_dealloc(uint32_t taddr, int ncols) {   // one whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Issue a read of 16 lanes x 8 columns from taddr (lanes 0..15 of the warp)
// and 8 columns further on (lanes 16..31); the values are valid only after
// tc5_ld_wait.
__device__ __forceinline__ void tc5_ld16(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.16x32bx2.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], 8;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Wait for the reads issued so far; each value then passes through an empty
// volatile asm placed after the wait, so no use of it can be scheduled before.
template <int U>
__device__ __forceinline__ void tc5_ld_wait(uint32_t (&r)[U][8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < 8; ++i) asm volatile("" : "+r"(r[u][i]));
}

// Bounded wait for a product commit (no sleep between polls: a product takes
// well under a microsecond).  Sets bit 2 of *flag when it gives up.
__device__ __forceinline__ bool tc5_wait(uint64_t* bar, uint32_t parity, int* flag) {
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) {
            atomicOr(flag, 2);
            return false;
        }
    }
}

// Per-CTA state of the tensor-core passes.
struct Tc5 {
    unsigned char* a1;        // stage-1 operand A: hi, then lo (TC5_A_BYTES each)
    unsigned char* a2;        // stage-2 operand A: hi, then lo (== a1 for 1024-point lines)
    unsigned char* b;         // operand B: hi, then lo (NC * 128 bytes each)
    uint64_t* bar;            // mbarrier of the product commits
    uint32_t tmem;            // accumulator (NC columns)
    uint32_t phase;           // parity of the next commit
    int* flag;                // device status (bit 2: a bounded wait ran out)
    bool ok;                  // false once a wait ran out: the rest of the work is skipped
};

// Issue D = A_hi B_hi + A_hi B_lo + A_lo B_hi (thread 0) and wait for it (all).
template <int PREC, int NC>
__device__ __forceinline__ void tc5_product(Tc5& t, const unsigned char* a) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // operands written: visible to the tensor cores
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    if (threadIdx.x == 0 && t.ok) {
        constexpr uint32_t idesc = tc5_idesc<PREC>(NC);
        const uint32_t ah = smem_addr(a), al = ah + TC5_A_BYTES;
        const uint32_t bh = smem_addr(t.b), bl = bh + NC * 128;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) tc5_mma(t.tmem, tc5_desc(ah + kk * 256), tc5_desc(bh + kk * 256), idesc, kk > 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) tc5_mma(t.tmem, tc5_desc(ah + kk * 256), tc5_desc(bl + kk * 256), idesc, 1u);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) tc5_mma(t.tmem, tc5_desc(al + kk * 256), tc5_desc(bh + kk * 256), idesc, 1u);
        tc5_commit(t.bar);
    }
    bool ok = t.ok && tc5_wait(t.bar, t.phase, t.flag);
    t.ok = __syncthreads_and(ok) != 0;                 // uniform: the read-back is warp-collective
    t.phase ^= 1u;
    tc5_fence_after();
}

// In-place DFT (direction DIR) of every column of the tile buf ([n][c], CX
// columns, plain layout in and out).  Starts and ends with the tile fully
// written (callers synchronise before).  cmx: column maxima of the float16
// form (SCAN: read them from the tile here; otherwise deposited by the caller
// before its barrier).
//
// Thread work: the stage-1 conversion gives a thread four inputs b = 4 bq .. 4 bq
// + 3 of one operand column, so it writes one 16-byte row of a core matrix
// (hi and lo), and a warp writes 512 contiguous bytes.  In the read-backs the
// two lanes that hold the real and imaginary rows of the same output swap
// halves of their eight columns (four shuffles), so each lane finishes four
// whole complex values.
template <int LOGN, int CX, int DIR, int THREADS, int PREC, bool SCAN = true>
__device__ __forceinline__ void tile_fft_tc5(float2* buf, Tc5& t, const float2* __restrict__ tw, TcColMax& cmx) {
    constexpr int N = 1 << LOGN;
    constexpr int N1 = N / 32;
    constexpr int NC = N1 * CX;                        // product columns
    constexpr int WG = THREADS / 128;                  // warps per tensor-memory quarter
    constexpr int NCW = NC / WG;                       // columns per warp in the read-back
    static_assert(LOGN >= 6 && LOGN <= 10 && THREADS % 128 == 0 && NCW % 16 == 0, "tile shape");
    static_assert((8 * NC) % THREADS == 0 && CX % 4 == 0, "operand conversion split");
    constexpr float CJ = DIR > 0 ? -1.0f : 1.0f;       // conjugation of the inverse transform
    unsigned int* colmax = cmx.m + 16 * cmx.cur;
    if constexpr (PREC == 2 && SCAN) {
        float m = 0.f;
#pragma unroll 4
        for (int i = threadIdx.x; i < N * CX; i += THREADS) {
            const float2 v = buf[i];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        tc_colmax_deposit<CX>(m, cmx);
        __syncthreads();
    }
    cmx.cur ^= 1;
    // ---- stage 1 operand: column a CX + c, rows 2b, 2b + 1 <- x[a + n1 b][c]
#pragma unroll
    for (int r = 0; r < 8 * NC / THREADS; ++r) {
        const int it = threadIdx.x + THREADS * r;
        const int col = (it >> 6) * 8 + (it & 7), bq = (it >> 3) & 7;
        const int a = col / CX, c = col % CX;
        float sc = 1.0f;
        if constexpr (PREC == 2) sc = col_scale(colmax[c], false);
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 v = buf[(a + N1 * (4 * bq + i)) * CX + c];
            split2<PREC>(v.x * sc, v.y * (sc * CJ), hi[i], lo[i]);
        }
        const int o = tc5_koff(col, 8 * bq);
        *reinterpret_cast<uint4*>(t.b + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(t.b + NC * 128 + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    tc5_product<PREC, NC>(t, t.a1);
    // ---- twiddle, stage 2 operand: D1 row 2 k2 + r, column a CX + c
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = w & 3, wg = w >> 2;
    const int m = 16 * q + (lane & 15);                // accumulator row of this lane
    const int k2 = m >> 1, ri = m & 1;
    const uint32_t lane_addr = t.tmem + ((uint32_t)(32 * q) << 16);
    // the twiddles (global loads) are issued before the tensor-memory reads and
    // their wait, so the two latencies overlap
    float2 wts[NCW / 16];
#pragma unroll
    for (int u = 0; u < NCW / 16; ++u) {
        const int a = (wg * NCW + 16 * u + 8 * (lane >> 4) + 4 * ri) / CX;
        wts[u] = twiddle1024<-1>(tw, (a * k2 * (1024 / N)) & 1023);
    }
    uint32_t rv[NCW / 16][8];
    if (t.ok) {
#pragma unroll
        for (int u = 0; u < NCW / 16; ++u) tc5_ld16(lane_addr + wg * NCW + 16 * u, rv[u]);
        tc5_ld_wait<NCW / 16>(rv);
    } else {
#pragma unroll
        for (int u = 0; u < NCW / 16; ++u)
#pragma unroll
            for (int e = 0; e < 8; ++e) rv[u][e] = 0u;
    }
#pragma unroll
    for (int u = 0; u < NCW / 16; ++u) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(rv[u][e]);
        // this lane finishes columns col0 .. col0 + 3 (even lane: the first four)
        const int col0 = wg * NCW + 16 * u + 8 * (lane >> 4) + 4 * ri;
        const int a = col0 / CX, c0 = col0 % CX;
        const float2 wt = wts[u];
        const int ob = tc5_koff((k2 % N1) * CX + c0, 2 * N1 * (k2 / N1) + 2 * a);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float o = __shfl_xor_sync(0xffffffffu, ri ? v[e] : v[e + 4], 1);
            float2 y = ri ? make_float2(o, v[e + 4]) : make_float2(v[e], o);
            y = cmul(y, wt);
            uint32_t hi, lo;
            split2<PREC>(y.x, y.y, hi, lo);
            // rows 2 n1 j + 2a (+1) of block j = k2 / n1, column (k2 mod n1) CX + c0 + e
            *reinterpret_cast<uint32_t*>(t.b + ob + 16 * e) = hi;
            *reinterpret_cast<uint32_t*>(t.b + NC * 128 + ob + 16 * e) = lo;
        }
    }
    tc5_product<PREC, NC>(t, t.a2);
    // ---- read-back: D2 row 2 n1 j + 2 k1 + r, column (k2 mod n1) CX + c -> X[k2 + 32 k1][c]
    // (the tile's last readers were the stage-1 conversions, before the first product)
    const int j = m / (2 * N1), k1 = (m % (2 * N1)) >> 1;
    if (t.ok) {
#pragma unroll
        for (int u = 0; u < NCW / 16; ++u) tc5_ld16(lane_addr + wg * NCW + 16 * u, rv[u]);
        tc5_ld_wait<NCW / 16>(rv);
    } else {
#pragma unroll
        for (int u = 0; u < NCW / 16; ++u)
#pragma unroll
            for (int e = 0; e < 8; ++e) rv[u][e] = 0u;
    }
#pragma unroll
    for (int u = 0; u < NCW / 16; ++u) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(rv[u][e]);
        const int col0 = wg * NCW + 16 * u + 8 * (lane >> 4) + 4 * ri;
        const int c0 = col0 % CX, kk = j * N1 + col0 / CX + 32 * k1;
        float2 z[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float o = __shfl_xor_sync(0xffffffffu, ri ? v[e] : v[e + 4], 1);
            float2 x = ri ? make_float2(o, v[e + 4]) : make_float2(v[e], o);
            float s = 1.0f;
            if constexpr (PREC == 2) s = col_scale(colmax[c0 + e], true);
            z[e] = make_float2(x.x * s, x.y * (s * CJ));
        }
        float4* dst = reinterpret_cast<float4*>(buf + kk * CX + c0);
        dst[0] = make_float4(z[0].x, z[0].y, z[1].x, z[1].y);
        dst[1] = make_float4(z[2].x, z[2].y, z[3].x, z[3].y);
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
}

}  // namespace kwgb
