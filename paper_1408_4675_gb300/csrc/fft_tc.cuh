// Split-precision tensor-core form of the strided FFT passes of 16- and
// 32-point lines (mma.sync; lines of 64 points and more run on tcgen05,
// fft_tc5.cuh, which reuses the operand splits and float16 column scales
// defined here).
//
// A tile (CX columns x N points, layout [e][c] in shared memory) is
// transformed in place.  Every radix-8 Stockham stage is written as a real
// matrix product on the tensor cores: the 8-point complex DFT in real form is
// the 16 x 16 matrix
//     W = [[C, -S], [S, C]],  C + iS = exp(DIR 2 pi i r k / 8),
// acting on columns [Re x_0..Re x_7, Im x_0..Im x_7] of 8 butterflies at a
// time (mma.sync m16n8k16: W as the A operand, the butterflies as B, float32
// accumulation).  Both operands are split into bfloat16 hi + lo parts
// (hi = bf16(v), lo = bf16(v - hi)) and the product is formed as
// W_hi X_hi + W_hi X_lo + W_lo X_hi, which keeps about 16 significant bits of
// every operand (the dropped W_lo X_lo term is of relative size 2^-16).
// PREC 2 uses float16 hi + lo instead (11 + 11 significant bits, relative
// residue 2^-22): float16 has a narrow exponent range, so each column is
// scaled by a power of two (exact) that brings its largest input to [32, 64);
// 8-point stages grow values at most 8x, so a column stays far below the
// float16 maximum 65504; outputs are scaled back before they are stored.
// A remaining radix-2 or radix-4 stage runs in float32 on the CUDA cores.
// Each thread reads its B fragment (two complex inputs of one butterfly)
// straight from the Stockham input positions, applies the stage twiddles, and
// writes its D fragment (one complex output of two butterflies) straight to
// the Stockham output positions, so no extra shuffles are needed.  Between
// passes the tile is XOR-swizzled so that the accesses are free of bank
// conflicts (TcSwz, TcXor).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fft_core.cuh"

namespace kwgb {

__device__ __forceinline__ uint32_t pack_bf16(float lo_half, float hi_half) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo_half, hi_half);   // .x in the low 16 bits
    return *reinterpret_cast<uint32_t*>(&v);
}

// split a pair (a, b) into packed bf16 hi and lo words
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const float ra = a - __bfloat162float(ha), rb = b - __bfloat162float(hb);
    __nv_bfloat162 h;
    h.x = ha;
    h.y = hb;
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = pack_bf16(ra, rb);
}

// split a pair (a, b) into packed float16 hi and lo words
__device__ __forceinline__ void split_f16(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    const float ra = a - __half2float(ha), rb = b - __half2float(hb);
    __half2 h;
    h.x = ha;
    h.y = hb;
    hi = *reinterpret_cast<uint32_t*>(&h);
    __half2 l = __floats2half2_rn(ra, rb);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (PREC == 2) split_f16(a, b, hi, lo);
    else split_bf16(a, b, hi, lo);
}

template <int PREC>
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (PREC == 2) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
            "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
            "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// A fragments (hi and lo) of the real 16 x 16 DFT-8 matrix for this lane:
// reg0 (row g, cols 2t, 2t+1) = C, reg1 (row g+8) = S, reg2 (row g, cols 2t+8..) = -S,
// reg3 (row g+8, cols 2t+8..) = C, with C + iS = exp(DIR 2 pi i g k / 8).
template <int DIR, int PREC>
__device__ __forceinline__ void dft8_matrix(int lane, uint32_t (&ah)[4], uint32_t (&al)[4]) {
    const int g = lane >> 2, t = lane & 3;
    float c[2], s[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int m = (2 * g * (2 * t + i)) & 15;             // 2 pi g k / 8 = 2 pi (2 g k) / 16
        c[i] = cos16(m);
        s[i] = DIR > 0 ? sin16(m) : -sin16(m);
    }
    split2<PREC>(c[0], c[1], ah[0], al[0]);
    split2<PREC>(s[0], s[1], ah[1], al[1]);
    split2<PREC>(-s[0], -s[1], ah[2], al[2]);
    split2<PREC>(c[0], c[1], ah[3], al[3]);
}

// Layout of a tile between two tensor-core stages (the first stage reads and
// the last writes the plain layout [e][c] that the TMA and the float32 code
// use).  A stage's lanes (g = lane / 4, t = lane % 4) read rows b + (2t + d) N/8
// of four columns and write rows base + g NS of four columns; in the plain
// layout the four rows of a half-warp fall on the same banks (64-bit accesses
// are served per half-warp: four-way conflicts).  Here element (e, c) sits at
// row e ^ P(e), column c ^ H(e), with P and H bits formed as parities of row
// bits:
//   A = bits {0, 3, 6, 9}     separates the rows g NS of a write (with C),
//   C = bits {1, 4, 7, 10}    (plus bit Q+1 when it holds neither Q nor Q+1),
//   B = bit Q or Q+1          separates the rows b + (2t + d) N/8 of a read
//                             (with C), Q = log2 N - 2;
// 16 columns: H = A | B << 2 | C << 3, P = 0; 8 columns (a row is 16 banks):
// H = A | B << 2 and P = C flips the row's bank half.  Every access of every
// stage of the tiles used here is then one wavefront per half-warp (checked by
// enumerating the accesses).  A, B, C are parities, hence XOR-linear: for rows
// whose parts occupy disjoint bits, H(x + y) = H(x) ^ H(y), so the per-lane
// parts are computed once.
template <int LOGN, int CX>
struct TcSwz {
    static_assert(CX == 8 || CX == 16, "tile width");
    static constexpr int Q = LOGN - 2;
    static constexpr uint32_t A = 0x249u;
    static constexpr uint32_t C0 = 0x492u;
    static constexpr uint32_t C = ((C0 >> Q) & 3u) ? C0 : (C0 | (1u << (Q + 1)));
    static constexpr uint32_t B = ((C >> (Q + 1)) & 1u) ? (1u << Q) : (1u << (Q + 1));
    __device__ __forceinline__ static int par(uint32_t m, int r) { return __popc((uint32_t)r & m) & 1; }
    __device__ __forceinline__ static int hcol(int r) {
        return par(A, r) | (par(B, r) << 2) | (CX == 16 ? (par(C, r) << 3) : 0);
    }
    __device__ __forceinline__ static int hrow(int r) { return CX == 8 ? par(C, r) : 0; }
    // index of (row, col) given the row's H and P
    __device__ __forceinline__ static int at(int row, int col, int h, int p) { return (row ^ p) * CX + (col ^ h); }
    __device__ __forceinline__ static int idx(int row, int col) { return at(row, col, hcol(row), hrow(row)); }
};

// A tile layout given by its masks: bit k of H is the parity of the row bits in
// Mk, P the parity of the row bits in MP (element (e, c) at row e ^ P(e),
// column c ^ H(e), as in TcSwz).  MP must not hold bit 0, so that the row map
// is a bijection.  All masks zero: the plain layout [e][c].
template <int CX, uint32_t M0, uint32_t M1, uint32_t M2, uint32_t M3, uint32_t MP>
struct TcXor {
    static_assert(CX == 8 || CX == 16, "tile width");
    static_assert((CX == 16 || M3 == 0) && (CX == 8 || MP == 0) && (MP & 1u) == 0, "layout masks");
    __device__ __forceinline__ static int par(uint32_t m, int r) { return m ? (__popc((uint32_t)r & m) & 1) : 0; }
    __device__ __forceinline__ static int hcol(int r) {
        return par(M0, r) | (par(M1, r) << 1) | (par(M2, r) << 2) | (par(M3, r) << 3);
    }
    __device__ __forceinline__ static int hrow(int r) { return par(MP, r); }
    __device__ __forceinline__ static int at(int row, int col, int h, int p) { return (row ^ p) * CX + (col ^ h); }
    __device__ __forceinline__ static int idx(int row, int col) { return at(row, col, hcol(row), hrow(row)); }
};
template <int CX>
using TcPlain = TcXor<CX, 0u, 0u, 0u, 0u, 0u>;

// Float16-split column scale from the bits of the column maximum m (a
// non-negative float, biased exponent ex): 2^k with k = 132 - ex, so that
// m 2^k lies in [32, 64), or 2^-k when `inverse`; k is clamped to [-100, 100]
// (a zero column takes 2^100, a non-finite one 2^-100: both stay what they
// are).  Branch-free: the result's biased exponent is 127 +- k.
__device__ __forceinline__ float col_scale(unsigned int mbits, bool inverse) {
    const int ex = (int)(mbits >> 23);                           // sign bit clear
    const int be = inverse ? ex - 5 : 259 - ex;
    return __int_as_float(max(27, min(227, be)) << 23);
}

// Column maxima of the float16-split form: two buffers of 16 words in shared
// memory that alternate between transforms (all zero at the start); a
// transform fills buffer `cur` and clears the other one for the next.
struct TcColMax {
    unsigned int* m;
    int cur;
};

// One radix-8 Stockham stage (stride NS) of a tile, on the tensor cores.
// Butterfly beta = 32 w + 8 G + n (column c = beta % CX, butterfly b = beta / CX).
// LI / LO: the layouts the stage reads and writes (TcSwz, TcXor).
template <int N, int CX, int NS, int DIR, int THREADS, int PREC, class LI, class LO>
__device__ __forceinline__ void tc_stage8(float2* buf, const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          const float2* __restrict__ tw, const unsigned int* colmax) {
    constexpr int NBF = CX * N / 8;                           // butterflies in the tile
    constexpr int WARPS = THREADS / 32;
    constexpr int GROUPS = NBF / (8 * WARPS);                 // 8-butterfly groups per warp
    static_assert(NBF % (8 * WARPS) == 0, "tile / warp split");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // per-lane parts of the layouts: read rows b + (2t + d) N/8, write rows base + g NS
    const int rr0 = (2 * t) * (N / 8), rr1 = (2 * t + 1) * (N / 8);
    const int hr0 = LI::hcol(rr0), pr0 = LI::hrow(rr0), hr1 = LI::hcol(rr1), pr1 = LI::hrow(rr1);
    const int hw = LO::hcol(g * NS), pw = LO::hrow(g * NS);
    float d[GROUPS][4];
#pragma unroll
    for (int G = 0; G < GROUPS; ++G) {
        const int beta = (w * GROUPS + G) * 8 + g;            // this lane's B column
        const int c = beta % CX, b = beta / CX;
        const int hb = LI::hcol(b), pb = LI::hrow(b);
        float2 x0 = buf[LI::at(b + rr0, c, hb ^ hr0, pb ^ pr0)];
        float2 x1 = buf[LI::at(b + rr1, c, hb ^ hr1, pb ^ pr1)];
        if (NS > 1) {
            const int k = b & (NS - 1);
            x0 = cmul(x0, twiddle1024<DIR>(tw, k * (2 * t) * (1024 / (NS * 8))));
            x1 = cmul(x1, twiddle1024<DIR>(tw, k * (2 * t + 1) * (1024 / (NS * 8))));
        }
        if (PREC == 2) {
            const float sc = col_scale(colmax[c], false);
            x0 = cscale(x0, sc);
            x1 = cscale(x1, sc);
        }
        uint32_t bh0, bl0, bh1, bl1;
        split2<PREC>(x0.x, x1.x, bh0, bl0);                   // rows 2t, 2t+1: real parts
        split2<PREC>(x0.y, x1.y, bh1, bl1);                   // rows 2t+8, 2t+9: imaginary parts
        d[G][0] = d[G][1] = d[G][2] = d[G][3] = 0.f;
        mma_16816<PREC>(d[G], al, bh0, bh1);
        mma_16816<PREC>(d[G], ah, bl0, bl1);
        mma_16816<PREC>(d[G], ah, bh0, bh1);
    }
    __syncthreads();                                          // all inputs read
#pragma unroll
    for (int G = 0; G < GROUPS; ++G) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {                         // output g of butterflies 2t, 2t+1
            const int beta = (w * GROUPS + G) * 8 + 2 * t + i;
            const int c = beta % CX, b = beta / CX;
            const int base = (b / NS) * NS * 8 + (b & (NS - 1));
            const float us = PREC == 2 ? col_scale(colmax[c], true) : 1.0f;
            const float2 o = make_float2(d[G][i] * us, d[G][2 + i] * us);
            buf[LO::at(base + g * NS, c, LO::hcol(base) ^ hw, LO::hrow(base) ^ pw)] = o;
        }
    }
    __syncthreads();
}

// A float32 radix-RP Stockham stage (RP = 2 or 4) on the tile in shared memory;
// the last stage of a transform: reads layout LI, writes the plain layout.
template <int N, int CX, int RP, int NS, int DIR, int THREADS, class LI>
__device__ __forceinline__ void f32_stage(float2* buf, const float2* __restrict__ tw) {
    constexpr int NBF = CX * N / RP;
    float2 o[(NBF + THREADS - 1) / THREADS][RP];
#pragma unroll
    for (int q = 0; q < (NBF + THREADS - 1) / THREADS; ++q) {
        const int beta = threadIdx.x + q * THREADS;
        if (beta < NBF) {
            const int c = beta % CX, b = beta / CX;
            float2 v[RP];
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const int row = b + r * (N / RP);
                v[r] = buf[LI::idx(row, c)];
            }
            if (NS > 1) {
                const int k = b & (NS - 1);
#pragma unroll
                for (int r = 1; r < RP; ++r) v[r] = cmul(v[r], twiddle1024<DIR>(tw, k * r * (1024 / (NS * RP))));
            }
            dft_reg<RP, DIR>(v);
#pragma unroll
            for (int r = 0; r < RP; ++r) o[q][r] = v[r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (NBF + THREADS - 1) / THREADS; ++q) {
        const int beta = threadIdx.x + q * THREADS;
        if (beta < NBF) {
            const int c = beta % CX, b = beta / CX;
            const int base = (b / NS) * NS * RP + (b & (NS - 1));
#pragma unroll
            for (int r = 0; r < RP; ++r) buf[(base + r * NS) * CX + c] = o[q][r];
        }
    }
    __syncthreads();
}

// Radix-8 tensor-core stages while they fit, then one float32 stage of the rest.
template <int LOGN, int CX, int DIR, int THREADS, int PREC, int NS>
struct TcChain {
    __device__ __forceinline__ static void run(float2* buf, const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                               const float2* __restrict__ tw, const unsigned int* colmax) {
        constexpr int N = 1 << LOGN;
        constexpr int REM = N / NS;
        if constexpr (REM >= 8) {
            using LI = std::conditional_t<(NS > 1), TcSwz<LOGN, CX>, TcPlain<CX>>;
            using LO = std::conditional_t<(NS * 8 < N), TcSwz<LOGN, CX>, TcPlain<CX>>;
            tc_stage8<N, CX, NS, DIR, THREADS, PREC, LI, LO>(buf, ah, al, tw, colmax);
            TcChain<LOGN, CX, DIR, THREADS, PREC, NS * 8>::run(buf, ah, al, tw, colmax);
        } else {
            using LI = std::conditional_t<(NS > 1), TcSwz<LOGN, CX>, TcPlain<CX>>;
            f32_stage<N, CX, (REM >= 4 ? 4 : 2), NS, DIR, THREADS, LI>(buf, tw);
        }
    }
};
template <int LOGN, int CX, int DIR, int THREADS, int PREC>
struct TcChain<LOGN, CX, DIR, THREADS, PREC, (1 << LOGN)> {
    __device__ __forceinline__ static void run(float2*, const uint32_t (&)[4], const uint32_t (&)[4],
                                               const float2*, const unsigned int*) {}
};

// Float16-split: a thread's maximum m of the column threadIdx.x % CX goes into
// the current buffer of cmx (a butterfly over the lanes of the same column, one
// shared atomic per column and warp), and the other buffer is cleared for the
// next transform (its last readers were the stages of the previous one).
template <int CX>
__device__ __forceinline__ void tc_colmax_deposit(float m, TcColMax& cmx) {
#pragma unroll
    for (int o = CX; o < 32; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) < CX) atomicMax(cmx.m + 16 * cmx.cur + (threadIdx.x % CX), __float_as_uint(m));   // non-negative floats order as integers
    if (threadIdx.x < CX) cmx.m[16 * (cmx.cur ^ 1) + threadIdx.x] = 0u;
}

// In-place unnormalised DFT of every column of the tile (natural order in and
// out; plain layout in and out).
// Starts and ends with the tile fully written (callers synchronise before).
// cmx: the column maxima of the float16-split form (PREC 2).  SCAN: the
// transform reads the tile for them; otherwise every thread has already
// deposited them (tc_colmax_deposit) before the caller's barrier.
template <int LOGN, int CX, int DIR, int THREADS, int PREC, bool SCAN = true>
__device__ __forceinline__ void tile_fft_tc(float2* buf, const float2* __restrict__ tw, TcColMax& cmx) {
    static_assert(LOGN <= 5, "16- and 32-point lines (longer lines: tile_fft_tc5)");
    uint32_t ah[4], al[4];
    dft8_matrix<DIR, PREC>(threadIdx.x & 31, ah, al);
    unsigned int* colmax = cmx.m + 16 * cmx.cur;
    if constexpr (PREC == 2 && SCAN) {
        // per column: largest |Re|, |Im| (each stage turns it into its power-of-two scale)
        constexpr int N = 1 << LOGN;
        static_assert(THREADS % CX == 0 && CX <= 16 && (N * CX) % THREADS == 0, "column of a thread");
        // every element a thread visits lies in column threadIdx.x % CX
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
    TcChain<LOGN, CX, DIR, THREADS, PREC, 1>::run(buf, ah, al, tw, colmax);
}

}  // namespace kwgb
