// Device building blocks of the FFT passes: complex helpers, in-register
// radix-2^k DFTs and a Stockham line FFT that exchanges through shared memory.
//
// Layout contract of line_fft: a line of N = 2^LOGN complex values is held by
// TL = N / E threads; thread j keeps element j + TL*m in register v[m]
// (m = 0..E-1).  That is the layout a coalesced load of the line gives (the
// threads of a warp touch consecutive elements), so the first pass reads
// straight from registers, and the Stockham last pass lands each output in
// the same layout (natural order), so no reordering exchange is needed before
// the store.  Only the passes in between go through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kwgb {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// cos(2 pi m / 16): the real parts of the 16th roots of unity.
__host__ __device__ constexpr float cos16(int m) {
    return (m & 15) == 0 ? 1.0f
         : (m & 15) == 1 || (m & 15) == 15 ? 0.92387953251128675613f
         : (m & 15) == 2 || (m & 15) == 14 ? 0.70710678118654752440f
         : (m & 15) == 3 || (m & 15) == 13 ? 0.38268343236508977173f
         : (m & 15) == 4 || (m & 15) == 12 ? 0.0f
         : (m & 15) == 5 || (m & 15) == 11 ? -0.38268343236508977173f
         : (m & 15) == 6 || (m & 15) == 10 ? -0.70710678118654752440f
         : (m & 15) == 7 || (m & 15) == 9 ? -0.92387953251128675613f
         : -1.0f;
}
__host__ __device__ constexpr float sin16(int m) { return cos16(m - 4); }

// d * exp(DIR * 2 pi i * m / 16) for a compile-time m (after unrolling).
template <int DIR>
__device__ __forceinline__ float2 rot16(float2 d, int m) {
    m &= 15;
    if (m == 0) return d;
    if (m == 4) return DIR > 0 ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    if (m == 8) return make_float2(-d.x, -d.y);
    if (m == 12) return DIR > 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    const float c = cos16(m), s = DIR > 0 ? sin16(m) : -sin16(m);
    return make_float2(fmaf(d.x, c, -d.y * s), fmaf(d.x, s, d.y * c));
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
// Bit reversal of the low `bits` (<= 4) bits of i, written without recursion
// so that it folds to a constant once the calling loop is unrolled.
__host__ __device__ constexpr int bitrev(int i, int bits) {
    return (((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3)) >> (4 - bits);
}

// In-register DFT of size R (2, 4, 8 or 16):
//   v[k] <- sum_r v[r] exp(DIR 2 pi i r k / R)
// as radix-2 decimation in frequency followed by a compile-time bit reversal.
// Every loop has a compile-time trip count (the stage loop runs over the
// stage index, not over a shifted span) so that it unrolls completely and
// the array stays in registers.
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v) {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "radix");
    constexpr int LR = ilog2c(R);
#pragma unroll
    for (int st = 0; st < LR; ++st) {
        const int span = R >> (st + 1);
#pragma unroll
        for (int g = 0; g < (1 << st); ++g) {
#pragma unroll
            for (int j = 0; j < (R >> (st + 1)); ++j) {
                const int start = g * 2 * span;
                const float2 a = v[start + j], b = v[start + j + span];
                v[start + j] = cadd(a, b);
                v[start + j + span] = rot16<DIR>(csub(a, b), j * (16 / (2 * span)));
            }
        }
    }
    if (R > 2) {
        float2 t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[bitrev(i, LR)];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = t[i];
    }
}

// The twiddle table (Tables::tw, float2, generated in float64) has three
// regions; every entry is exp(-2 pi i theta):
//   [0, 1024)            theta = t / 1024
//   stage blocks         one per (L, RP), at stw_off(L, RP): entry (r-1) L/RP + k
//                        holds theta = k r / L for k < L/RP, 1 <= r < RP -- the
//                        twiddles of a radix-RP Stockham pass that builds
//                        transforms of length L.  The lanes of a warp hold
//                        consecutive k, so they read consecutive entries (one or
//                        two L1 wavefronts per load instead of one per line touched
//                        by the strided index k r 1024/L).
//   row blocks           one per M (2 <= M <= 512), at rtw_off(M): entry k holds
//                        theta = k / (2 M), k < M (pre/post step of the real
//                        transforms of rows of 2M values)
__host__ __device__ constexpr int stw_off(int L, int RP) {
    int off = 1024;
    for (int l = 2; l < L; l *= 2)
        for (int rp = 2; rp <= 16 && rp <= l; rp *= 2) off += l - l / rp;
    for (int rp = 2; rp < RP; rp *= 2) off += L - L / rp;
    return off;
}
__host__ __device__ constexpr int rtw_off(int M) { return stw_off(2048, 2) + M - 2; }
constexpr int TW_TOTAL = rtw_off(1024);            // entries of the whole table

// exp(DIR 2 pi i k r / L) of a radix-RP pass building length-L transforms.
template <int DIR, int L, int RP>
__device__ __forceinline__ float2 stage_twiddle(const float2* __restrict__ tw, int k, int r) {
    constexpr int off = stw_off(L, RP);
    const float2 w = __ldg(tw + off + (r - 1) * (L / RP) + k);
    return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// exp(DIR 2 pi i k / (2 M)), k < M.
template <int DIR, int M>
__device__ __forceinline__ float2 row_twiddle(const float2* __restrict__ tw, int k) {
    constexpr int off = rtw_off(M);
    const float2 w = __ldg(tw + off + k);
    return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// exp(DIR 2 pi i t / 1024) from the table tw[t] = exp(-2 pi i t / 1024).
template <int DIR>
__device__ __forceinline__ float2 twiddle1024(const float2* __restrict__ tw, int t) {
    const float2 w = __ldg(tw + (t & 1023));
    return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// One Stockham pass of radix RP at stride NS on a line of N = 2^LOGN held in
// the register layout above (E elements per thread, TL threads per line).
// Butterfly b = j + TL*i (i < E/RP) reads elements b + r*N/RP (= register
// i + r*E/RP), multiplies input r by exp(DIR 2 pi i (b mod NS) r / (NS RP)),
// takes an RP-point DFT and sends output q to element
// (b / NS) * NS * RP + (b mod NS) + q * NS.
// LAST: that position is the thread's own register layout; otherwise the
// outputs go through shared memory (S.at(e) gives element e's slot; an Smem
// with PINGPONG has two buffers, S.at_pp<B>(e)).
template <int LOGN, int E, int RP, int NS, int DIR, bool LAST, class Smem>
__device__ __forceinline__ void stockham_pass(float2 (&v)[E], int j, Smem& S,
                                              const float2* __restrict__ tw) {
    constexpr int N = 1 << LOGN;
    constexpr int TL = N / E;
    constexpr int NB = E / RP;          // butterflies per thread
    float2 o[E];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        float2 w[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) w[r] = v[i + r * NB];
        const int b = j + TL * i;
        if (NS > 1) {
            const int k = b & (NS - 1);
#pragma unroll
            for (int r = 1; r < RP; ++r)
                w[r] = cmul(w[r], stage_twiddle<DIR, NS * RP, RP>(tw, k, r));
        }
        dft_reg<RP, DIR>(w);
#pragma unroll
        for (int q = 0; q < RP; ++q) o[i + q * NB] = w[q];
    }
    if (LAST) {
        // b < NS = N / RP: output q of butterfly b is element b + q*N/RP,
        // i.e. register i + q*NB of this thread.
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = o[m];
    } else if constexpr (Smem::PINGPONG) {
        // Two exchange buffers, chosen at compile time: exchange p (0-based,
        // this pass's index; all passes before the last have radix E) writes
        // the scratch buffer for even p and the arrived tile for odd p.  The
        // buffer written was last read before the previous exchange's barrier
        // (or, for p = 0, before the previous transform's second-last
        // barrier), so one barrier per exchange suffices -- except when a
        // transform has an odd number of exchanges: then its last exchange
        // and the next transform's first both write the scratch buffer.
        constexpr int P = ilog2c(NS) / ilog2c(E);
        constexpr int NX = (LOGN + ilog2c(E) - 1) / ilog2c(E) - 1;
        constexpr int B = (P & 1) ? 0 : 1;
        if constexpr (P == 0 && (NX & 1)) S.sync();
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int b = j + TL * i;
            const int base = (b / NS) * NS * RP + (b & (NS - 1));
#pragma unroll
            for (int q = 0; q < RP; ++q) S.template at_pp<B>(base + q * NS) = o[i + q * NB];
        }
        S.sync();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = S.template at_pp<B>(j + TL * m);
    } else {
        S.sync();
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int b = j + TL * i;
            const int base = (b / NS) * NS * RP + (b & (NS - 1));
#pragma unroll
            for (int q = 0; q < RP; ++q) S.at(base + q * NS) = o[i + q * NB];
        }
        S.sync();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = S.at(j + TL * m);
    }
}

// Passes of radix E while they fit, then one pass of the remaining radix.
template <int LOGN, int E, int DIR, int NS, class Smem>
struct StockhamChain {
    __device__ __forceinline__ static void run(float2 (&v)[E], int j, Smem& S,
                                               const float2* __restrict__ tw) {
        constexpr int N = 1 << LOGN;
        constexpr int REM = N / NS;                   // product of radices still to apply
        constexpr int RP = REM >= E ? E : REM;
        constexpr bool LAST = (NS * RP == N);
        stockham_pass<LOGN, E, RP, NS, DIR, LAST>(v, j, S, tw);
        StockhamChain<LOGN, E, DIR, (LAST ? N : NS * RP), Smem>::run_next(v, j, S, tw);
    }
    __device__ __forceinline__ static void run_next(float2 (&v)[E], int j, Smem& S,
                                                    const float2* __restrict__ tw) {
        if (NS < (1 << LOGN)) run(v, j, S, tw);
    }
};
template <int LOGN, int E, int DIR, class Smem>
struct StockhamChain<LOGN, E, DIR, (1 << LOGN), Smem> {
    __device__ __forceinline__ static void run(float2 (&)[E], int, Smem&, const float2*) {}
    __device__ __forceinline__ static void run_next(float2 (&)[E], int, Smem&, const float2*) {}
};

// Unnormalised DFT of the line, DIR = -1 forward, +1 inverse.
template <int LOGN, int E, int DIR, class Smem>
__device__ __forceinline__ void line_fft(float2 (&v)[E], int j, Smem& S,
                                         const float2* __restrict__ tw) {
    StockhamChain<LOGN, E, DIR, 1, Smem>::run(v, j, S, tw);
}

}  // namespace kwgb
