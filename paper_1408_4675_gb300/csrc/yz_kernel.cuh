#pragma once
// Strided-axis FFT passes on the half spectra [nz][ny][nhp] (complex64).
//
// Work item = a tile of CX consecutive x-columns times one whole line along
// y (y pass) or z (z pass).  The kernels are persistent: each CTA walks its
// share of the tiles with a two-stage shared-memory ring that the TMA unit
// fills (cp.async.bulk.tensor, box CX x 256 lines, completion on an
// mbarrier), so the HBM reads of tile t+1 run while tile t is transformed.
// The x extent of the tensor map is nh (not the padded pitch), so the ragged
// last tile reads no padding: the TMA zero-fills those columns.
//
// Thread (c, j) takes elements j + TL*m of column c into registers; the
// Stockham passes exchange through the stage buffer the tile arrived in, and
// results are stored from registers (a warp writes whole 64..128-byte row
// segments).
//
// The z pass is the fused spectral-operator pass: forward z FFT, the
// pointwise operator of Eq. 4a, 4c or 8 (all of kx, ky, kz are known here),
// inverse z FFT, store.  It plays the role of the paper's transposed-space
// spectral multiply (Sec. 3.2): the spectrum does not return to HBM between
// the forward and the inverse transform along z.
#include <algorithm>

#include "fft_core.cuh"
#include "fft_tc.cuh"
#include "fft_tc5.cuh"
#include "kwgb_internal.h"
#include "tma.cuh"

namespace kwgb {

enum { OP_Y_FWD = 0, OP_Y_INV = 1, OP_Z_GRAD_FWD = 2, OP_Z_GRAD_BWD = 3, OP_Z_DIV = 4, OP_Z_ABS = 5,
       OP_Z_DIV_FWD = 6, OP_Z_DIV_SUM = 7 };

// Column c of a tile in shared memory.  The TMA lands element e of every
// column as row e (CX float2, dense): raw(e).  The float32 passes (PP)
// exchange through two buffers, the arrived tile (B = 0) and a scratch tile
// (B = 1), one barrier per exchange (fft_core.cuh).  Rows stay in order: a
// swizzle against the bank conflicts of the first exchange cost more
// registers and address arithmetic than the conflicts cost.
template <int CX, bool PP>
struct TileSmem {
    float2* buf;              // the arrived tile
    float2* scr;              // scratch tile (PP)
    int c;
    static constexpr bool PINGPONG = PP;
    __device__ __forceinline__ float2& at(int e) { return buf[e * CX + c]; }
    __device__ __forceinline__ float2& raw(int e) { return buf[e * CX + c]; }
    template <int B>
    __device__ __forceinline__ float2& at_pp(int e) { return (B ? scr : buf)[e * CX + c]; }
    __device__ __forceinline__ void sync() { __syncthreads(); }
};

// MIXED: the tensor-core forms take 8-column tiles of 256 threads for 512-point
// y lines (64 KB per CTA: two CTAs per SM; the float32 y pass keeps 16 columns)
template <int LOGN, bool ISY, int MIXED = 0>
struct TShape {
    static constexpr int N = 1 << LOGN;
    // tensor-core form: lines of 64 points and more run on tcgen05 (fft_tc5.cuh),
    // shorter ones on mma.sync (fft_tc.cuh)
    static constexpr bool TC5 = MIXED != 0 && LOGN >= 6;
    // z: E = 8 keeps the operator pass spill-free at two CTAs per SM; 1024-point
    // lines take E = 16 so that a tile stays 8 columns (64-byte TMA rows) wide.
    // tcgen05 form: 16 values per thread (8 for 64-point lines, which need the
    // four warps of a tensor-memory read-back) and tiles of at most 256
    // threads (4 columns for 1024-point lines), so that two CTAs share an SM
    static constexpr int E = TC5 ? ((LOGN == 10 || LOGN == 7) ? 16 : 8) : (ISY ? (LOGN >= 8 ? 16 : 8) : (LOGN >= 10 ? 16 : 8));
    static constexpr int TL = N / E;
    static constexpr int MAXT = TC5 ? 256 : ((ISY && MIXED && LOGN == 9) ? 256 : 512);
    static constexpr int CX = (MAXT / TL) >= 16 ? 16 : (MAXT / TL);
    static constexpr int THREADS = CX * TL;
    static constexpr int BOX = N < 256 ? N : 256;
    static constexpr int NBOX = N / BOX;
    static constexpr int STAGE = N * CX;                       // complex elements per stage
    static constexpr int NST = TC5 ? 1 : 2;                    // TMA stages (tcgen05: one, two CTAs per SM)
    static constexpr int NC = (N / 32) * CX;                   // product columns of a tile
    static constexpr int TC5_TMEM = tc5_tmem_cols(NC);
    static constexpr int TC5_A = (LOGN == 10 ? 2 : 4) * TC5_A_BYTES;   // A operands (one set for 1024 points)
    // two TMA stages, plus the scratch exchange buffer of the float32 passes, or
    // (tcgen05) one stage, 1 KB of barriers, the A operands and the B operand (hi, lo)
    static constexpr int smem(int mixed) {
        return TC5 ? STAGE * (int)sizeof(float2) + 1024 + TC5_A + 2 * NC * 128
                   : (mixed ? 2 : 3) * STAGE * (int)sizeof(float2) + 64;
    }
};

struct alignas(64) YZK {
    CUtensorMap map[3];       // input tensor maps (box of the pass)
    GridC g;
    float2* out[3];
    int ncomp;                // y pass: components (items carry the component)
    int nloads;               // z pass: loads per item
    int load_comp[3];         // z pass: component of each load
    int* flag;
};

// sinc(x) = sin(x)/x with sinc(0) = 1 (kappa of Sec. 2.2), as a function of
// x^2 so that no square root is needed on the usual path: the Taylor series
// sum_n (-x^2)^n / (2n+1)! up to n = 5 for x^2 <= 2 (truncation error below
// 2^6/13! < 1.1e-8, under float32 rounding; every grid point at CFL <= 0.5
// takes this branch), up to n = 9 for x^2 <= 9 (below 3^20/21! < 7e-11),
// beyond that sin(x)/x directly.
__device__ __forceinline__ float sinc_sq(float x2) {
    if (x2 <= 2.0f) {
        float p = -1.0f / 39916800.0f;                // -1/11!
        p = fmaf(p, x2, 1.0f / 362880.0f);            //  1/9!
        p = fmaf(p, x2, -1.0f / 5040.0f);             // -1/7!
        p = fmaf(p, x2, 1.0f / 120.0f);               //  1/5!
        p = fmaf(p, x2, -1.0f / 6.0f);                // -1/3!
        return fmaf(p, x2, 1.0f);
    }
    if (x2 > 9.0f) {
        const float x = sqrtf(x2);
        return __fdividef(sinf(x), x);
    }
    float p = -1.0f / 121645100408832000.0f;          // -1/19!
    p = fmaf(p, x2, 1.0f / 355687428096000.0f);       //  1/17!
    p = fmaf(p, x2, -1.0f / 1307674368000.0f);        // -1/15!
    p = fmaf(p, x2, 1.0f / 6227020800.0f);            //  1/13!
    p = fmaf(p, x2, -1.0f / 39916800.0f);             // -1/11!
    p = fmaf(p, x2, 1.0f / 362880.0f);                //  1/9!
    p = fmaf(p, x2, -1.0f / 5040.0f);                 // -1/7!
    p = fmaf(p, x2, 1.0f / 120.0f);                   //  1/5!
    p = fmaf(p, x2, -1.0f / 6.0f);                    // -1/3!
    return fmaf(p, x2, 1.0f);
}

// a.out[i] for a run-time i without copying the parameter array to local memory
__device__ __forceinline__ float2* out_ptr(const YZK& a, int i) {
    return i == 0 ? a.out[0] : (i == 1 ? a.out[1] : a.out[2]);
}

// Inverse transform of the register layout v (element j + TL*m of column c):
// float32 register passes, or (MIXED) through the tile in shared memory.
template <int LOGN, int E, int CX, int THREADS, int MIXED>
__device__ __forceinline__ void inverse_tile(float2 (&v)[E], int j, TileSmem<CX, MIXED == 0>& S, float2* tile,
                                             const float2* __restrict__ tw, TcColMax& cmx, Tc5& t5) {
    constexpr int TL = (1 << LOGN) / E;
    if constexpr (MIXED == 0) {
        line_fft<LOGN, E, +1>(v, j, S, tw);
    } else {
        __syncthreads();                              // every thread is done reading the tile
#pragma unroll
        for (int m = 0; m < E; ++m) S.at(j + TL * m) = v[m];
        if constexpr (MIXED == 2) {                   // column maxima from the registers: no tile scan
            float mx = 0.f;
#pragma unroll
            for (int m = 0; m < E; ++m) mx = fmaxf(mx, fmaxf(fabsf(v[m].x), fabsf(v[m].y)));
            tc_colmax_deposit<CX>(mx, cmx);
        }
        __syncthreads();
        if constexpr (LOGN >= 6) {
            tile_fft_tc5<LOGN, CX, +1, THREADS, MIXED, false>(tile, t5, tw, cmx);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = tile[(j + TL * m) * CX + S.c];
        } else {
            tile_fft_tc<LOGN, CX, +1, THREADS, MIXED, false>(tile, tw, cmx);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = tile[(j + TL * m) * CX + S.c];
        }
    }
}

// MIXED = 1 / 2: the transforms run as bfloat16- / float16-split tensor-core
// products on the tile in shared memory (fft_tc.cuh) instead of the float32
// register passes.  Two CTAs per SM for the z passes of 512-point lines in
// both forms (the mixed form then spills a few words of its operator values,
// which costs less than the idle barrier time of one CTA per SM).
template <int LOGN, int OP, int MIXED>
constexpr int yz_min_blocks() {
    if (MIXED && LOGN >= 6) return (LOGN == 8 || LOGN == 9) ? 3 : 2;   // tcgen05 form: two or three CTAs per SM
    if (OP < 2) return (MIXED && LOGN == 9) ? 3 : 1;
    if (LOGN >= 10) return 1;
    return (MIXED && LOGN != 9) ? 1 : 2;
}

template <int LOGN, int OP, int MIXED>
__global__ void __launch_bounds__(TShape<LOGN, (OP < 2), MIXED>::THREADS, yz_min_blocks<LOGN, OP, MIXED>())
yz_kernel(const __grid_constant__ YZK a) {
    constexpr bool ISY = OP < 2;
    using Sh = TShape<LOGN, ISY, MIXED>;
    constexpr int E = Sh::E, TL = Sh::TL, CX = Sh::CX, STAGE = Sh::STAGE;
    extern __shared__ __align__(128) float2 smem[];
    __shared__ int abort_flag;
    __shared__ unsigned int colmax[32];              // column maxima of the float16-split form (2 buffers)
    constexpr int NST = Sh::NST;
    float2* scratch = smem + 2 * STAGE;             // float32 exchanges (not used by MIXED)
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (Sh::TC5 ? 1 : (MIXED ? 2 : 3)) * STAGE);
    const GridC& g = a.g;
    const int tid = threadIdx.x;
    const int c = tid % CX, j = tid / CX;
    const int nchunk = (g.nh + CX - 1) / CX;
    const int lines = ISY ? g.nz : g.ny;
    const int items = nchunk * lines * (ISY ? a.ncomp : 1);
    // loads per tile: compile-time where the operator fixes it, so that values kept
    // for the loads of a tile are provably dead at the end of the tile
    constexpr int LC = (ISY || OP == OP_Z_GRAD_FWD || OP == OP_Z_GRAD_BWD) ? 1
                       : ((OP == OP_Z_DIV || OP == OP_Z_DIV_FWD || OP == OP_Z_DIV_SUM) ? 3 : 0);
    const int L = LC ? LC : a.nloads;
    const int my = items > (int)blockIdx.x ? (items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my * L;

    constexpr bool TC5 = Sh::TC5;
    Tc5 t5{};
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    if constexpr (TC5) {
        // A operands from global memory (stage 1, then this axis's stage 2), the
        // product barrier, the accumulator in tensor memory
        unsigned char* base = reinterpret_cast<unsigned char*>(bar);
        t5.bar = bar + 2;
        t5.a1 = base + 1024;
        t5.a2 = LOGN == 10 ? t5.a1 : t5.a1 + 2 * TC5_A_BYTES;
        t5.b = t5.a1 + Sh::TC5_A;
        const uint4* s1 = reinterpret_cast<const uint4*>(g.t.tc5a);
        const uint4* s2 = reinterpret_cast<const uint4*>(g.t.tc5a + (ISY ? 2 : 4) * TC5_A_WORDS);
        for (int i = tid; i < 2 * TC5_A_BYTES / 16; i += Sh::THREADS) {
            reinterpret_cast<uint4*>(t5.a1)[i] = __ldg(s1 + i);
            if (LOGN != 10) reinterpret_cast<uint4*>(t5.a2)[i] = __ldg(s2 + i);
        }
        if (tid < 32) tc5_alloc(tslot, Sh::TC5_TMEM);
        t5.flag = a.flag;
        t5.ok = true;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if (TC5) mbar_init(t5.bar, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    if (tid < 32) colmax[tid] = 0u;
    TcColMax cmx{colmax, 0};
    if (TC5) tc5_fence_before();
    __syncthreads();
    if constexpr (TC5) {
        tc5_fence_after();
        t5.tmem = *tslot;
    }

    auto issue = [&](int q) {                 // thread 0 only
        const int item = (int)blockIdx.x + (q / L) * (int)gridDim.x;
        const int l = q % L;
        const int chunk = item % nchunk;
        const int line = (item / nchunk) % lines;
        const int mi = ISY ? item / (nchunk * lines) : (l == 0 ? a.load_comp[0] : (l == 1 ? a.load_comp[1] : a.load_comp[2]));
        const CUtensorMap* map = mi == 0 ? &a.map[0] : (mi == 1 ? &a.map[1] : &a.map[2]);
        float2* dst = smem + (q % NST) * STAGE;
        uint64_t* b = &bar[q % NST];
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(b, STAGE * (uint32_t)sizeof(float2) + g.wait_fault_tx);
#pragma unroll
        for (int k = 0; k < Sh::NBOX; ++k) {
            if (ISY) tma_load_3d(dst + k * Sh::BOX * CX, map, chunk * CX, k * Sh::BOX, line, b);
            else tma_load_3d(dst + k * Sh::BOX * CX, map, chunk * CX, line, k * Sh::BOX, b);
        }
    };

    if (tid == 0 && Q > 0) issue(0);
    float kap[E];
    float lg[E];
    float2 acc[E];                                   // OP_Z_DIV_SUM: the sum over the tile's loads
#pragma unroll
    for (int m = 0; m < E; ++m) { kap[m] = 0.f; lg[m] = 0.f; }

    for (int q = 0; q < Q; ++q) {
        const int s = q % NST;
        if (NST == 2 && tid == 0 && q + 1 < Q) issue(q + 1);
        const bool ok = mbar_wait_bounded(&bar[s], (q / NST) & 1, a.flag);
        if (!ok) abort_flag = 1;
        const int item = (int)blockIdx.x + (q / L) * (int)gridDim.x;
        const int l = q % L;
        const int chunk = item % nchunk;
        const int line = (item / nchunk) % lines;
        const int col = chunk * CX + c;
        const bool valid = ok && col < g.nh;
        TileSmem<CX, MIXED == 0> S{smem + s * STAGE, scratch, c};
        constexpr int THREADS = Sh::THREADS;
        float2 v[E];
        if constexpr (TC5) {
            tile_fft_tc5<LOGN, CX, (ISY ? (OP == OP_Y_FWD ? -1 : +1) : -1), THREADS, MIXED>(smem + s * STAGE, t5,
                                                                                          g.t.tw, cmx);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = smem[s * STAGE + (j + TL * m) * CX + c];
        } else if constexpr (MIXED != 0) {
            tile_fft_tc<LOGN, CX, (ISY ? (OP == OP_Y_FWD ? -1 : +1) : -1), THREADS, MIXED>(smem + s * STAGE, g.t.tw, cmx);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = smem[s * STAGE + (j + TL * m) * CX + c];
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = S.raw(j + TL * m);
        }

        if (ISY) {
            const int comp = item / (nchunk * lines);
            if (!MIXED) line_fft<LOGN, E, (OP == OP_Y_FWD ? -1 : +1)>(v, j, S, g.t.tw);
            if (valid) {
                float2* out = out_ptr(a, comp) + (size_t)line * g.ny * g.nhp + col;
#pragma unroll
                for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * g.nhp, v[m]);
            }
        } else {
            const int y = line;
            const size_t es = (size_t)g.ny * g.nhp;
            const size_t off = (size_t)y * g.nhp + col;
            const float kx = col < g.nh ? __ldg(g.t.kx + col) : 0.f;
            const float ky = __ldg(g.t.ky + y);
            if (l == 0) {                            // operator values of this tile, kept for its loads
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const float kz = __ldg(g.t.kz + j + TL * m);
                    const float k2 = fmaf(kx, kx, fmaf(ky, ky, kz * kz));
                    if (OP == OP_Z_ABS) lg[m] = k2 > 0.f ? log2f(k2 * g.inv_kmax2) : -INFINITY;
                    else kap[m] = sinc_sq(g.hk2 * k2) * g.scale;
                }
            }
            if (!MIXED) line_fft<LOGN, E, -1>(v, j, S, g.t.tw);
            if (OP == OP_Z_GRAD_FWD || OP == OP_Z_GRAD_BWD) {
                // kappa (and the 1/N normalisation) is common to the three outputs.
                // The x and y shift operators do not vary along z, so they commute
                // with the inverse z transform: outputs 0 and 1 are dx Q and dy Q
                // with Q = IFT_z{kappa P}, and only output 2 needs a second inverse
                // transform, of kappa dz P.
                float2 dx = col < g.nh ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
                float2 dy = __ldg(g.t.dfy + y);
                if (OP == OP_Z_GRAD_BWD) {                       // i k e^{-ikd/2}
                    dx = make_float2(-dx.x, dx.y);
                    dy = make_float2(-dy.x, dy.y);
                }
                float2 w[E];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    v[m] = cscale(v[m], kap[m]);
                    float2 d = __ldg(g.t.dfz + j + TL * m);
                    if (OP == OP_Z_GRAD_BWD) d = make_float2(-d.x, d.y);
                    w[m] = cmul(v[m], d);
                }
                float2* o0 = a.out[0];
                float2* o1 = a.out[1];
                float2* o2 = a.out[2];
                if (o0 != nullptr || o1 != nullptr) {           // uniform
                    inverse_tile<LOGN, E, CX, THREADS, MIXED>(v, j, S, smem + s * STAGE, g.t.tw, cmx, t5);
                    if (valid) {
#pragma unroll
                        for (int m = 0; m < E; ++m) {
                            const size_t o = off + (size_t)(j + TL * m) * es;
                            if (o0 != nullptr) __stcs(o0 + o, cmul(v[m], dx));
                            if (o1 != nullptr) __stcs(o1 + o, cmul(v[m], dy));
                        }
                    }
                }
                if (o2 != nullptr) {
                    inverse_tile<LOGN, E, CX, THREADS, MIXED>(w, j, S, smem + s * STAGE, g.t.tw, cmx, t5);
                    if (valid) {
#pragma unroll
                        for (int m = 0; m < E; ++m) __stcs(o2 + off + (size_t)(j + TL * m) * es, w[m]);
                    }
                }
            } else if (OP == OP_Z_DIV || OP == OP_Z_DIV_FWD) {
                const int xi = l;
                const float2 dx = col < g.nh ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
                const float2 dy = __ldg(g.t.dfy + y);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    float2 d = xi == 0 ? dx : (xi == 1 ? dy : __ldg(g.t.dfz + j + TL * m));
                    if (OP == OP_Z_DIV) d = make_float2(-d.x, d.y);   // Eq. 4c: i k e^{-ikd/2}
                    v[m] = cscale(cmul(v[m], d), kap[m]);            // OP_Z_DIV_FWD: Eq. 4a's operator
                }
                inverse_tile<LOGN, E, CX, THREADS, MIXED>(v, j, S, smem + s * STAGE, g.t.tw, cmx, t5);
                if (valid) {
                    float2* out = out_ptr(a, xi) + off;
#pragma unroll
                    for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, v[m]);
                }
            } else if (OP == OP_Z_DIV_SUM) {
                // sum over xi of the Eq. 4c operator on load xi, then one inverse transform
                const int xi = l;
                const float2 dx = col < g.nh ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
                const float2 dy = __ldg(g.t.dfy + y);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    float2 d = xi == 0 ? dx : (xi == 1 ? dy : __ldg(g.t.dfz + j + TL * m));
                    d = make_float2(-d.x, d.y);                      // i k e^{-ikd/2}
                    const float2 t = cscale(cmul(v[m], d), kap[m]);
                    acc[m] = xi == 0 ? t : cadd(acc[m], t);
                }
                if (xi == 2) {
                    inverse_tile<LOGN, E, CX, THREADS, MIXED>(acc, j, S, smem + s * STAGE, g.t.tw, cmx, t5);
                    if (valid) {
                        float2* out = a.out[0] + off;
#pragma unroll
                        for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, acc[m]);
                    }
                }
            } else {                                   // OP_Z_ABS
                const int t = l == 0 ? a.load_comp[0] : a.load_comp[1];
                const float e = g.abs_e[t], cst = g.abs_c[t] * g.scale;
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const float f = lg[m] > -INFINITY ? exp2f(e * lg[m]) * cst : 0.f;   // k^{y-2} / k^{y-1}, 0 at k = 0
                    v[m] = cscale(v[m], f);
                }
                inverse_tile<LOGN, E, CX, THREADS, MIXED>(v, j, S, smem + s * STAGE, g.t.tw, cmx, t5);
                if (valid) {
                    float2* out = out_ptr(a, t) + off;
#pragma unroll
                    for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, v[m]);
                }
            }
        }
        if (TC5 && !t5.ok && tid == 0) abort_flag = 1;
        __syncthreads();                          // stage s is free for the load of q + NST
        if (abort_flag) {
            if (NST == 2 && tid == 0 && q + 1 < Q) mbar_wait_bounded(&bar[(q + 1) & 1], ((q + 1) >> 1) & 1, a.flag);
            break;
        }
        if (NST == 1 && tid == 0 && q + 1 < Q) issue(q + 1);
    }
    if constexpr (TC5) {
        // a product whose wait ran out gets one more bounded wait before its
        // accumulator is freed
        if (!t5.ok && tid == 0) mbar_wait_bounded(t5.bar, t5.phase ^ 1u, a.flag);
        tc5_fence_before();
        __syncthreads();
        tc5_fence_after();
        if (tid < 32) tc5_dealloc(t5.tmem, Sh::TC5_TMEM);
    }
}


template <int LOGN, int OP, int MIXED>
inline cudaError_t launch_t(const YZK& a, int items, cudaStream_t s) {
    using Sh = TShape<LOGN, (OP < 2), MIXED>;
    auto k = yz_kernel<LOGN, OP, MIXED>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::smem(MIXED));
        if (e != cudaSuccess) return e;
        if (Sh::TC5) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
        }
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Sh::THREADS, Sh::smem(MIXED));
        if (e != cudaSuccess) return e;
        if (Sh::TC5) {
            // residency from the kernel's registers and shared memory (the query
            // has returned less than the hardware holds for the tensor-core form);
            // each resident CTA holds TC5_TMEM of the 512 tensor-memory columns
            cudaFuncAttributes fa;
            int dev = 0, smem_sm = 0, regs_sm = 0;
            if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess) {
                const int per_block = Sh::smem(MIXED) + (int)fa.sharedSizeBytes + 1024;
                const int regs = ((fa.numRegs + 7) / 8) * 8 * Sh::THREADS;
                int m = std::min(smem_sm / per_block, regs_sm / std::max(regs, 1));
                m = std::min(m, 512 / Sh::TC5_TMEM);
                per_sm = std::max(per_sm, m);
            }
        }
        if (per_sm < 1) per_sm = 1;
    }
    int grid = per_sm * a.g.num_sms;
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<grid, Sh::THREADS, Sh::smem(MIXED), s>>>(a);
    return cudaGetLastError();
}


#define KWGB_LOG_CASES(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)
#define KWGB_LOG_CASES_TC(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

// one translation unit per precision form instantiates these
cudaError_t yz_dispatch_f32(const YZK& a, int op, int logn, int items, cudaStream_t s);
cudaError_t yz_dispatch_bf16(const YZK& a, int op, int logn, int items, cudaStream_t s);
cudaError_t yz_dispatch_f16(const YZK& a, int op, int logn, int items, cudaStream_t s);

}  // namespace kwgb
