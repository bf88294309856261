#pragma once
// Float32 y and z passes with two adjacent x-columns per thread (256- to
// 1024-point lines).  Same tiles, TMA ring, operators and outputs as
// yz_kernel; the difference is the thread mapping: thread (cp, j) holds
// elements j + TL*m of columns 2cp and 2cp+1, so
//   * each twiddle loaded from the table serves two columns,
//   * every shared-memory access and every store moves both columns' values
//     as one float4 (half the load/store instructions of one column per
//     thread),
//   * the two columns' transforms are independent instruction streams
//     that the scheduler interleaves,
// at half the threads per tile (CTAs of CX/2 * TL threads).
#include "yz_kernel.cuh"

namespace kwgb {

// Column pair cp (columns 2cp, 2cp+1) of a tile: row e holds the pair as one float4.
template <int CX>
struct PairSmem {
    float2* buf;              // the arrived tile
    float2* scr;              // scratch tile
    int cp;
    __device__ __forceinline__ float4& raw(int e) { return reinterpret_cast<float4*>(buf)[e * (CX / 2) + cp]; }
    template <int B>
    __device__ __forceinline__ float4& at_pp(int e) {
        return reinterpret_cast<float4*>(B ? scr : buf)[e * (CX / 2) + cp];
    }
};

// One radix-RP Stockham pass (stride NS) on two lines held in the register
// layout of fft_core.cuh; the exchanges use the two buffers of PairSmem with
// one barrier each (buffer choice and barrier rule as in stockham_pass).
template <int LOGN, int E, int RP, int NS, int DIR, bool LAST, int CX>
__device__ __forceinline__ void pair_pass(float2 (&va)[E], float2 (&vb)[E], int j, PairSmem<CX>& S,
                                          const float2* __restrict__ tw) {
    constexpr int N = 1 << LOGN;
    constexpr int TL = N / E;
    constexpr int NB = E / RP;
    float2 oa[E], ob[E];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        float2 wa[RP], wb[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            wa[r] = va[i + r * NB];
            wb[r] = vb[i + r * NB];
        }
        if (NS > 1) {
            const int k = (j + TL * i) & (NS - 1);
#pragma unroll
            for (int r = 1; r < RP; ++r) {
                const float2 t = stage_twiddle<DIR, NS * RP, RP>(tw, k, r);
                wa[r] = cmul(wa[r], t);
                wb[r] = cmul(wb[r], t);
            }
        }
        dft_reg<RP, DIR>(wa);
        dft_reg<RP, DIR>(wb);
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            oa[i + q * NB] = wa[q];
            ob[i + q * NB] = wb[q];
        }
    }
    if constexpr (LAST) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            va[m] = oa[m];
            vb[m] = ob[m];
        }
    } else {
        constexpr int P = ilog2c(NS) / ilog2c(E);
        constexpr int NX = (LOGN + ilog2c(E) - 1) / ilog2c(E) - 1;
        constexpr int B = (P & 1) ? 0 : 1;
        if constexpr (P == 0 && (NX & 1)) __syncthreads();
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int b = j + TL * i;
            const int base = (b / NS) * NS * RP + (b & (NS - 1));
#pragma unroll
            for (int q = 0; q < RP; ++q)
                S.template at_pp<B>(base + q * NS) =
                    make_float4(oa[i + q * NB].x, oa[i + q * NB].y, ob[i + q * NB].x, ob[i + q * NB].y);
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const float4 t = S.template at_pp<B>(j + TL * m);
            va[m] = make_float2(t.x, t.y);
            vb[m] = make_float2(t.z, t.w);
        }
    }
}

template <int LOGN, int E, int DIR, int NS, int CX>
struct PairChain {
    __device__ __forceinline__ static void run(float2 (&va)[E], float2 (&vb)[E], int j, PairSmem<CX>& S,
                                               const float2* __restrict__ tw) {
        constexpr int N = 1 << LOGN;
        constexpr int REM = N / NS;
        constexpr int RP = REM >= E ? E : REM;
        constexpr bool LAST = (NS * RP == N);
        pair_pass<LOGN, E, RP, NS, DIR, LAST, CX>(va, vb, j, S, tw);
        if constexpr (!LAST) PairChain<LOGN, E, DIR, NS * RP, CX>::run(va, vb, j, S, tw);
    }
};

template <int LOGN, int E, int DIR, int CX>
__device__ __forceinline__ void line_fft_pair(float2 (&va)[E], float2 (&vb)[E], int j, PairSmem<CX>& S,
                                              const float2* __restrict__ tw) {
    PairChain<LOGN, E, DIR, 1, CX>::run(va, vb, j, S, tw);
}

// Tiles as in yz_kernel (CX columns, the same TMA boxes); 8 values per
// column per thread for every line length.
template <int LOGN, bool ISY>
struct PShape {
    using Sh = TShape<LOGN, ISY>;
    static constexpr int E = 8;
    static constexpr int TL = (1 << LOGN) / E;
    static constexpr int CP = Sh::CX / 2;                      // column pairs per tile
    static constexpr int THREADS = CP * TL;
    static constexpr int SMEM = 3 * Sh::STAGE * (int)sizeof(float2) + 64;
    static constexpr int MINB = 3 * Sh::STAGE * (int)sizeof(float2) > 100 * 1024 ? 1 : 2;
    static_assert(THREADS <= 1024, "tile too large");
};

// Store the pair (a, b) of row e: one float4 when both columns exist.
__device__ __forceinline__ void store_pair(float2* p, float2 a, float2 b, bool v0, bool v1) {
    if (v1) __stcs(reinterpret_cast<float4*>(p), make_float4(a.x, a.y, b.x, b.y));
    else if (v0) __stcs(p, a);
}

// OP_Y_FWD / OP_Y_INV: the y pass (transform only; items carry the component);
// z operators: as the z branch of yz_kernel.  (The kernel keeps its z name.)
template <int LOGN, int OP>
__global__ void __launch_bounds__(PShape<LOGN, (OP < 2)>::THREADS, PShape<LOGN, (OP < 2)>::MINB)
z_pair_kernel(const __grid_constant__ YZK a) {
    constexpr bool ISY = OP < 2;
    using Sh = TShape<LOGN, ISY>;
    using Ps = PShape<LOGN, ISY>;
    constexpr int E = Ps::E, TL = Ps::TL, CX = Sh::CX, STAGE = Sh::STAGE, CP = Ps::CP;
    extern __shared__ __align__(128) float2 smem[];
    __shared__ int abort_flag;
    float2* scratch = smem + 2 * STAGE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 3 * STAGE);
    const GridC& g = a.g;
    const int tid = threadIdx.x;
    const int cp = tid % CP, j = tid / CP;
    const int nchunk = (g.nh + CX - 1) / CX;
    const int lines = ISY ? g.nz : g.ny;
    const int items = nchunk * lines * (ISY ? a.ncomp : 1);
    constexpr int LC = (ISY || OP == OP_Z_GRAD_FWD || OP == OP_Z_GRAD_BWD) ? 1 : ((OP == OP_Z_DIV || OP == OP_Z_DIV_FWD) ? 3 : 0);
    const int L = LC ? LC : a.nloads;
    const int my = items > (int)blockIdx.x ? (items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my * L;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int q) {                 // thread 0 only
        const int item = (int)blockIdx.x + (q / L) * (int)gridDim.x;
        const int l = q % L;
        const int chunk = item % nchunk;
        const int line = (item / nchunk) % lines;
        const int mi = ISY ? item / (nchunk * lines) : (l == 0 ? a.load_comp[0] : (l == 1 ? a.load_comp[1] : a.load_comp[2]));
        const CUtensorMap* map = mi == 0 ? &a.map[0] : (mi == 1 ? &a.map[1] : &a.map[2]);
        float2* dst = smem + (q & 1) * STAGE;
        uint64_t* b = &bar[q & 1];
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(b, STAGE * (uint32_t)sizeof(float2) + g.wait_fault_tx);
#pragma unroll
        for (int k = 0; k < Sh::NBOX; ++k) {
            if (ISY) tma_load_3d(dst + k * Sh::BOX * CX, map, chunk * CX, k * Sh::BOX, line, b);
            else tma_load_3d(dst + k * Sh::BOX * CX, map, chunk * CX, line, k * Sh::BOX, b);
        }
    };

    if (tid == 0 && Q > 0) issue(0);
    float ka[E], kb[E];                       // kappa (or log2 k^2/kmax^2) of the tile's two columns
#pragma unroll
    for (int m = 0; m < E; ++m) { ka[m] = 0.f; kb[m] = 0.f; }

    for (int q = 0; q < Q; ++q) {
        const int s = q & 1;
        if (tid == 0 && q + 1 < Q) issue(q + 1);
        const bool ok = mbar_wait_bounded(&bar[s], (q >> 1) & 1, a.flag);
        if (!ok) abort_flag = 1;
        const int item = (int)blockIdx.x + (q / L) * (int)gridDim.x;
        const int l = q % L;
        const int chunk = item % nchunk;
        const int y = (item / nchunk) % lines;               // the line: y for the z pass, z for the y pass
        const int col = chunk * CX + 2 * cp;
        const bool v0 = ok && col < g.nh, v1 = ok && col + 1 < g.nh;
        PairSmem<CX> S{smem + s * STAGE, scratch, cp};
        float2 va[E], vb[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const float4 t = S.raw(j + TL * m);
            va[m] = make_float2(t.x, t.y);
            vb[m] = make_float2(t.z, t.w);
        }
        if constexpr (ISY) {
            const int comp = item / (nchunk * lines);
            line_fft_pair<LOGN, E, (OP == OP_Y_FWD ? -1 : +1), CX>(va, vb, j, S, g.t.tw);
            float2* out = out_ptr(a, comp) + (size_t)y * g.ny * g.nhp + col;
#pragma unroll
            for (int m = 0; m < E; ++m) store_pair(out + (size_t)(j + TL * m) * g.nhp, va[m], vb[m], v0, v1);
        } else {
        const size_t es = (size_t)g.ny * g.nhp;
        const size_t off = (size_t)y * g.nhp + col;
        const float kxa = col < g.nh ? __ldg(g.t.kx + col) : 0.f;
        const float kxb = col + 1 < g.nh ? __ldg(g.t.kx + col + 1) : 0.f;
        const float ky = __ldg(g.t.ky + y);
        if (!ISY && l == 0) {                    // operator values of this tile, kept for its loads
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const float kz = __ldg(g.t.kz + j + TL * m);
                const float kyz = fmaf(ky, ky, kz * kz);
                const float k2a = fmaf(kxa, kxa, kyz), k2b = fmaf(kxb, kxb, kyz);
                if (OP == OP_Z_ABS) {
                    ka[m] = k2a > 0.f ? log2f(k2a * g.inv_kmax2) : -INFINITY;
                    kb[m] = k2b > 0.f ? log2f(k2b * g.inv_kmax2) : -INFINITY;
                } else {
                    ka[m] = sinc_sq(g.hk2 * k2a) * g.scale;
                    kb[m] = sinc_sq(g.hk2 * k2b) * g.scale;
                }
            }
        }
        line_fft_pair<LOGN, E, -1, CX>(va, vb, j, S, g.t.tw);
        if (OP == OP_Z_GRAD_FWD || OP == OP_Z_GRAD_BWD) {
            // as in yz_kernel: outputs 0 and 1 are dx Q and dy Q with Q = IFT_z{kappa P},
            // output 2 the inverse transform of kappa dz P
            float2 dxa = col < g.nh ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
            float2 dxb = col + 1 < g.nh ? __ldg(g.t.dfx + col + 1) : make_float2(0.f, 0.f);
            float2 dy = __ldg(g.t.dfy + y);
            if (OP == OP_Z_GRAD_BWD) {                       // i k e^{-ikd/2}
                dxa = make_float2(-dxa.x, dxa.y);
                dxb = make_float2(-dxb.x, dxb.y);
                dy = make_float2(-dy.x, dy.y);
            }
            float2 wa[E], wb[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                va[m] = cscale(va[m], ka[m]);
                vb[m] = cscale(vb[m], kb[m]);
                float2 d = __ldg(g.t.dfz + j + TL * m);
                if (OP == OP_Z_GRAD_BWD) d = make_float2(-d.x, d.y);
                wa[m] = cmul(va[m], d);
                wb[m] = cmul(vb[m], d);
            }
            float2* o0 = a.out[0];
            float2* o1 = a.out[1];
            float2* o2 = a.out[2];
            if (o0 != nullptr || o1 != nullptr) {           // uniform
                line_fft_pair<LOGN, E, +1, CX>(va, vb, j, S, g.t.tw);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const size_t o = off + (size_t)(j + TL * m) * es;
                    if (o0 != nullptr) store_pair(o0 + o, cmul(va[m], dxa), cmul(vb[m], dxb), v0, v1);
                    if (o1 != nullptr) store_pair(o1 + o, cmul(va[m], dy), cmul(vb[m], dy), v0, v1);
                }
            }
            if (o2 != nullptr) {
                line_fft_pair<LOGN, E, +1, CX>(wa, wb, j, S, g.t.tw);
#pragma unroll
                for (int m = 0; m < E; ++m) store_pair(o2 + off + (size_t)(j + TL * m) * es, wa[m], wb[m], v0, v1);
            }
        } else if (OP == OP_Z_DIV || OP == OP_Z_DIV_FWD) {
            const int xi = l;
            float2 da, db;                                   // x / y shift operators (constant along z)
            if (xi == 0) {
                da = col < g.nh ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
                db = col + 1 < g.nh ? __ldg(g.t.dfx + col + 1) : make_float2(0.f, 0.f);
            } else {
                da = db = __ldg(g.t.dfy + y);
            }
#pragma unroll
            for (int m = 0; m < E; ++m) {
                float2 d0 = da, d1 = db;
                if (xi == 2) d0 = d1 = __ldg(g.t.dfz + j + TL * m);
                if (OP == OP_Z_DIV) {                        // Eq. 4c: i k e^{-ikd/2}
                    d0 = make_float2(-d0.x, d0.y);
                    d1 = make_float2(-d1.x, d1.y);
                }
                va[m] = cscale(cmul(va[m], d0), ka[m]);      // OP_Z_DIV_FWD: Eq. 4a's operator
                vb[m] = cscale(cmul(vb[m], d1), kb[m]);
            }
            line_fft_pair<LOGN, E, +1, CX>(va, vb, j, S, g.t.tw);
            float2* out = out_ptr(a, xi) + off;
#pragma unroll
            for (int m = 0; m < E; ++m) store_pair(out + (size_t)(j + TL * m) * es, va[m], vb[m], v0, v1);
        } else {                                             // OP_Z_ABS
            const int t = l == 0 ? a.load_comp[0] : a.load_comp[1];
            const float e = g.abs_e[t], cst = g.abs_c[t] * g.scale;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const float fa = ka[m] > -INFINITY ? exp2f(e * ka[m]) * cst : 0.f;   // k^{y-2} / k^{y-1}, 0 at k = 0
                const float fb = kb[m] > -INFINITY ? exp2f(e * kb[m]) * cst : 0.f;
                va[m] = cscale(va[m], fa);
                vb[m] = cscale(vb[m], fb);
            }
            line_fft_pair<LOGN, E, +1, CX>(va, vb, j, S, g.t.tw);
            float2* out = out_ptr(a, t) + off;
#pragma unroll
            for (int m = 0; m < E; ++m) store_pair(out + (size_t)(j + TL * m) * es, va[m], vb[m], v0, v1);
        }
        }
        __syncthreads();                          // stage s is free for the load of q + 2
        if (abort_flag) {
            if (tid == 0 && q + 1 < Q) mbar_wait_bounded(&bar[(q + 1) & 1], ((q + 1) >> 1) & 1, a.flag);
            return;
        }
    }
}

template <int LOGN, int OP>
inline cudaError_t launch_pair(const YZK& a, int items, cudaStream_t s) {
    using Ps = PShape<LOGN, (OP < 2)>;
    auto k = z_pair_kernel<LOGN, OP>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Ps::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Ps::THREADS, Ps::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    int grid = per_sm * a.g.num_sms;
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<grid, Ps::THREADS, Ps::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace kwgb
