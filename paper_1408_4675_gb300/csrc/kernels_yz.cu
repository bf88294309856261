// Strided-axis FFT passes on the half spectra [nz][ny][nhp] (complex64).
//
// A CTA owns a tile of CX consecutive x-columns times one whole line along
// y (y pass) or z (z pass).  Thread (c, j) loads elements j + TL*m of column c
// straight into registers: a warp reads 2 (CX = 16) or 4 (CX = 8) full
// 64..128-byte row segments per instruction, so the strided axis is read with
// coalesced accesses and each element crosses HBM once per pass.
//
// The z pass is the fused spectral-operator pass: forward z FFT, the
// pointwise operator of Eq. 4a, 4c or 8 (which needs kx, ky, kz, all known
// here), inverse z FFT, store.  It plays the role of the paper's
// "transposed-space" spectral multiply (Sec. 3.2): the spectrum never
// returns to HBM between the forward and the inverse transform along z.
#include "fft_core.cuh"
#include "kwgb_internal.h"

namespace kwgb {

template <int CX>
struct ColSmem {
    static constexpr int CXP = CX < 16 ? CX + 1 : CX;   // odd pitch for narrow tiles (banks)
    float2* buf;
    int c;
    __device__ __forceinline__ float2& at(int e) { return buf[e * CXP + c]; }
    __device__ __forceinline__ void sync() { __syncthreads(); }
};

template <int LOGN>
struct YZShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int E = LOGN >= 8 ? 16 : (N >= 8 ? 8 : N);
    static constexpr int TL = N / E;
    static constexpr int CX = (512 / TL) >= 16 ? 16 : (512 / TL);
    static constexpr int THREADS = CX * TL;
    static constexpr int SMEM = N * ColSmem<CX>::CXP * (int)sizeof(float2);
};

struct YArgs {
    GridC g;
    float2* in[3];
    float2* out[3];
};

template <int LOGN, int DIR>
__global__ void __launch_bounds__(YZShape<LOGN>::THREADS)
y_pass_kernel(const YArgs a) {
    using Sh = YZShape<LOGN>;
    constexpr int E = Sh::E, TL = Sh::TL, CX = Sh::CX;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % CX, j = threadIdx.x / CX;
    const int col = blockIdx.x * CX + c;
    const bool valid = col < a.g.nh;
    const size_t off = (size_t)blockIdx.y * a.g.ny * a.g.nhp + col;
    const size_t es = a.g.nhp;
    const float2* __restrict__ in = a.in[blockIdx.z] + off;
    float2* __restrict__ out = a.out[blockIdx.z] + off;
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = valid ? __ldcs(in + (size_t)(j + TL * m) * es) : make_float2(0.f, 0.f);
    ColSmem<CX> S{smem, c};
    line_fft<LOGN, E, DIR>(v, j, S, a.g.t.tw);
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, v[m]);
    }
}

struct ZArgs {
    GridC g;
    float2* in[3];
    float2* out[3];
};

// sinc(x) = sin(x)/x with sinc(0) = 1 (kappa of Sec. 2.2)
__device__ __forceinline__ float sinc_f(float x) {
    return fabsf(x) < 1e-4f ? 1.0f - x * x * (1.0f / 6.0f) : sinf(x) / x;
}

template <int LOGN, int OP>
__global__ void __launch_bounds__(YZShape<LOGN>::THREADS)
z_op_kernel(const ZArgs a) {
    using Sh = YZShape<LOGN>;
    constexpr int E = Sh::E, TL = Sh::TL, CX = Sh::CX;
    extern __shared__ float2 smem[];
    const GridC& g = a.g;
    const int c = threadIdx.x % CX, j = threadIdx.x / CX;
    const int col = blockIdx.x * CX + c;
    const int y = blockIdx.y;
    const bool valid = col < g.nh;
    const size_t off = (size_t)y * g.nhp + col;
    const size_t es = (size_t)g.ny * g.nhp;
    ColSmem<CX> S{smem, c};

    const float kx = valid ? __ldg(g.t.kx + col) : 0.f;
    const float ky = __ldg(g.t.ky + y);
    float k2[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const float kz = __ldg(g.t.kz + j + TL * m);
        k2[m] = fmaf(kx, kx, fmaf(ky, ky, kz * kz));
    }

    if (OP == Z_GRAD_FWD || OP == Z_GRAD_BWD) {
        float2 v[E];
        const float2* __restrict__ in = a.in[0] + off;
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = valid ? __ldcs(in + (size_t)(j + TL * m) * es) : make_float2(0.f, 0.f);
        line_fft<LOGN, E, -1>(v, j, S, g.t.tw);
        float kap[E];
#pragma unroll
        for (int m = 0; m < E; ++m) kap[m] = sinc_f(g.hk * sqrtf(k2[m])) * g.scale;
        const float2 dx = valid ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
        const float2 dy = __ldg(g.t.dfy + y);
#pragma unroll 1
        for (int xi = 0; xi < 3; ++xi) {
            float2* __restrict__ out = a.out[xi];
            if (out == nullptr) continue;          // uniform across the CTA
            out += off;
            float2 w[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                float2 d = xi == 0 ? dx : (xi == 1 ? dy : __ldg(g.t.dfz + j + TL * m));
                if (OP == Z_GRAD_BWD) d = make_float2(-d.x, d.y);   // i k e^{-ikd/2} = -conj(i k e^{+ikd/2})
                w[m] = cscale(cmul(v[m], d), kap[m]);
            }
            line_fft<LOGN, E, +1>(w, j, S, g.t.tw);
            if (valid) {
#pragma unroll
                for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, w[m]);
            }
        }
    } else if (OP == Z_DIV) {
        float kap[E];
#pragma unroll
        for (int m = 0; m < E; ++m) kap[m] = sinc_f(g.hk * sqrtf(k2[m])) * g.scale;
        const float2 dx = valid ? __ldg(g.t.dfx + col) : make_float2(0.f, 0.f);
        const float2 dy = __ldg(g.t.dfy + y);
#pragma unroll 1
        for (int xi = 0; xi < 3; ++xi) {
            const float2* __restrict__ in = a.in[xi] + off;
            float2* __restrict__ out = a.out[xi] + off;
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m)
                v[m] = valid ? __ldcs(in + (size_t)(j + TL * m) * es) : make_float2(0.f, 0.f);
            line_fft<LOGN, E, -1>(v, j, S, g.t.tw);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                float2 d = xi == 0 ? dx : (xi == 1 ? dy : __ldg(g.t.dfz + j + TL * m));
                d = make_float2(-d.x, d.y);        // Eq. 4c: i k e^{-ikd/2}
                v[m] = cscale(cmul(v[m], d), kap[m]);
            }
            line_fft<LOGN, E, +1>(v, j, S, g.t.tw);
            if (valid) {
#pragma unroll
                for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, v[m]);
            }
        }
    } else {  // Z_ABS
        float lg[E];
#pragma unroll
        for (int m = 0; m < E; ++m) lg[m] = k2[m] > 0.f ? log2f(k2[m] * g.inv_kmax2) : 0.f;
#pragma unroll 1
        for (int t = 0; t < 2; ++t) {
            if (a.in[t] == nullptr) continue;      // uniform
            const float2* __restrict__ in = a.in[t] + off;
            float2* __restrict__ out = a.out[t] + off;
            float2 v[E];
#pragma unroll
            for (int m = 0; m < E; ++m)
                v[m] = valid ? __ldcs(in + (size_t)(j + TL * m) * es) : make_float2(0.f, 0.f);
            line_fft<LOGN, E, -1>(v, j, S, g.t.tw);
            const float e = g.abs_e[t], cst = g.abs_c[t] * g.scale;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const float f = k2[m] > 0.f ? exp2f(e * lg[m]) * cst : 0.f;   // k^{y-2} or k^{y-1}, 0 at k = 0
                v[m] = cscale(v[m], f);
            }
            line_fft<LOGN, E, +1>(v, j, S, g.t.tw);
            if (valid) {
#pragma unroll
                for (int m = 0; m < E; ++m) __stcs(out + (size_t)(j + TL * m) * es, v[m]);
            }
        }
    }
}

template <int LOGN, int DIR>
static cudaError_t launch_y_t(const YArgs& a, int ncomp, cudaStream_t s) {
    using Sh = YZShape<LOGN>;
    auto k = y_pass_kernel<LOGN, DIR>;
    if (Sh::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.g.nh + Sh::CX - 1) / Sh::CX, a.g.nz, ncomp);
    k<<<grid, Sh::THREADS, Sh::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int LOGN, int OP>
static cudaError_t launch_z_t(const ZArgs& a, cudaStream_t s) {
    using Sh = YZShape<LOGN>;
    auto k = z_op_kernel<LOGN, OP>;
    if (Sh::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.g.nh + Sh::CX - 1) / Sh::CX, a.g.ny, 1);
    k<<<grid, Sh::THREADS, Sh::SMEM, s>>>(a);
    return cudaGetLastError();
}

#define KWGB_LOG_CASES(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

cudaError_t launch_y_pass(const GridC& g, int dir, float2* const* in, float2* const* out,
                          int ncomp, cudaStream_t s) {
    YArgs a;
    a.g = g;
    for (int i = 0; i < 3; ++i) {
        a.in[i] = i < ncomp ? in[i] : nullptr;
        a.out[i] = i < ncomp ? out[i] : nullptr;
    }
    switch (g.logny) {
#define CASE(L) case L: return dir < 0 ? launch_y_t<L, -1>(a, ncomp, s) : launch_y_t<L, +1>(a, ncomp, s);
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

template <int OP>
static cudaError_t launch_z_op_k(const ZArgs& a, cudaStream_t s) {
    switch (a.g.lognz) {
#define CASE(L) case L: return launch_z_t<L, OP>(a, s);
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_z_op(const GridC& g, int kind, float2* const* in, float2* const* out,
                        cudaStream_t s) {
    ZArgs a;
    a.g = g;
    for (int i = 0; i < 3; ++i) {
        a.in[i] = in[i];
        a.out[i] = out[i];
    }
    switch (kind) {
        case Z_GRAD_FWD: return launch_z_op_k<Z_GRAD_FWD>(a, s);
        case Z_GRAD_BWD: return launch_z_op_k<Z_GRAD_BWD>(a, s);
        case Z_DIV: return launch_z_op_k<Z_DIV>(a, s);
        case Z_ABS: return launch_z_op_k<Z_ABS>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kwgb
