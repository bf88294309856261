// Shared parts of the contiguous-axis (x) passes (kernels_xvel.cu,
// kernels_x.cu): complex-to-real and real-to-complex transforms
// of whole rows, fused with the pointwise work of the time step so that the
// real-space fields only ever exist in registers:
//
//   x_vel   C2R of the three gradient spectra (Eq. 4a) -> velocity update with
//           PML (Eq. 4b) -> R2C of the new u_xi (first stage of Eq. 4c)
//   x_dens  C2R of the three divergence spectra (Eq. 4c) -> split density
//           update with PML and nonlinear denominator (Eq. 4d) -> additive
//           mass source -> rho = sum rho_xi and rho0 sum d -> R2C of both
//           (first stage of Eq. 8); for a lossless medium the EOS (Eq. 6),
//           the sensors and the R2C of p are done here as well
//   x_eos   C2R of the two absorption spectra (Eq. 8) -> EOS (Eq. 6) ->
//           sensors -> R2C of p^{n+1} (first stage of the next Eq. 4a)
//
// A row of nx reals is treated as M = nx/2 complex values z[n] = x[2n] +
// i x[2n+1]; an M-point FFT plus one post-processing step pairing bins k and
// M-k gives the nx/2+1 bins of the real transform (and the reverse for C2R).
// TL = M/E threads own a row; thread j holds z[j + TL*m], i.e. the float2 at
// x = 2(j + TL*m), so every global access of a row is coalesced.  A "team"
// is the smallest set of whole warps that holds whole rows: one warp with
// 32/TL rows (TL <= 32), or the TL/32 warps of one row (1024-point rows:
// E = 8, TL = 64, two warps, so that the kernels keep two CTAs per SM
// instead of spilling 16 values per thread at one CTA).  All synchronisation
// is within a team (a warp barrier, or a named barrier per team), so the
// teams of a CTA stream their rows independently.
#pragma once

#include "fft_core.cuh"
#include "kwgb_internal.h"

namespace kwgb {

constexpr int XTHREADS = 256;

// Work row of a team in shared memory, and the team's barrier.
template <int TEAM>
struct RowSmem {
    float2* base;
    int bar;                                         // named barrier id (TEAM > 32)
    static constexpr bool PINGPONG = false;
    __device__ __forceinline__ float2& at(int e) { return base[e + (e >> 4)]; }
    __device__ __forceinline__ float& f(int x) { return reinterpret_cast<float*>(base)[x]; }
    __device__ __forceinline__ void sync() {
        if constexpr (TEAM <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(TEAM) : "memory");
    }
};

template <int LOGM>
struct XShape {
    static constexpr int M = 1 << LOGM;
    static constexpr int E = M >= 8 ? 8 : M;
    static constexpr int TL = M / E;
    static constexpr int TEAM = TL > 32 ? TL : 32;   // threads of a team
    static constexpr int RPT = TEAM / TL;            // rows per team
    static constexpr int TPB = XTHREADS / TEAM;      // teams per CTA
    static_assert(TPB >= 1 && TPB <= 15, "named barriers 1..15");
    static constexpr int MINB = 2;                   // resident CTAs per SM the fused kernels are compiled for
    static constexpr int RPB = XTHREADS / TL;        // rows per CTA
    static constexpr int PITCH = M + M / 16 + 2;     // complex slots per row (padded, + Nyquist)
    static constexpr int SMEM = RPB * PITCH * (int)sizeof(float2);
    using Smem = RowSmem<TEAM>;
    // the work row of row slot r (threads r*TL .. r*TL + TL - 1) of a CTA
    __device__ __forceinline__ static Smem row_smem(float2* smem, int r) {
        return Smem{smem + r * PITCH, 1 + (r * TL) / TEAM};
    }
};

// exp(DIR 2 pi i k / (2M)) for k = j + TL*m.  Rows of 1024 reals: one table
// load per thread (w0 = the value at k = j) times the compile-time root
// exp(DIR i pi m / E) (TL / M = 1 / E), instead of E loads (measured faster
// there); shorter rows: the table entry of k, loaded where it is used
// (measured faster at 512 reals).
template <int DIR, int M, int E>
__device__ __forceinline__ float2 row_tw(const float2* __restrict__ tw, float2 w0, int k, int m) {
    static_assert(E <= 8 && 8 % E == 0, "roots of 16");
    if constexpr (M >= 512) return rot16<DIR>(w0, m * (8 / E));
    else return row_twiddle<DIR, M>(tw, k);
}
template <int DIR, int M>
__device__ __forceinline__ float2 row_tw0(const float2* __restrict__ tw, int j) {
    if constexpr (M >= 512) return row_twiddle<DIR, M>(tw, j);
    else return make_float2(0.f, 0.f);
}

// Unnormalised C2R of one row: spec[0..M] (Hermitian half spectrum) ->
// z[m] = (x[2n], x[2n+1]) with n = j + TL*m and
// x[i] = sum_{k<nx} X[k] exp(+2 pi i k i / nx).
template <int LOGM>
__device__ __forceinline__ void row_c2r(const float2* __restrict__ spec, typename XShape<LOGM>::Smem& S, int j,
                                        bool valid, const float2* __restrict__ tw,
                                        float2 (&z)[XShape<LOGM>::E]) {
    using Sh = XShape<LOGM>;
    constexpr int M = Sh::M, E = Sh::E, TL = Sh::TL;
    // all E + 1 loads of the row are issued before the first one is used
    float2 t[E];
    float2 nyq = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < E; ++m) t[m] = valid ? __ldcs(spec + j + TL * m) : make_float2(0.f, 0.f);
    if (valid && j == 0) nyq = __ldcs(spec + M);
    S.sync();                                      // smem row free
#pragma unroll
    for (int m = 0; m < E; ++m) S.at(j + TL * m) = t[m];
    if (j == 0) S.at(M) = nyq;
    S.sync();
    const float2 w0 = row_tw0<+1, M>(tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = j + TL * m;
        const float2 xk = S.at(k), xm = cconj(S.at(M - k));
        const float2 a = cadd(xk, xm);
        const float2 b = cmul(csub(xk, xm), row_tw<+1, M, E>(tw, w0, k, m));   // exp(+2 pi i k / nx)
        z[m] = make_float2(a.x - b.y, a.y + b.x);                                // a + i b
    }
    line_fft<LOGM, E, +1>(z, j, S, tw);
}

// ---- asynchronous row staging (per-warp cp.async double buffer) ----------
// A warp's rows of one spectrum are copied into shared memory one item ahead
// of their use, so the global-memory latency of the row load overlaps the
// transform of the previous item.  Rows are copied as M + 2 complex values
// (a multiple of 16 bytes; the extra value lies in the row padding).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int LOGM>
struct XStage {
    static constexpr int M = 1 << LOGM;
    static constexpr int SROW = M + 2;                   // staged complex values per row
    static constexpr int RPT = XShape<LOGM>::RPT;        // rows per team
    static constexpr int TEAM = XShape<LOGM>::TEAM;
    static constexpr int TSTAGE = 2 * RPT * SROW;        // complex per team (two stages)
};

// Issue the copies of rows first_row .. first_row + RPT - 1 of `spec` into
// stage buffer `dst` (RPT * SROW complex).  All threads of the team take part.
template <int LOGM>
__device__ __forceinline__ void stage_rows(float2* dst, const float2* __restrict__ spec, int first_row,
                                           int nrows, int nhp, int lane) {
    using St = XStage<LOGM>;
    constexpr int CH = St::SROW / 2;                     // 16-byte chunks per row
#pragma unroll
    for (int t = 0; t < (St::RPT * CH + St::TEAM - 1) / St::TEAM; ++t) {
        const int c = lane + St::TEAM * t;
        if (c < St::RPT * CH) {
            const int r = c / CH, q = c % CH;
            if (first_row + r < nrows)
                cp_async16(dst + r * St::SROW + 2 * q, spec + (size_t)(first_row + r) * nhp + 2 * q);
        }
    }
}

// C2R of one row whose half spectrum X[0..M] is already in shared memory
// (srow, unpadded): same result as row_c2r.
template <int LOGM>
__device__ __forceinline__ void row_c2r_staged(const float2* srow, typename XShape<LOGM>::Smem& S, int j,
                                               const float2* __restrict__ tw,
                                               float2 (&z)[XShape<LOGM>::E]) {
    using Sh = XShape<LOGM>;
    constexpr int M = Sh::M, E = Sh::E, TL = Sh::TL;
    const float2 w0 = row_tw0<+1, M>(tw, j);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = j + TL * m;
        const float2 xk = srow[k], xm = cconj(srow[M - k]);
        const float2 a = cadd(xk, xm);
        const float2 b = cmul(csub(xk, xm), row_tw<+1, M, E>(tw, w0, k, m));   // exp(+2 pi i k / nx)
        z[m] = make_float2(a.x - b.y, a.y + b.x);                                // a + i b
    }
    S.sync();                                        // previous users of the work row are done
    line_fft<LOGM, E, +1>(z, j, S, tw);
}

// Unnormalised R2C of one row: z[m] = (x[2n], x[2n+1]) -> spec[0..M].
template <int LOGM>
__device__ __forceinline__ void row_r2c(float2 (&z)[XShape<LOGM>::E], typename XShape<LOGM>::Smem& S, int j,
                                        bool valid, const float2* __restrict__ tw,
                                        float2* __restrict__ spec) {
    using Sh = XShape<LOGM>;
    constexpr int M = Sh::M, E = Sh::E, TL = Sh::TL;
    line_fft<LOGM, E, -1>(z, j, S, tw);
    S.sync();
#pragma unroll
    for (int m = 0; m < E; ++m) S.at(j + TL * m) = z[m];
    S.sync();
    if (valid) {
        const float2 w0 = row_tw0<-1, M>(tw, j);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = j + TL * m;
            const float2 zk = z[m], zm = cconj(S.at((M - k) & (M - 1)));
            const float2 s = cadd(zk, zm), d = csub(zk, zm);
            const float2 xe = make_float2(0.5f * s.x, 0.5f * s.y);
            const float2 xo = make_float2(0.5f * d.y, -0.5f * d.x);              // d / (2i)
            const float2 x = cadd(xe, cmul(xo, row_tw<-1, M, E>(tw, w0, k, m)));   // exp(-2 pi i k / nx)
            __stcs(spec + k, x);
            if (k == 0) __stcs(spec + M, csub(xe, xo));
        }
    }
}

__device__ __forceinline__ float2 ld2(const float* p) { return __ldcs(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float2 ldg2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st2(float* p, float2 v) { __stcs(reinterpret_cast<float2*>(p), v); }

__device__ __forceinline__ float2 med2(const float* f, float s, size_t i) {
    return f ? ldg2(f + i) : make_float2(s, s);
}

// Sensors, non-finite watch and the R2C of p (shared by x_eos and the fused
// lossless x_dens).  p[m] holds p at x = 2n, 2n+1.
template <int LOGM>
__device__ __forceinline__ void finish_pressure(float2 (&p)[XShape<LOGM>::E], const GridC& g,
                                                const SensorC& sens, const StepC& st,
                                                typename XShape<LOGM>::Smem& S, int j, bool valid, int row,
                                                float2* __restrict__ P) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    const size_t rbase = (size_t)row * g.nx;
    if (valid) {
        bool bad = false;
#pragma unroll
        for (int m = 0; m < E; ++m) bad |= !(isfinite(p[m].x) && isfinite(p[m].y));
        if (bad) atomicOr(st.flag, 1);
        for (int k = 0; k < sens.nfull; ++k) {
            float* pm = sens.full_max[k] + rbase;
            double* p2 = sens.full_p2[k] + rbase;
            float* pn = sens.full_min[k] ? sens.full_min[k] + rbase : nullptr;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int x = 2 * (j + TL * m);
                float2 o = *reinterpret_cast<float2*>(pm + x);
                o.x = fmaxf(o.x, p[m].x);
                o.y = fmaxf(o.y, p[m].y);
                *reinterpret_cast<float2*>(pm + x) = o;
                double2 q = *reinterpret_cast<double2*>(p2 + x);
                q.x += (double)p[m].x * (double)p[m].x;
                q.y += (double)p[m].y * (double)p[m].y;
                *reinterpret_cast<double2*>(p2 + x) = q;
                if (pn) {
                    float2 w = *reinterpret_cast<float2*>(pn + x);
                    w.x = fminf(w.x, p[m].x);
                    w.y = fminf(w.y, p[m].y);
                    *reinterpret_cast<float2*>(pn + x) = w;
                }
            }
        }
    }
    if (sens.row_ptr) {                               // uniform over the launch
        S.sync();
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            S.f(x) = p[m].x;
            S.f(x + 1) = p[m].y;
        }
        S.sync();
        if (valid) {
            const int e0 = __ldg(sens.row_ptr + row), e1 = __ldg(sens.row_ptr + row + 1);
            for (int e = e0 + j; e < e1; e += TL) {
                const int slot = __ldg(sens.e_slot + e);
                const float v = S.f(__ldg(sens.e_x + e));
                sens.p_max[slot] = fmaxf(sens.p_max[slot], v);
                sens.p2[slot] += (double)v * (double)v;
                sens.p_sens[slot] = v;
            }

        }
    }
    row_r2c<LOGM>(p, S, j, valid, g.t.tw, P + (size_t)row * g.nhp);
}

// Dirichlet pressure sources of one row in step n: afterwards S.f(x) holds the
// summed sample of every point x of the row that is held in this step, and
// NaN at every other x.  All threads of the row's team call it (it contains
// the team barriers); the result says whether the row has source points
// (the same for the threads of one row).
template <int LOGM>
__device__ __forceinline__ bool dirichlet_row(const SourceC& ds, const GridC& g, typename XShape<LOGM>::Smem& S,
                                              int j, bool valid, int row, int64_t n) {
    constexpr int TL = XShape<LOGM>::TL;
    const int p0 = valid ? __ldg(ds.row_ptr + row) : 0, p1 = valid ? __ldg(ds.row_ptr + row + 1) : 0;
    S.sync();
    if (p1 > p0) {
        for (int x = j; x < g.nx; x += TL) S.f(x) = __int_as_float(0x7fc00000);    // quiet NaN: not held
    }
    S.sync();
    for (int p = p0 + j; p < p1; p += TL) {
        const int c0 = __ldg(ds.pt_c + p), c1 = __ldg(ds.pt_c + p + 1);
        float acc = 0.f;
        bool held = false;
        for (int c = c0; c < c1; ++c) {
            if (n < __ldg(ds.c_nt + c)) {
                acc += __ldg(ds.signal + __ldg(ds.c_off + c) + n) * __ldg(ds.c_scale + c);
                held = true;
            }
        }
        if (held) S.f(__ldg(ds.pt_x + p)) = acc;
    }
    S.sync();
    return p1 > p0;
}

// p[i] for a run-time i without copying the parameter array to local memory
__device__ __forceinline__ const float2* pick3(const float2* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}
__device__ __forceinline__ float* pick3f(float* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}
__device__ __forceinline__ const float* pick3c(const float* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}
__device__ __forceinline__ float2* pick3w(float2* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}

// ---------------------------------------------------------------- launchers
template <class Kern, class Args>
static cudaError_t launch_rows(Kern k, int rpb, int smem_bytes, const GridC& g, const Args& args,
                               cudaStream_t s) {
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (e != cudaSuccess) return e;
    }
    const int nrows = g.ny * g.nz;
    k<<<(nrows + rpb - 1) / rpb, XTHREADS, smem_bytes, s>>>(args);
    return cudaGetLastError();
}

// Persistent launch of a pipelined row kernel: one CTA per resident slot.
template <int LOGM, class Kern, class Args>
static cudaError_t launch_persistent(Kern k, const GridC& g, const Args& args, cudaStream_t s) {
    using Sh = XShape<LOGM>;
    using St = XStage<LOGM>;
    const int smem_bytes = (Sh::RPB * Sh::PITCH + Sh::TPB * St::TSTAGE) * (int)sizeof(float2);
    int per_sm = 0;
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, XTHREADS, smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int ngroups = (g.ny * g.nz + Sh::RPT - 1) / Sh::RPT;
    int blocks = (ngroups + Sh::TPB - 1) / Sh::TPB;
    if (blocks > per_sm * g.num_sms) blocks = per_sm * g.num_sms;
    k<<<blocks, XTHREADS, smem_bytes, s>>>(args);
    return cudaGetLastError();
}

#define KWGB_LOGM_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9)

}  // namespace kwgb
