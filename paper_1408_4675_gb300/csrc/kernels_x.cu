// Contiguous-axis (x) passes: complex-to-real and real-to-complex transforms
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
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = j + TL * m;
        const float2 xk = S.at(k), xm = cconj(S.at(M - k));
        const float2 a = cadd(xk, xm);
        const float2 b = cmul(csub(xk, xm), row_twiddle<+1, M>(tw, k));   // exp(+2 pi i k / nx)
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
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = j + TL * m;
        const float2 xk = srow[k], xm = cconj(srow[M - k]);
        const float2 a = cadd(xk, xm);
        const float2 b = cmul(csub(xk, xm), row_twiddle<+1, M>(tw, k));   // exp(+2 pi i k / nx)
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
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = j + TL * m;
            const float2 zk = z[m], zm = cconj(S.at((M - k) & (M - 1)));
            const float2 s = cadd(zk, zm), d = csub(zk, zm);
            const float2 xe = make_float2(0.5f * s.x, 0.5f * s.y);
            const float2 xo = make_float2(0.5f * d.y, -0.5f * d.x);              // d / (2i)
            const float2 x = cadd(xe, cmul(xo, row_twiddle<-1, M>(tw, k)));
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

// ---------------------------------------------------------------- x_vel
// p[i] for a run-time i without copying the parameter array to local memory
__device__ __forceinline__ const float2* pick3(const float2* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}
__device__ __forceinline__ float* pick3f(float* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}
__device__ __forceinline__ float2* pick3w(float2* const (&p)[3], int i) {
    return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}

// x_dens is persistent: team w of the grid handles row groups w, w + W,
// w + 2W, ... (a group is the rows one team transforms at once), and walks
// the components of each group as a sequence of items; the spectrum rows of
// item i+1 are staged while item i is processed.  x_vel and x_eos take one
// row per TL threads per launch slot.
struct XVelK {
    GridC g;
    Medium md;
    XVelArgs a;
};

template <int LOGM, int MODE>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) x_vel_kernel(const XVelK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const GridC& g = K.g;
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int nrows = g.ny * g.nz;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < nrows;
    const int rr = valid ? row : 0;
    const int y = rr % g.ny, z = rr / g.ny;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    const size_t rb = (size_t)rr * g.nx;
    const float* rho0 = K.md.rho0;
    const float rho0s = K.md.rho0_s;

    float2 r0[E];                                     // rho0 of this row (x = 2n, 2n+1)
#pragma unroll
    for (int m = 0; m < E; ++m) r0[m] = rho0 ? ldg2(rho0 + rb + 2 * (j + TL * m)) : make_float2(rho0s, rho0s);
#pragma unroll
    for (int xi = 0; xi < 3; ++xi) {
        // issue this component's field loads before the row transform
        size_t nb;                                    // row base of the +1 neighbour along y / z
        if (xi == 1) nb = (size_t)(((y + 1) & (g.ny - 1)) + g.ny * z) * g.nx;
        else nb = (size_t)(y + g.ny * ((z + 1) & (g.nz - 1))) * g.nx;
        float2 uo[E], r1[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            uo[m] = (MODE != XV_INIT && valid) ? ld2(K.a.u[xi] + rb + x) : make_float2(0.f, 0.f);
            if (!rho0) r1[m] = make_float2(rho0s, rho0s);
            else if (xi == 0) r1[m] = make_float2(__ldg(rho0 + rb + ((x + 2) & (g.nx - 1))), 0.f);
            else r1[m] = ldg2(rho0 + nb + x);
        }
        float2 v[E];
        row_c2r<LOGM>(K.a.G[xi] + (size_t)rr * g.nhp, S, j, valid, g.t.tw, v);
        const float fyz = xi == 1 ? __ldg(g.t.pml_sg[1] + y) : __ldg(g.t.pml_sg[2] + z);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            // staggered-grid density: mean of the two neighbours along xi
            float2 rs;
            if (xi == 0) rs = make_float2(0.5f * (r0[m].x + r0[m].y), 0.5f * (r0[m].y + (rho0 ? r1[m].x : rho0s)));
            else rs = make_float2(0.5f * (r0[m].x + r1[m].x), 0.5f * (r0[m].y + r1[m].y));
            const float2 f = xi == 0 ? ldg2(g.t.pml_sg[0] + x) : make_float2(fyz, fyz);
            const float2 gr = v[m];
            float2 un;
            if (MODE == XV_INIT) {
                // u^{-1/2} = +dt / (2 rho0_sg) d/dxi p0
                un = make_float2(__fdividef(0.5f * g.dt * gr.x, rs.x), __fdividef(0.5f * g.dt * gr.y, rs.y));
            } else {
                // Eq. 4b with the PML: u <- f (f u - dt grad p / rho0_sg)
                un = make_float2(f.x * (f.x * uo[m].x - __fdividef(g.dt * gr.x, rs.x)),
                                 f.y * (f.y * uo[m].y - __fdividef(g.dt * gr.y, rs.y)));
            }
            if (valid) {
                if (MODE == XV_TAIL) st2(K.a.tail[xi] + (size_t)rr * 2 * g.nhp + x, un);
                else st2(K.a.u[xi] + rb + x, un);
            }
            v[m] = un;
        }
        if (MODE == XV_STEP) row_r2c<LOGM>(v, S, j, valid, g.t.tw, K.a.U[xi] + (size_t)rr * g.nhp);
    }
}

// ---------------------------------------------------------------- x_dens
struct XDensK {
    GridC g;
    Medium md;
    SourceC src;
    SensorC sens;
    StepC st;
    XDensArgs a;
};


template <int LOGM, bool FUSED_EOS>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) x_dens_kernel(const XDensK K) {
    using Sh = XShape<LOGM>;
    using St = XStage<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL, RPW = Sh::RPT, TPB = Sh::TPB;
    extern __shared__ __align__(16) float2 smem[];
    const GridC& g = K.g;
    const Medium& md = K.md;
    const int team = threadIdx.x / Sh::TEAM, lane = threadIdx.x % Sh::TEAM;
    const int r = lane / TL, j = lane % TL;
    typename Sh::Smem S = Sh::row_smem(smem, team * RPW + r);
    float2* stage = smem + Sh::RPB * Sh::PITCH + team * St::TSTAGE;
    const int nrows = g.ny * g.nz;
    const int ngroups = (nrows + RPW - 1) / RPW;
    const int gw = blockIdx.x * TPB + team, nw = gridDim.x * TPB;
    const int mygroups = gw < ngroups ? (ngroups - 1 - gw) / nw + 1 : 0;

    if (mygroups > 0) stage_rows<LOGM>(stage, K.a.D[0], gw * RPW, nrows, g.nhp, lane);
    cp_async_commit();
    for (int gi = 0; gi < mygroups; ++gi) {
        const int grp = gw + gi * nw;
        const int row = grp * RPW + r;
        const bool valid = row < nrows;
        const int rr = valid ? row : 0;
        const int y = rr % g.ny, z = rr / g.ny;
        const size_t rb = (size_t)rr * g.nx;

        float2 s[E], rt[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            s[m] = make_float2(0.f, 0.f);
            rt[m] = make_float2(0.f, 0.f);
        }
        const float fy = __ldg(g.t.pml[1] + y), fz = __ldg(g.t.pml[2] + z);
#pragma unroll 1
        for (int xi = 0; xi < 3; ++xi) {
            const int it = 3 * gi + xi;
            S.sync();
            if (xi < 2) stage_rows<LOGM>(stage + ((it + 1) & 1) * RPW * St::SROW, pick3(K.a.D, xi + 1), grp * RPW,
                                         nrows, g.nhp, lane);
            else if (gi + 1 < mygroups)
                stage_rows<LOGM>(stage + ((it + 1) & 1) * RPW * St::SROW, K.a.D[0], (grp + nw) * RPW, nrows,
                                 g.nhp, lane);
            cp_async_commit();
            float* rho_xi = pick3f(K.a.rho, xi);
            float2 ro_[E], r0[E];                     // issued before the row transform (rho0: L1/L2 hits)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                ro_[m] = valid ? ld2(rho_xi + rb + 2 * (j + TL * m)) : make_float2(0.f, 0.f);
                r0[m] = med2(md.rho0, md.rho0_s, rb + 2 * (j + TL * m));
            }
            cp_async_wait1();
            S.sync();
            float2 d[E];
            row_c2r_staged<LOGM>(stage + (it & 1) * RPW * St::SROW + r * St::SROW, S, j, g.t.tw, d);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int x = 2 * (j + TL * m);
                const float2 ro = ro_[m];
                const float2 f = xi == 0 ? ldg2(g.t.pml[0] + x) : (xi == 1 ? make_float2(fy, fy) : make_float2(fz, fz));
                // Eq. 4d with the PML: rho_xi <- f (f rho_xi - dt rho0 d) / (1 + 2 dt d)
                float nx_ = f.x * (f.x * ro.x - g.dt * r0[m].x * d[m].x);
                float ny_ = f.y * (f.y * ro.y - g.dt * r0[m].y * d[m].y);
                if (md.nonlinear) {
                    nx_ = __fdividef(nx_, 1.0f + 2.0f * g.dt * d[m].x);
                    ny_ = __fdividef(ny_, 1.0f + 2.0f * g.dt * d[m].y);
                }
                const float2 rn = make_float2(nx_, ny_);
                if (valid) st2(rho_xi + rb + x, rn);
                rt[m] = cadd(rt[m], rn);
                s[m] = make_float2(fmaf(r0[m].x, d[m].x, s[m].x), fmaf(r0[m].y, d[m].y, s[m].y));
            }
        }
        // additive mass source (dt M_xi, identical for every xi), applied after the
        // component loop: rho += 3 dt M, and rho_xi += dt M at the (few) source points
        if (K.src.row_ptr) {                           // uniform over the launch
            const int p0 = valid ? __ldg(K.src.row_ptr + rr) : 0;
            const int p1 = valid ? __ldg(K.src.row_ptr + rr + 1) : 0;
            const int64_t n = *K.st.step;
            S.sync();
            if (p1 > p0) {
                for (int x = j; x < g.nx; x += TL) S.f(x) = 0.f;
            }
            S.sync();
            for (int p = p0 + j; p < p1; p += TL) {
                const int c0 = __ldg(K.src.pt_c + p), c1 = __ldg(K.src.pt_c + p + 1);
                float acc = 0.f;
                for (int c = c0; c < c1; ++c) {
                    if (n < __ldg(K.src.c_nt + c))
                        acc += __ldg(K.src.signal + __ldg(K.src.c_off + c) + n) * __ldg(K.src.c_scale + c);
                }
                const int x = __ldg(K.src.pt_x + p);
                const float c = md.c0 ? __ldg(md.c0 + rb + x) : md.c0_s;
                S.f(x) = __fdividef(acc, c);           // dt * 2 s / (3 c0 dx)
            }
            S.sync();
            if (p1 > p0) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int x = 2 * (j + TL * m);
                    const float2 sv = make_float2(S.f(x), S.f(x + 1));
                    if (sv.x != 0.f || sv.y != 0.f) {
#pragma unroll
                        for (int xi = 0; xi < 3; ++xi) {
                            float* q = pick3f(K.a.rho, xi) + rb + x;
                            float2 o = *reinterpret_cast<float2*>(q);
                            *reinterpret_cast<float2*>(q) = make_float2(o.x + sv.x, o.y + sv.y);
                        }
                        rt[m] = make_float2(rt[m].x + 3.0f * sv.x, rt[m].y + 3.0f * sv.y);
                    }
                }
            }
        }
        if (FUSED_EOS) {
            // Eq. 6 without absorption: p = c0^2 (rho + B/2A rho^2 / rho0)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const size_t i = rb + 2 * (j + TL * m);
                const float2 c = med2(md.c0, md.c0_s, i);
                float2 rho = rt[m];
                float2 q = rho;
                if (md.nonlinear) {
                    const float2 ba = med2(md.bona, md.bona_s, i);
                    const float2 r0 = med2(md.rho0, md.rho0_s, i);
                    q.x += __fdividef(0.5f * ba.x * rho.x * rho.x, r0.x);
                    q.y += __fdividef(0.5f * ba.y * rho.y * rho.y, r0.y);
                }
                s[m] = make_float2(c.x * c.x * q.x, c.y * c.y * q.y);
            }
            finish_pressure<LOGM>(s, g, K.sens, K.st, S, j, valid, rr, K.a.P);
        } else {
            if (valid) {
#pragma unroll
                for (int m = 0; m < E; ++m)
                    st2(K.a.rho_tot + (size_t)rr * 2 * g.nhp + 2 * (j + TL * m), rt[m]);
            }
            row_r2c<LOGM>(s, S, j, valid, g.t.tw, K.a.S + (size_t)rr * g.nhp);
            row_r2c<LOGM>(rt, S, j, valid, g.t.tw, K.a.R + (size_t)rr * g.nhp);
        }
    }
}

// ---------------------------------------------------------------- x_eos
struct XEosK {
    GridC g;
    Medium md;
    SensorC sens;
    StepC st;
    XEosArgs a;
};

// Copy rows first_row .. first_row + RPT - 1 of a real field (nx = 2M floats
// per row, row pitch `pitch` floats) into dst (M float2 per row).
template <int LOGM>
__device__ __forceinline__ void stage_real_rows(float2* dst, const float* __restrict__ src, size_t pitch,
                                                int first_row, int nrows, int lane) {
    using Sh = XShape<LOGM>;
    constexpr int CH = Sh::M / 2;                        // 16-byte chunks per row
#pragma unroll
    for (int t = 0; t < (Sh::RPT * CH + Sh::TEAM - 1) / Sh::TEAM; ++t) {
        const int c = lane + Sh::TEAM * t;
        if (c < Sh::RPT * CH) {
            const int r = c / CH, q = c % CH;
            if (first_row + r < nrows) cp_async16(dst + r * Sh::M + 2 * q, src + (size_t)(first_row + r) * pitch + 4 * q);
        }
    }
}

// x_eos loads: the two absorption spectra rows and the rows of rho, rho0 and
// B/A are copied into shared memory (cp.async) at the start; c0 and alpha0
// go to registers and are consumed after the first row transform, so every
// global load overlaps transform work.
template <int LOGM>
struct XEosStage {
    static constexpr int RPT = XShape<LOGM>::RPT;
    static constexpr int A = RPT * XStage<LOGM>::SROW;   // one spectrum's rows of a team
    static constexpr int R = RPT * XShape<LOGM>::M;      // one real field's rows of a team (float2)
    static constexpr int TEAM = 2 * A + 3 * R;          // per team
};

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) x_eos_kernel(const XEosK K) {
    using Sh = XShape<LOGM>;
    using St = XStage<LOGM>;
    using Es = XEosStage<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL, M = Sh::M;
    extern __shared__ __align__(16) float2 smem[];
    const GridC& g = K.g;
    const Medium& md = K.md;
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int team = threadIdx.x / Sh::TEAM, lane = threadIdx.x % Sh::TEAM;
    const int nrows = g.ny * g.nz;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < nrows;
    const int rr = valid ? row : 0;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    float2* stage = smem + Sh::RPB * Sh::PITCH + team * Es::TEAM;
    const int first = blockIdx.x * Sh::RPB + team * Sh::RPT;
    const bool nl = md.nonlinear;
    stage_rows<LOGM>(stage, K.a.A1, first, nrows, g.nhp, lane);
    stage_rows<LOGM>(stage + Es::A, K.a.A2, first, nrows, g.nhp, lane);
    stage_real_rows<LOGM>(stage + 2 * Es::A, K.a.rho_tot, 2 * (size_t)g.nhp, first, nrows, lane);
    if (nl && md.rho0) stage_real_rows<LOGM>(stage + 2 * Es::A + Es::R, md.rho0, g.nx, first, nrows, lane);
    if (nl && md.bona) stage_real_rows<LOGM>(stage + 2 * Es::A + 2 * Es::R, md.bona, g.nx, first, nrows, lane);
    cp_async_commit();
    const size_t rb = (size_t)rr * g.nx;
    const int lr = r % Sh::RPT;                          // this row within the team's stage
    // Eq. 6 with Eq. 8 and Eq. 3:
    //   p = c0^2 (rho + B/2A rho^2/rho0) + c0^2 tau a1 - c0^2 eta a2,
    //   a1 = IFT{k^{y-2} FT{rho0 sum d}}, a2 = IFT{k^{y-1} FT{rho}},
    //   tau = -2 alpha0 c0^{y-1}, eta = 2 alpha0 c0^y tan(pi y / 2),
    // so with ct = c0^2 tau: p = c0^2 (...) + ct (a1 + c0 tan(pi y/2) a2).
    float2 c[E], al[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const size_t i = rb + 2 * (j + TL * m);
        c[m] = med2(md.c0, md.c0_s, i);
        al[m] = med2(md.alpha0, md.alpha0_s, i);
    }
    cp_async_wait0();
    S.sync();
    const float2* cur = stage + lr * St::SROW;
    float2 a[E];
    row_c2r_staged<LOGM>(cur, S, j, g.t.tw, a);
    const float ym1 = md.y - 1.0f;
    float2 acc[E], ce[E], c2[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const float px = exp2f(ym1 * log2f(c[m].x)), py = exp2f(ym1 * log2f(c[m].y));   // c0^{y-1}
        c2[m] = make_float2(c[m].x * c[m].x, c[m].y * c[m].y);
        const float2 ct = make_float2(c2[m].x * (-2.0f * al[m].x * px), c2[m].y * (-2.0f * al[m].y * py));
        acc[m] = make_float2(ct.x * a[m].x, ct.y * a[m].y);
        ce[m] = make_float2(ct.x * c[m].x * md.tan_pi_y_2, ct.y * c[m].y * md.tan_pi_y_2);   // -c0^2 eta
    }
    row_c2r_staged<LOGM>(cur + Es::A, S, j, g.t.tw, a);
    const float2* rho_s = stage + 2 * Es::A + lr * M;
    const float2* r0_s = stage + 2 * Es::A + Es::R + lr * M;
    const float2* ba_s = stage + 2 * Es::A + 2 * Es::R + lr * M;
    float2 p[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int e = j + TL * m;
        const float2 rho = rho_s[e];
        float2 q = rho;
        if (nl) {
            const float2 r0 = md.rho0 ? r0_s[e] : make_float2(md.rho0_s, md.rho0_s);
            const float2 ba = md.bona ? ba_s[e] : make_float2(md.bona_s, md.bona_s);
            q.x += __fdividef(0.5f * ba.x * rho.x * rho.x, r0.x);
            q.y += __fdividef(0.5f * ba.y * rho.y * rho.y, r0.y);
        }
        p[m] = make_float2(fmaf(c2[m].x, q.x, fmaf(ce[m].x, a[m].x, acc[m].x)),
                           fmaf(c2[m].y, q.y, fmaf(ce[m].y, a[m].y, acc[m].y)));
    }
    finish_pressure<LOGM>(p, g, K.sens, K.st, S, j, valid, rr, K.a.P);
}

// ---------------------------------------------------------------- plain x
struct XPlainK {
    GridC g;
    const float* rin;
    int rpitch;
    float2* cout;
    const float2* cin;
    float* rout;
};

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS) x_r2c_kernel(const XPlainK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < K.g.ny * K.g.nz;
    const int rr = valid ? row : 0;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = valid ? ld2(K.rin + (size_t)rr * K.rpitch + 2 * (j + TL * m)) : make_float2(0.f, 0.f);
    row_r2c<LOGM>(v, S, j, valid, K.g.t.tw, K.cout + (size_t)rr * K.g.nhp);
}

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS) x_c2r_kernel(const XPlainK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < K.g.ny * K.g.nz;
    const int rr = valid ? row : 0;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    float2 v[E];
    row_c2r<LOGM>(K.cin + (size_t)rr * K.g.nhp, S, j, valid, K.g.t.tw, v);
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) st2(K.rout + (size_t)rr * K.rpitch + 2 * (j + TL * m), v[m]);
    }
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

cudaError_t launch_x_vel(const GridC& g, const Medium& m, int mode, const XVelArgs& a,
                         cudaStream_t s) {
    XVelK K{g, m, a};
    switch (g.lognx - 1) {
#define CASE(L)                                                                                   \
    case L:                                                                                       \
        if (mode == XV_STEP) return launch_rows(x_vel_kernel<L, XV_STEP>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        if (mode == XV_TAIL) return launch_rows(x_vel_kernel<L, XV_TAIL>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        return launch_rows(x_vel_kernel<L, XV_INIT>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_x_dens(const GridC& g, const Medium& m, const SourceC& src,
                          const SensorC& sens, const StepC& st, const XDensArgs& a,
                          cudaStream_t s) {
    XDensK K{g, m, src, sens, st, a};
    const bool fused = !m.absorbing;
    switch (g.lognx - 1) {
#define CASE(L)                                                                                   \
    case L:                                                                                       \
        if (fused) return launch_persistent<L>(x_dens_kernel<L, true>, g, K, s); \
        return launch_persistent<L>(x_dens_kernel<L, false>, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_x_eos(const GridC& g, const Medium& m, const SensorC& sens,
                         const StepC& st, const XEosArgs& a, cudaStream_t s) {
    XEosK K{g, m, sens, st, a};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(x_eos_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM + XShape<L>::TPB * XEosStage<L>::TEAM * (int)sizeof(float2), g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_x_r2c(const GridC& g, const float* in, int in_pitch, float2* out,
                         cudaStream_t s) {
    XPlainK K{g, in, in_pitch, out, nullptr, nullptr};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(x_r2c_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_x_c2r(const GridC& g, const float2* in, float* out, int out_pitch,
                         cudaStream_t s) {
    XPlainK K{g, nullptr, out_pitch, nullptr, in, out};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(x_c2r_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace kwgb
