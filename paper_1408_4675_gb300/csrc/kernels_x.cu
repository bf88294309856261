// x_dens, x_eos and the plain x transforms.  Row layout and helpers:
// x_rows.cuh.
#include "x_rows.cuh"

namespace kwgb {

// ---------------------------------------------------------------- x_dens
// x_dens is persistent: team w of the grid handles row groups w, w + W,
// w + 2W, ... (a group is the rows one team transforms at once), and walks
// the components of each group as a sequence of items; the spectrum rows of
// item i+1 are staged while item i is processed.
struct XDensK {
    GridC g;
    Medium md;
    SourceC src;
    SourceC dsrc;             // Dirichlet pressure sources
    SensorC sens;
    StepC st;
    XDensArgs a;
};


// DIRICHLET: the launch has Dirichlet pressure sources; DOUT: it also writes
// the Eq. 4c derivatives d_xi, the densities it read and the new total
// density (the adjoint's recomputation).  Separate
// instantiations, so that the common path carries no code for them.
template <int LOGM, bool FUSED_EOS, bool DIRICHLET, bool DOUT>
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

    const size_t NN = (size_t)g.nx * g.ny * g.nz;
    float* kp = nullptr;                               // this step's kept fields
    if (DOUT) kp = K.a.keep + (size_t)(*K.st.step % K.a.keep_period) * 7 * NN;
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
                if (DOUT && valid) {
                    st2(kp + (3 + xi) * NN + rb + x, d[m]);
                    st2(kp + xi * NN + rb + x, ro);
                }
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
        // Dirichlet pressure sources: rho_xi = s / (3 c0^2) at the held points
        bool drow = false;
        float2 dv[E];
        if (DIRICHLET) {
            drow = dirichlet_row<LOGM>(K.dsrc, g, S, j, valid, rr, *K.st.step);
            if (drow) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int x = 2 * (j + TL * m);
                    dv[m] = make_float2(S.f(x), S.f(x + 1));
                    const float2 c = med2(md.c0, md.c0_s, rb + x);
                    if (valid && dv[m].x == dv[m].x) {
                        const float rx = __fdividef(dv[m].x, c.x * c.x);
#pragma unroll
                        for (int xi = 0; xi < 3; ++xi) pick3f(K.a.rho, xi)[rb + x] = rx * (1.0f / 3.0f);
                        rt[m].x = rx;
                    }
                    if (valid && dv[m].y == dv[m].y) {
                        const float ry = __fdividef(dv[m].y, c.y * c.y);
#pragma unroll
                        for (int xi = 0; xi < 3; ++xi) pick3f(K.a.rho, xi)[rb + x + 1] = ry * (1.0f / 3.0f);
                        rt[m].y = ry;
                    }
                }
            }
        }
        if (DOUT && valid) {
#pragma unroll
            for (int m = 0; m < E; ++m) st2(kp + 6 * NN + rb + 2 * (j + TL * m), rt[m]);
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
                if (DIRICHLET && drow) {                   // p = s at the held points
                    if (dv[m].x == dv[m].x) s[m].x = dv[m].x;
                    if (dv[m].y == dv[m].y) s[m].y = dv[m].y;
                }
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
    SourceC dsrc;             // Dirichlet pressure sources
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

template <int LOGM, bool DIRICHLET>
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
    if (DIRICHLET) {                                     // p = s at the held points
        if (dirichlet_row<LOGM>(K.dsrc, g, S, j, valid, rr, *K.st.step)) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int x = 2 * (j + TL * m);
                const float2 dv = make_float2(S.f(x), S.f(x + 1));
                if (dv.x == dv.x) p[m].x = dv.x;
                if (dv.y == dv.y) p[m].y = dv.y;
            }
        }
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

cudaError_t launch_x_dens(const GridC& g, const Medium& m, const SourceC& src, const SourceC& dsrc,
                          const SensorC& sens, const StepC& st, const XDensArgs& a,
                          cudaStream_t s) {
    XDensK K{g, m, src, dsrc, sens, st, a};
    const bool fused = !m.absorbing;
    const bool dir = dsrc.row_ptr != nullptr;
    const bool dout = a.keep != nullptr;
    if (dout && a.keep_period <= 0) return cudaErrorInvalidValue;
    if (dout && dir) return cudaErrorInvalidValue;          // the adjoint takes no Dirichlet sources
    switch (g.lognx - 1) {
#define CASE(L)                                                                                          \
    case L:                                                                                              \
        if (dout && fused) return launch_persistent<L>(x_dens_kernel<L, true, false, true>, g, K, s);   \
        if (dout) return launch_persistent<L>(x_dens_kernel<L, false, false, true>, g, K, s);           \
        if (fused && dir) return launch_persistent<L>(x_dens_kernel<L, true, true, false>, g, K, s);    \
        if (fused) return launch_persistent<L>(x_dens_kernel<L, true, false, false>, g, K, s);          \
        if (dir) return launch_persistent<L>(x_dens_kernel<L, false, true, false>, g, K, s);            \
        return launch_persistent<L>(x_dens_kernel<L, false, false, false>, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_x_eos(const GridC& g, const Medium& m, const SourceC& dsrc, const SensorC& sens,
                         const StepC& st, const XEosArgs& a, cudaStream_t s) {
    XEosK K{g, m, dsrc, sens, st, a};
    const bool dir = dsrc.row_ptr != nullptr;
    switch (g.lognx - 1) {
#define CASE(L)                                                                                            \
    case L: {                                                                                              \
        const int smem = XShape<L>::SMEM + XShape<L>::TPB * XEosStage<L>::TEAM * (int)sizeof(float2);      \
        if (dir) return launch_rows(x_eos_kernel<L, true>, XShape<L>::RPB, smem, g, K, s);                 \
        return launch_rows(x_eos_kernel<L, false>, XShape<L>::RPB, smem, g, K, s);                         \
    }
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
