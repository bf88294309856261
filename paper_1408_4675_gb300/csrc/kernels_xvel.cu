// x_vel: C2R of the three gradient spectra (Eq. 4a) -> velocity update with
// PML (Eq. 4b) and force sources -> R2C of the new u_xi (first stage of
// Eq. 4c).  Row layout and helpers: x_rows.cuh.
#include "x_rows.cuh"

namespace kwgb {

// One row per TL threads per launch slot (not persistent).
struct XVelK {
    GridC g;
    Medium md;
    XVelArgs a;
};

// FORCE: the launch has force sources (a separate instantiation, so that the
// common path carries no code for them).
template <int LOGM, int MODE, bool FORCE>
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
        if (FORCE && MODE != XV_INIT && K.a.f[xi].row_ptr) {   // force sources along xi (uniform over the launch)
            // u_xi += dt F / rho0_sg at the row's source points, after Eq. 4b; the
            // point's value (already stored above) is stored again by its thread
            const SourceC& fs = K.a.f[xi];
            const int p0 = valid ? __ldg(fs.row_ptr + rr) : 0, p1 = valid ? __ldg(fs.row_ptr + rr + 1) : 0;
            S.sync();
            if (p1 > p0) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int x = 2 * (j + TL * m);
                    S.f(x) = v[m].x;
                    S.f(x + 1) = v[m].y;
                }
            }
            S.sync();
            if (p1 > p0) {
                const int64_t n = *K.a.step;
                for (int p = p0 + j; p < p1; p += TL) {
                    const int ca = __ldg(fs.pt_c + p), cb = __ldg(fs.pt_c + p + 1);
                    float acc = 0.f;
                    for (int c = ca; c < cb; ++c)
                        if (n < __ldg(fs.c_nt + c)) acc += __ldg(fs.signal + __ldg(fs.c_off + c) + n) * __ldg(fs.c_scale + c);
                    const int x = __ldg(fs.pt_x + p);
                    float rsx = rho0s;                    // rho0 at the staggered point x + 1/2 along xi
                    if (rho0) {
                        const size_t other = xi == 0 ? rb + ((x + 1) & (g.nx - 1))
                                           : xi == 1 ? (size_t)(((y + 1) & (g.ny - 1)) + g.ny * z) * g.nx + x
                                                     : (size_t)(y + g.ny * ((z + 1) & (g.nz - 1))) * g.nx + x;
                        rsx = 0.5f * (__ldg(rho0 + rb + x) + __ldg(rho0 + other));
                    }
                    const float un = S.f(x) + __fdividef(acc, rsx);
                    S.f(x) = un;
                    if (MODE == XV_TAIL) K.a.tail[xi][(size_t)rr * 2 * g.nhp + x] = un;
                    else K.a.u[xi][rb + x] = un;
                }
            }
            S.sync();
            if (p1 > p0) {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int x = 2 * (j + TL * m);
                    v[m] = make_float2(S.f(x), S.f(x + 1));
                }
            }
        }
        if (MODE == XV_STEP) row_r2c<LOGM>(v, S, j, valid, g.t.tw, K.a.U[xi] + (size_t)rr * g.nhp);
    }
}

cudaError_t launch_x_vel(const GridC& g, const Medium& m, int mode, const XVelArgs& a,
                         cudaStream_t s) {
    XVelK K{g, m, a};
    const bool force = a.f[0].row_ptr || a.f[1].row_ptr || a.f[2].row_ptr;
    switch (g.lognx - 1) {
#define CASE(L)                                                                                   \
    case L:                                                                                       \
        if (mode == XV_STEP && force) return launch_rows(x_vel_kernel<L, XV_STEP, true>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        if (mode == XV_STEP) return launch_rows(x_vel_kernel<L, XV_STEP, false>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        if (mode == XV_TAIL && force) return launch_rows(x_vel_kernel<L, XV_TAIL, true>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        if (mode == XV_TAIL) return launch_rows(x_vel_kernel<L, XV_TAIL, false>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        return launch_rows(x_vel_kernel<L, XV_INIT, false>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace kwgb
