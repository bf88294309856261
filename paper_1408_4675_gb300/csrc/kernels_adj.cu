// The adjoint (reverse-mode) time step.  The spectral parts reuse the
// forward y and z passes: the adjoint of IFT{O FT{.}} on real fields is
// IFT{conj(O) FT{.}}, and conj(i k kappa e^{-ikd/2}) = -(i k kappa e^{+ikd/2}),
// so the transpose of Eq. 4c's operator is minus Eq. 4a's and vice versa.
// The pointwise parts run inside x passes, between the C2R and the R2C of a
// row (as the forward's x_vel and x_dens do), so the adjoint fields cross HBM
// once per reverse step and no real-space temporary is stored.
//
// One backward step n (the forward step maps n -> n+1), lossless medium:
//   lambda_rho   = c0^2 (1 + (B/A) rho^{n+1} / rho0) lambda_p         (Eq. 6)
//   lambda_rho_xi' = lambda_rho_xi + lambda_rho
//   lambda_rho_xi <- lambda_rho_xi' f^2 / (1 + 2 dt d_xi)            (Eq. 4d)
//   lambda_d_xi   = -lambda_rho_xi' f dt (rho0 + 2 f rho_xi^n) / (1 + 2 dt d_xi)^2
//   lambda_u_xi'  = lambda_u_xi - (Eq. 4a op) lambda_d_xi
//   lambda_u_xi  <- f_sg^2 lambda_u_xi'                               (Eq. 4b)
//   lambda_g_xi   = -f_sg dt / rho0_sg lambda_u_xi'
//   lambda_p      = -sum_xi (Eq. 4c op) lambda_g_xi
// (linear medium: no (B/A) term and a denominator of 1).  Absorbing medium
// (Eq. 8, p gains c0^2 tau a1 - c0^2 eta a2 with a1 = IFT{k^{y-2} FT{rho0
// sum d}}, a2 = IFT{k^{y-1} FT{rho}}): the two operators are real and even,
// hence self-adjoint, so
//   lambda_rho   += IFT{k^{y-1} FT{-c0^2 eta lambda_p}}            (a2)
//   lambda_d_xi  += rho0 IFT{k^{y-2} FT{c0^2 tau lambda_p}}         (rho0 a1)
//
// Kernels of one reverse step (x passes; y, z as in the forward):
//   adj_x_absprep (absorbing)  lambda_p -> R2C of c0^2 tau lambda_p (sp[0])
//                              and of -c0^2 eta lambda_p (sp[1]);
//                              then y, z (k^{y-2}, k^{y-1}), y
//   adj_x_dens   [C2R of sp[0], sp[1]] -> Eq. 6 / 4d backwards -> lambda_rho,
//                lambda_src, R2C of lambda_d_xi -> sp[xi]; then y, z (Eq. 4a
//                op per component), y
//   adj_x_vel    C2R of sp[xi] -> Eq. 4b backwards -> lambda_u, R2C of
//                lambda_g_xi -> sp[xi]; then y (3 spectra), z (Eq. 4c op on
//                each, summed into sp[0]), y (1 spectrum)
//   adj_x_p      C2R of sp[0] -> lambda_p; steps the reverse-step counter back
// Every kernel reads a row's spectra before it writes that row's spectra, so
// the spectra can be read and written in place.
#include "x_rows.cuh"

namespace kwgb {

struct AdjXK {
    GridC g;
    Medium md;
    AdjX a;
};

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) adj_x_absprep_kernel(const AdjXK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const GridC& g = K.g;
    const Medium& md = K.md;
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < g.ny * g.nz;
    const int rr = valid ? row : 0;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    const size_t rb = (size_t)rr * g.nx;
    const float ym1 = md.y - 1.0f;
    float2 q1[E], q2[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const size_t i = rb + 2 * (j + TL * m);
        const float2 l = valid ? ld2(K.a.lam_p + i) : make_float2(0.f, 0.f);
        const float2 c = med2(md.c0, md.c0_s, i);
        const float2 al = med2(md.alpha0, md.alpha0_s, i);
        // c0^2 tau = -2 alpha0 c0^{y+1};  -c0^2 eta = c0^2 tau c0 tan(pi y / 2)
        const float2 ct = make_float2(c.x * c.x * (-2.0f * al.x * exp2f(ym1 * log2f(c.x))),
                                      c.y * c.y * (-2.0f * al.y * exp2f(ym1 * log2f(c.y))));
        q1[m] = make_float2(ct.x * l.x, ct.y * l.y);
        q2[m] = make_float2(ct.x * c.x * md.tan_pi_y_2 * l.x, ct.y * c.y * md.tan_pi_y_2 * l.y);
    }
    row_r2c<LOGM>(q1, S, j, valid, g.t.tw, K.a.sp[0] + (size_t)rr * g.nhp);
    row_r2c<LOGM>(q2, S, j, valid, g.t.tw, K.a.sp[1] + (size_t)rr * g.nhp);
}

template <int LOGM, bool ABS>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) adj_x_dens_kernel(const AdjXK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const GridC& g = K.g;
    const Medium& md = K.md;
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < g.ny * g.nz;
    const int rr = valid ? row : 0;
    const int y = rr % g.ny, z = rr / g.ny;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    const size_t rb = (size_t)rr * g.nx;
    const bool nl = md.nonlinear;
    const size_t NN = (size_t)g.nx * g.ny * g.nz;
    const float* kp = K.a.keep + (size_t)(*K.a.nrev % K.a.keep_period) * 7 * NN;   // step n's kept fields

    float2 lrt[E], labs[E], r0[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const size_t i = rb + 2 * (j + TL * m);
        const float2 l = valid ? ld2(K.a.lam_p + i) : make_float2(0.f, 0.f);
        const float2 c = med2(md.c0, md.c0_s, i);
        r0[m] = med2(md.rho0, md.rho0_s, i);
        float2 w = make_float2(c.x * c.x, c.y * c.y);
        if (nl) {                                     // dp/drho = c0^2 (1 + (B/A) rho / rho0)
            const float2 ba = med2(md.bona, md.bona_s, i);
            const float2 rt = valid ? ld2(kp + 6 * NN + i) : make_float2(0.f, 0.f);
            w.x *= 1.0f + __fdividef(ba.x * rt.x, r0[m].x);
            w.y *= 1.0f + __fdividef(ba.y * rt.y, r0[m].y);
        }
        lrt[m] = make_float2(w.x * l.x, w.y * l.y);
        labs[m] = make_float2(0.f, 0.f);
    }
    if (ABS) {                                        // Eq. 8 backwards: a1 -> lambda_d, a2 -> lambda_rho
        float2 a[E];
        row_c2r<LOGM>(K.a.sp[0] + (size_t)rr * g.nhp, S, j, valid, g.t.tw, a);
#pragma unroll
        for (int m = 0; m < E; ++m) labs[m] = make_float2(r0[m].x * a[m].x, r0[m].y * a[m].y);
        row_c2r<LOGM>(K.a.sp[1] + (size_t)rr * g.nhp, S, j, valid, g.t.tw, a);
#pragma unroll
        for (int m = 0; m < E; ++m) lrt[m] = cadd(lrt[m], a[m]);
    }
    float2 src[E];
#pragma unroll
    for (int m = 0; m < E; ++m) src[m] = make_float2(0.f, 0.f);
    const float fy = __ldg(g.t.pml[1] + y), fz = __ldg(g.t.pml[2] + z);
#pragma unroll 1
    for (int xi = 0; xi < 3; ++xi) {
        const float* lrho = pick3f(K.a.lam_rho, xi);
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            const size_t i = rb + x;
            const float2 lr = valid ? ld2(lrho + i) : make_float2(0.f, 0.f);
            const float2 d = valid ? ld2(kp + (3 + xi) * NN + i) : make_float2(0.f, 0.f);
            const float2 f = xi == 0 ? ldg2(g.t.pml[0] + x) : (xi == 1 ? make_float2(fy, fy) : make_float2(fz, fz));
            const float2 lrp = cadd(lr, lrt[m]);
            src[m] = cadd(src[m], lrp);
            float2 nlr, ld;
            if (nl) {
                const float2 rb_ = valid ? ld2(kp + xi * NN + i) : make_float2(0.f, 0.f);
                const float dx_ = __fdividef(1.0f, 1.0f + 2.0f * g.dt * d.x);
                const float dy_ = __fdividef(1.0f, 1.0f + 2.0f * g.dt * d.y);
                nlr = make_float2(lrp.x * f.x * f.x * dx_, lrp.y * f.y * f.y * dy_);
                ld = make_float2(labs[m].x - lrp.x * f.x * g.dt * (r0[m].x + 2.0f * f.x * rb_.x) * dx_ * dx_,
                                 labs[m].y - lrp.y * f.y * g.dt * (r0[m].y + 2.0f * f.y * rb_.y) * dy_ * dy_);
            } else {
                nlr = make_float2(lrp.x * f.x * f.x, lrp.y * f.y * f.y);
                ld = make_float2(labs[m].x - lrp.x * f.x * g.dt * r0[m].x, labs[m].y - lrp.y * f.y * g.dt * r0[m].y);
            }
            if (valid) st2(pick3f(K.a.lam_rho, xi) + i, nlr);
            v[m] = ld;
        }
        row_r2c<LOGM>(v, S, j, valid, g.t.tw, pick3w(K.a.sp, xi) + (size_t)rr * g.nhp);
    }
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) st2(K.a.lam_src + rb + 2 * (j + TL * m), src[m]);
    }
}

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) adj_x_vel_kernel(const AdjXK K) {
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

    float2 r0[E];
#pragma unroll
    for (int m = 0; m < E; ++m) r0[m] = rho0 ? ldg2(rho0 + rb + 2 * (j + TL * m)) : make_float2(rho0s, rho0s);
#pragma unroll
    for (int xi = 0; xi < 3; ++xi) {
        size_t nb;                                    // row base of the +1 neighbour along y / z
        if (xi == 1) nb = (size_t)(((y + 1) & (g.ny - 1)) + g.ny * z) * g.nx;
        else nb = (size_t)(y + g.ny * ((z + 1) & (g.nz - 1))) * g.nx;
        float* lu = pick3f(K.a.lam_u, xi);
        float2 lo[E], r1[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            lo[m] = valid ? ld2(lu + rb + x) : make_float2(0.f, 0.f);
            if (!rho0) r1[m] = make_float2(rho0s, rho0s);
            else if (xi == 0) r1[m] = make_float2(__ldg(rho0 + rb + ((x + 2) & (g.nx - 1))), 0.f);
            else r1[m] = ldg2(rho0 + nb + x);
        }
        float2 v[E];
        row_c2r<LOGM>(pick3w(K.a.sp, xi) + (size_t)rr * g.nhp, S, j, valid, g.t.tw, v);
        const float fyz = xi == 1 ? __ldg(g.t.pml_sg[1] + y) : __ldg(g.t.pml_sg[2] + z);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int x = 2 * (j + TL * m);
            float2 rs;                                // rho0 at the staggered point (mean along xi)
            if (xi == 0) rs = make_float2(0.5f * (r0[m].x + r0[m].y), 0.5f * (r0[m].y + (rho0 ? r1[m].x : rho0s)));
            else rs = make_float2(0.5f * (r0[m].x + r1[m].x), 0.5f * (r0[m].y + r1[m].y));
            const float2 f = xi == 0 ? ldg2(g.t.pml_sg[0] + x) : make_float2(fyz, fyz);
            const float2 lup = csub(lo[m], v[m]);
            if (valid) st2(lu + rb + x, make_float2(f.x * f.x * lup.x, f.y * f.y * lup.y));
            v[m] = make_float2(-__fdividef(f.x * g.dt * lup.x, rs.x), -__fdividef(f.y * g.dt * lup.y, rs.y));
        }
        row_r2c<LOGM>(v, S, j, valid, g.t.tw, pick3w(K.a.sp, xi) + (size_t)rr * g.nhp);
    }
}

template <int LOGM>
__global__ void __launch_bounds__(XTHREADS, XShape<LOGM>::MINB) adj_x_p_kernel(const AdjXK K) {
    using Sh = XShape<LOGM>;
    constexpr int E = Sh::E, TL = Sh::TL;
    extern __shared__ float2 smem[];
    const GridC& g = K.g;
    const int r = threadIdx.x / TL, j = threadIdx.x % TL;
    const int row = blockIdx.x * Sh::RPB + r;
    const bool valid = row < g.ny * g.nz;
    const int rr = valid ? row : 0;
    typename Sh::Smem S = Sh::row_smem(smem, r);
    float2 v[E];
    row_c2r<LOGM>(K.a.sp[0] + (size_t)rr * g.nhp, S, j, valid, g.t.tw, v);
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m)
            st2(K.a.lam_p + (size_t)rr * g.nx + 2 * (j + TL * m), make_float2(-v[m].x, -v[m].y));
    }
    // the last kernel of a reverse step: its readers of the step index (the
    // objective and the source gradient) have finished, so step it back here
    if (K.a.nrev && blockIdx.x == 0 && threadIdx.x == 0) *K.a.nrev -= 1;
}

__device__ __forceinline__ float medv(const float* f, float s, int64_t i) { return f ? f[i] : s; }

// The reverse step's index n is read from the device counter nrev (so that a
// captured segment of reverse steps serves every segment), and lowered by
// adj_x_p_kernel at the end of each reverse step.
__global__ void adj_obj_kernel(int64_t n_obj, const int64_t* __restrict__ idx, const float* __restrict__ pobj,
                               const int64_t* __restrict__ nrev, double weight, float* lam_p) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_obj) return;
    const float v = pobj[*nrev * n_obj + k];                  // p^{n+1} at objective point k
    const float sgn = v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f);   // d|p|/dp
    lam_p[idx[k]] += (float)(weight * sgn);
}

// One warp per signal row: the lanes stride over the row's points and the
// partial sums meet in a fixed butterfly, so the result does not depend on
// scheduling (the gradient is bitwise reproducible).
__global__ void adj_src_kernel(int rows, const int32_t* __restrict__ row_ptr, const int64_t* __restrict__ pts,
                               const float* __restrict__ scale, const int32_t* __restrict__ nt,
                               const float* __restrict__ lam_src, Medium md, double* grad, int64_t stride,
                               const int64_t* __restrict__ nrev) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= rows) return;                                     // whole warps
    const int64_t n = *nrev;
    if (n >= nt[r]) return;
    double acc = 0.0;
    for (int k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int64_t L = pts[k];
        acc += (double)lam_src[L] * (double)scale[k] / (double)medv(md.c0, md.c0_s, L);   // dt 2 / (3 c0 dx)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) grad[r * stride + n] += acc;
}

cudaError_t launch_adj_x_absprep(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s) {
    AdjXK K{g, m, a};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(adj_x_absprep_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj_x_dens(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s) {
    AdjXK K{g, m, a};
    switch (g.lognx - 1) {
#define CASE(L)                                                                                          \
    case L:                                                                                              \
        if (m.absorbing) return launch_rows(adj_x_dens_kernel<L, true>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s); \
        return launch_rows(adj_x_dens_kernel<L, false>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj_x_vel(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s) {
    AdjXK K{g, m, a};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(adj_x_vel_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj_x_p(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s) {
    AdjXK K{g, m, a};
    switch (g.lognx - 1) {
#define CASE(L) \
    case L: return launch_rows(adj_x_p_kernel<L>, XShape<L>::RPB, XShape<L>::SMEM, g, K, s);
        KWGB_LOGM_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj_obj(int64_t n_obj, const int64_t* idx, const float* pobj, const int64_t* nrev, double weight,
                           float* lam_p, cudaStream_t s) {
    if (n_obj <= 0) return cudaSuccess;
    adj_obj_kernel<<<(unsigned)((n_obj + 255) / 256), 256, 0, s>>>(n_obj, idx, pobj, nrev, weight, lam_p);
    return cudaGetLastError();
}

cudaError_t launch_adj_src(int rows, const int32_t* row_ptr, const int64_t* pts, const float* scale,
                           const int32_t* nt, const float* lam_src, const Medium& m, double* grad,
                           int64_t stride, const int64_t* nrev, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    adj_src_kernel<<<(rows + 7) / 8, 256, 0, s>>>(rows, row_ptr, pts, scale, nt, lam_src, m, grad, stride, nrev);
    return cudaGetLastError();
}

}  // namespace kwgb
