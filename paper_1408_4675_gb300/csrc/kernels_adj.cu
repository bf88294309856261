// Pointwise parts of the adjoint (reverse-mode) time step.  The spectral
// parts reuse the forward passes: the adjoint of IFT{O FT{.}} on real fields
// is IFT{conj(O) FT{.}}, and conj(i k kappa e^{-ikd/2}) = -(i k kappa e^{+ikd/2}),
// so the transpose of Eq. 4c's operator is minus Eq. 4a's and vice versa.
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
//   lambda_rho   += IFT{k^{y-1} FT{-c0^2 eta lambda_p}}            (abs2)
//   lambda_d_xi  += rho0 IFT{k^{y-2} FT{c0^2 tau lambda_p}}         (rho0 abs1)
#include "kwgb_internal.h"

namespace kwgb {

__device__ __forceinline__ float medv(const float* f, float s, int64_t i) { return f ? f[i] : s; }

__global__ void adj_dens_kernel(GridC g, Medium md, AdjFields a) {
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((int64_t)g.nx * g.ny));
        const float c = medv(md.c0, md.c0_s, i);
        const float r0 = medv(md.rho0, md.rho0_s, i);
        float lrt = c * c * a.lam_p[i];
        if (md.nonlinear) {
            const float rho = a.rho_after[0][i] + a.rho_after[1][i] + a.rho_after[2][i];
            lrt *= 1.0f + medv(md.bona, md.bona_s, i) * rho / r0;
        }
        float ld_abs = 0.f;
        if (a.abs1) {
            lrt += a.abs2[i];
            ld_abs = r0 * a.abs1[i];
        }
        float src = 0.f;
#pragma unroll
        for (int xi = 0; xi < 3; ++xi) {
            const float f = xi == 0 ? g.t.pml[0][x] : (xi == 1 ? g.t.pml[1][y] : g.t.pml[2][z]);
            const float lrp = a.lam_rho[xi][i] + lrt;
            src += lrp;
            const float d = a.w[xi][i];
            if (md.nonlinear) {
                const float den = 1.0f + 2.0f * g.dt * d;
                a.lam_rho[xi][i] = lrp * f * f / den;
                a.w[xi][i] = ld_abs - lrp * f * g.dt * (r0 + 2.0f * f * a.rho_before[xi][i]) / (den * den);
            } else {
                a.lam_rho[xi][i] = lrp * f * f;
                a.w[xi][i] = ld_abs - lrp * f * g.dt * r0;
            }
        }
        a.lam_src[i] = src;
    }
}

__global__ void adj_absprep_kernel(GridC g, Medium md, const float* __restrict__ lam_p, float* q1, float* q2) {
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    const float ym1 = md.y - 1.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float c = medv(md.c0, md.c0_s, i);
        const float al = medv(md.alpha0, md.alpha0_s, i);
        const float ct = c * c * (-2.0f * al * exp2f(ym1 * log2f(c)));    // c0^2 tau, tau = -2 alpha0 c0^{y-1}
        const float l = lam_p[i];
        q1[i] = ct * l;
        q2[i] = ct * c * md.tan_pi_y_2 * l;                               // -c0^2 eta = c0^2 tau c0 tan(pi y/2)
    }
}

__global__ void adj_vel_kernel(GridC g, Medium md, AdjFields a) {
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((int64_t)g.nx * g.ny));
        const float r0 = medv(md.rho0, md.rho0_s, i);
#pragma unroll
        for (int xi = 0; xi < 3; ++xi) {
            // rho0 at the staggered point: mean with the +1 neighbour along xi (periodic)
            int64_t nb;
            if (xi == 0) nb = i - x + ((x + 1) % g.nx);
            else if (xi == 1) nb = i + (int64_t)(((y + 1) % g.ny) - y) * g.nx;
            else nb = i + (int64_t)(((z + 1) % g.nz) - z) * g.nx * g.ny;
            const float rs = 0.5f * (r0 + medv(md.rho0, md.rho0_s, nb));
            const float fs = xi == 0 ? g.t.pml_sg[0][x] : (xi == 1 ? g.t.pml_sg[1][y] : g.t.pml_sg[2][z]);
            const float lup = a.lam_u[xi][i] - a.w[xi][i];
            a.lam_u[xi][i] = fs * fs * lup;
            a.w[xi][i] = -fs * g.dt / rs * lup;
        }
    }
}

__global__ void adj_psum_kernel(GridC g, AdjFields a) {
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        a.lam_p[i] = -(a.w[0][i] + a.w[1][i] + a.w[2][i]);
}

__global__ void adj_obj_kernel(int64_t n, const int64_t* __restrict__ idx, const float* __restrict__ p,
                               double weight, float* lam_p) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float v = p[k];
    const float sgn = v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f);   // d|p|/dp
    lam_p[idx[k]] += (float)(weight * sgn);
}

__global__ void adj_src_kernel(int rows, const int32_t* __restrict__ row_ptr, const int64_t* __restrict__ pts,
                               const float* __restrict__ scale, const int32_t* __restrict__ nt,
                               const float* __restrict__ lam_src, Medium md, double* grad, int64_t stride,
                               int64_t n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows || n >= nt[r]) return;
    double acc = 0.0;
    for (int k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
        const int64_t L = pts[k];
        acc += (double)lam_src[L] * (double)scale[k] / (double)medv(md.c0, md.c0_s, L);   // dt 2 / (3 c0 dx)
    }
    grad[r * stride + n] += acc;
}

static int blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b > 4864 ? 4864 : (b < 1 ? 1 : b));
}

cudaError_t launch_adj_dens(const GridC& g, const Medium& m, const AdjFields& a, cudaStream_t s) {
    adj_dens_kernel<<<blocks_for((int64_t)g.nx * g.ny * g.nz), 256, 0, s>>>(g, m, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_absprep(const GridC& g, const Medium& m, const float* lam_p, float* q1, float* q2,
                               cudaStream_t s) {
    adj_absprep_kernel<<<blocks_for((int64_t)g.nx * g.ny * g.nz), 256, 0, s>>>(g, m, lam_p, q1, q2);
    return cudaGetLastError();
}

cudaError_t launch_adj_vel(const GridC& g, const Medium& m, const AdjFields& a, cudaStream_t s) {
    adj_vel_kernel<<<blocks_for((int64_t)g.nx * g.ny * g.nz), 256, 0, s>>>(g, m, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_psum(const GridC& g, const AdjFields& a, cudaStream_t s) {
    adj_psum_kernel<<<blocks_for((int64_t)g.nx * g.ny * g.nz), 256, 0, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_obj(int64_t n, const int64_t* idx, const float* p, double weight, float* lam_p,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    adj_obj_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, idx, p, weight, lam_p);
    return cudaGetLastError();
}

cudaError_t launch_adj_src(int rows, const int32_t* row_ptr, const int64_t* pts, const float* scale,
                           const int32_t* nt, const float* lam_src, const Medium& m, double* grad,
                           int64_t stride, int64_t n, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    adj_src_kernel<<<(rows + 127) / 128, 128, 0, s>>>(rows, row_ptr, pts, scale, nt, lam_src, m, grad, stride, n);
    return cudaGetLastError();
}

}  // namespace kwgb
