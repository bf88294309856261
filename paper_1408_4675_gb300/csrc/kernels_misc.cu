// Small kernels around the FFT passes: initial density, the device step
// counter (keeps every launch of a step identical, so a step can be captured
// in a CUDA graph once and replayed), and the sparse intensity sensors.
#include <cmath>

#include "kwgb_internal.h"

namespace kwgb {

// exp(-2 pi i a / b) rounded to float, a reduced modulo b first
static float2 unit_root(long a, long b) {
    const double t = 2.0 * 3.14159265358979323846 * (double)(a % b) / (double)b;
    return make_float2((float)std::cos(t), (float)-std::sin(t));
}

void fill_twiddle_table(float2* out) {
    for (int t = 0; t < 1024; ++t) out[t] = unit_root(t, 1024);
    for (int L = 2; L <= 1024; L *= 2)
        for (int rp = 2; rp <= 16 && rp <= L; rp *= 2) {
            const int off = stw_off(L, rp), ns = L / rp;
            for (int r = 1; r < rp; ++r)
                for (int k = 0; k < ns; ++k) out[off + (r - 1) * ns + k] = unit_root((long)k * r, L);
        }
    for (int M = 2; M <= 512; M *= 2)
        for (int k = 0; k < M; ++k) out[rtw_off(M) + k] = unit_root(k, 2 * M);
}

__global__ void init_rho_kernel(GridC g, Medium md, const float* __restrict__ p0, int pitch,
                                float* rx, float* ry, float* rz) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / g.nx, x = i % g.nx;
        const float c = md.c0 ? md.c0[i] : md.c0_s;
        const float v = p0[row * pitch + x] / (3.0f * c * c);   // rho_xi^0 = p0 / (3 c0^2)
        rx[i] = v;
        ry[i] = v;
        rz[i] = v;
    }
}

cudaError_t launch_init_rho(const GridC& g, const Medium& m, const float* p0, int p0_pitch,
                            float* rho[3], cudaStream_t s) {
    init_rho_kernel<<<1216, 256, 0, s>>>(g, m, p0, p0_pitch, rho[0], rho[1], rho[2]);
    return cudaGetLastError();
}

__global__ void advance_step_kernel(int64_t* step) { *step += 1; }

// Per-step work of the p_min / series sensors, after the pressure pass (which
// leaves p^{n+1} of every masked sensor slot in p_sens): slots k < n_slots
// update p_min and write sample n of their p series; points k < n_u write
// u_xi^{n+1/2} into their u series.
__global__ void series_kernel(int64_t n_slots, const float* __restrict__ p_sens, float* p_min,
                              const SeriesSlot* __restrict__ ser, float* series, int64_t n_u,
                              const int64_t* __restrict__ idx, const SeriesSlot* __restrict__ uq,
                              const float* __restrict__ ux, const float* __restrict__ uy,
                              const float* __restrict__ uz, float* useries, const int64_t* __restrict__ step) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = *step;
    if (k < n_slots) {
        const float v = p_sens[k];
        if (p_min) p_min[k] = fminf(p_min[k], v);
        if (ser) {
            const SeriesSlot q = ser[k];
            if (q.base >= 0) series[q.base + (n % q.cap) * q.stride] = v;
        }
    }
    if (k < n_u) {
        const SeriesSlot q = uq[k];
        const int64_t L = idx[k];
        const int64_t o = q.base + (n % q.cap) * 3 * (int64_t)q.stride;
        useries[o] = ux[L];
        useries[o + q.stride] = uy[L];
        useries[o + 2 * (int64_t)q.stride] = uz[L];
    }
}

cudaError_t launch_series(int64_t n_slots, const float* p_sens, float* p_min, const SeriesSlot* ser, float* series,
                          int64_t n_u, const int64_t* idx, const SeriesSlot* uq, float* const* u, float* useries,
                          const int64_t* step, cudaStream_t s) {
    const int64_t n = n_slots > n_u ? n_slots : n_u;
    if (n <= 0) return cudaSuccess;
    series_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_slots, p_sens, p_min, ser, series, n_u, idx, uq,
                                                               u[0], u[1], u[2], useries, step);
    return cudaGetLastError();
}

cudaError_t launch_advance_step(int64_t* step, cudaStream_t s) {
    advance_step_kernel<<<1, 1, 0, s>>>(step);
    return cudaGetLastError();
}

__global__ void fill_f32_kernel(float* p, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4864) blocks = 4864;
    fill_f32_kernel<<<blocks, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

// u_xi at the sensor point s and at s - e_xi (periodic), the two staggered
// values whose mean is the velocity on the regular grid.
__device__ __forceinline__ void neighbours(int64_t s, const GridC& g, int64_t (&nb)[3]) {
    const int64_t x = s % g.nx, y = (s / g.nx) % g.ny, z = s / ((int64_t)g.nx * g.ny);
    nb[0] = ((x + g.nx - 1) % g.nx) + g.nx * (y + (int64_t)g.ny * z);
    nb[1] = x + g.nx * (((y + g.ny - 1) % g.ny) + (int64_t)g.ny * z);
    nb[2] = x + g.nx * (y + (int64_t)g.ny * ((z + g.nz - 1) % g.nz));
}

__device__ __forceinline__ int64_t pitched(int64_t i, const GridC& g, int pitch) {
    return (i / g.nx) * pitch + (i % g.nx);
}

struct UPtrs {
    const float* u[3];
};

__global__ void intensity_gather_kernel(int64_t n, const int64_t* __restrict__ idx, GridC g,
                                        UPtrs u, int pitch, float* __restrict__ ubuf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = idx[i];
    int64_t nb[3];
    neighbours(s, g, nb);
#pragma unroll
    for (int xi = 0; xi < 3; ++xi) {
        ubuf[6 * i + 2 * xi] = u.u[xi][pitched(s, g, pitch)];
        ubuf[6 * i + 2 * xi + 1] = u.u[xi][pitched(nb[xi], g, pitch)];
    }
}

cudaError_t launch_intensity_gather(int64_t n, const int64_t* idx, const GridC& g,
                                    float* const* u, int pitch, float* ubuf, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    UPtrs up{{u[0], u[1], u[2]}};
    intensity_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, idx, g, up, pitch, ubuf);
    return cudaGetLastError();
}

// I_xi += p^n * (ubar^{n-1/2} + ubar^{n+1/2}) / 2, ubar = mean of u_xi at s - e_xi and s
__global__ void intensity_accum_kernel(int64_t n, const int64_t* __restrict__ idx, GridC g,
                                       UPtrs u, int pitch, const float* __restrict__ ubuf,
                                       const float* __restrict__ p_sens,
                                       const int32_t* __restrict__ slot, double* __restrict__ I,
                                       const int64_t* __restrict__ step, int skip_first) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (skip_first && *step == 0) return;           // p^0 is not a sample
    const int64_t s = idx[i];
    int64_t nb[3];
    neighbours(s, g, nb);
    const double p = p_sens[slot[i]];
#pragma unroll
    for (int xi = 0; xi < 3; ++xi) {
        const double un = (double)u.u[xi][pitched(s, g, pitch)] + (double)u.u[xi][pitched(nb[xi], g, pitch)];
        const double uo = (double)ubuf[6 * i + 2 * xi] + (double)ubuf[6 * i + 2 * xi + 1];
        I[xi * n + i] += p * 0.25 * (uo + un);
    }
}

cudaError_t launch_intensity_accum(int64_t n, const int64_t* idx, const GridC& g,
                                   float* const* u, int pitch, const float* ubuf,
                                   const float* p_sens, const int32_t* slot, double* I,
                                   const int64_t* step, int skip_first, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    UPtrs up{{u[0], u[1], u[2]}};
    intensity_accum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, idx, g, up, pitch, ubuf,
                                                                       p_sens, slot, I, step, skip_first);
    return cudaGetLastError();
}

}  // namespace kwgb
