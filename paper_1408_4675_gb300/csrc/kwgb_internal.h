// Internal declarations shared by the kernel translation units and the C-ABI
// implementation: parameter blocks passed by value to the kernels and the
// host-side launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace kwgb {

// Fill the TW_TOTAL-entry twiddle table (layout in fft_core.cuh) in float64.
void fill_twiddle_table(float2* out);

// 1-D tables in device memory (generated on the host in float64, stored as float).
struct Tables {
    const float2* tw;         // FFT twiddles, TW_TOTAL entries (regions: fft_core.cuh)
    const float* kx;          // Eq. 5 wavenumbers: kx for the half spectrum (nh values)
    const float* ky;          //   ky (ny), kz (nz), FFT storage order
    const float* kz;
    const float2* dfx;        // i k exp(+i k d / 2) per axis (Eq. 4a shift operator, no kappa)
    const float2* dfy;
    const float2* dfz;
    const float* pml[3];      // PML factor exp(-a dt / 2) on the regular grid, per axis
    const float* pml_sg[3];   // ... on the staggered grid i + 1/2
    // tensor-core forms: 64 x 64 DFT operands (hi, lo; fft_tc5.cuh layout) of the
    // radix-32 stage, then of the second stage of y lines, then of z lines
    const uint32_t* tc5a;
};

struct GridC {
    int nx, ny, nz;           // grid
    int nh;                   // nx / 2 + 1 (half-spectrum length along x)
    int nhp;                  // row pitch of spectra, complex elements (multiple of 16)
    int lognx, logny, lognz;
    float dt;
    float scale;              // 1 / (nx ny nz): inverse-FFT normalisation
    float hk;                 // c_ref dt / 2, argument factor of kappa
    float hk2;                // hk^2 (kappa is evaluated from (hk k)^2)
    float inv_kmax2;          // 1 / max k^2
    float abs_e[2];           // (y-2)/2, (y-1)/2: powers of k^2 / kmax^2 in Eq. 8
    float abs_c[2];           // kmax^(y-2), kmax^(y-1)
    int num_sms;              // SMs of the device (persistent grids)
    int mixed;                // strided passes: 0 float32, 1 bfloat16-split, 2 float16-split tensor-core products
    uint32_t wait_fault_tx;   // test hook (kwgb_debug_wait_fault): extra bytes each tile load expects, 0 normally
    Tables t;
};

// A spectrum buffer with the TMA tensor maps of its y-pass and z-pass tiles.
struct SpecBuf {
    float2* p;
    CUtensorMap ymap;
    CUtensorMap zmap;
};
// Encode the two tensor maps of a spectrum buffer (0 on success).
int make_spec_maps(const GridC& g, float2* ptr, SpecBuf* out);

struct Medium {
    const float* c0;          // NULL -> scalar value below
    const float* rho0;
    const float* bona;
    const float* alpha0;
    float c0_s, rho0_s, bona_s, alpha0_s;
    float y;                  // power-law exponent
    float tan_pi_y_2;         // tan(pi y / 2)
    int nonlinear, absorbing;
};

// Sources: unique points per row (CSR over rows), each with a range of
// contributions (signal row, per-point scale dt * 2 / (3 c0 dx)).
struct SourceC {
    const int32_t* row_ptr;   // nrows + 1, NULL when there are no sources
    const int32_t* pt_x;      // x of each unique point
    const int32_t* pt_c;      // npts + 1 contribution ranges
    const int64_t* c_off;     // start of the contribution's signal samples
    const int32_t* c_nt;      // number of samples
    const float* c_scale;     // per contribution: dt * 2 / (3 dx) (mass), dt (force), 1 (Dirichlet)
    const float* signal;      // all signal samples
};

// Masked sensor points (CSR over rows) and full-grid sensors.
// Where the samples of one sensor point go in a series ring buffer:
// sample n at base + (n mod cap) * stride (u series: base + ((n mod cap) * 3 + xi) * stride).
struct SeriesSlot {
    int64_t base;             // < 0: the point records no series
    int32_t stride;           // points of its sensor
    int32_t cap;              // ring length
};

struct SensorC {
    const int32_t* row_ptr;   // nrows + 1, NULL when no masked sensor points
    const int32_t* e_x;       // x of each entry
    const int32_t* e_slot;    // slot of each entry
    float* p_max;             // per slot
    double* p2;               // per slot, sum of p^2
    float* p_sens;            // per slot, last p (intensity)
    float* p_min;             // per slot (NULL when no sensor records P_MIN); updated by launch_series
    const SeriesSlot* ser;    // per slot (NULL when no sensor records a p series)
    float* series;            // p series ring buffers
    int nfull;                // full-grid sensors (<= 4)
    float* full_max[4];
    double* full_p2[4];
    float* full_min[4];       // NULL unless that sensor records P_MIN
};

struct StepC {
    const int64_t* step;      // device step counter n (the step maps n -> n+1)
    int* flag;                // device status bits (1 = non-finite pressure)
};

// ---- launchers (return the launch error) --------------------------------
// y pass on ncomp spectra: in[c] -> out[c] (in place allowed); dir -1 forward, +1 inverse.
// flag receives bit 2 if a bounded TMA wait runs out.
cudaError_t launch_y_pass(const GridC& g, int dir, const SpecBuf* const* in, float2* const* out,
                          int ncomp, int* flag, cudaStream_t s);

enum ZOpKind { Z_GRAD_FWD = 0, Z_GRAD_BWD = 1, Z_DIV = 2, Z_ABS = 3, Z_DIV_FWD = 4, Z_DIV_SUM = 5 };
// z forward FFT -> operator -> z inverse FFT:
//   Z_GRAD_*: in[0] -> out[xi] (NULL skips a component)
//   Z_DIV:    in[xi] -> out[xi]  (Eq. 4c operator)
//   Z_DIV_FWD: in[xi] -> out[xi] (Eq. 4a operator per component; adjoint pass)
//   Z_DIV_SUM: in[0..2] -> out[0] = sum over xi of the Eq. 4c operator on in[xi] (adjoint pass)
//   Z_ABS:    in[0] -> out[0] with k^{y-2}, in[1] -> out[1] with k^{y-1} (NULL skips)
cudaError_t launch_z_op(const GridC& g, int kind, const SpecBuf* const* in, float2* const* out,
                        int* flag, cudaStream_t s);

enum XVelMode { XV_STEP = 0, XV_TAIL = 1, XV_INIT = 2 };
struct XVelArgs {
    const float2* G[3];       // gradient spectra (Eq. 4a, after y/z inverse)
    float* u[3];              // velocity (pitch nx)
    float2* U[3];             // XV_STEP: x-R2C of the new velocity (may alias G)
    float* tail[3];           // XV_TAIL: u^{Nt+1/2} written as real rows of pitch 2*nhp
    SourceC f[3];             // force sources along x, y, z (row_ptr NULL: none)
    const int64_t* step;      // device step counter (force samples)
};
cudaError_t launch_x_vel(const GridC& g, const Medium& m, int mode, const XVelArgs& a,
                         cudaStream_t s);

struct XDensArgs {
    const float2* D[3];       // divergence spectra (Eq. 4c)
    float* rho[3];            // split density (pitch nx)
    float2* S;                // x-R2C of rho0 sum d  (absorbing only)
    float2* R;                // x-R2C of rho         (absorbing only)
    float* rho_tot;           // rho as real rows of pitch 2*nhp (absorbing only)
    float2* P;                // non-absorbing: x-R2C of p (EOS fused here)
    // adjoint: with keep set, the step also writes, at keep + k 7 N (k = step
    // index mod keep_period, N = nx ny nz, pitch nx): rho_xi^n as read
    // (+ xi N), the Eq. 4c derivative d_xi (+ (3 + xi) N) and
    // rho^{n+1} = sum rho_xi after the sources (+ 6 N)
    float* keep;
    int64_t keep_period;
};
cudaError_t launch_x_dens(const GridC& g, const Medium& m, const SourceC& src, const SourceC& dsrc,
                          const SensorC& sens, const StepC& st, const XDensArgs& a,
                          cudaStream_t s);

struct XEosArgs {
    const float2* A1;         // IFT_yz{k^{y-2} ...} of S (x still spectral)
    const float2* A2;         // ... k^{y-1} of R
    const float* rho_tot;     // pitch 2*nhp
    float2* P;                // x-R2C of p^{n+1}
};
cudaError_t launch_x_eos(const GridC& g, const Medium& m, const SourceC& dsrc, const SensorC& sens,
                         const StepC& st, const XEosArgs& a, cudaStream_t s);

// plain x transforms: real rows (pitch in floats) <-> half spectra (pitch nhp)
cudaError_t launch_x_r2c(const GridC& g, const float* in, int in_pitch, float2* out,
                         cudaStream_t s);
cudaError_t launch_x_c2r(const GridC& g, const float2* in, float* out, int out_pitch,
                         cudaStream_t s);

// small kernels
cudaError_t launch_init_rho(const GridC& g, const Medium& m, const float* p0, int p0_pitch,
                            float* rho[3], cudaStream_t s);
cudaError_t launch_advance_step(int64_t* step, cudaStream_t s);
// p_min and series sensors of one step: masked slots (p from p_sens) and u-series points
cudaError_t launch_series(int64_t n_slots, const float* p_sens, float* p_min, const SeriesSlot* ser, float* series,
                          int64_t n_u, const int64_t* idx, const SeriesSlot* uq, float* const* u, float* useries,
                          const int64_t* step, cudaStream_t s);
cudaError_t launch_intensity_gather(int64_t n, const int64_t* idx, const GridC& g,
                                    float* const* u, int pitch, float* ubuf, cudaStream_t s);
cudaError_t launch_intensity_accum(int64_t n, const int64_t* idx, const GridC& g,
                                   float* const* u, int pitch, const float* ubuf,
                                   const float* p_sens, const int32_t* slot, double* I,
                                   const int64_t* step, int skip_first, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t s);

// ---- adjoint (reverse-mode) step ---------------------------------------
// Fields of one reverse step; the x passes read and write the spectra sp[]
// in place (kernels_adj.cu).
struct AdjX {
    float* lam_p;             // lambda of p^{n+1} (adj_x_dens in), of p^n (adj_x_p out)
    float* lam_u[3];          // lambda of u^{n+1/2} -> of u^{n-1/2}
    float* lam_rho[3];        // lambda of rho_xi^{n+1} -> of rho_xi^n
    float* lam_src;           // sum_xi lambda of rho_xi^{n+1} (source gradient)
    // the forward step's kept fields, laid out as XDensArgs::keep: rho_xi^n,
    // d_xi (Eq. 4c derivative), rho^{n+1}; step n's at keep + (n mod keep_period) 7 N
    const float* keep;
    int64_t keep_period;
    float2* sp[3];            // spectra (x transformed), pitch nhp
    int64_t* nrev;            // reverse-step counter n, lowered by adj_x_p
};
// absorbing: R2C of c0^2 tau lambda_p -> sp[0] and of -c0^2 eta lambda_p -> sp[1]
cudaError_t launch_adj_x_absprep(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s);
// [absorbing: C2R of the k^{y-2} / k^{y-1} results in sp[0], sp[1]] -> Eq. 6 / 4d backwards
// -> lambda_rho, lambda_src -> R2C of lambda_d_xi -> sp[xi]
cudaError_t launch_adj_x_dens(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s);
// C2R of sp[xi] (Eq. 4a op of lambda_d) -> Eq. 4b backwards -> lambda_u -> R2C of lambda_g_xi -> sp[xi]
cudaError_t launch_adj_x_vel(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s);
// lambda_p = -C2R sp[0] (sp[0]: the transpose of Eq. 4a, its three terms summed); then *nrev -= 1 (if nrev)
cudaError_t launch_adj_x_p(const GridC& g, const Medium& m, const AdjX& a, cudaStream_t s);
// lambda_p[idx_k] += weight * sign(p^{n+1}_k), n = *nrev, samples pobj[n * n_obj + k]
cudaError_t launch_adj_obj(int64_t n_obj, const int64_t* idx, const float* pobj, const int64_t* nrev, double weight,
                           float* lam_p, cudaStream_t s);
// per signal row r: grad[r * stride + n] += sum over its points of lambda_src * scale / c0 (n = *nrev < nt_r)
cudaError_t launch_adj_src(int rows, const int32_t* row_ptr, const int64_t* pts, const float* scale,
                           const int32_t* nt, const float* lam_src, const Medium& m, double* grad,
                           int64_t stride, const int64_t* nrev, cudaStream_t s);

}  // namespace kwgb
