// C-ABI implementation: validation, device buffers, the 1-D tables (built on
// the host in float64), the sparse source/sensor structures, and the launch
// sequence of one time step.
//
// Device memory of a simulation (F = nx*ny*nz floats, S = nz*ny*nhp complex):
//   u_x, u_y, u_z, rho_x, rho_y, rho_z        6 F   state
//   c0, rho0, B/A, alpha0                     <= 4 F (scalars take no memory)
//   P (x-transformed p^n), T1, T2, T3         4 S   spectra; T1/T2 hold the
//                                                   step's temporaries, T3 is
//                                                   scratch for reads and
//                                                   kwgb_apply_operator
//   sensors, sources, 1-D tables              small
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/kwgb.h"
#include "fft_tc5.cuh"
#include "kwgb_internal.h"

using namespace kwgb;

static constexpr double kPi = 3.14159265358979323846;

namespace {

struct HostSource {
    std::vector<int64_t> idx;
    std::vector<float> sig;
    int64_t nsig, nt;
    int mode = KWGB_ADDITIVE_MASS;
};

struct HostSensor {
    bool full;
    std::vector<int64_t> idx;   // masked points
    uint32_t record;
    int64_t n;                  // number of points
    int64_t slot0;              // first slot (masked)
    int full_k;                 // index into the full-grid arrays
    int64_t i0;                 // first entry in the intensity list (-1: none)
    int64_t cap = 0;            // series ring length (kwgb_set_series_capacity)
    int64_t pser0 = -1;         // p series: offset of its ring in the p series buffer
    int64_t user0 = -1;         // u series: offset of its ring in the u series buffer
};

thread_local std::string g_create_error;

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) ++l; return l; }

}  // namespace

struct kwgb_sim {
    kwgb_grid_desc d;
    GridC g;
    Medium md;
    std::string err;
    void* (*alloc)(size_t, void*) = nullptr;
    void (*freef)(void*, void*) = nullptr;
    void* actx = nullptr;
    std::vector<void*> allocs;
    int64_t bytes = 0;
    bool medium_set = false;
    bool frozen = false;
    int64_t steps = 0;
    int64_t N = 0;              // grid points
    size_t spec_elems = 0;      // complex elements per spectrum

    float* u[3] = {nullptr, nullptr, nullptr};
    float* rho[3] = {nullptr, nullptr, nullptr};
    float2* P = nullptr;
    float2* T1 = nullptr;
    float2* T2 = nullptr;
    float2* T3 = nullptr;
    SpecBuf bP{}, b1{}, b2{}, b3{};     // the same buffers with their TMA tensor maps
    int64_t* d_step = nullptr;
    int* d_flag = nullptr;

    std::vector<HostSource> hsrc;
    std::vector<HostSensor> hsens;
    SourceC src{};              // additive mass sources
    SourceC fsrc[3] = {};       // force sources along x, y, z
    SourceC dsrc{};             // Dirichlet pressure sources
    bool any_force = false;
    SensorC sens{};
    int64_t n_slots = 0;
    int64_t n_i = 0;            // intensity points
    int64_t* i_idx = nullptr;
    int32_t* i_slot = nullptr;
    double* I = nullptr;
    double* I_tail = nullptr;
    float* ubuf = nullptr;
    int64_t series_elems = 0;   // p series buffer (floats)
    int64_t n_u = 0;            // points recording a u series
    int64_t* u_idx = nullptr;
    SeriesSlot* u_q = nullptr;
    float* useries = nullptr;
    int64_t useries_elems = 0;
    cudaStream_t last_stream = nullptr;
    int64_t launches = 0;       // kernels launched so far
    bool adjoint_done = false;
    // adjoint: kwgb_adjoint_forward keeps what kwgb_adjoint_backward needs
    // x_dens keeps rho_xi^n, d_xi and rho^{n+1} of step n at
    // adj_keep + (n mod adj_period) 7 N when set (XDensArgs::keep)
    float* adj_keep = nullptr;
    int64_t adj_period = 0;
    struct AdjRun {
        bool pending = false;            // forward with checkpoints done, reverse pass not yet run
        bool keep_all = false;           // K >= n_steps: the forward run kept every step's fields
        float* seg = nullptr;            // kept fields (keep_all: of every step, written by the forward run)
        int64_t n_steps = 0, K = 0, n_obj = 0;
        double w = 0.0;                  // 1 / (n_obj n_steps)
        char* ck = nullptr;              // checkpoints (u, rho_xi, P) every K steps
        char* fin = nullptr;             // forward end state
        float* pobj = nullptr;           // p at the objective points, every step
        int64_t* d_obj = nullptr;        // objective points
        char* snap = nullptr;            // sensor accumulators after the forward run
        std::vector<std::pair<void*, size_t>> sarr;
    } adj;
    // one captured step, replayed by kwgb_step (CUDA graph)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;         // stream the step is captured on
    int64_t glaunches = 0;              // kernels in the captured step
    bool graph_off = false;             // capture not possible: launch directly
    bool warmed = false;                // a step has run directly (one-time set-up done)
    // per-launch event timing (kwgb_step_profiled)
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int32_t> ev_kind;
};

// ------------------------------------------------------------------ helpers
// NVTX range over one C-ABI call (visible to Nsight tools; a no-op without one)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static int fail(kwgb_sim* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(sim, KWGB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void* dalloc(kwgb_sim* sim, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (sim->alloc) {
        p = sim->alloc(bytes, sim->actx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        sim->allocs.push_back(p);
        sim->bytes += (int64_t)bytes;
    }
    return p;
}

template <class T>
static T* dalloc_t(kwgb_sim* sim, size_t n) { return static_cast<T*>(dalloc(sim, n * sizeof(T))); }

#define DALLOC(ptr, T, n)                                                              \
    do {                                                                               \
        ptr = dalloc_t<T>(sim, (size_t)(n));                                           \
        if (!ptr) return fail(sim, KWGB_ERR_OOM, "device allocation failed: " #ptr);   \
    } while (0)

template <class T>
static int upload(kwgb_sim* sim, T** dst, const std::vector<T>& src) {
    DALLOC(*dst, T, src.size());
    if (!src.empty()) CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return KWGB_OK;
}

// Eq. 5 wavenumber of DFT bin j of an axis with n points and spacing d
static double wavenumber(int64_t j, int64_t n, double d) {
    const int64_t m = (n % 2 == 0) ? (j < n / 2 ? j : j - n) : (j <= (n - 1) / 2 ? j : j - n);
    return (double)m * 2.0 * kPi / (d * (double)n);
}

// PML factor exp(-a dt / 2), a = alpha * (c_ref / d) * (depth / size)^4
static double pml_factor(double s, int64_t n, int size, double alpha, double c_ref, double d, double dt) {
    if (size <= 0) return 1.0;
    const double depth = std::max(0.0, std::max((double)size - s, s - (double)(n - 1 - size)));
    const double a = alpha * (c_ref / d) * std::pow(depth / size, 4.0);
    return std::exp(-a * dt / 2.0);
}

// ------------------------------------------------------------------ create
extern "C" int kwgb_create(const kwgb_grid_desc* desc, kwgb_sim** out) {
    g_create_error.clear();
    auto bad = [&](int code, const char* m) { g_create_error = m; if (out) *out = nullptr; return code; };
    if (!desc || !out) return bad(KWGB_ERR_ARG, "null argument");
    const int64_t n[3] = {desc->nx, desc->ny, desc->nz};
    const double dd[3] = {desc->dx, desc->dy, desc->dz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] <= 0) return bad(KWGB_ERR_ARG, "grid sizes must be positive");
        if (!is_pow2(n[a]) || n[a] < 8 || n[a] > 1024)
            return bad(KWGB_ERR_UNSUPPORTED, "grid sizes must be powers of two in [8, 1024]");
        if (!(dd[a] > 0) || !std::isfinite(dd[a])) return bad(KWGB_ERR_ARG, "spacing must be positive");
        if (desc->pml_size[a] < 0 || 2 * (int64_t)desc->pml_size[a] >= n[a])
            return bad(KWGB_ERR_ARG, "pml_size must be >= 0 and leave an interior");
        if (!(desc->pml_alpha[a] >= 0) || !std::isfinite(desc->pml_alpha[a]))
            return bad(KWGB_ERR_ARG, "pml_alpha must be >= 0");
    }
    if (!(desc->dt > 0) || !std::isfinite(desc->dt)) return bad(KWGB_ERR_ARG, "dt must be positive");
    if (!(desc->c_ref > 0) || !std::isfinite(desc->c_ref)) return bad(KWGB_ERR_ARG, "c_ref must be positive");
    if (desc->flags & ~(KWGB_NONLINEAR | KWGB_ABSORBING | KWGB_MIXED_BF16 | KWGB_MIXED_F16))
        return bad(KWGB_ERR_ARG, "unknown flag bits");
    if ((desc->flags & KWGB_MIXED_BF16) && (desc->flags & KWGB_MIXED_F16))
        return bad(KWGB_ERR_ARG, "choose one tensor-core form");
    if ((desc->flags & (KWGB_MIXED_BF16 | KWGB_MIXED_F16)) && (desc->ny < 16 || desc->nz < 16))
        return bad(KWGB_ERR_UNSUPPORTED, "the tensor-core form needs ny, nz >= 16");
    if (desc->flags & KWGB_ABSORBING) {
        const double y = desc->alpha_power;
        if (!(y > 0 && y < 3) || y == 1.0) return bad(KWGB_ERR_ARG, "alpha_power must be in (0,3), != 1");
    }
    kwgb_sim* sim = new (std::nothrow) kwgb_sim();
    if (!sim) return bad(KWGB_ERR_OOM, "host allocation failed");
    sim->d = *desc;
    GridC& g = sim->g;
    std::memset(&g, 0, sizeof(g));
    g.nx = (int)n[0]; g.ny = (int)n[1]; g.nz = (int)n[2];
    g.nh = g.nx / 2 + 1;
    g.nhp = (g.nh + 15) / 16 * 16;
    g.lognx = ilog2(n[0]); g.logny = ilog2(n[1]); g.lognz = ilog2(n[2]);
    g.dt = (float)desc->dt;
    sim->N = n[0] * n[1] * n[2];
    g.scale = (float)(1.0 / (double)sim->N);
    g.hk = (float)(desc->c_ref * desc->dt / 2.0);
    g.hk2 = (float)((desc->c_ref * desc->dt / 2.0) * (desc->c_ref * desc->dt / 2.0));
    const double y = desc->alpha_power;
    double kmax2 = 0;
    for (int a = 0; a < 3; ++a) kmax2 += (kPi / dd[a]) * (kPi / dd[a]);
    g.inv_kmax2 = (float)(1.0 / kmax2);
    g.abs_e[0] = (float)((y - 2.0) / 2.0);
    g.abs_e[1] = (float)((y - 1.0) / 2.0);
    g.abs_c[0] = (float)std::pow(std::sqrt(kmax2), y - 2.0);
    g.abs_c[1] = (float)std::pow(std::sqrt(kmax2), y - 1.0);
    sim->spec_elems = (size_t)g.nhp * g.ny * g.nz;
    Medium& md = sim->md;
    std::memset(&md, 0, sizeof(md));
    md.y = (float)y;
    md.tan_pi_y_2 = (float)std::tan(kPi * y / 2.0);
    md.nonlinear = (desc->flags & KWGB_NONLINEAR) ? 1 : 0;
    md.absorbing = (desc->flags & KWGB_ABSORBING) ? 1 : 0;
    g.mixed = (desc->flags & KWGB_MIXED_BF16) ? 1 : ((desc->flags & KWGB_MIXED_F16) ? 2 : 0);
    *out = sim;
    return KWGB_OK;
}

extern "C" int kwgb_set_allocator(kwgb_sim* sim, void* (*alloc)(size_t, void*),
                                  void (*free_fn)(void*, void*), void* ctx) {
    if (!sim) return KWGB_ERR_ARG;
    if (sim->medium_set) return fail(sim, KWGB_ERR_STATE, "allocator must be set before kwgb_set_medium");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(sim, KWGB_ERR_ARG, "alloc and free go together");
    sim->alloc = alloc;
    sim->freef = free_fn;
    sim->actx = ctx;
    return KWGB_OK;
}

// ------------------------------------------------------------------ medium
// One 64 x 64 operand of the tensor-core form (layout tc5_koff): `blocks`
// copies on the diagonal of the L-point forward DFT in real form (row
// 2k + r, column 2b + s; L = 64 / (2 blocks)), split into hi = round(a) and
// lo = round(a - hi) in float16 (prec 2) or bfloat16 (prec 1), generated in
// float64.
static void tc5_dft_operand(int prec, int L, uint16_t* hi, uint16_t* lo) {
    for (int m = 0; m < 64; ++m)
        for (int k = 0; k < 64; ++k) {
            double v = 0.0;
            if (m / (2 * L) == k / (2 * L)) {
                const int kk = (m % (2 * L)) / 2, b = (k % (2 * L)) / 2;
                const double th = -2.0 * kPi * (double)((kk * b) % L) / (double)L;
                const int r = m & 1, c = k & 1;
                // (x_re + i x_im)(cos th + i sin th): re row [cos, -sin], im row [sin, cos]
                v = r == 0 ? (c == 0 ? std::cos(th) : -std::sin(th)) : (c == 0 ? std::sin(th) : std::cos(th));
            }
            uint16_t h, l;
            if (prec == 2) {
                const __half hh = __float2half_rn((float)v);
                const __half ll = __float2half_rn((float)(v - (double)__half2float(hh)));
                std::memcpy(&h, &hh, 2);
                std::memcpy(&l, &ll, 2);
            } else {
                const __nv_bfloat16 hh = __float2bfloat16_rn((float)v);
                const __nv_bfloat16 ll = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hh)));
                std::memcpy(&h, &hh, 2);
                std::memcpy(&l, &ll, 2);
            }
            const int o = tc5_koff(m, k) / 2;
            hi[o] = h;
            lo[o] = l;
        }
}

// The operands of the tcgen05 passes: the 32-point DFT (stage 1), then the
// stage-2 operand of y lines and of z lines (32 / n1 copies of the n1-point
// DFT, n1 = n / 32; unused for n < 64); each as hi then lo.
static void tc5_operands(int prec, int ny, int nz, std::vector<uint32_t>& out) {
    out.assign(6 * TC5_A_WORDS, 0u);
    uint16_t* p = reinterpret_cast<uint16_t*>(out.data());
    const int per = TC5_A_BYTES / 2;
    tc5_dft_operand(prec, 32, p, p + per);
    const int n1[2] = {ny / 32, nz / 32};
    for (int i = 0; i < 2; ++i)
        if (n1[i] >= 2) tc5_dft_operand(prec, n1[i], p + (2 + 2 * i) * per, p + (3 + 2 * i) * per);
}

static int build_tables(kwgb_sim* sim) {
    const kwgb_grid_desc& d = sim->d;
    GridC& g = sim->g;
    const int64_t n[3] = {d.nx, d.ny, d.nz};
    const double dd[3] = {d.dx, d.dy, d.dz};
    std::vector<float2> tw(TW_TOTAL);
    fill_twiddle_table(tw.data());
    float2* dtw;
    if (int e = upload(sim, &dtw, tw)) return e;
    g.t.tw = dtw;
    const int64_t klen[3] = {g.nh, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
        std::vector<float> k(klen[a]);
        std::vector<float2> df(klen[a]);
        for (int64_t j = 0; j < klen[a]; ++j) {
            const double kk = wavenumber(j, n[a], dd[a]);
            k[j] = (float)kk;
            // i k exp(+i k d / 2) = (-k sin(k d / 2), k cos(k d / 2))
            df[j] = make_float2((float)(-kk * std::sin(kk * dd[a] / 2.0)), (float)(kk * std::cos(kk * dd[a] / 2.0)));
        }
        float* dk;
        float2* ddf;
        if (int e = upload(sim, &dk, k)) return e;
        if (int e = upload(sim, &ddf, df)) return e;
        if (a == 0) { g.t.kx = dk; g.t.dfx = ddf; }
        if (a == 1) { g.t.ky = dk; g.t.dfy = ddf; }
        if (a == 2) { g.t.kz = dk; g.t.dfz = ddf; }
        std::vector<float> f(n[a]), fs(n[a]);
        for (int64_t i = 0; i < n[a]; ++i) {
            f[i] = (float)pml_factor((double)i, n[a], d.pml_size[a], d.pml_alpha[a], d.c_ref, dd[a], d.dt);
            fs[i] = (float)pml_factor((double)i + 0.5, n[a], d.pml_size[a], d.pml_alpha[a], d.c_ref, dd[a], d.dt);
        }
        float *df1, *df2;
        if (int e = upload(sim, &df1, f)) return e;
        if (int e = upload(sim, &df2, fs)) return e;
        g.t.pml[a] = df1;
        g.t.pml_sg[a] = df2;
    }
    if (g.mixed) {
        std::vector<uint32_t> a;
        tc5_operands(g.mixed, (int)d.ny, (int)d.nz, a);
        uint32_t* da;
        if (int e = upload(sim, &da, a)) return e;
        g.t.tc5a = da;
    }
    return KWGB_OK;
}

static int set_field(kwgb_sim* sim, const float* src, bool scalar, bool dev, float* scal_out,
                     const float** field_out, float dflt) {
    *field_out = nullptr;
    if (src == nullptr) { *scal_out = dflt; return KWGB_OK; }
    if (scalar) {
        *scal_out = *src;
        if (!std::isfinite(*scal_out)) return fail(sim, KWGB_ERR_ARG, "non-finite medium scalar");
        return KWGB_OK;
    }
    float* p;
    DALLOC(p, float, sim->N);
    CK(cudaMemcpy(p, src, sim->N * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    *field_out = p;
    *scal_out = 0.f;
    return KWGB_OK;
}

extern "C" int kwgb_set_medium(kwgb_sim* sim, const float* c0, const float* rho0,
                               const float* b_on_a, const float* alpha0, uint32_t scalar_mask) {
    NvtxRange nvtx_("kwgb_set_medium");
    if (!sim) return KWGB_ERR_ARG;
    if (sim->medium_set) return fail(sim, KWGB_ERR_STATE, "medium already set");
    if (!c0 || !rho0) return fail(sim, KWGB_ERR_ARG, "c0 and rho0 are required");
    const bool dev = (scalar_mask & KWGB_INPUT_DEVICE) != 0;
    if ((scalar_mask & KWGB_SCALAR_C0) && !(*c0 > 0)) return fail(sim, KWGB_ERR_ARG, "c0 must be positive");
    if ((scalar_mask & KWGB_SCALAR_RHO0) && !(*rho0 > 0)) return fail(sim, KWGB_ERR_ARG, "rho0 must be positive");
    int dev_id = 0;
    CK(cudaGetDevice(&dev_id));
    Medium& md = sim->md;
    int e;
    if ((e = set_field(sim, c0, scalar_mask & KWGB_SCALAR_C0, dev, &md.c0_s, &md.c0, 0.f))) return e;
    if ((e = set_field(sim, rho0, scalar_mask & KWGB_SCALAR_RHO0, dev, &md.rho0_s, &md.rho0, 0.f))) return e;
    if ((e = set_field(sim, b_on_a, scalar_mask & KWGB_SCALAR_BONA, dev, &md.bona_s, &md.bona, 0.f))) return e;
    if ((e = set_field(sim, alpha0, scalar_mask & KWGB_SCALAR_ALPHA0, dev, &md.alpha0_s, &md.alpha0, 0.f))) return e;
    if ((e = build_tables(sim))) return e;
    const size_t N = (size_t)sim->N;
    for (int a = 0; a < 3; ++a) {
        DALLOC(sim->u[a], float, N);
        DALLOC(sim->rho[a], float, N);
        CK(cudaMemset(sim->u[a], 0, N * sizeof(float)));
        CK(cudaMemset(sim->rho[a], 0, N * sizeof(float)));
    }
    DALLOC(sim->P, float2, sim->spec_elems);
    DALLOC(sim->T1, float2, sim->spec_elems);
    DALLOC(sim->T2, float2, sim->spec_elems);
    DALLOC(sim->T3, float2, sim->spec_elems);
    CK(cudaMemset(sim->P, 0, sim->spec_elems * sizeof(float2)));
    {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
        sim->g.num_sms = sms;
        float2* bufs[4] = {sim->P, sim->T1, sim->T2, sim->T3};
        SpecBuf* sb[4] = {&sim->bP, &sim->b1, &sim->b2, &sim->b3};
        for (int i = 0; i < 4; ++i)
            if (make_spec_maps(sim->g, bufs[i], sb[i]) != 0)
                return fail(sim, KWGB_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
    DALLOC(sim->d_step, int64_t, 1);
    DALLOC(sim->d_flag, int, 1);
    CK(cudaMemset(sim->d_step, 0, sizeof(int64_t)));
    CK(cudaMemset(sim->d_flag, 0, sizeof(int)));
    CK(cudaDeviceSynchronize());
    sim->medium_set = true;
    return KWGB_OK;
}

// ------------------------------------------------------------------ launch helpers
#define LK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(sim, KWGB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static const char* const kKernelNames[] = {
    "y_fwd_p", "z_grad", "y_inv_grad", "x_vel", "y_fwd_u", "z_div", "y_inv_div", "x_dens",
    "y_fwd_abs", "z_abs", "y_inv_abs", "x_eos", "intensity_gather", "intensity_accum", "advance_step",
    "series"};
enum { K_Y_FWD_P, K_Z_GRAD, K_Y_INV_GRAD, K_X_VEL, K_Y_FWD_U, K_Z_DIV, K_Y_INV_DIV, K_X_DENS,
       K_Y_FWD_ABS, K_Z_ABS, K_Y_INV_ABS, K_X_EOS, K_I_GATHER, K_I_ACCUM, K_ADVANCE, K_SERIES, K_COUNT };

// Count a launch; when profiling, record an event after it on the launch stream.
static int mark(kwgb_sim* sim, int kind, cudaStream_t s) {
    sim->launches++;
    if (!sim->prof) return KWGB_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    CK(cudaEventRecord(e, s));
    sim->ev.push_back(e);
    sim->ev_kind.push_back(kind);
    return KWGB_OK;
}

#define LKM(call, kind)                                                                \
    do {                                                                               \
        LK(call);                                                                      \
        if (int e2_ = mark(sim, kind, s)) return e2_;                                  \
    } while (0)

// spectrum buffer -> its TMA descriptors
static const SpecBuf* spec(kwgb_sim* sim, const float2* p) {
    if (p == sim->P) return &sim->bP;
    if (p == sim->T1) return &sim->b1;
    if (p == sim->T2) return &sim->b2;
    if (p == sim->T3) return &sim->b3;
    return nullptr;
}

static cudaError_t ypass(kwgb_sim* sim, int dir, float2* const* in, float2* const* out, int n,
                         cudaStream_t s) {
    const SpecBuf* b[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < n; ++i) b[i] = spec(sim, in[i]);
    return launch_y_pass(sim->g, dir, b, out, n, sim->d_flag, s);
}

static cudaError_t zop(kwgb_sim* sim, int kind, float2* const* in, float2* const* out, cudaStream_t s) {
    const SpecBuf* b[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i) b[i] = in[i] ? spec(sim, in[i]) : nullptr;
    return launch_z_op(sim->g, kind, b, out, sim->d_flag, s);
}

// spectrum -> gradient spectra (x still transformed): y fwd, z op, y inv
static int grad_chain(kwgb_sim* sim, float2* in, float2* const out[3], int kind, cudaStream_t s) {
    float2* i1[1] = {in};
    LK(ypass(sim, -1, i1, i1, 1, s));
    float2* zin[3] = {in, nullptr, nullptr};
    LK(zop(sim, kind, zin, out, s));
    LK(ypass(sim, +1, out, out, 3, s));
    return KWGB_OK;
}

static SensorC sensor_c(kwgb_sim* sim) { return sim->sens; }

static int launch_step(kwgb_sim* sim, cudaStream_t s) {
    const GridC& g = sim->g;
    float2* sp[3] = {sim->P, sim->T1, sim->T2};
    StepC st{sim->d_step, sim->d_flag};
    // Eq. 4a: y fwd of x-transformed p, z fwd + operator + z inv (3 outputs), y inv
    {
        float2* i1[1] = {sim->P};
        LKM(ypass(sim, -1, i1, i1, 1, s), K_Y_FWD_P);
        float2* zin[3] = {sim->P, nullptr, nullptr};
        LKM(zop(sim, Z_GRAD_FWD, zin, sp, s), K_Z_GRAD);
        LKM(ypass(sim, +1, sp, sp, 3, s), K_Y_INV_GRAD);
    }
    if (sim->n_i) LKM(launch_intensity_gather(sim->n_i, sim->i_idx, g, sim->u, g.nx, sim->ubuf, s), K_I_GATHER);
    // Eq. 4b (+ x R2C of u), Eq. 4c (y fwd, z fwd + operator + z inv, y inv)
    XVelArgs va{};
    for (int a = 0; a < 3; ++a) { va.G[a] = sp[a]; va.u[a] = sim->u[a]; va.U[a] = sp[a]; va.f[a] = sim->fsrc[a]; }
    va.step = sim->d_step;
    LKM(launch_x_vel(g, sim->md, XV_STEP, va, s), K_X_VEL);
    if (sim->n_i)
        LKM(launch_intensity_accum(sim->n_i, sim->i_idx, g, sim->u, g.nx, sim->ubuf, sim->sens.p_sens,
                                   sim->i_slot, sim->I, sim->d_step, 1, s), K_I_ACCUM);
    LKM(ypass(sim, -1, sp, sp, 3, s), K_Y_FWD_U);
    LKM(zop(sim, Z_DIV, sp, sp, s), K_Z_DIV);
    LKM(ypass(sim, +1, sp, sp, 3, s), K_Y_INV_DIV);
    // Eq. 4d + source; lossless: Eq. 6 + sensors + R2C of p here
    XDensArgs da{};
    for (int a = 0; a < 3; ++a) {
        da.D[a] = sp[a];
        da.rho[a] = sim->rho[a];
    }
    da.keep = sim->adj_keep;
    da.keep_period = sim->adj_period;
    const SensorC sens = sensor_c(sim);
    if (sim->md.absorbing) {
        da.S = sim->P;
        da.R = sim->T1;
        da.rho_tot = reinterpret_cast<float*>(sim->T2);
        LKM(launch_x_dens(g, sim->md, sim->src, sim->dsrc, sens, st, da, s), K_X_DENS);
        // Eq. 8: y fwd, z fwd + k^{y-2} / k^{y-1} + z inv, y inv, then Eq. 6
        float2* ab[3] = {sim->P, sim->T1, nullptr};
        LKM(ypass(sim, -1, ab, ab, 2, s), K_Y_FWD_ABS);
        LKM(zop(sim, Z_ABS, ab, ab, s), K_Z_ABS);
        LKM(ypass(sim, +1, ab, ab, 2, s), K_Y_INV_ABS);
        XEosArgs ea{sim->P, sim->T1, reinterpret_cast<float*>(sim->T2), sim->P};
        LKM(launch_x_eos(g, sim->md, sim->dsrc, sens, st, ea, s), K_X_EOS);
    } else {
        da.P = sim->P;
        LKM(launch_x_dens(g, sim->md, sim->src, sim->dsrc, sens, st, da, s), K_X_DENS);
    }
    if (sim->n_u || sim->sens.p_min || sim->sens.ser) {
        const SensorC& sc = sim->sens;
        const int64_t np = (sc.p_min || sc.ser) ? sim->n_slots : 0;
        LKM(launch_series(np, sc.p_sens, sc.p_min, sc.ser, sc.series, sim->n_u, sim->u_idx, sim->u_q, sim->u,
                          sim->useries, sim->d_step, s), K_SERIES);
    }
    LKM(launch_advance_step(sim->d_step, s), K_ADVANCE);
    return KWGB_OK;
}

// Capture one step into a CUDA graph (once; every launch argument of a step
// is fixed after freeze(), and the time-dependent parts read the device step
// counter), so that a step is one graph launch instead of 13-15 kernel
// launches.  Called after the first step has run directly (one-time kernel
// attribute set-up stays outside the capture).  If capture or instantiation
// fails the simulation keeps launching kernels directly.
static void capture_step(kwgb_sim* sim) {
    if (sim->gexec || sim->graph_off) return;
    sim->graph_off = true;
    if (!sim->cap && cudaStreamCreateWithFlags(&sim->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaStreamBeginCapture(sim->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const int64_t l0 = sim->launches;
    const bool prof = sim->prof;
    const std::string err = sim->err;
    sim->prof = false;
    const int e = launch_step(sim, sim->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(sim->cap, &graph);
    sim->prof = prof;
    sim->glaunches = sim->launches - l0;
    sim->launches = l0;
    sim->err = err;
    if (e == KWGB_OK && ce == cudaSuccess && graph &&
        cudaGraphInstantiate(&sim->gexec, graph, 0) == cudaSuccess)
        sim->graph_off = false;
    else
        sim->gexec = nullptr;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
}

// One step on stream s: the captured graph when there is one, else direct launches.
static int run_step(kwgb_sim* sim, cudaStream_t s) {
    if (sim->warmed && !sim->prof) capture_step(sim);
    if (sim->gexec && !sim->prof) {
        CK(cudaGraphLaunch(sim->gexec, s));
        sim->launches += sim->glaunches;
        return KWGB_OK;
    }
    const int e = launch_step(sim, s);
    if (e == KWGB_OK) sim->warmed = true;
    return e;
}

// ------------------------------------------------------------------ initial pressure
extern "C" int kwgb_set_initial_pressure(kwgb_sim* sim, const float* p0) {
    NvtxRange nvtx_("kwgb_set_initial_pressure");
    if (!sim) return KWGB_ERR_ARG;
    if (!p0) return fail(sim, KWGB_ERR_ARG, "p0 is null");
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (sim->steps > 0) return fail(sim, KWGB_ERR_STATE, "initial pressure after stepping");
    const GridC& g = sim->g;
    cudaStream_t s = nullptr;
    float* real3 = reinterpret_cast<float*>(sim->T3);
    const int rp = 2 * g.nhp;
    CK(cudaMemcpy2D(real3, rp * sizeof(float), p0, g.nx * sizeof(float), g.nx * sizeof(float),
                    (size_t)g.ny * g.nz, cudaMemcpyHostToDevice));
    LK(launch_init_rho(g, sim->md, real3, rp, sim->rho, s));
    // u^{-1/2} = +dt / (2 rho0_sg) d/dxi p0
    LK(launch_x_r2c(g, real3, rp, sim->P, s));
    float2* out[3] = {sim->T3, sim->T1, sim->T2};
    if (int e = grad_chain(sim, sim->P, out, Z_GRAD_FWD, s)) return e;
    XVelArgs va{};
    for (int a = 0; a < 3; ++a) { va.G[a] = out[a]; va.u[a] = sim->u[a]; }
    LK(launch_x_vel(g, sim->md, XV_INIT, va, s));
    // P = x-R2C of p0 again (the chain above consumed it)
    CK(cudaMemcpy2D(real3, rp * sizeof(float), p0, g.nx * sizeof(float), g.nx * sizeof(float),
                    (size_t)g.ny * g.nz, cudaMemcpyHostToDevice));
    LK(launch_x_r2c(g, real3, rp, sim->P, s));
    CK(cudaDeviceSynchronize());
    return KWGB_OK;
}

// ------------------------------------------------------------------ sources and sensors
extern "C" int kwgb_add_source(kwgb_sim* sim, const int64_t* idx, int64_t n_idx,
                               const float* signal, int64_t n_signals, int64_t n_t,
                               int mode, int32_t* source_id) {
    if (!sim) return KWGB_ERR_ARG;
    if (sim->frozen || sim->steps > 0) return fail(sim, KWGB_ERR_STATE, "sources must be added before stepping");
    if (mode != KWGB_ADDITIVE_MASS && mode != KWGB_FORCE_X && mode != KWGB_FORCE_Y && mode != KWGB_FORCE_Z &&
        mode != KWGB_DIRICHLET_P)
        return fail(sim, KWGB_ERR_ARG, "unknown source mode");
    if (n_idx < 0 || n_t < 0) return fail(sim, KWGB_ERR_ARG, "negative size");
    if (n_idx > 0 && (!idx || (n_t > 0 && !signal))) return fail(sim, KWGB_ERR_ARG, "null idx or signal");
    if (!(n_signals == 1 || n_signals == n_idx)) return fail(sim, KWGB_ERR_ARG, "n_signals must be 1 or n_idx");
    HostSource hs;
    hs.idx.assign(idx, idx + n_idx);
    for (int64_t v : hs.idx)
        if (v < 0 || v >= sim->N) return fail(sim, KWGB_ERR_ARG, "source index out of range");
    hs.nsig = n_signals;
    hs.nt = n_t;
    hs.mode = mode;
    if (n_t > 0 && n_idx > 0) hs.sig.assign(signal, signal + n_signals * n_t);
    sim->hsrc.push_back(std::move(hs));
    if (source_id) *source_id = (int32_t)sim->hsrc.size() - 1;
    return KWGB_OK;
}

extern "C" int kwgb_add_sensor(kwgb_sim* sim, const int64_t* idx, int64_t n_idx,
                               uint32_t record, int32_t* sensor_id) {
    if (!sim) return KWGB_ERR_ARG;
    if (sim->frozen || sim->steps > 0) return fail(sim, KWGB_ERR_STATE, "sensors must be added before stepping");
    const uint32_t all = KWGB_P_MAX | KWGB_P_RMS | KWGB_I_AVG | KWGB_P_MIN | KWGB_P_SERIES | KWGB_U_SERIES;
    if (record == 0 || (record & ~all)) return fail(sim, KWGB_ERR_ARG, "bad record flags");
    HostSensor hs{};
    hs.record = record;
    hs.i0 = -1;
    if (idx == nullptr) {
        int nfull = 0;
        for (auto& o : sim->hsens) nfull += o.full ? 1 : 0;
        if ((record & (KWGB_I_AVG | KWGB_P_SERIES | KWGB_U_SERIES)) || nfull >= 4) {
            // full-grid intensity or series (or a fifth full-grid sensor): list every point
            hs.full = false;
            hs.idx.resize(sim->N);
            std::iota(hs.idx.begin(), hs.idx.end(), int64_t(0));
        } else {
            hs.full = true;
        }
        hs.n = sim->N;
    } else {
        if (n_idx < 0) return fail(sim, KWGB_ERR_ARG, "negative size");
        hs.full = false;
        hs.idx.assign(idx, idx + n_idx);
        for (int64_t v : hs.idx)
            if (v < 0 || v >= sim->N) return fail(sim, KWGB_ERR_ARG, "sensor index out of range");
        hs.n = n_idx;
    }
    sim->hsens.push_back(std::move(hs));
    if (sensor_id) *sensor_id = (int32_t)sim->hsens.size() - 1;
    return KWGB_OK;
}

extern "C" int kwgb_set_series_capacity(kwgb_sim* sim, int32_t sensor_id, int64_t n_t) {
    if (!sim) return KWGB_ERR_ARG;
    if (sim->frozen || sim->steps > 0) return fail(sim, KWGB_ERR_STATE, "series capacity must be set before stepping");
    if (sensor_id < 0 || sensor_id >= (int32_t)sim->hsens.size()) return fail(sim, KWGB_ERR_ARG, "bad sensor id");
    if (n_t <= 0 || n_t > INT32_MAX) return fail(sim, KWGB_ERR_ARG, "capacity must be in [1, 2^31)");
    HostSensor& h = sim->hsens[sensor_id];
    if (!(h.record & (KWGB_P_SERIES | KWGB_U_SERIES))) return fail(sim, KWGB_ERR_ARG, "sensor records no series");
    h.cap = n_t;
    return KWGB_OK;
}

// Stable sort of entries (member L, a linear index x + nx row) by L: a
// counting sort by row, then a stable sort by x inside each row (insertion
// sort for short rows, std::stable_sort for long unsorted ones).  The order
// is that of std::stable_sort by L; the cost is O(n + rows) when the entries
// of each row arrive in x order (masks built from boxes and planes).
template <typename T>
static void sort_by_index(std::vector<T>& v, int64_t nx, int64_t nrows) {
    if (v.size() < 2) return;
    std::vector<int64_t> begin(nrows + 1, 0);
    for (const T& e : v) begin[e.L / nx + 1]++;
    for (int64_t r = 0; r < nrows; ++r) begin[r + 1] += begin[r];
    std::vector<int64_t> cur(begin.begin(), begin.end() - 1);
    std::vector<T> out(v.size());
    for (const T& e : v) out[cur[e.L / nx]++] = e;
    auto lessL = [](const T& a, const T& b) { return a.L < b.L; };
    for (int64_t r = 0; r < nrows; ++r) {
        T* lo = out.data() + begin[r];
        T* hi = out.data() + begin[r + 1];
        if (hi - lo < 2 || std::is_sorted(lo, hi, lessL)) continue;
        if (hi - lo > 32) {
            std::stable_sort(lo, hi, lessL);
            continue;
        }
        for (T* p = lo + 1; p < hi; ++p) {
            const T e = *p;
            T* k = p;
            for (; k > lo && (k - 1)->L > e.L; --k) *k = *(k - 1);
            *k = e;
        }
    }
    v.swap(out);
}

// Row-CSR device lists of the sources of one kind (unique points per grid
// row, each with its contributions: signal offset, length and scale sc).
static int build_sources(kwgb_sim* sim, int mode, float sc, SourceC* out) {
    *out = SourceC{};
    const int64_t nx = sim->g.nx;
    const int64_t nrows = (int64_t)sim->g.ny * sim->g.nz;
    struct Contrib { int64_t L; int64_t off; int32_t nt; };
    std::vector<Contrib> cs;
    std::vector<float> sig;
    {
        size_t nc = 0, ns = 0;
        for (auto& s : sim->hsrc)
            if (s.mode == mode) {
                nc += s.idx.size();
                ns += s.sig.size();
            }
        cs.reserve(nc);
        sig.reserve(ns);
    }
    for (auto& s : sim->hsrc) {
        if (s.mode != mode) continue;
        const int64_t base = (int64_t)sig.size();
        sig.insert(sig.end(), s.sig.begin(), s.sig.end());
        for (size_t i = 0; i < s.idx.size(); ++i)
            cs.push_back({s.idx[i], base + (s.nsig == 1 ? 0 : (int64_t)i * s.nt), (int32_t)s.nt});
    }
    if (!cs.empty()) {
        sort_by_index(cs, nx, nrows);
        std::vector<int32_t> row_ptr(nrows + 1, 0), pt_x, pt_c;
        std::vector<int64_t> c_off;
        std::vector<int32_t> c_nt;
        std::vector<float> c_scale;
        for (size_t i = 0; i < cs.size(); ++i) {
            if (i == 0 || cs[i].L != cs[i - 1].L) {
                pt_x.push_back((int32_t)(cs[i].L % nx));
                pt_c.push_back((int32_t)c_off.size());
                row_ptr[cs[i].L / nx + 1]++;
            }
            c_off.push_back(cs[i].off);
            c_nt.push_back(cs[i].nt);
            c_scale.push_back(sc);
        }
        pt_c.push_back((int32_t)c_off.size());
        for (int64_t r = 0; r < nrows; ++r) row_ptr[r + 1] += row_ptr[r];
        int32_t *d_rp, *d_px, *d_pc, *d_cnt;
        int64_t* d_coff;
        float *d_cs, *d_sig;
        if (int e = upload(sim, &d_rp, row_ptr)) return e;
        if (int e = upload(sim, &d_px, pt_x)) return e;
        if (int e = upload(sim, &d_pc, pt_c)) return e;
        if (int e = upload(sim, &d_coff, c_off)) return e;
        if (int e = upload(sim, &d_cnt, c_nt)) return e;
        if (int e = upload(sim, &d_cs, c_scale)) return e;
        if (sig.empty()) sig.push_back(0.f);
        if (int e = upload(sim, &d_sig, sig)) return e;
        *out = SourceC{d_rp, d_px, d_pc, d_coff, d_cnt, d_cs, d_sig};
    }
    return KWGB_OK;
}

// Build the device source/sensor structures (once, at the first step).
static int freeze(kwgb_sim* sim) {
    if (sim->frozen) return KWGB_OK;
    const int64_t nx = sim->g.nx;
    const int64_t nrows = (int64_t)sim->g.ny * sim->g.nz;
    // ---- sources: per kind, contributions sorted by grid index, unique points per row
    // mass: dt M_xi = dt * 2 s / (3 c0 dx), the kernel divides by c0;
    // force along xi: dt F / rho0_sg, the kernel divides by rho0_sg
    if (int e = build_sources(sim, KWGB_ADDITIVE_MASS, (float)(sim->d.dt * 2.0 / (3.0 * sim->d.dx)), &sim->src)) return e;
    for (int a = 0; a < 3; ++a) {
        if (int e = build_sources(sim, KWGB_FORCE_X + a, (float)sim->d.dt, &sim->fsrc[a])) return e;
        sim->any_force |= sim->fsrc[a].row_ptr != nullptr;
    }
    // Dirichlet: the summed samples themselves
    if (int e = build_sources(sim, KWGB_DIRICHLET_P, 1.0f, &sim->dsrc)) return e;
    // ---- sensors
    SensorC& sc = sim->sens;
    sc = SensorC{};
    struct Entry { int64_t L; int32_t slot; };
    std::vector<Entry> es;
    std::vector<int64_t> ii;
    std::vector<int32_t> islot;
    int64_t slots = 0;
    {
        int64_t ne = 0, ni = 0;
        for (auto& h : sim->hsens)
            if (!h.full) {
                ne += h.n;
                ni += (h.record & KWGB_I_AVG) ? h.n : 0;
            }
        es.reserve(ne);
        ii.reserve(ni);
        islot.reserve(ni);
    }
    for (auto& h : sim->hsens) {
        if (h.full) {
            h.full_k = sc.nfull;
            DALLOC(sc.full_max[sc.nfull], float, sim->N);
            DALLOC(sc.full_p2[sc.nfull], double, sim->N);
            LK(launch_fill_f32(sc.full_max[sc.nfull], sim->N, -INFINITY, nullptr));
            CK(cudaMemset(sc.full_p2[sc.nfull], 0, sim->N * sizeof(double)));
            if (h.record & KWGB_P_MIN) {
                DALLOC(sc.full_min[sc.nfull], float, sim->N);
                LK(launch_fill_f32(sc.full_min[sc.nfull], sim->N, INFINITY, nullptr));
            }
            sc.nfull++;
            continue;
        }
        h.slot0 = slots;
        for (int64_t i = 0; i < h.n; ++i) es.push_back({h.idx[i], (int32_t)(slots + i)});
        if (h.record & KWGB_I_AVG) {
            h.i0 = (int64_t)ii.size();
            for (int64_t i = 0; i < h.n; ++i) { ii.push_back(h.idx[i]); islot.push_back((int32_t)(slots + i)); }
        }
        slots += h.n;
    }
    sim->n_slots = slots;
    if (!es.empty()) {
        sort_by_index(es, nx, nrows);
        std::vector<int32_t> row_ptr(nrows + 1, 0), ex(es.size()), eslot(es.size());
        for (size_t i = 0; i < es.size(); ++i) {
            row_ptr[es[i].L / nx + 1]++;
            ex[i] = (int32_t)(es[i].L % nx);
            eslot[i] = es[i].slot;
        }
        for (int64_t r = 0; r < nrows; ++r) row_ptr[r + 1] += row_ptr[r];
        int32_t *d_rp, *d_ex, *d_es;
        if (int e = upload(sim, &d_rp, row_ptr)) return e;
        if (int e = upload(sim, &d_ex, ex)) return e;
        if (int e = upload(sim, &d_es, eslot)) return e;
        sc.row_ptr = d_rp;
        sc.e_x = d_ex;
        sc.e_slot = d_es;
        DALLOC(sc.p_max, float, slots);
        DALLOC(sc.p2, double, slots);
        DALLOC(sc.p_sens, float, slots);
        LK(launch_fill_f32(sc.p_max, slots, -INFINITY, nullptr));
        CK(cudaMemset(sc.p2, 0, slots * sizeof(double)));
        CK(cudaMemset(sc.p_sens, 0, slots * sizeof(float)));
        // p_min and the series rings (time-varying outputs at the sensor mask, Sec. 3.4)
        bool any_min = false, any_pser = false;
        std::vector<SeriesSlot> ser;                     // built when a sensor records the p series
        std::vector<int64_t> uidx;
        std::vector<SeriesSlot> uq;
        int64_t ptot = 0, utot = 0;
        for (auto& h : sim->hsens) {
            if (h.full) continue;
            any_min |= (h.record & KWGB_P_MIN) != 0;
            if ((h.record & (KWGB_P_SERIES | KWGB_U_SERIES)) && h.cap <= 0)
                return fail(sim, KWGB_ERR_ARG, "a series sensor needs kwgb_set_series_capacity before stepping");
            if (h.record & KWGB_P_SERIES) {
                if (!any_pser) ser.assign(slots, SeriesSlot{-1, 0, 1});
                any_pser = true;
                h.pser0 = ptot;
                for (int64_t i = 0; i < h.n; ++i) ser[h.slot0 + i] = SeriesSlot{ptot + i, (int32_t)h.n, (int32_t)h.cap};
                ptot += h.cap * h.n;
            }
            if (h.record & KWGB_U_SERIES) {
                h.user0 = utot;
                for (int64_t i = 0; i < h.n; ++i) {
                    uidx.push_back(h.idx[i]);
                    uq.push_back(SeriesSlot{utot + i, (int32_t)h.n, (int32_t)h.cap});
                }
                utot += 3 * h.cap * h.n;
            }
        }
        if (any_min) {
            DALLOC(sc.p_min, float, slots);
            LK(launch_fill_f32(sc.p_min, slots, INFINITY, nullptr));
        }
        if (any_pser) {
            SeriesSlot* d_ser;
            if (int e = upload(sim, &d_ser, ser)) return e;
            sc.ser = d_ser;
            DALLOC(sc.series, float, ptot);
            CK(cudaMemset(sc.series, 0, ptot * sizeof(float)));
            sim->series_elems = ptot;
        }
        if (!uidx.empty()) {
            if (int e = upload(sim, &sim->u_idx, uidx)) return e;
            if (int e = upload(sim, &sim->u_q, uq)) return e;
            DALLOC(sim->useries, float, utot);
            CK(cudaMemset(sim->useries, 0, utot * sizeof(float)));
            sim->n_u = (int64_t)uidx.size();
            sim->useries_elems = utot;
        }
    }
    sim->n_i = (int64_t)ii.size();
    if (sim->n_i) {
        if (int e = upload(sim, &sim->i_idx, ii)) return e;
        if (int e = upload(sim, &sim->i_slot, islot)) return e;
        DALLOC(sim->I, double, 3 * sim->n_i);
        DALLOC(sim->I_tail, double, 3 * sim->n_i);
        DALLOC(sim->ubuf, float, 6 * sim->n_i);
        CK(cudaMemset(sim->I, 0, 3 * sim->n_i * sizeof(double)));
    }
    CK(cudaDeviceSynchronize());
    sim->frozen = true;
    return KWGB_OK;
}

// ------------------------------------------------------------------ stepping
extern "C" int kwgb_step(kwgb_sim* sim, int64_t n_steps, void* cuda_stream) {
    NvtxRange nvtx_("kwgb_step");
    if (!sim) return KWGB_ERR_ARG;
    if (n_steps < 0) return fail(sim, KWGB_ERR_ARG, "n_steps < 0");
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (n_steps == 0) return KWGB_OK;
    if (int e = freeze(sim)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sim->last_stream = s;
    for (int64_t i = 0; i < n_steps; ++i) {
        if (int e = run_step(sim, s)) return e;
        sim->steps++;
    }
    return KWGB_OK;
}

// ------------------------------------------------------------------ checkpoint / restart
namespace {
struct StateHeader {
    char magic[8];
    int64_t nx, ny, nz, nhp, n_slots, nfull, n_i, steps, bytes;
};
constexpr char kStateMagic[8] = {'K', 'W', 'G', 'B', 'S', 'T', '0', '1'};
}  // namespace

// The device blocks of a snapshot, in order.
static std::vector<std::pair<void*, size_t>> state_blocks(kwgb_sim* sim) {
    std::vector<std::pair<void*, size_t>> b;
    const size_t F = (size_t)sim->N * sizeof(float);
    for (int a = 0; a < 3; ++a) b.push_back({sim->u[a], F});
    for (int a = 0; a < 3; ++a) b.push_back({sim->rho[a], F});
    b.push_back({sim->P, sim->spec_elems * sizeof(float2)});
    const SensorC& sc = sim->sens;
    if (sim->n_slots) {
        b.push_back({sc.p_max, sim->n_slots * sizeof(float)});
        b.push_back({sc.p2, sim->n_slots * sizeof(double)});
        b.push_back({sc.p_sens, sim->n_slots * sizeof(float)});
        if (sc.p_min) b.push_back({sc.p_min, sim->n_slots * sizeof(float)});
    }
    for (int k = 0; k < sc.nfull; ++k) {
        b.push_back({sc.full_max[k], (size_t)sim->N * sizeof(float)});
        b.push_back({sc.full_p2[k], (size_t)sim->N * sizeof(double)});
        if (sc.full_min[k]) b.push_back({sc.full_min[k], (size_t)sim->N * sizeof(float)});
    }
    if (sim->n_i) b.push_back({sim->I, 3 * sim->n_i * sizeof(double)});
    if (sim->series_elems) b.push_back({sc.series, sim->series_elems * sizeof(float)});
    if (sim->useries_elems) b.push_back({sim->useries, sim->useries_elems * sizeof(float)});
    return b;
}

static int64_t state_size(kwgb_sim* sim) {
    int64_t n = sizeof(StateHeader);
    for (auto& b : state_blocks(sim)) n += (int64_t)b.second;
    return n;
}

static StateHeader state_header(kwgb_sim* sim) {
    StateHeader h;
    std::memcpy(h.magic, kStateMagic, 8);
    h.nx = sim->g.nx; h.ny = sim->g.ny; h.nz = sim->g.nz; h.nhp = sim->g.nhp;
    h.n_slots = sim->n_slots; h.nfull = sim->sens.nfull; h.n_i = sim->n_i;
    h.steps = sim->steps;
    h.bytes = state_size(sim);
    return h;
}

extern "C" int64_t kwgb_state_bytes(kwgb_sim* sim) {
    if (!sim || !sim->medium_set) return 0;
    if (freeze(sim)) return 0;
    return state_size(sim);
}

extern "C" int kwgb_save_state(kwgb_sim* sim, void* buf, int64_t len) {
    NvtxRange nvtx_("kwgb_save_state");
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (int e = freeze(sim)) return e;
    const StateHeader h = state_header(sim);
    if (!buf || len < h.bytes) return fail(sim, KWGB_ERR_ARG, "state buffer too small");
    CK(cudaDeviceSynchronize());
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (auto& b : state_blocks(sim)) {
        CK(cudaMemcpy(out + off, b.first, b.second, cudaMemcpyDeviceToHost));
        off += b.second;
    }
    return KWGB_OK;
}

extern "C" int kwgb_load_state(kwgb_sim* sim, const void* buf, int64_t len) {
    NvtxRange nvtx_("kwgb_load_state");
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (int e = freeze(sim)) return e;
    if (!buf || len < (int64_t)sizeof(StateHeader)) return fail(sim, KWGB_ERR_ARG, "not a snapshot");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const StateHeader mine = state_header(sim);
    if (std::memcmp(h.magic, kStateMagic, 8) != 0) return fail(sim, KWGB_ERR_ARG, "not a snapshot");
    if (h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz || h.nhp != mine.nhp || h.n_slots != mine.n_slots ||
        h.nfull != mine.nfull || h.n_i != mine.n_i || h.bytes != mine.bytes || len < h.bytes || h.steps < 0)
        return fail(sim, KWGB_ERR_ARG, "snapshot of a different grid or sensor layout");
    CK(cudaDeviceSynchronize());
    const char* in = static_cast<const char*>(buf);
    size_t off = sizeof(h);
    for (auto& b : state_blocks(sim)) {
        CK(cudaMemcpy(b.first, in + off, b.second, cudaMemcpyHostToDevice));
        off += b.second;
    }
    CK(cudaMemcpy(sim->d_step, &h.steps, sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemset(sim->d_flag, 0, sizeof(int)));
    sim->steps = h.steps;
    return KWGB_OK;
}

extern "C" int64_t kwgb_steps_done(const kwgb_sim* sim) { return sim ? sim->steps : 0; }

extern "C" int64_t kwgb_launch_count(const kwgb_sim* sim) { return sim ? sim->launches : 0; }

extern "C" const char* kwgb_kernel_name(int32_t kind) {
    return (kind >= 0 && kind < K_COUNT) ? kKernelNames[kind] : "";
}

extern "C" int kwgb_step_profiled(kwgb_sim* sim, void* cuda_stream, int32_t* kinds, float* ms,
                                  int32_t capacity, int32_t* n_launches) {
    if (!sim) return KWGB_ERR_ARG;
    if (!kinds || !ms || !n_launches || capacity <= 0) return fail(sim, KWGB_ERR_ARG, "null output");
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (int e = freeze(sim)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sim->last_stream = s;
    cudaEvent_t start;
    CK(cudaEventCreate(&start));
    CK(cudaEventRecord(start, s));
    sim->prof = true;
    sim->ev.clear();
    sim->ev_kind.clear();
    int rc = launch_step(sim, s);
    sim->prof = false;
    if (rc == KWGB_OK) {
        sim->steps++;
        cudaError_t e = cudaEventSynchronize(sim->ev.empty() ? start : sim->ev.back());
        if (e != cudaSuccess) rc = fail(sim, KWGB_ERR_CUDA, cudaGetErrorString(e));
    }
    int32_t n = 0;
    cudaEvent_t prev = start;
    for (size_t i = 0; i < sim->ev.size(); ++i) {
        if (rc == KWGB_OK && n < capacity) {
            float t = 0.f;
            cudaEventElapsedTime(&t, prev, sim->ev[i]);
            kinds[n] = sim->ev_kind[i];
            ms[n] = t;
            ++n;
        }
        prev = sim->ev[i];
    }
    for (cudaEvent_t e : sim->ev) cudaEventDestroy(e);
    cudaEventDestroy(start);
    sim->ev.clear();
    sim->ev_kind.clear();
    *n_launches = n;
    return rc;
}

static int sync_and_flag(kwgb_sim* sim) {
    CK(cudaStreamSynchronize(sim->last_stream));
    CK(cudaDeviceSynchronize());
    int flag = 0;
    if (sim->d_flag) CK(cudaMemcpy(&flag, sim->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 2) return fail(sim, KWGB_ERR_TIMEOUT, "a bounded device wait ran out (TMA tile load)");
    if (flag & 1) return fail(sim, KWGB_ERR_NONFINITE, "pressure became non-finite");
    return KWGB_OK;
}

extern "C" int kwgb_status(kwgb_sim* sim) {
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return KWGB_OK;
    return sync_and_flag(sim);
}

// ------------------------------------------------------------------ reading
extern "C" int kwgb_read(kwgb_sim* sim, int32_t sensor_id, uint32_t which, double* host_out, int64_t n) {
    NvtxRange nvtx_("kwgb_read");
    if (!sim) return KWGB_ERR_ARG;
    if (sensor_id < 0 || sensor_id >= (int32_t)sim->hsens.size()) return fail(sim, KWGB_ERR_ARG, "bad sensor id");
    if (!host_out) return fail(sim, KWGB_ERR_ARG, "null output");
    HostSensor& h = sim->hsens[sensor_id];
    if (!(which == KWGB_P_MAX || which == KWGB_P_RMS || which == KWGB_I_AVG || which == KWGB_P_MIN ||
          which == KWGB_P_SERIES || which == KWGB_U_SERIES))
        return fail(sim, KWGB_ERR_ARG, "which must be one of P_MAX, P_RMS, I_AVG, P_MIN, P_SERIES, U_SERIES");
    if (!(h.record & which)) return fail(sim, KWGB_ERR_ARG, "output not recorded by this sensor");
    const int64_t nt = sim->steps;
    const int64_t m = (nt == 0 || !sim->frozen) ? 0 : std::min<int64_t>(nt, h.cap);   // series samples kept
    const int64_t need = which == KWGB_I_AVG ? 3 * h.n
                       : which == KWGB_P_SERIES ? m * h.n
                       : which == KWGB_U_SERIES ? 3 * m * h.n : h.n;
    if (n < need) return fail(sim, KWGB_ERR_ARG, "output buffer too small");
    if (nt == 0 || !sim->frozen) {
        const double v = which == KWGB_P_MAX ? -INFINITY : (which == KWGB_P_MIN ? INFINITY : 0.0);
        for (int64_t i = 0; i < need; ++i) host_out[i] = v;
        return KWGB_OK;
    }
    int status = sync_and_flag(sim);
    if (status == KWGB_ERR_CUDA) return status;
    const SensorC& sc = sim->sens;
    if (which == KWGB_P_MAX || which == KWGB_P_MIN) {
        std::vector<float> t(h.n);
        const float* src = which == KWGB_P_MAX ? (h.full ? sc.full_max[h.full_k] : sc.p_max + h.slot0)
                                               : (h.full ? sc.full_min[h.full_k] : sc.p_min + h.slot0);
        CK(cudaMemcpy(t.data(), src, h.n * sizeof(float), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < h.n; ++i) host_out[i] = t[i];
    } else if (which == KWGB_P_SERIES || which == KWGB_U_SERIES) {
        // ring row of sample t is t mod cap; the last m samples, oldest first
        const int64_t w = which == KWGB_P_SERIES ? h.n : 3 * h.n;
        const float* src = which == KWGB_P_SERIES ? sc.series + h.pser0 : sim->useries + h.user0;
        std::vector<float> t((size_t)h.cap * w);
        CK(cudaMemcpy(t.data(), src, t.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < m; ++r) {
            const int64_t row = (nt - m + r) % h.cap;
            for (int64_t i = 0; i < w; ++i) host_out[r * w + i] = t[row * w + i];
        }
    } else if (which == KWGB_P_RMS) {
        const double* src = h.full ? sc.full_p2[h.full_k] : sc.p2 + h.slot0;
        CK(cudaMemcpy(host_out, src, h.n * sizeof(double), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < h.n; ++i) host_out[i] = std::sqrt(host_out[i] / (double)nt);
    } else {
        // tail term p^{Nt} (ubar^{Nt-1/2} + ubar^{Nt+1/2}) / 2 with u^{Nt+1/2} from one
        // velocity update that is not stored
        const GridC& g = sim->g;
        cudaStream_t s = nullptr;
        float2* out[3] = {sim->T3, sim->T1, sim->T2};
        float2* yi[1] = {sim->T3};
        float2* pin[1] = {sim->P};
        LK(ypass(sim, -1, pin, yi, 1, s));                  // out of place: P is kept
        float2* zin[3] = {sim->T3, nullptr, nullptr};
        LK(zop(sim, Z_GRAD_FWD, zin, out, s));
        LK(ypass(sim, +1, out, out, 3, s));
        XVelArgs va{};
        va.step = sim->d_step;
        for (int a = 0; a < 3; ++a) {
            va.f[a] = sim->fsrc[a];
            va.G[a] = out[a];
            va.u[a] = sim->u[a];
            va.tail[a] = reinterpret_cast<float*>(out[a]);
        }
        LK(launch_x_vel(g, sim->md, XV_TAIL, va, s));
        CK(cudaMemset(sim->I_tail, 0, 3 * sim->n_i * sizeof(double)));
        LK(launch_intensity_gather(sim->n_i, sim->i_idx, g, sim->u, g.nx, sim->ubuf, s));
        float* tails[3] = {reinterpret_cast<float*>(out[0]), reinterpret_cast<float*>(out[1]),
                           reinterpret_cast<float*>(out[2])};
        LK(launch_intensity_accum(sim->n_i, sim->i_idx, g, tails, 2 * g.nhp, sim->ubuf, sc.p_sens,
                                  sim->i_slot, sim->I_tail, sim->d_step, 0, s));
        CK(cudaDeviceSynchronize());
        std::vector<double> a(3 * sim->n_i), b(3 * sim->n_i);
        CK(cudaMemcpy(a.data(), sim->I, a.size() * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(b.data(), sim->I_tail, b.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int xi = 0; xi < 3; ++xi)
            for (int64_t i = 0; i < h.n; ++i) {
                const int64_t k = xi * sim->n_i + h.i0 + i;
                host_out[xi * h.n + i] = (a[k] + b[k]) / (double)nt;
            }
    }
    return status;
}

extern "C" int kwgb_read_field(kwgb_sim* sim, int field, float* host_out, int64_t n) {
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "no state yet");
    if (!host_out || n < sim->N) return fail(sim, KWGB_ERR_ARG, "output buffer too small");
    if (field < KWGB_FIELD_P || field > KWGB_FIELD_RHOZ) return fail(sim, KWGB_ERR_ARG, "bad field");
    int status = sync_and_flag(sim);
    if (status == KWGB_ERR_CUDA) return status;
    const GridC& g = sim->g;
    if (field == KWGB_FIELD_P) {
        float* real3 = reinterpret_cast<float*>(sim->T3);
        LK(launch_x_c2r(g, sim->P, real3, 2 * g.nhp, nullptr));
        CK(cudaDeviceSynchronize());
        // the C2R is unnormalised along x: divide by nx
        std::vector<float> rows((size_t)g.ny * g.nz * g.nx);
        CK(cudaMemcpy2D(rows.data(), g.nx * sizeof(float), real3, 2 * g.nhp * sizeof(float),
                        g.nx * sizeof(float), (size_t)g.ny * g.nz, cudaMemcpyDeviceToHost));
        const float inv = 1.0f / (float)g.nx;
        for (size_t i = 0; i < rows.size(); ++i) host_out[i] = rows[i] * inv;
    } else {
        const float* src = field <= KWGB_FIELD_UZ ? sim->u[field - 1] : sim->rho[field - 4];
        CK(cudaMemcpy(host_out, src, sim->N * sizeof(float), cudaMemcpyDeviceToHost));
    }
    return status;
}

extern "C" int kwgb_apply_operator(kwgb_sim* sim, int op, const float* in, float* out0,
                                   float* out1, float* out2, void* cuda_stream) {
    NvtxRange nvtx_("kwgb_apply_operator");
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (!in || !out0) return fail(sim, KWGB_ERR_ARG, "null field");
    const GridC& g = sim->g;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sim->last_stream = s;
    if (op == KWGB_OP_GRAD_FWD || op == KWGB_OP_GRAD_BWD) {
        if (!out1 || !out2) return fail(sim, KWGB_ERR_ARG, "gradient needs three outputs");
        LK(launch_x_r2c(g, in, g.nx, sim->T3, s));
        float2* outs[3] = {sim->T3, sim->T1, sim->T2};
        if (int e = grad_chain(sim, sim->T3, outs, op == KWGB_OP_GRAD_FWD ? Z_GRAD_FWD : Z_GRAD_BWD, s)) return e;
        float* r[3] = {out0, out1, out2};
        for (int a = 0; a < 3; ++a) LK(launch_x_c2r(g, outs[a], r[a], g.nx, s));
        return KWGB_OK;
    }
    if (op == KWGB_OP_ABS_TAU || op == KWGB_OP_ABS_ETA) {
        LK(launch_x_r2c(g, in, g.nx, sim->T3, s));
        float2* a1[1] = {sim->T3};
        LK(ypass(sim, -1, a1, a1, 1, s));
        float2* zin[3] = {nullptr, nullptr, nullptr};
        zin[op == KWGB_OP_ABS_TAU ? 0 : 1] = sim->T3;
        LK(zop(sim, Z_ABS, zin, zin, s));
        LK(ypass(sim, +1, a1, a1, 1, s));
        LK(launch_x_c2r(g, sim->T3, out0, g.nx, s));
        return KWGB_OK;
    }
    return fail(sim, KWGB_ERR_ARG, "unknown operator");
}


// ------------------------------------------------------------------ adjoint
static int copy_dev(kwgb_sim* sim, void* dst, const void* src, size_t bytes, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return KWGB_OK;
}

static size_t ck_bytes(kwgb_sim* sim) {
    return 6 * (size_t)sim->N * sizeof(float) + sim->spec_elems * sizeof(float2);
}

// state (u, rho_xi, P) <-> a checkpoint slot
static int save_ck(kwgb_sim* sim, char* dst, cudaStream_t s) {
    const size_t F = (size_t)sim->N * sizeof(float);
    for (int a = 0; a < 3; ++a) {
        if (int e = copy_dev(sim, dst + a * F, sim->u[a], F, s)) return e;
        if (int e = copy_dev(sim, dst + (3 + a) * F, sim->rho[a], F, s)) return e;
    }
    return copy_dev(sim, dst + 6 * F, sim->P, sim->spec_elems * sizeof(float2), s);
}

static int load_ck(kwgb_sim* sim, const char* src, int64_t step, cudaStream_t s) {
    const size_t F = (size_t)sim->N * sizeof(float);
    for (int a = 0; a < 3; ++a) {
        if (int e = copy_dev(sim, sim->u[a], src + a * F, F, s)) return e;
        if (int e = copy_dev(sim, sim->rho[a], src + (3 + a) * F, F, s)) return e;
    }
    if (int e = copy_dev(sim, sim->P, src + 6 * F, sim->spec_elems * sizeof(float2), s)) return e;
    CK(cudaMemcpyAsync(sim->d_step, &step, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));              // the host value of step goes out of scope
    return KWGB_OK;
}

extern "C" int kwgb_adjoint_forward(kwgb_sim* sim, const int64_t* obj_idx, int64_t n_obj, int objective,
                                    int64_t n_steps, int64_t checkpoint_every, double* J_out,
                                    void* cuda_stream) {
    NvtxRange nvtx_("kwgb_adjoint_forward");
    if (!sim) return KWGB_ERR_ARG;
    if (!sim->medium_set) return fail(sim, KWGB_ERR_STATE, "set the medium first");
    if (sim->steps != 0 || sim->frozen || sim->adjoint_done)
        return fail(sim, KWGB_ERR_STATE, "the adjoint needs a simulation that has not stepped");
    if (objective != KWGB_OBJ_MEAN_ABS_P) return fail(sim, KWGB_ERR_ARG, "unknown objective");
    if (checkpoint_every > 0)
        for (auto& h : sim->hsrc)
            if (h.mode != KWGB_ADDITIVE_MASS)
                return fail(sim, KWGB_ERR_UNSUPPORTED, "the adjoint differentiates additive mass sources only");
    if (!obj_idx || n_obj <= 0 || n_steps <= 0 || checkpoint_every < 0 || !J_out)
        return fail(sim, KWGB_ERR_ARG, "bad objective, step count or checkpoint interval");
    {
        std::vector<int64_t> u(obj_idx, obj_idx + n_obj);
        std::sort(u.begin(), u.end());
        for (size_t i = 0; i < u.size(); ++i)
            if (u[i] < 0 || u[i] >= sim->N || (i && u[i] == u[i - 1]))
                return fail(sim, KWGB_ERR_ARG, "objective indices must be unique and inside the grid");
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sim->last_stream = s;
    auto& A = sim->adj;
    const int64_t K = checkpoint_every;
    // the objective points become an internal p-series sensor of n_steps samples:
    // the step itself (its series kernel, inside the captured step) records
    // p^{n+1} at the points as sample n, laid out [n][point]
    int32_t osid = -1;
    if (int e = kwgb_add_sensor(sim, obj_idx, n_obj, KWGB_P_SERIES, &osid)) return e;
    if (int e = kwgb_set_series_capacity(sim, osid, n_steps)) return e;
    if (int e = freeze(sim)) return e;
    sim->adjoint_done = true;
    A.pobj = sim->sens.series + sim->hsens[osid].pser0;
    const size_t F = (size_t)sim->N * sizeof(float);
    A.keep_all = K >= n_steps;
    if (A.keep_all) {
        if (sim->gexec) {                      // a captured step without the kept fields
            cudaGraphExecDestroy(sim->gexec);
            sim->gexec = nullptr;
        }
        // every step's fields (7 N floats a step) instead of checkpoints: the
        // reverse pass recomputes nothing
        A.seg = static_cast<float*>(dalloc(sim, (size_t)n_steps * 7 * F));
        if (!A.seg)
            return fail(sim, KWGB_ERR_OOM, "keeping every step's fields for the adjoint (28 N bytes a step); "
                                           "give a checkpoint interval below the step count");
        sim->adj_keep = A.seg;
        sim->adj_period = n_steps;
    } else if (K > 0) {
        const int64_t nck = (n_steps + K - 1) / K;
        A.ck = static_cast<char*>(dalloc(sim, (size_t)nck * ck_bytes(sim)));
        A.fin = static_cast<char*>(dalloc(sim, ck_bytes(sim)));
        if (!A.ck || !A.fin) return fail(sim, KWGB_ERR_OOM, "adjoint checkpoints");
    }
    if (K > 0) {
        std::vector<int64_t> ov(obj_idx, obj_idx + n_obj);
        if (int e = upload(sim, &A.d_obj, ov)) return e;
    }
    // ---- forward run, a checkpoint every K steps (or every step's fields kept)
    auto stop_keeping = [&]() {               // later steps keep nothing: drop the step that writes the fields
        if (!A.keep_all) return;
        sim->adj_keep = nullptr;
        sim->adj_period = 0;
        if (sim->gexec) {
            cudaGraphExecDestroy(sim->gexec);
            sim->gexec = nullptr;
        }
    };
    for (int64_t n = 0; n < n_steps; ++n) {
        int e = KWGB_OK;
        if (K > 0 && !A.keep_all && n % K == 0) e = save_ck(sim, A.ck + (size_t)(n / K) * ck_bytes(sim), s);
        if (!e) e = run_step(sim, s);
        if (e) {
            stop_keeping();
            return e;
        }
        sim->steps++;
    }
    stop_keeping();
    if (K > 0 && !A.keep_all) {
        if (int e = save_ck(sim, A.fin, s)) return e;
        // sensor accumulators as the forward run left them (the recomputation steps again)
        const SensorC& sc_ = sim->sens;
        const size_t N = (size_t)sim->N;
        auto& sarr = A.sarr;
        sarr.clear();
        if (sim->n_slots) {
            sarr.push_back({sc_.p_max, sim->n_slots * sizeof(float)});
            sarr.push_back({sc_.p2, sim->n_slots * sizeof(double)});
            sarr.push_back({sc_.p_sens, sim->n_slots * sizeof(float)});
            if (sc_.p_min) sarr.push_back({sc_.p_min, sim->n_slots * sizeof(float)});
        }
        for (int k = 0; k < sc_.nfull; ++k) {
            sarr.push_back({sc_.full_max[k], N * sizeof(float)});
            sarr.push_back({sc_.full_p2[k], N * sizeof(double)});
            if (sc_.full_min[k]) sarr.push_back({sc_.full_min[k], N * sizeof(float)});
        }
        if (sim->n_i) sarr.push_back({sim->I, 3 * sim->n_i * sizeof(double)});
        if (sim->series_elems) sarr.push_back({sc_.series, sim->series_elems * sizeof(float)});
        if (sim->useries_elems) sarr.push_back({sim->useries, sim->useries_elems * sizeof(float)});
        size_t sbytes = 0;
        for (auto& q : sarr) sbytes += q.second;
        A.snap = static_cast<char*>(dalloc(sim, std::max<size_t>(sbytes, 16)));
        if (!A.snap) return fail(sim, KWGB_ERR_OOM, "sensor snapshot");
        size_t off = 0;
        for (auto& q : sarr) {
            if (int e = copy_dev(sim, A.snap + off, q.first, q.second, s)) return e;
            off += q.second;
        }
    }
    // ---- objective value (float64 on the host)
    std::vector<float> hp((size_t)n_steps * n_obj);
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(hp.data(), A.pobj, hp.size() * sizeof(float), cudaMemcpyDeviceToHost));
    A.w = 1.0 / ((double)n_obj * (double)n_steps);
    double J = 0.0;
    for (float v : hp) J += std::fabs((double)v);
    *J_out = J * A.w;
    A.n_steps = n_steps;
    A.K = K;
    A.n_obj = n_obj;
    A.pending = K > 0;
    return sync_and_flag(sim);
}

extern "C" int kwgb_adjoint_backward(kwgb_sim* sim, double* grad_out, int64_t grad_len, void* cuda_stream) {
    NvtxRange nvtx_("kwgb_adjoint_backward");
    if (!sim) return KWGB_ERR_ARG;
    auto& A = sim->adj;
    if (!A.pending)
        return fail(sim, KWGB_ERR_STATE, "kwgb_adjoint_backward needs kwgb_adjoint_forward with checkpoints first");
    int64_t rows = 0, need = 0, max_nt = 1;
    for (auto& h : sim->hsrc) {
        rows += h.nsig;
        need += h.nsig * h.nt;
        max_nt = std::max(max_nt, h.nt);
    }
    if (grad_len < need || (need > 0 && !grad_out)) return fail(sim, KWGB_ERR_ARG, "gradient buffer too small");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sim->last_stream = s;
    const size_t N = (size_t)sim->N;
    const size_t F = N * sizeof(float);
    const int64_t n_steps = A.n_steps, K = A.K, n_obj = A.n_obj;
    const bool keep_all = A.keep_all;
    // steps per segment: a checkpoint interval, or (every step kept) a graph's worth of reverse steps
    const int64_t L = keep_all ? std::min<int64_t>(n_steps, 64) : K;
    const int64_t nseg = (n_steps + L - 1) / L;
    // kept fields, per step: rho_xi^n, d_xi, rho^{n+1} (of every step, or of one
    // segment's steps, recomputed); adjoint fields
    float* seg = keep_all ? A.seg : static_cast<float*>(dalloc(sim, (size_t)std::min(K, n_steps) * 7 * F));
    float* lam = static_cast<float*>(dalloc(sim, 8 * F));
    double* grad = static_cast<double*>(dalloc(sim, (size_t)std::max<int64_t>(rows, 1) * max_nt * sizeof(double)));
    if (!seg || !lam || !grad) return fail(sim, KWGB_ERR_OOM, "adjoint buffers");
    // per signal row: its points and the source scale dt 2 / (3 dx) (the kernel divides by c0)
    std::vector<int32_t> rptr(1, 0), rnt;
    std::vector<int64_t> rpts;
    std::vector<float> rscale;
    const float sc = (float)(sim->d.dt * 2.0 / (3.0 * sim->d.dx));
    for (auto& h : sim->hsrc)
        for (int64_t r = 0; r < h.nsig; ++r) {
            if (h.nsig == 1) {
                for (int64_t v : h.idx) { rpts.push_back(v); rscale.push_back(sc); }
            } else {
                rpts.push_back(h.idx[r]);
                rscale.push_back(sc);
            }
            rptr.push_back((int32_t)rpts.size());
            rnt.push_back((int32_t)h.nt);
        }
    int32_t *d_rptr = nullptr, *d_rnt = nullptr;
    int64_t* d_rpts = nullptr;
    float* d_rscale = nullptr;
    if (rows > 0) {
        if (int e = upload(sim, &d_rptr, rptr)) return e;
        if (int e = upload(sim, &d_rnt, rnt)) return e;
        if (int e = upload(sim, &d_rpts, rpts)) return e;
        if (int e = upload(sim, &d_rscale, rscale)) return e;
    }
    int64_t* d_rev = static_cast<int64_t*>(dalloc(sim, sizeof(int64_t)));
    if (!d_rev) return fail(sim, KWGB_ERR_OOM, "adjoint step counter");
    CK(cudaMemsetAsync(lam, 0, 8 * F, s));
    CK(cudaMemsetAsync(grad, 0, (size_t)std::max<int64_t>(rows, 1) * max_nt * sizeof(double), s));
    const GridC& g = sim->g;
    const bool absorbing = sim->md.absorbing != 0;
    AdjX ax{};
    ax.keep = seg;
    ax.keep_period = keep_all ? n_steps : K;
    ax.lam_p = lam;
    for (int a = 0; a < 3; ++a) {
        ax.lam_u[a] = lam + (1 + a) * N;
        ax.lam_rho[a] = lam + (4 + a) * N;
    }
    ax.lam_src = lam + 7 * N;
    ax.nrev = d_rev;
    float2* sp[3] = {sim->T1, sim->T2, sim->T3};
    for (int a = 0; a < 3; ++a) ax.sp[a] = sp[a];
    float2* ab[3] = {sim->T1, sim->T2, nullptr};
    // One segment of len steps (device reverse counter at its last step): with
    // checkpoints, recompute it from its loaded checkpoint (device step counter
    // at its first step), x_dens keeping every step's fields; then step it
    // backwards.  The kernels index the kept fields by the device counters, so
    // a full segment can be captured once and replayed for the others.
    auto segment = [&](cudaStream_t st, int64_t len) -> int {
        if (!keep_all) {
            sim->adj_keep = seg;
            sim->adj_period = K;
            int e = KWGB_OK;
            for (int64_t k = 0; k < len && !e; ++k) e = launch_step(sim, st);
            sim->adj_keep = nullptr;
            sim->adj_period = 0;
            if (e) return e;
        }
        cudaStream_t s = st;                                                  // for LK
        for (int64_t k = len - 1; k >= 0; --k) {
            LK(launch_adj_obj(n_obj, A.d_obj, A.pobj, d_rev, A.w, ax.lam_p, s));
            if (absorbing) {                                                  // Eq. 8 backwards
                LK(launch_adj_x_absprep(g, sim->md, ax, s));
                LK(ypass(sim, -1, ab, ab, 2, s));
                LK(zop(sim, Z_ABS, ab, ab, s));
                LK(ypass(sim, +1, ab, ab, 2, s));
            }
            LK(launch_adj_x_dens(g, sim->md, ax, s));                        // Eqs. 6, 4d backwards
            LK(launch_adj_src((int)rows, d_rptr, d_rpts, d_rscale, d_rnt, ax.lam_src, sim->md, grad, max_nt, d_rev, s));
            LK(ypass(sim, -1, sp, sp, 3, s));                                 // transpose of Eq. 4c
            LK(zop(sim, Z_DIV_FWD, sp, sp, s));
            LK(ypass(sim, +1, sp, sp, 3, s));
            LK(launch_adj_x_vel(g, sim->md, ax, s));                         // Eq. 4b backwards
            LK(ypass(sim, -1, sp, sp, 3, s));                                 // transpose of Eq. 4a:
            LK(zop(sim, Z_DIV_SUM, sp, sp, s));                               // the three terms summed
            LK(ypass(sim, +1, sp, sp, 1, s));                                 // into sp[0]
            LK(launch_adj_x_p(g, sim->md, ax, s));                           // (steps d_rev back)
        }
        return KWGB_OK;
    };
    cudaGraphExec_t seg_exec = nullptr;
    bool direct_done = false;                  // a full segment has run directly (one-time set-up done)
    int64_t seg_launches = 0;
    for (int64_t c = nseg - 1; c >= 0; --c) {
        const int64_t n0 = c * L, n1 = std::min(n0 + L, n_steps);
        if (!keep_all)
            if (int e = load_ck(sim, A.ck + (size_t)c * ck_bytes(sim), n0, s)) return e;
        const int64_t nr = n1 - 1;
        CK(cudaMemcpyAsync(d_rev, &nr, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));          // the host value nr goes out of scope
        if (n1 - n0 == L && direct_done && !seg_exec && sim->cap) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(sim->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int64_t l0 = sim->launches;
                const std::string err = sim->err;
                const int e = segment(sim->cap, L);
                const cudaError_t ce = cudaStreamEndCapture(sim->cap, &graph);
                seg_launches = sim->launches - l0;
                sim->launches = l0;
                sim->err = err;
                if (e != KWGB_OK || ce != cudaSuccess || !graph ||
                    cudaGraphInstantiate(&seg_exec, graph, 0) != cudaSuccess)
                    seg_exec = nullptr;
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();
        }
        if (n1 - n0 == L && seg_exec) {
            CK(cudaGraphLaunch(seg_exec, s));
            sim->launches += seg_launches;
        } else {
            if (int e = segment(s, n1 - n0)) return e;
            if (n1 - n0 == L) direct_done = true;
        }
    }
    if (seg_exec) cudaGraphExecDestroy(seg_exec);
    // ---- put back the forward end state and the sensors (the recomputation stepped them)
    if (!keep_all) {
        if (int e = load_ck(sim, A.fin, n_steps, s)) return e;
        size_t off = 0;
        for (auto& q : A.sarr) {
            if (int e = copy_dev(sim, q.first, A.snap + off, q.second, s)) return e;
            off += q.second;
        }
    }
    std::vector<double> hg((size_t)std::max<int64_t>(rows, 1) * max_nt);
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(hg.data(), grad, hg.size() * sizeof(double), cudaMemcpyDeviceToHost));
    int64_t o = 0, r = 0;
    for (auto& h : sim->hsrc)
        for (int64_t q = 0; q < h.nsig; ++q, ++r)
            for (int64_t n = 0; n < h.nt; ++n) grad_out[o++] = hg[(size_t)r * max_nt + n];
    A.pending = false;
    return sync_and_flag(sim);
}

extern "C" int kwgb_adjoint(kwgb_sim* sim, const int64_t* obj_idx, int64_t n_obj, int objective,
                            int64_t n_steps, int64_t checkpoint_every, double* J_out, double* grad_out,
                            int64_t grad_len, void* cuda_stream) {
    NvtxRange nvtx_("kwgb_adjoint");
    if (!sim) return KWGB_ERR_ARG;
    if (checkpoint_every <= 0) return fail(sim, KWGB_ERR_ARG, "bad objective, step count or checkpoint interval");
    int64_t need = 0;
    for (auto& h : sim->hsrc) need += h.nsig * h.nt;
    if (grad_len < need || (need > 0 && !grad_out)) return fail(sim, KWGB_ERR_ARG, "gradient buffer too small");
    if (int e = kwgb_adjoint_forward(sim, obj_idx, n_obj, objective, n_steps, checkpoint_every, J_out, cuda_stream))
        return e;
    return kwgb_adjoint_backward(sim, grad_out, grad_len, cuda_stream);
}

extern "C" int kwgb_debug_wait_fault(kwgb_sim* sim, int on) {
    if (!sim) return KWGB_ERR_ARG;
    sim->g.wait_fault_tx = on ? 16u : 0u;
    if (sim->gexec) {                          // the captured step holds the old parameters
        cudaGraphExecDestroy(sim->gexec);
        sim->gexec = nullptr;
    }
    sim->graph_off = false;
    return KWGB_OK;
}

extern "C" int64_t kwgb_device_bytes(const kwgb_sim* sim) { return sim ? sim->bytes : 0; }

extern "C" const char* kwgb_last_error(const kwgb_sim* sim) {
    return sim ? sim->err.c_str() : g_create_error.c_str();
}

extern "C" void kwgb_destroy(kwgb_sim* sim) {
    if (!sim) return;
    if (sim->medium_set) cudaDeviceSynchronize();
    if (sim->gexec) cudaGraphExecDestroy(sim->gexec);
    if (sim->cap) cudaStreamDestroy(sim->cap);
    for (void* p : sim->allocs) {
        if (sim->freef) sim->freef(p, sim->actx);
        else cudaFree(p);
    }
    delete sim;
}
