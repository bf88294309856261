// Allocation-free staggered spectral gradient (kwgb_gradient_static).
//
// Some callers cannot allocate device memory when they need this operation:
// code whose device memory is owned entirely by another allocator (a
// framework's memory pool, or a fixed arena sized once at start-up), and
// code paths that must not allocate after initialisation, because cudaMalloc
// can synchronise the device and can fail once memory has been committed
// elsewhere.  This entry point therefore takes its scratch space from one
// file-scope __device__ array instead of allocating: about 4.7 MB, enough for
// grids up to 64 x 64 x 64, which every GPU that loads the library's device
// code holds until the process exits.  With CUDA's lazy module loading that
// code (and the array) is loaded on the first call on each device, so that
// first call should be made at start-up.
//
// The operation is the same chain kwgb_apply_operator runs for
// KWGB_OP_GRAD_FWD / KWGB_OP_GRAD_BWD (x R2C, y FFT, z FFT + operator + z
// inverse, y inverse, x C2R) through the same kernels; only the scratch
// spectra and the small tables live in the static array.  The twiddle table
// is uploaded once per device at set-up; the per-grid wavenumber and shift
// tables are computed on the device in float64 by a small kernel, so a call
// after the first enqueues kernels and one memset and copies nothing from
// the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/kwgb.h"
#include "kwgb_internal.h"

using namespace kwgb;

namespace {

constexpr int kMaxN = 64;                                          // largest nx, ny, nz
constexpr int kMaxNhp = ((kMaxN / 2 + 1) + 15) / 16 * 16;          // padded spectrum pitch
constexpr size_t kSpec = (size_t)kMaxNhp * kMaxN * kMaxN;          // complex per spectrum
// layout of the scratch array, in float2 units (every block 256-byte aligned)
constexpr size_t kOffSpec = 0;                                     // 3 spectra
constexpr size_t kOffTw = 3 * kSpec;                               // TW_TOTAL twiddles
constexpr size_t kOffK = kOffTw + (TW_TOTAL + 31) / 32 * 32;       // kx, ky, kz (float)
constexpr size_t kOffDf = kOffK + 128;                             // dfx, dfy, dfz (kx.. take 256 floats)
constexpr size_t kOffFlag = kOffDf + 256;                          // device status word
constexpr size_t kTotal = kOffFlag + 32;
constexpr int kMaxDevices = 64;
constexpr double kPi = 3.14159265358979323846;

// Copy msg into the caller's optional error buffer and return code.
int report(char* buf, size_t len, int code, const char* msg) {
    if (buf && len > 0) {
        std::strncpy(buf, msg, len - 1);
        buf[len - 1] = 0;
    }
    return code;
}

std::mutex g_setup_mu;
float2* g_base[kMaxDevices];     // device address of the scratch array, per device
int g_sms[kMaxDevices];
bool g_wait_fault = false;       // test hook: tile loads expect 16 bytes more than they receive

}  // namespace

// The scratch: three spectra plus the tables of the chain.  Host code must not
// pass this symbol to a kernel (on the host it only stands in for the device
// array); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_static_scratch[kTotal];

// Once per device, with that device current: look up the scratch array's
// device address and the SM count, and upload the (grid-independent) twiddle
// table.  Synchronises the device once.
static int static_setup(int dev, float2** base, int* sms, char* err, size_t errlen) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_base[dev] == nullptr) {
        float2* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return report(err, errlen, KWGB_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return report(err, errlen, KWGB_ERR_CUDA, "cudaDeviceGetAttribute failed");
        static float2 tw[TW_TOTAL];               // the same on every device
        static bool filled = false;
        if (!filled) fill_twiddle_table(tw);
        filled = true;
        e = cudaMemcpy(p + kOffTw, tw, sizeof(tw), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return report(err, errlen, KWGB_ERR_CUDA, "uploading the twiddle table into the static scratch failed");
        }
        g_sms[dev] = n;
        g_base[dev] = p;
    }
    *base = g_base[dev];
    *sms = g_sms[dev];
    return KWGB_OK;
}

// Per-grid tables, computed in float64 on the device: for each axis a the
// wavenumbers k_j (FFT storage order, the Nyquist bin at -n/2) and the shift
// operator i k exp(+i k d / 2) of the staggered gradient, stored as float.
// One block; thread j serves entry j of every axis.
struct StaticTableArgs {
    int len[3];       // entries per axis: nx/2 + 1, ny, nz
    int n[3];
    double d[3];
    float* k[3];
    float2* df[3];
};

__global__ void static_tables_kernel(StaticTableArgs a) {
    const int j = threadIdx.x;
    for (int ax = 0; ax < 3; ++ax) {
        if (j >= a.len[ax]) continue;
        const int m = j < a.n[ax] / 2 ? j : j - a.n[ax];
        const double k = (double)m * 2.0 * kPi / (a.d[ax] * (double)a.n[ax]);
        double sn, cs;
        sincos(k * a.d[ax] / 2.0, &sn, &cs);
        a.k[ax][j] = (float)k;
        a.df[ax][j] = make_float2((float)(-k * sn), (float)(k * cs));
    }
}

static int ilog2_static(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

extern "C" int kwgb_gradient_static(const kwgb_grid_desc* desc, int op, const float* in,
                                    float* out_x, float* out_y, float* out_z, void* cuda_stream,
                                    char* err, size_t errlen) {
    report(err, errlen, KWGB_OK, "");
    if (!desc || !in || !out_x || !out_y || !out_z) return report(err, errlen, KWGB_ERR_ARG, "null argument");
    if (op != KWGB_OP_GRAD_FWD && op != KWGB_OP_GRAD_BWD)
        return report(err, errlen, KWGB_ERR_ARG, "op must be KWGB_OP_GRAD_FWD or KWGB_OP_GRAD_BWD");
    const int64_t n[3] = {desc->nx, desc->ny, desc->nz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 8 || n[a] > kMaxN || (n[a] & (n[a] - 1)))
            return report(err, errlen, KWGB_ERR_UNSUPPORTED,
                               "kwgb_gradient_static serves nx, ny, nz powers of two in [8, 64] only");
    }
    const double dd[3] = {desc->dx, desc->dy, desc->dz};
    for (int a = 0; a < 3; ++a)
        if (!(dd[a] > 0) || !std::isfinite(dd[a])) return report(err, errlen, KWGB_ERR_ARG, "spacing must be positive");
    if (!(desc->dt > 0) || !(desc->c_ref > 0) || !std::isfinite(desc->dt) || !std::isfinite(desc->c_ref))
        return report(err, errlen, KWGB_ERR_ARG, "dt and c_ref must be positive and finite");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(err, errlen, KWGB_ERR_CUDA, "no usable current device");
    float2* base = nullptr;
    int sms = 0;
    if (int e = static_setup(dev, &base, &sms, err, errlen)) return e;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    GridC g;
    std::memset(&g, 0, sizeof(g));
    g.nx = (int)n[0]; g.ny = (int)n[1]; g.nz = (int)n[2];
    g.nh = g.nx / 2 + 1;
    g.nhp = (g.nh + 15) / 16 * 16;
    g.lognx = ilog2_static(g.nx); g.logny = ilog2_static(g.ny); g.lognz = ilog2_static(g.nz);
    g.dt = (float)desc->dt;
    g.scale = (float)(1.0 / ((double)g.nx * g.ny * g.nz));
    g.hk = (float)(desc->c_ref * desc->dt / 2.0);
    g.hk2 = (float)((desc->c_ref * desc->dt / 2.0) * (desc->c_ref * desc->dt / 2.0));
    g.num_sms = sms;

    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        g.wait_fault_tx = g_wait_fault ? 16u : 0u;
    }

    // per-grid tables on the device, the status word cleared
    float* kbase = reinterpret_cast<float*>(base + kOffK);
    const int koff[3] = {0, kMaxN / 2 + 1, kMaxN / 2 + 1 + kMaxN};
    const int doff[3] = {0, 64, 128};
    StaticTableArgs ta;
    const int klen[3] = {g.nh, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        ta.len[a] = klen[a];
        ta.n[a] = (int)n[a];
        ta.d[a] = dd[a];
        ta.k[a] = kbase + koff[a];
        ta.df[a] = base + kOffDf + doff[a];
    }
    static_tables_kernel<<<1, kMaxN, 0, s>>>(ta);
    if (cudaGetLastError() != cudaSuccess || cudaMemsetAsync(base + kOffFlag, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return report(err, errlen, KWGB_ERR_CUDA, "preparing the tables in the static scratch failed");
    }
    g.t.tw = base + kOffTw;
    g.t.kx = kbase + koff[0];
    g.t.ky = kbase + koff[1];
    g.t.kz = kbase + koff[2];
    g.t.dfx = base + kOffDf + doff[0];
    g.t.dfy = base + kOffDf + doff[1];
    g.t.dfz = base + kOffDf + doff[2];
    int* flag = reinterpret_cast<int*>(base + kOffFlag);

    // the three scratch spectra, with the tensor maps of their y and z tiles
    SpecBuf sb[3];
    for (int i = 0; i < 3; ++i)
        if (make_spec_maps(g, base + kOffSpec + i * kSpec, &sb[i]) != 0)
            return report(err, errlen, KWGB_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    float2* sp[3] = {sb[0].p, sb[1].p, sb[2].p};
    const SpecBuf* in0[3] = {&sb[0], nullptr, nullptr};
    const SpecBuf* all[3] = {&sb[0], &sb[1], &sb[2]};
    float* outs[3] = {out_x, out_y, out_z};
    cudaError_t e = launch_x_r2c(g, in, g.nx, sp[0], s);
    if (e == cudaSuccess) e = launch_y_pass(g, -1, in0, sp, 1, flag, s);
    if (e == cudaSuccess) e = launch_z_op(g, op == KWGB_OP_GRAD_FWD ? Z_GRAD_FWD : Z_GRAD_BWD, in0, sp, flag, s);
    if (e == cudaSuccess) e = launch_y_pass(g, +1, all, sp, 3, flag, s);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = launch_x_c2r(g, sp[a], outs[a], g.nx, s);
    if (e != cudaSuccess) return report(err, errlen, KWGB_ERR_CUDA, cudaGetErrorString(e));
    return KWGB_OK;
}

extern "C" int kwgb_gradient_static_status(void* cuda_stream, char* err, size_t errlen) {
    report(err, errlen, KWGB_OK, "");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(err, errlen, KWGB_ERR_CUDA, "no usable current device");
    float2* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        base = g_base[dev];
    }
    if (base == nullptr)
        return report(err, errlen, KWGB_ERR_STATE, "no kwgb_gradient_static call on this device yet");
    int flag = 0;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e == cudaSuccess) e = cudaMemcpy(&flag, base + kOffFlag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return report(err, errlen, KWGB_ERR_CUDA, cudaGetErrorString(e));
    if (flag & 2) return report(err, errlen, KWGB_ERR_TIMEOUT, "a bounded device wait ran out (TMA tile load)");
    if (flag & 1) return report(err, errlen, KWGB_ERR_NONFINITE, "non-finite value");
    return KWGB_OK;
}

extern "C" int kwgb_gradient_static_debug_wait_fault(int on) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    g_wait_fault = on != 0;
    return KWGB_OK;
}
