// Host side of the strided-axis passes: tensor-map encoding and launch
// dispatch (the kernels are in yz_kernel.cuh, instantiated per precision form
// in yz_f32.cu, yz_bf16.cu and yz_f16.cu).
#include "yz_kernel.cuh"

namespace kwgb {

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <int LOGN, bool ISY, int MIXED>
static int encode_box(const GridC& g, float2* ptr, CUtensorMap* map) {
    using Sh = TShape<LOGN, ISY, MIXED>;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return -1;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nh, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nhp * 8, (cuuint64_t)g.ny * g.nhp * 8};
    const cuuint32_t box[3] = {(cuuint32_t)Sh::CX, ISY ? (cuuint32_t)Sh::BOX : 1u, ISY ? 1u : (cuuint32_t)Sh::BOX};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, ptr, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}


int make_spec_maps(const GridC& g, float2* ptr, SpecBuf* out) {
    out->p = ptr;
    int e = -3;
    switch (g.logny) {
#define CASE(L) case L: e = g.mixed ? encode_box<L, true, 1>(g, ptr, &out->ymap) : encode_box<L, true, 0>(g, ptr, &out->ymap); break;
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    if (e) return e;
    switch (g.lognz) {
#define CASE(L) case L: e = g.mixed ? encode_box<L, false, 1>(g, ptr, &out->zmap) : encode_box<L, false, 0>(g, ptr, &out->zmap); break;
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    return e;
}

static cudaError_t launch_op(int op, const YZK& a, int logn, int items, cudaStream_t s) {
    if (a.g.mixed == 2) return yz_dispatch_f16(a, op, logn, items, s);
    if (a.g.mixed == 1) return yz_dispatch_bf16(a, op, logn, items, s);
    return yz_dispatch_f32(a, op, logn, items, s);
}

static int chunk_count(int nh, int cx) { return (nh + cx - 1) / cx; }

// tile width of the pass (the tensor-core forms share one shape)
template <bool ISY>
static int cx_of(int logn, int mixed) {
    switch (logn) {
#define CASE(L) case L: return mixed ? TShape<L, ISY, 1>::CX : TShape<L, ISY, 0>::CX;
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    return 16;
}

cudaError_t launch_y_pass(const GridC& g, int dir, const SpecBuf* const* in, float2* const* out,
                          int ncomp, int* flag, cudaStream_t s) {
    YZK a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    for (int i = 0; i < ncomp; ++i) {
        a.map[i] = in[i]->ymap;
        a.out[i] = out[i];
    }
    a.ncomp = ncomp;
    a.nloads = 1;
    a.flag = flag;
    const int items = chunk_count(g.nh, cx_of<true>(g.logny, g.mixed)) * g.nz * ncomp;
    return launch_op(dir < 0 ? OP_Y_FWD : OP_Y_INV, a, g.logny, items, s);
}

cudaError_t launch_z_op(const GridC& g, int kind, const SpecBuf* const* in, float2* const* out, int* flag,
                        cudaStream_t s) {
    YZK a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.flag = flag;
    for (int i = 0; i < 3; ++i) a.out[i] = out[i];
    if (kind == Z_GRAD_FWD || kind == Z_GRAD_BWD) {
        a.map[0] = in[0]->zmap;
        a.nloads = 1;
        a.load_comp[0] = 0;
    } else if (kind == Z_DIV || kind == Z_DIV_FWD || kind == Z_DIV_SUM) {
        for (int i = 0; i < 3; ++i) {
            a.map[i] = in[i]->zmap;
            a.load_comp[i] = i;
        }
        a.nloads = 3;
    } else {
        int n = 0;
        for (int t = 0; t < 2; ++t)
            if (in[t]) {
                a.map[t] = in[t]->zmap;
                a.load_comp[n++] = t;
            }
        a.nloads = n;
        if (n == 0) return cudaSuccess;
    }
    const int items = chunk_count(g.nh, cx_of<false>(g.lognz, g.mixed)) * g.ny;
    switch (kind) {
        case Z_GRAD_FWD: return launch_op(OP_Z_GRAD_FWD, a, g.lognz, items, s);
        case Z_GRAD_BWD: return launch_op(OP_Z_GRAD_BWD, a, g.lognz, items, s);
        case Z_DIV: return launch_op(OP_Z_DIV, a, g.lognz, items, s);
        case Z_DIV_FWD: return launch_op(OP_Z_DIV_FWD, a, g.lognz, items, s);
        case Z_DIV_SUM: return launch_op(OP_Z_DIV_SUM, a, g.lognz, items, s);
        case Z_ABS: return launch_op(OP_Z_ABS, a, g.lognz, items, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kwgb
