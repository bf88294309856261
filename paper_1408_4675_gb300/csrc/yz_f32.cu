// Instantiations of the strided-axis passes: float32 register passes.  The y
// and z passes of 256- to 1024-point lines use the two-columns-per-thread
// kernel (z_pair.cuh); shorter lines, and the y and absorption passes of
// 1024-point lines, the one-column form of yz_kernel.
#include "z_pair.cuh"

namespace kwgb {

template <int L, int OP>
static cudaError_t launch_f32(const YZK& a, int items, cudaStream_t s) {
    // (1024-point y passes and absorption pass: the one-column form measured faster;
    // the summing divergence pass of the adjoint exists in the one-column form only)
    if constexpr (L >= 8 && !(L == 10 && (OP == OP_Z_ABS || OP < 2)) && OP != OP_Z_DIV_SUM)
        return launch_pair<L, OP>(a, items, s);
    else return launch_t<L, OP, 0>(a, items, s);
}

template <int OP>
static cudaError_t by_size(const YZK& a, int logn, int items, cudaStream_t s) {
    switch (logn) {
#define CASE(L) case L: return launch_f32<L, OP>(a, items, s);
        KWGB_LOG_CASES(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t yz_dispatch_f32(const YZK& a, int op, int logn, int items, cudaStream_t s) {
    switch (op) {
        case OP_Y_FWD: return by_size<OP_Y_FWD>(a, logn, items, s);
        case OP_Y_INV: return by_size<OP_Y_INV>(a, logn, items, s);
        case OP_Z_GRAD_FWD: return by_size<OP_Z_GRAD_FWD>(a, logn, items, s);
        case OP_Z_GRAD_BWD: return by_size<OP_Z_GRAD_BWD>(a, logn, items, s);
        case OP_Z_DIV: return by_size<OP_Z_DIV>(a, logn, items, s);
        case OP_Z_ABS: return by_size<OP_Z_ABS>(a, logn, items, s);
        case OP_Z_DIV_FWD: return by_size<OP_Z_DIV_FWD>(a, logn, items, s);
        case OP_Z_DIV_SUM: return by_size<OP_Z_DIV_SUM>(a, logn, items, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kwgb
