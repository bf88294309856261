// Instantiations of the strided-axis passes: float16-split tensor-core stages.
#include "yz_kernel.cuh"

namespace kwgb {

template <int OP>
static cudaError_t by_size(const YZK& a, int logn, int items, cudaStream_t s) {
    switch (logn) {
#define CASE(L) case L: return launch_t<L, OP, 2>(a, items, s);
        KWGB_LOG_CASES_TC(CASE)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t yz_dispatch_f16(const YZK& a, int op, int logn, int items, cudaStream_t s) {
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
