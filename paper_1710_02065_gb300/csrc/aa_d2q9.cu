// aa_d2q9.cu -- instantiations of the in-place AA stream + collide kernels
// for D2Q9 (one translation unit per lattice so the library builds in parallel).
#include "step.cuh"
#include "dispatch.h"

namespace rr {

cudaError_t step_aa_d2q9(int precision, const StepParams &p, void *f, int block, bool loc, cudaStream_t st)
{
    switch (precision) {
    case PREC_FP64: return launch_stream_collide_aa<D2Q9, double, double>(p, f, block, loc, st);
    case PREC_FP32: return launch_stream_collide_aa<D2Q9, float, float>(p, f, block, loc, st);
    case PREC_FP16: return launch_stream_collide_aa<D2Q9, __half, float>(p, f, block, loc, st);
    case PREC_BF16: return launch_stream_collide_aa<D2Q9, __nv_bfloat16, float>(p, f, block, loc, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t aa_unswap_d2q9(int precision, const StepParams &p, void *f, cudaStream_t st)
{
    switch (precision) {
    case PREC_FP64: return launch_aa_unswap<D2Q9, double>(p, f, st);
    case PREC_FP32: return launch_aa_unswap<D2Q9, float>(p, f, st);
    case PREC_FP16: return launch_aa_unswap<D2Q9, __half>(p, f, st);
    case PREC_BF16: return launch_aa_unswap<D2Q9, __nv_bfloat16>(p, f, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rr
