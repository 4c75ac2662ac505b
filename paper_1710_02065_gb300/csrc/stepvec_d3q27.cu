// stepvec_d3q27.cu -- instantiations of the vectorised stream + collide kernel
// for D3Q27 (two cells per thread; a request for four runs the general kernel).
#include "step_vec.cuh"
#include "dispatch.h"

namespace rr {

cudaError_t stepvec_d3q27(int precision, int vec, const StepParams &p, const void *fin, void *fout,
                       int block, cudaStream_t st, int sp)
{
    if (vec != 2) return step_d3q27(precision, p, fin, fout, block, st);
    switch (precision) {
    case PREC_FP64: return launch_stream_collide_vec<D3Q27, double, double, 2>(p, fin, fout, block, st, sp);
    case PREC_FP32: return launch_stream_collide_vec<D3Q27, float, float, 2>(p, fin, fout, block, st, sp);
    case PREC_FP16: return launch_stream_collide_vec<D3Q27, __half, float, 2>(p, fin, fout, block, st, sp);
    case PREC_BF16: return launch_stream_collide_vec<D3Q27, __nv_bfloat16, float, 2>(p, fin, fout, block, st, sp);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rr
