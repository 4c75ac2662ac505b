// stepvec_d2q9.cu -- instantiations of the vectorised stream + collide kernel for D2Q9.
#include "step_vec.cuh"
#include "dispatch.h"

namespace rr {

cudaError_t stepvec_d2q9(int precision, int vec, const StepParams &p, const void *fin, void *fout,
                       int block, cudaStream_t st, int sp)
{
    switch (precision) {
    case PREC_FP64:
        if (vec == 2) return launch_stream_collide_vec<D2Q9, double, double, 2>(p, fin, fout, block, st, sp);
        break;
    case PREC_FP32:
        if (vec == 4) return launch_stream_collide_vec<D2Q9, float, float, 4>(p, fin, fout, block, st, sp);
        if (vec == 2) return launch_stream_collide_vec<D2Q9, float, float, 2>(p, fin, fout, block, st, sp);
        break;
    case PREC_FP16:
        if (vec == 4) return launch_stream_collide_vec<D2Q9, __half, float, 4>(p, fin, fout, block, st, sp);
        if (vec == 2) return launch_stream_collide_vec<D2Q9, __half, float, 2>(p, fin, fout, block, st, sp);
        break;
    case PREC_BF16:
        if (vec == 4) return launch_stream_collide_vec<D2Q9, __nv_bfloat16, float, 4>(p, fin, fout, block, st, sp);
        if (vec == 2) return launch_stream_collide_vec<D2Q9, __nv_bfloat16, float, 2>(p, fin, fout, block, st, sp);
        break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace rr
