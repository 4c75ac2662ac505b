// step_d3q27.cu -- instantiations of the fused stream + collide kernel for D3Q27
// (one translation unit per lattice so the library builds in parallel).
#include "step.cuh"
#include "dispatch.h"

namespace rr {

cudaError_t step_d3q27(int precision, const StepParams &p, const void *fin, void *fout, int block,
                    cudaStream_t st)
{
    switch (precision) {
    case PREC_FP64: return launch_stream_collide<D3Q27, double, double>(p, fin, fout, block, st);
    case PREC_FP32: return launch_stream_collide<D3Q27, float, float>(p, fin, fout, block, st);
    case PREC_FP16: return launch_stream_collide<D3Q27, __half, float>(p, fin, fout, block, st);
    case PREC_BF16: return launch_stream_collide<D3Q27, __nv_bfloat16, float>(p, fin, fout, block, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rr
