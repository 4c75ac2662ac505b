// rows_d2q9.cu -- instantiations of the row-staged stream + collide kernel for D2Q9.
#include "step_rows.cuh"
#include "dispatch.h"

namespace rr {

cudaError_t rows_d2q9(int precision, const StepParams &p, const void *fin, void *fout, int block, int stages,
                       unsigned *err, uint64_t wait_ns, cudaStream_t st)
{
    switch (precision) {
    case PREC_FP32: return launch_stream_collide_rows<D2Q9, float, float>(p, fin, fout, block, stages, err, wait_ns, st);
    case PREC_FP16: return launch_stream_collide_rows<D2Q9, __half, float>(p, fin, fout, block, stages, err, wait_ns, st);
    case PREC_BF16:
        return launch_stream_collide_rows<D2Q9, __nv_bfloat16, float>(p, fin, fout, block, stages, err, wait_ns, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t rows_plan_d2q9(int precision, const StepParams &p, const void *fin, const void *fout, int block,
                            int stages, RowsPlan &pl)
{
    switch (precision) {
    case PREC_FP32: return rows_plan<D2Q9, float, float>(p, fin, fout, block, stages, pl);
    case PREC_FP16: return rows_plan<D2Q9, __half, float>(p, fin, fout, block, stages, pl);
    case PREC_BF16: return rows_plan<D2Q9, __nv_bfloat16, float>(p, fin, fout, block, stages, pl);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace rr
