// dispatch.h -- entry points of the per-lattice kernel translation units.
#pragma once
#include <cuda_runtime.h>

namespace rr {

struct StepParams;

enum { PREC_FP64 = 0, PREC_FP32 = 1, PREC_FP16 = 2, PREC_BF16 = 3 };

cudaError_t step_d2q9(int precision, const StepParams &p, const void *fin, void *fout, int block,
                      cudaStream_t st);
cudaError_t step_d3q19(int precision, const StepParams &p, const void *fin, void *fout, int block,
                       cudaStream_t st);

}  // namespace rr
