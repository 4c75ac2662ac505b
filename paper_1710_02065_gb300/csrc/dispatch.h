// dispatch.h -- entry points of the per-lattice kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace rr {

struct StepParams;

enum { PREC_FP64 = 0, PREC_FP32 = 1, PREC_FP16 = 2, PREC_BF16 = 3 };

cudaError_t step_d2q9(int precision, const StepParams &p, const void *fin, void *fout, int block,
                      cudaStream_t st);
cudaError_t step_d3q19(int precision, const StepParams &p, const void *fin, void *fout, int block,
                       cudaStream_t st);
cudaError_t step_d3q27(int precision, const StepParams &p, const void *fin, void *fout, int block,
                       cudaStream_t st);

// In-place AA streaming on one lattice f: one step (loc: the local step, else
// gather-push) and the conversion of the push layout to the standard one
cudaError_t step_aa_d2q9(int precision, const StepParams &p, void *f, int block, bool loc, cudaStream_t st);
cudaError_t step_aa_d3q19(int precision, const StepParams &p, void *f, int block, bool loc, cudaStream_t st);
cudaError_t step_aa_d3q27(int precision, const StepParams &p, void *f, int block, bool loc, cudaStream_t st);
cudaError_t aa_unswap_d2q9(int precision, const StepParams &p, void *f, cudaStream_t st);
cudaError_t aa_unswap_d3q19(int precision, const StepParams &p, void *f, cudaStream_t st);
cudaError_t aa_unswap_d3q27(int precision, const StepParams &p, void *f, cudaStream_t st);

}  // namespace rr

namespace rr {

// Message returned by lbm_last_error(NULL) (for calls without a handle)
void rr_set_global_error(const char *msg);

// Vectorised kernel (no cell-type mask, nx % vec == 0).  Supported (precision,
// vec): FP64 2; FP32 2, 4; FP16 2, 4; BF16 2, 4.  sp: 0 the two-lattice pull
// (fin read, fout written), 1 / 2 the AA gather-push / local step (in place,
// fin == fout).
cudaError_t stepvec_d2q9(int precision, int vec, const StepParams &p, const void *fin, void *fout,
                         int block, cudaStream_t st, int sp = 0);
cudaError_t stepvec_d3q19(int precision, int vec, const StepParams &p, const void *fin, void *fout,
                          int block, cudaStream_t st, int sp = 0);
// D3Q27: two cells per thread (four fall back to the general kernel)
cudaError_t stepvec_d3q27(int precision, int vec, const StepParams &p, const void *fin, void *fout,
                          int block, cudaStream_t st, int sp = 0);

// Cells per thread the vectorised kernel supports for a precision (0: none)
inline bool vec_supported(int precision, int vec)
{
    switch (precision) {
    case PREC_FP64: return vec == 2;
    case PREC_FP32: return vec == 2 || vec == 4;
    case PREC_FP16:
    case PREC_BF16: return vec == 2 || vec == 4;
    }
    return false;
}
// Default cells per thread, measured on GB300 (round jet 384 x 256 x 256,
// G cell updates/s, one cell per thread vs two): D3Q19 FP16 52.9 vs 63.2,
// FP64 2.05 vs 2.00, FP32 at the copy bandwidth either way; D3Q27 FP32 31.4
// vs 32.4, FP16 38.0 vs 44.5; D2Q9 (1600 x 800) FP32 89 vs 81, FP16 96 vs 83.
inline int vec_default(int lattice, int precision)
{
    if (lattice == 0 /* D2Q9 */ || precision == PREC_FP64) return 1;
    if (precision == PREC_FP32) return lattice == 2 /* D3Q27 */ ? 2 : 1;
    return 2;
}
inline int block_default(int vec) { return vec == 1 ? 128 : 64; }

// Row-staged kernel (bulk copies of whole rows into shared memory; FP32,
// FP16, BF16; no cell-type mask; nx * element size a multiple of 16 bytes).
struct RowsPlan {
    int R;        // rows per tile
    int RS;       // elements per direction and stage (R nx)
    int stages;   // shared-memory stages
    int block;    // threads per CTA
    int grid;     // CTAs (resident: SMs x CTAs per SM, at most the tile count)
    int per_sm;   // CTAs resident per SM
    size_t smem;  // dynamic shared memory per CTA, bytes
};
// cudaErrorNotSupported (nothing launched, no CUDA error state): not eligible
// wait_ns: limit of each wait for a tile's bulk copies (0: one non-blocking
// test, for failure-path tests)
cudaError_t rows_d2q9(int precision, const StepParams &p, const void *fin, void *fout, int block, int stages,
                      unsigned *err, uint64_t wait_ns, cudaStream_t st);
cudaError_t rows_d3q19(int precision, const StepParams &p, const void *fin, void *fout, int block, int stages,
                       unsigned *err, uint64_t wait_ns, cudaStream_t st);
cudaError_t rows_plan_d2q9(int precision, const StepParams &p, const void *fin, const void *fout, int block,
                           int stages, RowsPlan &pl);
cudaError_t rows_plan_d3q19(int precision, const StepParams &p, const void *fin, const void *fout, int block,
                            int stages, RowsPlan &pl);

}  // namespace rr
