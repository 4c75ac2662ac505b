// lbm_noalloc.cu -- lbm_reduce_noalloc: the FP64 mass / momentum totals of a
// caller-owned population field, computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need
// the totals: a loop that must never enter an allocator (real-time or
// memory-accounted code), or a host that owns a fixed device-memory budget
// and hands the library only its own buffers.  This entry point serves them:
// the per-block partial sums live in one file-scope static device array,
// sized for at most LBM_NOALLOC_MAX_CELLS cells, that every GPU which loads
// the library holds until the process exits.  Nothing here calls cudaMalloc,
// cudaFree or an allocating library routine.
#include <cstdio>
#include <mutex>
#include <string>

#include "lbm.h"
#include "aux_kernels.cuh"
#include "dispatch.h"

using namespace rr;

namespace {

constexpr int NOALLOC_CELLS_PER_THREAD = 64;
constexpr int NOALLOC_MAX_BLOCKS =
    (int)((LBM_NOALLOC_MAX_CELLS + (int64_t)RED_BLOCK * NOALLOC_CELLS_PER_THREAD - 1) /
          ((int64_t)RED_BLOCK * NOALLOC_CELLS_PER_THREAD));
constexpr int MAX_DEVICES = 64;

// Per-block partials of the reduction, shared by every call on this device.
// Each call's blocks overwrite their own slots, so nothing has to be cleared
// between calls; calls that overlap on the GPU would race on it.
__device__ __align__(256) double g_reduce_scratch[NOALLOC_MAX_BLOCKS * RED_FIELDS];

std::mutex g_mu;
double *g_scratch_addr[MAX_DEVICES] = {};

// sum rho = fluid cells + sum (rho - 1), after the totals are written
__global__ void k_reduce_mass(double *__restrict__ out) { out[0] += out[4]; }

template <class L, class S>
cudaError_t launch(const void *f, int64_t ncell, const uint8_t *mask, double *scratch, int nblocks,
                   double *out, cudaStream_t st)
{
    k_reduce<L, S><<<nblocks, RED_BLOCK, 0, st>>>(ncell, (const S *)f, mask, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, 32 * RED_FIELDS, 0, st>>>(nblocks, scratch, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_mass<<<1, 1, 0, st>>>(out);
    return cudaGetLastError();
}

int set_error(int code, const char *msg)
{
    rr_set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int lbm_reduce_noalloc(int lattice, int precision, const void *f, int64_t ncell,
                                  const uint8_t *cell_type, double *out, void *cuda_stream)
{
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q27)
        return set_error(LBM_EINVAL, "lbm_reduce_noalloc: unknown lattice");
    if (precision < LBM_FP64 || precision > LBM_BF16_SHIFTED)
        return set_error(LBM_EINVAL, "lbm_reduce_noalloc: unknown precision");
    if (!f || !out) return set_error(LBM_EINVAL, "lbm_reduce_noalloc: f and out are required");
    if (ncell < 1) return set_error(LBM_EINVAL, "lbm_reduce_noalloc: ncell must be >= 1");
    if (ncell > LBM_NOALLOC_MAX_CELLS) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "lbm_reduce_noalloc: ncell = %lld exceeds the static scratch limit of %lld cells",
                      (long long)ncell, (long long)LBM_NOALLOC_MAX_CELLS);
        return set_error(LBM_EINVAL, buf);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(LBM_EINVAL, "lbm_reduce_noalloc: device index too large");
    double *scratch = nullptr;
    {
        // Once per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_reduce_scratch);
            if (e != cudaSuccess) return set_error(LBM_ECUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = (double *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    const int nblocks =
        (int)((ncell + (int64_t)RED_BLOCK * NOALLOC_CELLS_PER_THREAD - 1) / ((int64_t)RED_BLOCK * NOALLOC_CELLS_PER_THREAD));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (lattice == LBM_D2Q9) {
        switch (precision) {
        case LBM_FP64: e = launch<D2Q9, double>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP32: e = launch<D2Q9, float>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP16_SHIFTED: e = launch<D2Q9, __half>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        default: e = launch<D2Q9, __nv_bfloat16>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        }
    } else if (lattice == LBM_D3Q19) {
        switch (precision) {
        case LBM_FP64: e = launch<D3Q19, double>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP32: e = launch<D3Q19, float>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP16_SHIFTED: e = launch<D3Q19, __half>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        default: e = launch<D3Q19, __nv_bfloat16>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        }
    } else {
        switch (precision) {
        case LBM_FP64: e = launch<D3Q27, double>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP32: e = launch<D3Q27, float>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        case LBM_FP16_SHIFTED: e = launch<D3Q27, __half>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        default: e = launch<D3Q27, __nv_bfloat16>(f, ncell, cell_type, scratch, nblocks, out, st); break;
        }
    }
    if (e != cudaSuccess) return set_error(LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}
