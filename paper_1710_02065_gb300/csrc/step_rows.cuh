// step_rows.cuh -- row-staged fused stream + collide kernel (same update as
// step.cuh) for lattices without a cell-type mask.
//
// A persistent grid (CTAs resident on every SM) walks over tiles of R whole
// x rows at one z.  For each tile the populations every cell pulls are staged
// in shared memory by bulk asynchronous copies (cp.async.bulk, one copy per
// direction and run of contiguous source rows, completion counted in bytes on
// an mbarrier) while the CTA updates the previous tile: the tensor-memory
// accelerator moves the data, the threads only read shared memory and write
// their cells.  Shared memory holds NS stages of [Q][R nx] populations of the
// storage type; the row a cell streams from on a non-periodic y / z face and
// the rows above and below it (with wrap-around on periodic axes) are what a
// direction's copy brings, so streaming in y and z is resolved by the copies
// and streaming in x by the index (x - xi_x, wrapped) into the staged row.
//
// Requirements (checked by the launcher): no cell-type mask, nx * sizeof(S)
// a multiple of 16 bytes, 16-byte aligned population arrays, one tile of
// Q * nx * sizeof(S) bytes per stage fitting in shared memory.
//
// Every wait on an mbarrier is bounded (2 s of global time): a CTA whose copy
// does not arrive sets p.err, waits (bounded) for the copies it still has in
// flight and returns, so the host sees an error instead of a hung kernel.
#pragma once

#include <cstdint>

#include "dispatch.h"
#include "step.cuh"

namespace rr {

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier and bulk asynchronous copy global -> shared (sm_90+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive (the barrier's one expected arrival) and announce `bytes` of copies.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Non-blocking test of the phase of `parity`
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete; false after `limit_ns`.  A limit
// of 0 tests once without blocking (the failure path of the bounded wait,
// exercised by tests: the copies of a tile just issued are still in flight).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    if (limit_ns == 0) return mbar_test_wait(bar, parity);
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr uint64_t kRowsWaitLimitNs = 2000000000ull;  // 2 s

// Populations read from shared memory and converted to the compute type
template <class S>
__device__ __forceinline__ float lds_pop(const S *p);
template <>
__device__ __forceinline__ float lds_pop<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float lds_pop<__half>(const __half *p)
{
    return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short *>(p)));
}
template <>
__device__ __forceinline__ float lds_pop<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __uint_as_float((unsigned)*reinterpret_cast<const unsigned short *>(p) << 16);
}

// Row a node streams from on y / z (its inward neighbour on a non-periodic
// face) and the first boundary role of its row (y faces before z faces).
struct RowRole {
    int sy, sz, inlet;
};

template <class L>
__device__ __forceinline__ RowRole row_role(const StepParams &p, int y, int z)
{
    RowRole r{y, z, -1};
    const int ny = p.n[1], nz = p.n[2];
    if (!p.periodic[1]) {
        if (y == 0) { r.sy = 1; if (p.kind[2] != BC_OUTFLOW) r.inlet = 2; }
        if (y == ny - 1) { r.sy = ny - 2; if (p.kind[3] != BC_OUTFLOW && r.inlet < 0) r.inlet = 3; }
    }
    if (L::D == 3 && !p.periodic[2]) {
        if (z == 0) { r.sz = 1; if (p.kind[4] != BC_OUTFLOW && r.inlet < 0) r.inlet = 4; }
        if (z == nz - 1) { r.sz = nz - 2; if (p.kind[5] != BC_OUTFLOW && r.inlet < 0) r.inlet = 5; }
    }
    return r;
}

// Component `axis` of xi_i for a direction index known only at run time: the
// components + 1 packed two bits per direction in one constant.
template <class L>
__host__ __device__ constexpr uint64_t pack_xi(int axis)
{
    uint64_t m = 0;
    for (int i = 0; i < L::Q; ++i)
        m |= (uint64_t)((axis == 0 ? L::cx(i) : axis == 1 ? L::cy(i) : L::cz(i)) + 1) << (2 * i);
    return m;
}

template <class L, int AXIS>
__device__ __forceinline__ int xi_rt(int i)
{
    constexpr uint64_t m = pack_xi<L>(AXIS);
    return (int)((m >> (2 * i)) & 3u) - 1;
}

// Source row (y coordinate) of direction i for destination row y
template <class L>
__device__ __forceinline__ int src_row_y(const StepParams &p, int i, int y)
{
    const int ny = p.n[1];
    int sy = y;
    if (!p.periodic[1]) {
        if (y == 0) sy = 1;
        if (y == ny - 1) sy = ny - 2;
    }
    int Y = sy - xi_rt<L, 1>(i);
    if (Y < 0) Y += ny;
    if (Y >= ny) Y -= ny;
    return Y;
}

// Tile geometry shared by the issuing lanes and the computing threads
struct RowsTile {
    int z, y0, rows;  // rows y0 .. y0 + rows - 1 at this z
};

__device__ __forceinline__ RowsTile rows_tile(const StepParams &p, int t, int R)
{
    const int tiles_y = (p.n[1] + R - 1) / R;
    RowsTile tl;
    tl.z = t / tiles_y;
    tl.y0 = (t - tl.z * tiles_y) * R;
    tl.rows = p.n[1] - tl.y0 < R ? p.n[1] - tl.y0 : R;
    return tl;
}

// Issue the copies of tile t into one stage (warp 0; lane i < Q copies
// direction i in runs of contiguous source rows).  Lane 0 arrives on the
// stage's barrier with the tile's byte count before any copy is issued.
template <class L, class S>
__device__ __forceinline__ void issue_tile(const StepParams &p, S *stage, int RS, uint64_t *bar, int t, int R)
{
    const int lane = threadIdx.x & 31;
    const RowsTile tl = rows_tile(p, t, R);
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const unsigned row_bytes = (unsigned)nx * sizeof(S);
    if (lane == 0) mbar_arrive_expect_tx(bar, row_bytes * (unsigned)tl.rows * L::Q);
    __syncwarp();
    if (lane >= L::Q) return;
    const int i = lane;
    int sz = tl.z;
    if (L::D == 3 && !p.periodic[2]) {
        if (tl.z == 0) sz = 1;
        if (tl.z == nz - 1) sz = nz - 2;
    }
    int Z = L::D == 3 ? sz - xi_rt<L, 2>(i) : 0;
    if (Z < 0) Z += nz;
    if (Z >= nz) Z -= nz;
    const S *plane = (const S *)p.in[i] + (size_t)Z * nx * ny;
    S *dst = stage + (size_t)i * RS;
    int j = 0;
    while (j < tl.rows) {
        const int Y0 = src_row_y<L>(p, i, tl.y0 + j);
        int run = 1;
        while (j + run < tl.rows && src_row_y<L>(p, i, tl.y0 + j + run) == Y0 + run) ++run;
        bulk_g2s(dst + (size_t)j * nx, plane + (size_t)Y0 * nx, row_bytes * (unsigned)run, bar);
        j += run;
    }
}

// One cell's update from a staged tile: row j of the tile, column x.
template <class L, class S, class C>
__device__ __forceinline__ void update_cell_staged(const StepParams &p, const S *st, int RS, int j, int x, int y,
                                                   int z, int inlet_row, bool bulk_row, C chirow)
{
    const int nx = p.n[0];
    int sx = x, inlet = -1;
    if (!p.periodic[0]) {
        if (x == 0) { sx = 1; if (p.kind[0] != BC_OUTFLOW) inlet = 0; }
        if (x == nx - 1) { sx = nx - 2; if (p.kind[1] != BC_OUTFLOW && inlet < 0) inlet = 1; }
    }
    if (inlet < 0) inlet = inlet_row;
    const int xm = sx == 0 ? nx - 1 : sx - 1, xp = sx == nx - 1 ? 0 : sx + 1;
    const S *row = st + j * nx;

    C g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        g[i] = lds_pop<S>(row + i * RS + (L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : sx)));

    const Mom<C> m = moments_pairs<L, C>(g);
    const bool bulk = bulk_row && x >= p.blo[0] && x < p.bhi[0];
    const C chi = (bulk || inlet >= 0) ? C(0) : chi_cell<L, C>(p, chirow, x, y, z);
    const Coef<C> k = cell_coefficients<L, C>(p, m, chi, x, y, z, inlet);

    const unsigned cell = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)p.n[1] * (unsigned)z);
    const RebuildPre<C> r = rebuild_prep<L, C>(k);
    Store<S>::st((S *)p.out[0] + cell, rebuild_rest<L, C>(k, r));
#pragma unroll
    for (int i = 1; i <= L::HALF; ++i) {
        C gp, gm;
        rebuild_pair<L, C>(k, r, i, gp, gm);
        Store<S>::st((S *)p.out[i] + cell, gp);
        Store<S>::st((S *)p.out[i + L::HALF] + cell, gm);
    }
}

// The kernel.  Dynamic shared memory: NS barriers (padded to 128 bytes), then
// NS stages of Q directions x RS elements (RS = R nx rounded up to 16 bytes).
// wait_ns bounds each wait for a tile's copies (kRowsWaitLimitNs unless a
// test asks for less); the copies still in flight after a wait gave up are
// always awaited with kRowsWaitLimitNs before the CTA exits.
template <class L, class S, class C>
__global__ void __launch_bounds__(384, 2) k_stream_collide_rows(const __grid_constant__ StepParams p, int R, int RS,
                                                             int NS, unsigned *err, uint64_t wait_ns)
{
    extern __shared__ __align__(128) unsigned char rows_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(rows_smem);
    S *stages = reinterpret_cast<S *>(rows_smem + 128);
    const size_t stage_elems = (size_t)L::Q * RS;

    const int nx = p.n[0];
    const int tiles = p.n[2] * ((p.n[1] + R - 1) / R);
    const int tid = threadIdx.x, nthr = blockDim.x;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid < 32) {
        for (int s = 0; s < NS; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < tiles) issue_tile<L, S>(p, stages + s * stage_elems, RS, &bar[s], t, R);
        }
    }

    // this thread's first cell of a tile and its stride, as (row, column)
    const int x_first = tid % nx, j_first = tid / nx;
    const int dx = nthr % nx, dj = nthr / nx;

    int bad = 0, s = 0, k = 0;
    unsigned phase = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
        if (!mbar_wait_bounded(&bar[s], phase, wait_ns)) bad = 1;
        const RowsTile tl = rows_tile(p, t, R);
        const S *st = stages + s * stage_elems;
        int x = x_first, j = j_first, jc = -1;
        int inlet_row = -1;
        bool bulk_row = false;
        C chirow = C(0);
        while (j < tl.rows) {
            const int y = tl.y0 + j;
            if (j != jc) {
                jc = j;
                inlet_row = row_role<L>(p, y, tl.z).inlet;
                bulk_row = y >= p.blo[1] && y < p.bhi[1] && tl.z >= p.blo[2] && tl.z < p.bhi[2];
                chirow = bulk_row ? C(0) : chi_row<L, C>(p, y, tl.z);
            }
            update_cell_staged<L, S, C>(p, st, RS, j, x, y, tl.z, inlet_row, bulk_row, chirow);
            x += dx;
            j += dj;
            if (x >= nx) { x -= nx; ++j; }
        }
        // every thread is done with this stage: refill it with tile t + NS G
        if (__syncthreads_or(bad)) { bad = 1; break; }
        const int tn = t + NS * gridDim.x;
        if (tid < 32 && tn < tiles) issue_tile<L, S>(p, stages + s * stage_elems, RS, &bar[s], tn, R);
        if (++s == NS) { s = 0; phase ^= 1u; }
    }
    if (bad && tid == 0) {
        // a copy did not arrive in time: wait (bounded) for every copy this
        // CTA still has in flight, then report
        int ss = s;
        unsigned ph = phase;
        for (int q = 0; q < NS; ++q) {
            const int t = blockIdx.x + (k + q) * gridDim.x;
            if (t < tiles) mbar_wait_bounded(&bar[ss], ph, kRowsWaitLimitNs);
            if (++ss == NS) { ss = 0; ph ^= 1u; }
        }
        atomicOr(err, 1u);
    }
}

// Plan: cudaErrorNotSupported (nothing launched, no CUDA error state) when
// the lattice is not eligible -- a cell-type mask, nx sizeof(S) not a
// multiple of 16 bytes, unaligned arrays, or two stages of one row exceeding
// shared memory.  R rows per tile fill about 100 KB with the stages (at least
// one row, at most ny); `stages` >= 2 (0: 2); `block` threads (0: one thread
// per cell of a tile up to 384 threads, split evenly; the kernel is compiled
// for at most 384 threads and two CTAs per SM).
template <class L, class S, class C>
cudaError_t rows_plan(const StepParams &p, const void *fin, const void *fout, int block, int stages, RowsPlan &pl)
{
    const size_t row_bytes = (size_t)p.n[0] * sizeof(S);
    if (p.solid || row_bytes % 16 != 0) return cudaErrorNotSupported;
    if (((uintptr_t)fin | (uintptr_t)fout) % 16 != 0) return cudaErrorNotSupported;
    int dev = 0, nsm = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int NS = stages < 2 ? 2 : stages;
    if (128 + (size_t)NS * L::Q * row_bytes > (size_t)max_smem) return cudaErrorNotSupported;
    int R = (int)((100 * 1024 - 128) / ((size_t)NS * L::Q * row_bytes));
    if (R < 1) R = 1;
    if (R > p.n[1]) R = p.n[1];
    const int nx = p.n[0];
    int b = block;
    if (b <= 0) {
        const int cells = R * nx;
        const int per = (cells + 383) / 384;
        b = ((cells + per - 1) / per + 31) / 32 * 32;
    }
    if (b < 32 || b > 384 || b % 32 != 0) return cudaErrorInvalidValue;
    pl.R = R;
    pl.RS = R * nx;  // R nx sizeof(S) is a multiple of 16 bytes
    pl.stages = NS;
    pl.block = b;
    pl.smem = 128 + (size_t)NS * L::Q * (size_t)pl.RS * sizeof(S);
    auto kern = k_stream_collide_rows<L, S, C>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl.per_sm, kern, b, pl.smem);
    if (e != cudaSuccess) return e;
    if (pl.per_sm < 1) return cudaErrorNotSupported;
    const int tiles = p.n[2] * ((p.n[1] + R - 1) / R);
    pl.grid = tiles < nsm * pl.per_sm ? tiles : nsm * pl.per_sm;
    return cudaSuccess;
}

template <class L, class S, class C>
cudaError_t launch_stream_collide_rows(const StepParams &p, const void *fin, void *fout, int block, int stages,
                                       unsigned *err, uint64_t wait_ns, cudaStream_t st)
{
    RowsPlan pl;
    const cudaError_t e = rows_plan<L, S, C>(p, fin, fout, block, stages, pl);
    if (e != cudaSuccess) return e;
    StepParams q = p;
    set_bases<L, S>(q, fin, fout);
    k_stream_collide_rows<L, S, C><<<pl.grid, pl.block, pl.smem, st>>>(q, pl.R, pl.RS, pl.stages, err, wait_ns);
    return cudaGetLastError();
}

}  // namespace rr
