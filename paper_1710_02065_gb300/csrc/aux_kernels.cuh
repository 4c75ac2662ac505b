// aux_kernels.cuh -- initialisation, conversion and diagnostic kernels.
//
//   k_init_eq     : f = feqH(rho, u)  (Eq. eqH) into both lattices
//   k_set_dir     : one direction of a caller field, f_i - w_i, into both lattices
//   k_get_dir     : one direction of the stored field as plain FP64 f_i
//   k_moments     : rho, u, Pi^neq per cell, FP64 outputs (Eq. moments, Sec. II.A)
//   k_reduce      : FP64 per-block totals of rho - 1, rho u, fluid count and
//                   unstable count (non-finite, rho <= 0 or |u| >= c_s; warp
//                   shuffles, then a fixed-order pass)
//   k_probe       : rho at listed cells
//   k_rho_accumulate : running FP64 sum of rho per cell (temporal mean of p)
//   k_pressure_fluct : Delta p~ = c_s^2 (rho - mean rho) per cell
#pragma once

#include "rr.cuh"

namespace rr {

template <class L>
__device__ __forceinline__ double weight_rt(int i)
{
    double w = 0.0;
#pragma unroll
    for (int k = 0; k < L::Q; ++k)
        if (k == i) w = weight<L>(k);
    return w;
}

// The host-transfer kernels work on cells c0 .. c0 + n - 1 of an N-cell
// field (direction-major, stride N), with their host-side arrays staged for
// just those cells (index t = cell - c0), so that transfers go through a
// bounded staging buffer in chunks.

// bad (nullable): lowest index of a cell whose rho is not finite and > 0, or
// (2D) whose u_z is not 0; such cells are still written
// dsh (nullable, here and below): per-direction storage shift of a handle
// storing f_i - feqH_i(1, u_s) instead of f_i - w_i, dsh[i] = feqH_i(1, u_s) - w_i;
// stored value + dsh[i] is the population in the w_i-shifted convention the
// arithmetic uses.
// T: the host arrays' type (FP64, or FP32 for the single-precision transfer calls)
//
// The per-cell vectors (u: 3 values, Pi^neq: 6) are interleaved by cell, so
// a thread's own components lie 12-48 bytes apart from its neighbour's.  The
// kernels move a block's slice of them through shared memory with
// contiguous loads / stores (consecutive threads, consecutive elements): the
// host arrays may be page-locked host memory accessed over the host link,
// where three strided accesses per value cost three transfers of the same
// lines.  Blocks of at most kXferBlock threads.
constexpr int kXferBlock = 256;

template <class T, int M>
__device__ __forceinline__ void stage_in(const T *__restrict__ src, int count, T *sm)
{
    for (int k = threadIdx.x; k < M * count; k += blockDim.x) sm[k] = src[k];
}
template <class T, int M>
__device__ __forceinline__ void stage_out(T *__restrict__ dst, int count, const T *sm)
{
    for (int k = threadIdx.x; k < M * count; k += blockDim.x) dst[k] = sm[k];
}

template <class L, class S, class T = double>
__global__ void __launch_bounds__(kXferBlock) k_init_eq(int64_t N, int64_t c0, int64_t n,
                                                          const T *__restrict__ rho, const T *__restrict__ u,
                                                          S *__restrict__ f0, S *__restrict__ f1, int order4,
                                                          unsigned long long *__restrict__ bad,
                                                          const double *__restrict__ dsh = nullptr)
{
    using C = typename StoreC<S>::C;  // FP32 arithmetic for FP32/FP16/BF16 storage
    __shared__ T su[3 * kXferBlock];
    const int64_t b0 = blockIdx.x * (int64_t)blockDim.x;
    const int cnt = (int)(n - b0 < (int64_t)blockDim.x ? n - b0 : (int64_t)blockDim.x);
    stage_in<T, 3>(u + 3 * b0, cnt, su);
    __syncthreads();
    const int tid = threadIdx.x;
    if (tid >= cnt) return;
    const int64_t t = b0 + tid;
    const int64_t cell = c0 + t;
    const double r = rho[t];
    const T ux = su[3 * tid], uy = su[3 * tid + 1], uz = su[3 * tid + 2];
    if (bad && (!(r > 0.0) || !isfinite(r) || (L::D == 2 && uz != T(0))))
        atomicMin(bad, (unsigned long long)cell);
    Coef<C> k{};
    add_eq<C, L::D, true, full_third_order<L>()>(k, C(1), C(r - 1.0), C(r), C(ux), C(uy),
                                                  L::D == 3 ? C(uz) : C(0), order4 != 0);
    if (dsh) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const S v = Store<S>::from(rebuild<L, C>(k, i) - C(dsh[i]));
            f0[(int64_t)i * N + cell] = v;
            f1[(int64_t)i * N + cell] = v;
        }
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const S v = Store<S>::from(rebuild<L, C>(k, i));
            f0[(int64_t)i * N + cell] = v;
            f1[(int64_t)i * N + cell] = v;
        }
    }
}

// Change of the storage shift of one direction's values in place:
// stored + delta, delta = dsh_old[i] - dsh_new[i] (rounded once to the storage format)
template <class S>
__global__ void k_shift_values(int64_t n, S *__restrict__ f, double delta)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    f[t] = Store<S>::from((double)Store<S>::ld(f + t) + delta);
}

template <class L, class S>
__global__ void k_set_dir(int64_t N, int64_t c0, int64_t n, int i, const double *__restrict__ src,
                          S *__restrict__ f0, S *__restrict__ f1, const double *__restrict__ dsh = nullptr)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const S v = Store<S>::from(src[t] - weight_rt<L>(i) - (dsh ? dsh[i] : 0.0));
    f0[(int64_t)i * N + c0 + t] = v;
    f1[(int64_t)i * N + c0 + t] = v;
}

template <class L, class S>
__global__ void k_get_dir(int64_t N, int64_t c0, int64_t n, int i, const S *__restrict__ f,
                          double *__restrict__ dst, const double *__restrict__ dsh = nullptr)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    dst[t] = (double)Store<S>::ld(f + (int64_t)i * N + c0 + t) + (dsh ? dsh[i] : 0.0) + weight_rt<L>(i);
}

template <class L, class S>
__device__ __forceinline__ void load_cell_fp64(const S *__restrict__ f, int64_t N, int64_t cell,
                                               double (&g)[L::Q])
{
#pragma unroll
    for (int i = 0; i < L::Q; ++i) g[i] = (double)Store<S>::ld(f + (int64_t)i * N + cell);
}

// The Q populations of a cell in the compute type, the storage shift added
// when the handle has one (a uniform branch: the per-direction conversion of
// dsh to the compute type is not executed for the default shift)
template <class L, class S, class C>
__device__ __forceinline__ void load_cell(const S *__restrict__ f, int64_t N, int64_t cell,
                                          const double *__restrict__ dsh, C (&g)[L::Q])
{
    if (dsh) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = Store<S>::ld(f + (int64_t)i * N + cell) + C(dsh[i]);
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = Store<S>::ld(f + (int64_t)i * N + cell);
    }
}

// Moments in the kernel's compute type (FP32 for FP32/FP16/BF16 storage,
// whose values carry FP32 precision at most; FP64 for FP64 storage), stored
// as FP64: rho = 1 + dr keeps dr's relative precision.
template <class L, class S, class T = double>
__global__ void __launch_bounds__(kXferBlock) k_moments(int64_t N, int64_t c0, int64_t n, const S *__restrict__ f,
                                                          T *__restrict__ rho, T *__restrict__ u,
                                                          T *__restrict__ pn, const double *__restrict__ dsh = nullptr)
{
    using C = typename StoreC<S>::C;
    __shared__ T sm[6 * kXferBlock];  // u (3 per cell), then Pi^neq (6 per cell)
    const int64_t b0 = blockIdx.x * (int64_t)blockDim.x;
    const int cnt = (int)(n - b0 < (int64_t)blockDim.x ? n - b0 : (int64_t)blockDim.x);
    const int tid = threadIdx.x;
    const bool live = tid < cnt;
    const int64_t t = b0 + tid;
    Mom<C> m{};
    C r = C(1), ux = C(0), uy = C(0), uz = C(0);
    if (live) {
        C g[L::Q];
        load_cell<L, S, C>(f, N, c0 + t, dsh, g);
        m = moments<L, C>(g);
        r = C(1) + m.dr;
        ux = m.jx / r;
        uy = m.jy / r;
        uz = L::D == 3 ? m.jz / r : C(0);
        if (rho) rho[t] = T(1.0 + (double)m.dr);
    }
    if (u) {  // uniform: a kernel argument
        if (live) {
            sm[3 * tid] = ux;
            sm[3 * tid + 1] = uy;
            sm[3 * tid + 2] = uz;
        }
        __syncthreads();
        stage_out<T, 3>(u + 3 * b0, cnt, sm);
    }
    if (pn) {
        __syncthreads();
        if (live) {
            const Sym2<C> p = pi_neq<C>(m, m.dr, r, ux, uy, uz, L::D);
            sm[6 * tid + 0] = p.xx;
            sm[6 * tid + 1] = p.xy;
            sm[6 * tid + 2] = p.xz;
            sm[6 * tid + 3] = p.yy;
            sm[6 * tid + 4] = p.yz;
            sm[6 * tid + 5] = p.zz;
        }
        __syncthreads();
        stage_out<T, 6>(pn + 6 * b0, cnt, sm);
    }
}

// Per-block partial sums: [sum dr, sum jx, sum jy, sum jz, fluid cells, unstable cells]
constexpr int RED_FIELDS = 6;
constexpr int RED_BLOCK = 256;

template <class L, class S>
__global__ void __launch_bounds__(RED_BLOCK) k_reduce(int64_t N, const S *__restrict__ f,
                                                      const uint8_t *__restrict__ solid,
                                                      double *__restrict__ partial,
                                                      const double *__restrict__ dsh = nullptr)
{
    // Per-cell moments in the compute type (FP32 for FP32/FP16/BF16 storage,
    // whose values carry FP32 precision at most; FP64 for FP64 storage), the
    // running totals in FP64: GB300's FP64 rate is a small fraction of its
    // FP32 rate, and FP64 per-cell sums made this pass ALU-bound.
    using C = typename StoreC<S>::C;
    double acc[RED_FIELDS] = {0, 0, 0, 0, 0, 0};
    int fluid = 0, unstable = 0;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < N;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if (solid && (solid[cell] & MASK_TYPE)) continue;  // fluid cells only
        C g[L::Q];
        load_cell<L, S, C>(f, N, cell, dsh, g);
        bool finite = true;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) finite = finite && isfinite(g[i]);
        const Mom<C> m = moments<L, C>(g);
        if (finite) {
            acc[0] += (double)m.dr;
            acc[1] += (double)m.jx;
            acc[2] += (double)m.jy;
            acc[3] += (double)m.jz;
        }
        // unstable: non-finite, non-positive density, or |u| >= c_s
        const C rho = C(1) + m.dr, j2 = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
        if (!finite || !(rho > C(0)) || !(j2 < rho * rho * C(1.0 / 3.0))) ++unstable;
        ++fluid;
    }
    acc[4] = fluid;
    acc[5] = unstable;
    // warp, then block, in a fixed order
    __shared__ double sh[RED_BLOCK / 32][RED_FIELDS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RED_FIELDS; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < RED_FIELDS) {
        double v = 0.0;
        for (int w = 0; w < RED_BLOCK / 32; ++w) v += sh[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * RED_FIELDS + threadIdx.x] = v;
    }
}

// Final pass: one warp per field, strided then shuffled: fixed order, deterministic.
static __global__ void k_reduce_final(int nblocks, const double *__restrict__ partial,
                               double *__restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= RED_FIELDS) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partial[(int64_t)b * RED_FIELDS + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[k] = v;
}

// Momentum-exchange force on solid cells: every fluid cell x and direction i
// with x + xi_i solid adds 2 xi_i f*_i(x) (halfway bounce-back link).
// Per-block partials in the reduction layout: [Fx, Fy, Fz, 0, 0, 0].
template <class L, class S>
__global__ void __launch_bounds__(RED_BLOCK) k_force(int nx, int ny, int nz, int px, int py, int pz,
                                                     const S *__restrict__ f, const uint8_t *__restrict__ mask,
                                                     double *__restrict__ partial,
                                                     const double *__restrict__ dsh = nullptr)
{
    const int64_t N = (int64_t)nx * ny * nz;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < N;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if ((mask[cell] & MASK_TYPE) || !(mask[cell] & MASK_NEAR_SOLID)) continue;
        const int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((int64_t)nx * ny));
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            int X = x + L::cx(i), Y = y + L::cy(i), Z = z + L::cz(i);
            if (px) X = X < 0 ? X + nx : (X >= nx ? X - nx : X);
            if (py) Y = Y < 0 ? Y + ny : (Y >= ny ? Y - ny : Y);
            if (pz) Z = Z < 0 ? Z + nz : (Z >= nz ? Z - nz : Z);
            if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
            if ((mask[X + (int64_t)nx * (Y + (int64_t)ny * Z)] & MASK_TYPE) != MASK_SOLID) continue;
            const double fi = (double)Store<S>::ld(f + (int64_t)i * N + cell) + (dsh ? dsh[i] : 0.0) + weight<L>(i);
            acc[0] += 2.0 * L::cx(i) * fi;
            acc[1] += 2.0 * L::cy(i) * fi;
            acc[2] += 2.0 * L::cz(i) * fi;
        }
    }
    __shared__ double sh[RED_BLOCK / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < RED_FIELDS) {
        double v = 0.0;
        if (threadIdx.x < 3)
            for (int w = 0; w < RED_BLOCK / 32; ++w) v += sh[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * RED_FIELDS + threadIdx.x] = v;
    }
}

// rho at the listed cells; pressure = 1: p' = c_s^2 (rho - rho_ref) instead.
// A cell index outside [0, N) gives NaN (device-side lists are not checked
// on the host).
template <class L, class S>
__global__ void k_probe(int n, const int64_t *__restrict__ cells, int64_t N, const S *__restrict__ f,
                        double *__restrict__ rho, int pressure, double rho_ref)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t c = cells[t];
    if (c < 0 || c >= N) {
        rho[t] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double g[L::Q];
    load_cell_fp64<L, S>(f, N, c, g);
    double dr = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) dr += g[i];
    rho[t] = pressure ? (1.0 + dr - rho_ref) / 3.0 : 1.0 + dr;
}

// Running sum of rho per cell of the stored field (FP64), for the temporal
// mean of the pressure (Sec. III: Delta p~ = Delta p - Delta p_mean)
template <class L, class S>
__global__ void k_rho_accumulate(int64_t N, const S *__restrict__ f, double *__restrict__ acc)
{
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= N) return;
    double dr = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) dr += (double)Store<S>::ld(f + (int64_t)i * N + cell);
    acc[cell] += 1.0 + dr;
}

// Delta p~ = c_s^2 (rho - acc / count) of the stored field, and optionally the
// mean Delta p = c_s^2 (acc / count - 1) (ambient rho = 1)
template <class L, class S>
__global__ void k_pressure_fluct(int64_t N, const S *__restrict__ f, const double *__restrict__ acc, double count,
                                 double *__restrict__ dp, double *__restrict__ dp_mean)
{
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= N) return;
    double dr = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) dr += (double)Store<S>::ld(f + (int64_t)i * N + cell);
    const double mean = acc[cell] / count;
    dp[cell] = (1.0 + dr - mean) * (1.0 / 3.0);
    if (dp_mean) dp_mean[cell] = (mean - 1.0) * (1.0 / 3.0);
}

}  // namespace rr
