// step_vec.cuh -- vectorised fused stream + collide kernel (same update as
// step.cuh) for lattices without a cell-type mask.
//
// Each thread owns V consecutive cells of one x row.  Populations with
// xi_x = 0 move as one aligned V-wide load per direction (128-bit for FP32
// V = 4 and FP64 V = 2; 32-bit for FP16/BF16 V = 2).  Populations streamed
// along x (xi_x = +-1) sit one cell off that alignment: they are read as V
// scalar loads of the shifted cells (the sectors are the ones the warp's
// aligned loads touch, so DRAM traffic is unchanged; measured on GB300 this
// beats completing the aligned vector by a warp shuffle plus a scalar load
// at the warp's edge lanes).  Stores are aligned V-wide vectors of the
// thread's own cells.  Boundary roles are the ones of step.cuh: a node on a non-periodic
// y/z face streams the row of its inward neighbour (uniform for a thread); a
// node on a non-periodic x face takes the streamed populations of its x
// neighbour, which lives in the same thread.
//
// Reconstruction uses the parity of the Hermite terms: for an opposite pair
// (i, i + Q/2) the even part E = a0 + H2:A2 / (2 c_s^4) is shared and the
// odd part O = xi.a1 / c_s^2 + T3(A3) changes sign, so f_i = w (E + O) and
// f_opp = w (E - O).
#pragma once

#include <type_traits>

#include "step.cuh"

namespace rr {

// Two FP32 lanes computed by one packed instruction (add / mul / fma .f32x2
// of sm_100+): the rebuild of a thread's two cells with the same code.
// Measured on GB300 for the D3Q19 jet: BF16 storage 59.6 -> 64.2 G cell
// updates/s, FP16 63.1 -> 61.5, FP32 46.2 -> 44.7; so only the BF16
// two-cell kernel uses it.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float2 a) : v(a) {}
    __device__ __forceinline__ F2(double c) : v(make_float2((float)c, (float)c)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { a = a + b; return a; }
__device__ __forceinline__ F2 fmac(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ Coef<F2> pack_coef(const Coef<float> &a, const Coef<float> &b)
{
    Coef<F2> k;
    k.a0 = F2(a.a0, b.a0); k.a1x = F2(a.a1x, b.a1x); k.a1y = F2(a.a1y, b.a1y); k.a1z = F2(a.a1z, b.a1z);
    k.xx = F2(a.xx, b.xx); k.yy = F2(a.yy, b.yy); k.zz = F2(a.zz, b.zz);
    k.xy = F2(a.xy, b.xy); k.xz = F2(a.xz, b.xz); k.yz = F2(a.yz, b.yz);
    k.xxy = F2(a.xxy, b.xxy); k.xyy = F2(a.xyy, b.xyy); k.xxz = F2(a.xxz, b.xxz);
    k.xzz = F2(a.xzz, b.xzz); k.yyz = F2(a.yyz, b.yyz); k.yzz = F2(a.yzz, b.yzz);
    k.xyz = F2(a.xyz, b.xyz); k.xxyy = F2(a.xxyy, b.xxyy);
    return k;
}

// ---------------------------------------------------------------------------
// V-wide aligned loads / stores converting to / from the compute type C
// ---------------------------------------------------------------------------
template <class S, int V>
struct VecIO;

template <>
struct VecIO<float, 4> {
    __device__ static void ld(const float *p, float (&o)[4])
    {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static void st(float *p, const float (&o)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct VecIO<float, 2> {
    __device__ static void ld(const float *p, float (&o)[2])
    {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static void st(float *p, const float (&o)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    }
};
template <>
struct VecIO<double, 2> {
    __device__ static void ld(const double *p, double (&o)[2])
    {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static void st(double *p, const double (&o)[2])
    {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
};

// 16-bit pairs move as one 32-bit word; the paired conversion intrinsics
// unpack / pack (round to nearest) both halves of a word at once.
__device__ __forceinline__ float2 unpack_h2(unsigned v)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&v));
}
__device__ __forceinline__ unsigned pack_h2(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ float2 unpack_b2(unsigned v)
{
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
__device__ __forceinline__ unsigned pack_b2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}

template <>
struct VecIO<__half, 4> {
    __device__ static void ld(const __half *p, float (&o)[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = unpack_h2(v.x), b = unpack_h2(v.y);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    __device__ static void st(__half *p, const float (&o)[4])
    {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack_h2(o[0], o[1]), pack_h2(o[2], o[3]));
    }
};
template <>
struct VecIO<__half, 2> {
    __device__ static void ld(const __half *p, float (&o)[2])
    {
        const float2 a = unpack_h2(__ldg(reinterpret_cast<const unsigned *>(p)));
        o[0] = a.x; o[1] = a.y;
    }
    __device__ static void st(__half *p, const float (&o)[2])
    {
        *reinterpret_cast<unsigned *>(p) = pack_h2(o[0], o[1]);
    }
};
template <>
struct VecIO<__nv_bfloat16, 2> {
    __device__ static void ld(const __nv_bfloat16 *p, float (&o)[2])
    {
        const float2 a = unpack_b2(__ldg(reinterpret_cast<const unsigned *>(p)));
        o[0] = a.x; o[1] = a.y;
    }
    __device__ static void st(__nv_bfloat16 *p, const float (&o)[2])
    {
        *reinterpret_cast<unsigned *>(p) = pack_b2(o[0], o[1]);
    }
};
template <>
struct VecIO<__nv_bfloat16, 4> {
    __device__ static void ld(const __nv_bfloat16 *p, float (&o)[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = unpack_b2(v.x), b = unpack_b2(v.y);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    __device__ static void st(__nv_bfloat16 *p, const float (&o)[4])
    {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack_b2(o[0], o[1]), pack_b2(o[2], o[3]));
    }
};

// ---------------------------------------------------------------------------
// The kernel.  Block = one warp-multiple of threads along one x row.
// Requires: no cell-type mask, nx % V == 0.
// ---------------------------------------------------------------------------
// One thread's V cells of a row (x0raw = first cell, a multiple of V); the
// lanes of a warp hold consecutive V-cell groups of the same row.  Lanes past
// the row end do nothing.
template <class L, class S, class C, int V>
__device__ __forceinline__ void update_vec(const StepParams &p, const char *const *in, char *const *out, int x0raw,
                                           int y, int z)
{
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    if (x0raw >= nx) return;  // lanes past the row end
    const int x0 = x0raw;
    const unsigned nxy = (unsigned)nx * ny;

    // rows streamed from (uniform per thread): inward neighbour on non-periodic y/z faces
    int sy = y, sz = z, inlet_row = -1;
    if (!p.periodic[1]) {
        if (y == 0) { sy = 1; if (p.kind[2] != BC_OUTFLOW) inlet_row = 2; }
        if (y == ny - 1) { sy = ny - 2; if (p.kind[3] != BC_OUTFLOW && inlet_row < 0) inlet_row = 3; }
    }
    if (L::D == 3 && !p.periodic[2]) {
        if (z == 0) { sz = 1; if (p.kind[4] != BC_OUTFLOW && inlet_row < 0) inlet_row = 4; }
        if (z == nz - 1) { sz = nz - 2; if (p.kind[5] != BC_OUTFLOW && inlet_row < 0) inlet_row = 5; }
    }
    const int ym = sy == 0 ? ny - 1 : sy - 1, yp = sy == ny - 1 ? 0 : sy + 1;
    const int zm = sz == 0 ? nz - 1 : sz - 1, zp = sz == nz - 1 ? 0 : sz + 1;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;        // cell left of the vector (wrapped)
    const int xr = x0 + V == nx ? 0 : x0 + V;        // cell right of the vector (wrapped)

#ifdef LBM_BOUNDS_CHECK
    {
        // every row this thread reads (x0 - 1 .. x0 + V, wrapped) and writes
        bool bad = x0 < 0 || x0 + V > nx || xl >= nx || xr >= nx || sy >= ny || sz >= nz ||
                   (unsigned)nx * y + nxy * z + x0 + V > (unsigned)p.ncell;
        for (int i = 0; i < L::Q; ++i) {
            const int Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
            const int Z = L::D == 2 ? 0 : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
            bad = bad || Y < 0 || Y >= ny || Z < 0 || Z >= nz ||
                  (unsigned)nx * Y + nxy * Z + (unsigned)nx > (unsigned)p.ncell;
        }
        if (index_fault(p, bad)) return;
    }
#endif

    // ---- gather
    C g[L::Q][V];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
        const int Z = L::D == 2 ? 0 : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
        const S *row = (const S *)in[i] + ((unsigned)nx * Y + nxy * Z);
        if (L::cx(i) == 0) {
            C v[V];
            VecIO<S, V>::ld(row + x0, v);
#pragma unroll
            for (int k = 0; k < V; ++k) g[i][k] = v[k];
        } else if (L::cx(i) > 0) {
            // f_i(x) = f*_i(x - 1): cells x0 - 1 (wrapped) .. x0 + V - 2
            g[i][0] = Store<S>::ld(row + xl);
#pragma unroll
            for (int k = 1; k < V; ++k) g[i][k] = Store<S>::ld(row + x0 + k - 1);
        } else {
            // f_i(x) = f*_i(x + 1): cells x0 + 1 .. x0 + V (wrapped)
#pragma unroll
            for (int k = 0; k < V - 1; ++k) g[i][k] = Store<S>::ld(row + x0 + k + 1);
            g[i][V - 1] = Store<S>::ld(row + xr);
        }
    }

    // non-periodic x: boundary nodes take their x neighbour's streamed populations
    const bool xlo = !p.periodic[0] && x0 == 0, xhi = !p.periodic[0] && x0 + V == nx;
    if (xlo) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i][0] = g[i][1];
    }
    if (xhi) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i][V - 1] = g[i][V - 2];
    }

    // ---- collision coefficients of the V cells
    const bool bulk_row = y >= p.blo[1] && y < p.bhi[1] && z >= p.blo[2] && z < p.bhi[2];
    const C chirow = bulk_row ? C(0) : chi_row<L, C>(p, y, z);
    Coef<C> cf[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        C gk[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) gk[i] = g[i][k];
        const Mom<C> m = moments_pairs<L, C>(gk);
        int inlet = -1;
        if (k == 0 && xlo && p.kind[0] != BC_OUTFLOW) inlet = 0;
        else if (k == V - 1 && xhi && p.kind[1] != BC_OUTFLOW) inlet = 1;
        if (inlet < 0) inlet = inlet_row;
        const bool bulk = bulk_row && x0 + k >= p.blo[0] && x0 + k < p.bhi[0];
        const C chi = (bulk || inlet >= 0) ? C(0) : chi_cell<L, C>(p, chirow, x0 + k, y, z);
        cf[k] = cell_coefficients<L, C>(p, m, chi, x0 + k, y, z, inlet);
    }

    // ---- rebuild and store, one direction pair at a time
    const unsigned base = (unsigned)nx * y + nxy * z + x0;
    if constexpr (V == 2 && std::is_same<S, __nv_bfloat16>::value) {
        const Coef<F2> c2 = pack_coef(cf[0], cf[1]);
        const RebuildPre<F2> r2 = rebuild_prep<L, F2>(c2);
        {
            const F2 g0 = rebuild_rest<L, F2>(c2, r2);
            C o[V] = {g0.v.x, g0.v.y};
            VecIO<S, V>::st((S *)out[0] + base, o);
        }
#pragma unroll
        for (int i = 1; i <= L::HALF; ++i) {
            F2 p2, m2;
            rebuild_pair<L, F2>(c2, r2, i, p2, m2);
            C op[V] = {p2.v.x, p2.v.y}, om[V] = {m2.v.x, m2.v.y};
            VecIO<S, V>::st((S *)out[i] + base, op);
            VecIO<S, V>::st((S *)out[i + L::HALF] + base, om);
        }
        return;
    }
    RebuildPre<C> rp[V];
#pragma unroll
    for (int k = 0; k < V; ++k) rp[k] = rebuild_prep<L, C>(cf[k]);
    {
        C o[V];
#pragma unroll
        for (int k = 0; k < V; ++k) o[k] = rebuild_rest<L, C>(cf[k], rp[k]);
        VecIO<S, V>::st((S *)out[0] + base, o);
    }
#pragma unroll
    for (int i = 1; i <= L::HALF; ++i) {
        C op[V], om[V];
#pragma unroll
        for (int k = 0; k < V; ++k) rebuild_pair<L, C>(cf[k], rp[k], i, op[k], om[k]);
        VecIO<S, V>::st((S *)out[i] + base, op);
        VecIO<S, V>::st((S *)out[i + L::HALF] + base, om);
    }
}

// Minimum resident 256-thread blocks per SM asked of the compiler: 16-bit
// storage with 2 cells per thread is issue-bound, and capping it at 64
// registers (4 x 256 threads per SM, a few bytes of spill) measured 3%
// faster on GB300; every other instantiation keeps its natural allocation.
template <class S, int V>
struct VecMinBlocks {
    static constexpr int value = (sizeof(S) == 2 && V == 2) ? 4 : 1;
};

template <class L, class S, class C, int V>
__global__ void __launch_bounds__(256, (VecMinBlocks<S, V>::value)) k_stream_collide_vec(const __grid_constant__ StepParams p)
{
    update_vec<L, S, C, V>(p, p.in, p.out, (blockIdx.x * blockDim.x + threadIdx.x) * V, blockIdx.y, blockIdx.z);
}

template <class L, class S, class C, int V>
cudaError_t launch_stream_collide_vec(const StepParams &p, const void *fin, void *fout, int block,
                                      cudaStream_t st)
{
    const int threads_per_row = (p.n[0] / V + 31) / 32 * 32;
    const int b = block < threads_per_row ? block : threads_per_row;
    dim3 bd(b, 1, 1);
    dim3 g((p.n[0] / V + b - 1) / b, p.n[1], p.n[2]);
    StepParams q = p;
    set_bases<L, S>(q, fin, fout);
    k_stream_collide_vec<L, S, C, V><<<g, bd, 0, st>>>(q);
    return cudaGetLastError();
}

}  // namespace rr
