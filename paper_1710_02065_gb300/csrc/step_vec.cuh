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
// thread's own cells (the AA gather-push step stores its xi_x = +-1
// populations one cell at a time).  Boundary roles are the ones of step.cuh:
// rows on (or, for the AA steps, next to) a non-periodic y / z face take the
// general update; a node on a non-periodic x face takes the streamed
// populations of its x neighbour, which lives in the same thread, and its
// velocity / pressure / free-slip role is applied to their moments in
// registers.
//
// Reconstruction uses the parity of the Hermite terms: for an opposite pair
// (i, i + Q/2) the even part E = a0 + H2:A2 / (2 c_s^4) is shared and the
// odd part O = xi.a1 / c_s^2 + T3(A3) changes sign, so f_i = w (E + O) and
// f_opp = w (E - O).
#pragma once

#include <type_traits>

#include "step.cuh"

namespace rr {

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
// Raw V-wide words of the storage format (one aligned load) and the
// conversion of element k to the compute type.
// ---------------------------------------------------------------------------
template <class S, int V>
struct Raw;
template <>
struct Raw<double, 2> {
    using T = double2;
    __device__ static T ld(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
    __device__ static double get(const T &v, int k) { return k == 0 ? v.x : v.y; }
};
template <>
struct Raw<float, 2> {
    using T = float2;
    __device__ static T ld(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    __device__ static float get(const T &v, int k) { return k == 0 ? v.x : v.y; }
};
template <>
struct Raw<float, 4> {
    using T = float4;
    __device__ static T ld(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    __device__ static float get(const T &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }
};
__device__ __forceinline__ float half_lo(unsigned w) { return __low2float(*reinterpret_cast<const __half2 *>(&w)); }
__device__ __forceinline__ float half_hi(unsigned w) { return __high2float(*reinterpret_cast<const __half2 *>(&w)); }
template <>
struct Raw<__half, 2> {
    using T = unsigned;
    __device__ static T ld(const __half *p) { return __ldg(reinterpret_cast<const unsigned *>(p)); }
    __device__ static float get(const T &v, int k) { return k == 0 ? half_lo(v) : half_hi(v); }
};
template <>
struct Raw<__half, 4> {
    using T = uint2;
    __device__ static T ld(const __half *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float get(const T &v, int k)
    {
        return k == 0 ? half_lo(v.x) : (k == 1 ? half_hi(v.x) : (k == 2 ? half_lo(v.y) : half_hi(v.y)));
    }
};
__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
template <>
struct Raw<__nv_bfloat16, 2> {
    using T = unsigned;
    __device__ static T ld(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const unsigned *>(p)); }
    __device__ static float get(const T &v, int k) { return k == 0 ? bf_lo(v) : bf_hi(v); }
};
template <>
struct Raw<__nv_bfloat16, 4> {
    using T = uint2;
    __device__ static T ld(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float get(const T &v, int k)
    {
        return k == 0 ? bf_lo(v.x) : (k == 1 ? bf_hi(v.x) : (k == 2 ? bf_lo(v.y) : bf_hi(v.y)));
    }
};

// Store G consecutive values (aligned): one G-wide store, 16-bit pairs packed
// with one rounding conversion each
template <class S, int G>
struct GroupSt;
template <>
struct GroupSt<double, 2> {
    __device__ static void st(double *p, const double *o) { *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]); }
};
template <>
struct GroupSt<float, 2> {
    __device__ static void st(float *p, const float *o) { *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]); }
};
template <>
struct GroupSt<float, 4> {
    __device__ static void st(float *p, const float *o)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct GroupSt<__half, 2> {
    __device__ static void st(__half *p, const float *o) { *reinterpret_cast<unsigned *>(p) = pack_h2(o[0], o[1]); }
};
template <>
struct GroupSt<__half, 4> {
    __device__ static void st(__half *p, const float *o)
    {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack_h2(o[0], o[1]), pack_h2(o[2], o[3]));
    }
};
template <>
struct GroupSt<__nv_bfloat16, 2> {
    __device__ static void st(__nv_bfloat16 *p, const float *o)
    {
        *reinterpret_cast<unsigned *>(p) = pack_b2(o[0], o[1]);
    }
};
template <>
struct GroupSt<__nv_bfloat16, 4> {
    __device__ static void st(__nv_bfloat16 *p, const float *o)
    {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack_b2(o[0], o[1]), pack_b2(o[2], o[3]));
    }
};

// ---------------------------------------------------------------------------
// Rows whose y / z neighbour rows do not wrap around and that are not on a
// non-periodic y / z face (1 <= y <= ny - 2, 1 <= z <= nz - 2): every
// population is pulled from a fixed offset of the thread's own cell -- the
// row x - xi_i in direction i's array, i times the direction stride
// (p.st_off[1] bytes) from the lattice: one V-wide aligned load per
// direction plus, for xi_x = +-1, one scalar load of the cell just outside
// the vector (x0 - 1 or x0 + V, wrapped around on a periodic x axis).  The V
// cells' populations are then taken element by element; a node on a
// non-periodic x face takes its x neighbour's streamed populations (same
// thread) and its boundary role.  Cells are collided and stored G at a time.
// An interior cell is bulk or a sponge cell: layers relaxing to the rest
// state use the closed form of coef_interior (which gives the bulk
// coefficients bit for bit at chi = 0), other references and velocity /
// free-slip / pressure nodes the general coefficients.
//
// Streaming patterns (SP): kPull reads one lattice and writes the other;
// the two in-place AA step types of update_cell_aa work on one lattice:
// kAAPush pulls as kPull does and pushes each o_i to P_opp(i)[x + xi_i]
// (back to P_i[x] outside a non-periodic x face), kAALocal reads the V-wide
// word of P_opp(i) at the thread's own cells and writes P_i there.  The AA
// vector path takes rows whose y / z neighbours are not face rows either
// (a face node is updated with the node it takes populations from).
// ---------------------------------------------------------------------------
enum { kPull = 0, kAAPush = 1, kAALocal = 2 };

template <class L, class S, class C, int V>
struct VecIn {
    typename Raw<S, V>::T v[L::Q];  // V-wide words, all directions
    C e[L::Q];                      // edge values, xi_x = +-1 directions (pulls)
};

// Populations streamed into cell k of a thread's vector: element k of the
// V-wide load for xi_x = 0 (every direction for the local AA step), the
// neighbouring element (or the scalar edge value) for xi_x = +-1
template <class L, class S, class C, int V, int SP>
__device__ __forceinline__ void gather_vec(const VecIn<L, S, C, V> &r, int k, C *g)
{
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (SP == kAALocal || L::cx(i) == 0) g[i] = Raw<S, V>::get(r.v[i], k);
        else if (L::cx(i) > 0) g[i] = k == 0 ? r.e[i] : Raw<S, V>::get(r.v[i], k - 1);
        else g[i] = k == V - 1 ? r.e[i] : Raw<S, V>::get(r.v[i], k + 1);
    }
}

// Cell offsets from a row to the rows a pull reads: ym / yp for directions
// with c_y > 0 / < 0 (the rows y - 1 / y + 1), zm / zp likewise in z.  WR = 0:
// rows whose neighbours do not wrap (-nx, +nx, -nx ny, +nx ny); WR = 1: any
// row of a lattice periodic in y and z, the neighbours of the first and last
// rows wrapped around.  A push to the row y + c_y uses yp for c_y > 0 and ym
// for c_y < 0.
struct RowOff {
    int ym, yp, zm, zp;
};

template <class L, int WR>
__device__ __forceinline__ RowOff row_offsets(const StepParams &p, int y, int z)
{
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2], nxy = nx * ny;
    RowOff o;
    if (WR) {
        o.ym = y == 0 ? (ny - 1) * nx : -nx;
        o.yp = y == ny - 1 ? -(ny - 1) * nx : nx;
        o.zm = L::D == 2 ? 0 : (z == 0 ? (nz - 1) * nxy : -nxy);
        o.zp = L::D == 2 ? 0 : (z == nz - 1 ? -(nz - 1) * nxy : nxy);
    } else {
        o.ym = -nx;
        o.yp = nx;
        o.zm = -nxy;
        o.zp = nxy;
    }
    return o;
}

// Offset (cells) from a cell to the cell direction i pulls from, in its row
// pattern: -c_y(i), -c_z(i) rows away
template <class L>
__device__ __forceinline__ int pull_off(const RowOff &o, int i)
{
    return (L::cy(i) > 0 ? o.ym : (L::cy(i) < 0 ? o.yp : 0)) + (L::cz(i) > 0 ? o.zm : (L::cz(i) < 0 ? o.zp : 0));
}

// Address of the row direction i of a cell pulls from, in direction i's
// array (i times the direction stride in bytes).  The vector path runs on
// lattices that span less than 2 GB, and the address lies inside the lattice
// past the thread's cell, so the pull step forms the byte offset from the
// cell in 32-bit arithmetic (one 64-bit add: measured 1-2 % faster at 16-bit
// storage); the AA gather-push step keeps the 64-bit form, which measured
// faster there.
template <class L, class S, int SP>
__device__ __forceinline__ const S *vec_row_ptr(const char *bin, int i, const RowOff &o, unsigned dstride)
{
    if (SP == kPull)
        return reinterpret_cast<const S *>(bin + ((unsigned)i * dstride + (unsigned)(pull_off<L>(o, i) * (int)sizeof(S))));
    const char *rb = bin + (long long)pull_off<L>(o, i) * (long long)sizeof(S);
    return reinterpret_cast<const S *>(rb + (size_t)i * dstride);
}

// Loads of one thread's vector (x0, y, z) of such a row; false when a
// checked build finds an index outside the lattice (nothing loaded).
template <class L, class S, class C, int V, int SP>
__device__ __forceinline__ bool vec_load(const StepParams &p, const char *in0, int x0, int y, int z,
                                         const RowOff &ro, VecIn<L, S, C, V> &r)
{
    using RW = Raw<S, V>;
    const int nx = p.n[0];
    const unsigned nxy = (unsigned)nx * (unsigned)p.n[1];
    const unsigned cell = (unsigned)x0 + (unsigned)nx * y + nxy * z;
    // cells just left / right of the vector, relative to x0, on a periodic x
    // axis (wrapped around)
    const int dl = x0 > 0 ? -1 : nx - 1;
    const int dr = x0 + V < nx ? V : -x0;
#ifdef LBM_BOUNDS_CHECK
    {
        // every value used lies in its direction's lattice; the unused edge
        // reads of non-periodic x faces stay inside the allocation
        const int64_t N = p.ncell;
        bool bad = (int64_t)cell + V > N;
        for (int i = 0; i < L::Q && SP != kAALocal; ++i) {
            const int64_t src = (int64_t)cell + pull_off<L>(ro, i);
            bad = bad || src < 0 || src + V > N;
            if (p.periodic[0]) {
                if (L::cx(i) > 0) bad = bad || src + dl < 0 || src + dl >= N;
                if (L::cx(i) < 0) bad = bad || src + dr < 0 || src + dr >= N;
            } else {
                if (L::cx(i) > 0) bad = bad || i * N + src - 1 < 0 || (x0 > 0 && src - 1 < 0);
                if (L::cx(i) < 0) bad = bad || i * N + src + V >= L::Q * N || (x0 + V < nx && src + V >= N);
            }
        }
        if (index_fault(p, bad)) return false;
    }
#endif
    const char *bin = in0 + (size_t)cell * sizeof(S);
    const unsigned dstride = (unsigned)p.st_off[1];
    if (SP == kAALocal) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            r.v[i] = RW::ld(reinterpret_cast<const S *>(bin + (size_t)opp<L>(i) * dstride));
    } else if (!p.periodic[0]) {
        // The edge values at x0 - 1 / x0 + V are read unconditionally: on the
        // x faces (x0 = 0, x0 + V = nx) they are not used (the face node takes
        // its neighbour's populations), and the addresses stay inside the
        // lattice's allocation -- direction i >= 1 with xi_x > 0 reads at
        // index i ncell + src - 1 >= 0, and the last direction with xi_x < 0
        // (D2Q9 7, D3Q19 16, D3Q27 26) pulls from a row before the last one,
        // so i ncell + src + V < Q ncell.  A uniform branch, so no warp
        // diverges on it.
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const S *row = vec_row_ptr<L, S, SP>(bin, i, ro, dstride);
            r.v[i] = RW::ld(row);
            if (L::cx(i) > 0) r.e[i] = Store<S>::ld(row - 1);
            if (L::cx(i) < 0) r.e[i] = Store<S>::ld(row + V);
        }
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const S *row = vec_row_ptr<L, S, SP>(bin, i, ro, dstride);
            r.v[i] = RW::ld(row);
            if (L::cx(i) > 0) r.e[i] = Store<S>::ld(row + dl);
            if (L::cx(i) < 0) r.e[i] = Store<S>::ld(row + dr);
        }
    }
    return true;
}

// Store the rebuilt populations o[kk][i] of the group's cells k0 .. k0 + G - 1.
// kPull / kAALocal: direction i's array at the cells themselves (G-wide).
// kAAPush: o_i of cell x goes to P_opp(i)[x + xi_i]: a G-wide store in the
// row y + c_y, z + c_z for xi_x = 0; single values for xi_x = +-1, wrapped
// around a periodic x axis, kept in P_i at the node when they would leave
// through a non-periodic x face.
template <class L, class S, class C, int V, int G, int SP>
__device__ __forceinline__ void vec_store(const StepParams &p, char *bout, int x0, int k0, const RowOff &ro,
                                          const C (&o)[G][L::Q])
{
    const unsigned dstride = (unsigned)p.st_off[1];
    if (SP != kAAPush) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            C w[G];
#pragma unroll
            for (int kk = 0; kk < G; ++kk) w[kk] = o[kk][i];
            GroupSt<S, G>::st(reinterpret_cast<S *>(bout + (size_t)i * dstride) + k0, w);
        }
        return;
    }
    const int nx = p.n[0];
    // A value leaves the row only from its ends (nx is a multiple of V): the
    // first cell of the row's first thread moving -x, the last cell of its
    // last thread moving +x.
    const bool first = x0 == 0, last = x0 + V >= nx;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int j = opp<L>(i);
        // the row y + c_y(i), z + c_z(i): the row direction j = opp(i) pulls from
        // (32-bit byte offset from the cell, as the pull step's loads)
        S *dst = reinterpret_cast<S *>(bout + ((unsigned)j * dstride + (unsigned)(pull_off<L>(ro, j) * (int)sizeof(S)))) + k0;
        if (L::cx(i) == 0) {
            C w[G];
#pragma unroll
            for (int kk = 0; kk < G; ++kk) w[kk] = o[kk][i];
            GroupSt<S, G>::st(dst, w);
        } else {
#pragma unroll
            for (int kk = 0; kk < G; ++kk) {
                S *t = dst + kk + L::cx(i);
                if (L::cx(i) > 0 ? (k0 + kk == V - 1 && last) : (k0 + kk == 0 && first)) {
                    // wrapped around a periodic x axis; out through a
                    // non-periodic x face: kept in P_i at the node
                    t = p.periodic[0] ? t + (L::cx(i) < 0 ? nx : -nx)
                                      : reinterpret_cast<S *>(bout + (size_t)i * dstride) + k0 + kk;
                }
                Store<S>::st(t, o[kk][i]);
            }
        }
    }
}

// Collide the V cells of a loaded vector and store them, one cell at a time
// (gather, moments, coefficients, rebuild).  all_bulk: every cell of the
// vector is bulk (no sponge, no boundary role), decided by the caller for a
// whole warp so that the warp runs one code path; otherwise each cell takes
// its sponge strength from the per-axis tables (0 in the bulk) and the
// closed-form coefficients of a rest-state reference.  A node on a
// non-periodic x face collides its neighbour's streamed populations: as they
// are (outflow face) or with the face's density / velocity substituted.
template <class L, class S, class C, int V, int G, int SP>
__device__ __forceinline__ void vec_collide_store(const StepParams &p, char *out0, int x0, int y, int z,
                                                  const RowOff &ro, const VecIn<L, S, C, V> &r, bool all_bulk)
{
    const int nx = p.n[0];
    const unsigned nxy = (unsigned)nx * (unsigned)p.n[1];
    const unsigned cell = (unsigned)x0 + (unsigned)nx * y + nxy * z;
    char *bout = out0 + (size_t)cell * sizeof(S);
    const C om = C(p.omega);
    const bool bulk_row = y >= p.blo[1] && y < p.bhi[1] && z >= p.blo[2] && z < p.bhi[2];
    const C chirow = bulk_row ? C(0) : chi_row<L, C>(p, y, z);
    const bool xlo = !p.periodic[0] && x0 == 0, xhi = !p.periodic[0] && x0 + V == nx;
#pragma unroll
    for (int k0 = 0; k0 < V; k0 += G) {
        C o[G][L::Q];
#pragma unroll
        for (int kk = 0; kk < G; ++kk) {
            const int k = k0 + kk;
            C g[L::Q];
            Coef<C> cf;
            if (all_bulk) {
                gather_vec<L, S, C, V, SP>(r, k, g);
                cf = coef_interior<L, C, false>(moments_pairs<L, C>(g), om, C(0));
            } else {
                // a node on a non-periodic x face collides the populations
                // streamed into its neighbour (same thread), with its own role
                const bool face = (k == 0 && xlo) || (k == V - 1 && xhi);
                if (face)
                    gather_vec<L, S, C, V, SP>(r, k == 0 ? 1 : V - 2, g);
                else
                    gather_vec<L, S, C, V, SP>(r, k, g);
                Mom<C> m = moments_pairs<L, C>(g);
                const int x = x0 + k;
                const int inlet = !face ? -1 : (k == 0 ? (p.kind[0] != BC_OUTFLOW ? 0 : -1)
                                                        : (p.kind[1] != BC_OUTFLOW ? 1 : -1));
                C chi = C(0);
                if (inlet >= 0) {
                    m = face_moments<L, C>(p, m, inlet, x, y, z);
                } else {
                    chi = chirow;
                    if (!(x >= p.blo[0] && x < p.bhi[0]) && p.any_sponge) {
                        const C v = chi_tab<C>(p, x);
                        chi = v > chi ? v : chi;
                    }
                }
                cf = coef_interior<L, C, true>(m, om, chi);
            }
            rebuild_all<L, C, false>(cf, o[kk]);
        }
        vec_store<L, S, C, V, G, SP>(p, bout, x0, k0, ro, o);
    }
}

// Whether the vector path applies to row (y, z): its y / z neighbour rows do
// not wrap and it is not on a non-periodic y / z face; for the AA steps its
// neighbours are not face rows either.  The handle's sponge layers relax to
// the rest state (the vector path's closed form) -- launch_update checks it.
template <class L, int SP>
__device__ __forceinline__ bool vec_row(const StepParams &p, int y, int z)
{
    const int ny = p.n[1], nz = p.n[2];
    bool ok = p.off32 && !p.order4 && y > 0 && y < ny - 1 && (L::D == 2 || (z > 0 && z < nz - 1));
    if (SP != kPull) {
        if (!p.periodic[1]) ok = ok && y > 1 && y < ny - 2;
        if (L::D == 3 && !p.periodic[2]) ok = ok && z > 1 && z < nz - 2;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// One thread's V cells of a row (x0 = first cell, a multiple of V); lanes
// past the row end do nothing.  Rows outside the vector path update their
// cells one by one with the general update (the same arithmetic).  in / out:
// per-direction bases of the lattices (one lattice for the AA steps).  Used
// by the single-lattice kernel and by the batched serving kernel.
//
// A node on a non-periodic x face takes the populations streamed into its
// neighbour, which lives in the same thread; a velocity / free-slip /
// pressure face node becomes an interior collision of substituted moments
// (face_moments) -- in the AA steps too, since the neighbour's populations
// are the thread's own -- so the vector path carries no general-coefficient code:
// measured on GB300 (D3Q19 FP16 jet), general-update code in the path, even
// where it ran only for face cells, cost 13-17% of the whole kernel, and
// updating the face cells in threads or a launch of their own (one cell per
// row, so every access its own cache sector) cost more.
//
// WR = 1: a lattice periodic on every axis whose direction arrays span less
// than 2 GB (32-bit offsets), as the serving engine's domains are: every row
// takes the vector path, the first and last rows' neighbours wrapped
// (row_offsets), and no general update is compiled in.
// ---------------------------------------------------------------------------
template <class L, class S, class C, int V, int G, int SP = kPull, int WR = 0>
__device__ __forceinline__ void update_vec(const StepParams &p, const char *const *in, char *const *out, int x0,
                                           int y, int z)
{
    const int nx = p.n[0];
    if (x0 >= nx) return;  // lanes past the row end
    if (WR || vec_row<L, SP>(p, y, z)) {
        const RowOff ro = row_offsets<L, WR>(p, y, z);
        VecIn<L, S, C, V> r;
        if (!vec_load<L, S, C, V, SP>(p, in[0], x0, y, z, ro, r)) return;
        const bool bulk = y >= p.blo[1] && y < p.bhi[1] && z >= p.blo[2] && z < p.bhi[2] && x0 >= p.blo[0] &&
                          x0 + V <= p.bhi[0];
        vec_collide_store<L, S, C, V, G, SP>(p, out[0], x0, y, z, ro, r, bulk);
        return;
    }
    if constexpr (!WR) {
#pragma unroll 1
        for (int k = 0; k < V; ++k) {
            if (SP == kPull)
                update_cell<L, S, C, false, kMaskNone>(p, in, out, x0 + k, y, z);
            else
                update_cell_aa<L, S, C, false, kMaskNone, SP == kAALocal>(p, out, x0 + k, y, z);
        }
    }
}

// Minimum resident 256-thread blocks per SM asked of the compiler: 16-bit
// storage with 2 cells per thread is issue-bound, and 64 registers (4 x 256
// threads per SM) keep enough warps resident to hide the loads; on D3Q27
// (27 populations) 64 registers spill, and 3 blocks (80 registers) measured
// fastest (FP16 jet 45.5 -> 48.7 G cell updates/s; 2 blocks 48.0); the wider
// types and 4 cells per thread take 128.
template <class L, class S, int V, int SP = kPull>
struct VecMinBlocks {
    static constexpr int value = (sizeof(S) == 2 && V == 2) ? (L::Q > 19 ? 3 : 4) : 2;
};

// Cells collided and stored together (one G-wide store per direction)
template <class S, int V>
struct VecGroup {
    static constexpr int value = 2;
};

// ---------------------------------------------------------------------------
// The kernel: blocks along x rows (blockIdx.y = y, blockIdx.z = z), V cells
// per thread.  Requires: no cell-type mask, nx % V == 0.
// ---------------------------------------------------------------------------
// Grid (x blocks of a row, ny, nz)
template <class L, class S, class C, int V, int SP>
__global__ void __launch_bounds__(256, (VecMinBlocks<L, S, V, SP>::value)) k_stream_collide_vec(const __grid_constant__ StepParams p)
{
    update_vec<L, S, C, V, VecGroup<S, V>::value, SP>(p, p.in, p.out, (blockIdx.x * blockDim.x + threadIdx.x) * V,
                                                      blockIdx.y, blockIdx.z);
}

// sp: kPull (fin read, fout written) or an AA step type (fin == fout)
template <class L, class S, class C, int V>
cudaError_t launch_stream_collide_vec(const StepParams &p, const void *fin, void *fout, int block,
                                      cudaStream_t st, int sp = kPull)
{
    const int threads_per_row = (p.n[0] / V + 31) / 32 * 32;
    const int b = block < threads_per_row ? block : threads_per_row;
    dim3 bd(b, 1, 1);
    dim3 g((p.n[0] / V + b - 1) / b, p.n[1], p.n[2]);
    StepParams q = p;
    set_bases<L, S>(q, fin, fout);
    if (sp == kAAPush)
        k_stream_collide_vec<L, S, C, V, kAAPush><<<g, bd, 0, st>>>(q);
    else if (sp == kAALocal)
        k_stream_collide_vec<L, S, C, V, kAALocal><<<g, bd, 0, st>>>(q);
    else
        k_stream_collide_vec<L, S, C, V, kPull><<<g, bd, 0, st>>>(q);
    return cudaGetLastError();
}

}  // namespace rr
