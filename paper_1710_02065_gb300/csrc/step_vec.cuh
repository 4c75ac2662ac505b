// step_vec.cuh -- vectorised fused stream + collide kernel (same update as
// step.cuh) for lattices without a cell-type mask.
//
// Each thread owns V consecutive cells of one x row and moves them with one
// V-wide load per direction (128-bit for FP32 V = 4 and FP64 V = 2; 64-bit for
// FP16/BF16 V = 4).  Populations streamed along x (xi_x = +-1) are the same
// aligned vector shifted by one cell: the missing end element comes from the
// neighbouring lane by a warp shuffle, or, at a warp's first / last lane, from
// one scalar load.  Stores are aligned V-wide vectors of the thread's own
// cells.  Boundary roles are the ones of step.cuh: a node on a non-periodic
// y/z face streams the row of its inward neighbour (uniform for a thread); a
// node on a non-periodic x face takes the streamed populations of its x
// neighbour, which lives in the same thread.
//
// Reconstruction uses the parity of the Hermite terms: for an opposite pair
// (i, i + Q/2) the even part E = a0 + H2:A2 / (2 c_s^4) is shared and the
// odd part O = xi.a1 / c_s^2 + T3(A3) changes sign, so f_i = w (E + O) and
// f_opp = w (E - O).
#pragma once

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

__device__ __forceinline__ float h2f(unsigned short b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ unsigned short f2h(float v) { return __half_as_ushort(__float2half_rn(v)); }
__device__ __forceinline__ float b2f(unsigned short b) { return __uint_as_float((unsigned)b << 16); }
__device__ __forceinline__ unsigned short f2b(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <>
struct VecIO<__half, 4> {
    __device__ static void ld(const __half *p, float (&o)[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        o[0] = h2f(v.x & 0xffffu); o[1] = h2f(v.x >> 16);
        o[2] = h2f(v.y & 0xffffu); o[3] = h2f(v.y >> 16);
    }
    __device__ static void st(__half *p, const float (&o)[4])
    {
        uint2 v;
        v.x = (unsigned)f2h(o[0]) | ((unsigned)f2h(o[1]) << 16);
        v.y = (unsigned)f2h(o[2]) | ((unsigned)f2h(o[3]) << 16);
        *reinterpret_cast<uint2 *>(p) = v;
    }
};
template <>
struct VecIO<__nv_bfloat16, 4> {
    __device__ static void ld(const __nv_bfloat16 *p, float (&o)[4])
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xffff0000u);
        o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xffff0000u);
    }
    __device__ static void st(__nv_bfloat16 *p, const float (&o)[4])
    {
        uint2 v;
        v.x = (unsigned)f2b(o[0]) | ((unsigned)f2b(o[1]) << 16);
        v.y = (unsigned)f2b(o[2]) | ((unsigned)f2b(o[3]) << 16);
        *reinterpret_cast<uint2 *>(p) = v;
    }
};

// ---------------------------------------------------------------------------
// Moments from direction pairs: s = g_i + g_opp (even), d = g_i - g_opp (odd)
// ---------------------------------------------------------------------------
template <class L, class C>
__device__ __forceinline__ Mom<C> moments_pairs(const C *g)
{
    Mom<C> m{};
    m.dr = g[0];
#pragma unroll
    for (int i = 1; i <= L::HALF; ++i) {
        const C s = g[i] + g[i + L::HALF], d = g[i] - g[i + L::HALF];
        const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
        m.dr += s;
        if (x) m.jx += x > 0 ? d : -d;
        if (y) m.jy += y > 0 ? d : -d;
        if (z) m.jz += z > 0 ? d : -d;
        if (x) m.sxx += s;
        if (y) m.syy += s;
        if (z) m.szz += s;
        if (x && y) m.sxy += x * y > 0 ? s : -s;
        if (x && z) m.sxz += x * z > 0 ? s : -s;
        if (y && z) m.syz += y * z > 0 ? s : -s;
    }
    return m;
}

// Even (E) and odd (O) parts of the rebuilt population of direction i (1 <= i <= HALF)
template <class L, class C>
__device__ __forceinline__ void rebuild_pair(const Coef<C> &k, int i, C &even, C &odd)
{
    constexpr double cs2 = 1.0 / 3.0;
    const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
    C f2 = C(x * x - cs2) * k.xx + C(y * y - cs2) * k.yy;
    if (L::D == 3) f2 += C(z * z - cs2) * k.zz;
    if (x * y) f2 += C(2 * x * y) * k.xy;
    if (L::D == 3 && x * z) f2 += C(2 * x * z) * k.xz;
    if (L::D == 3 && y * z) f2 += C(2 * y * z) * k.yz;
    even = k.a0 + C(4.5) * f2;
    C f1 = C(0);
    if (x) f1 += x > 0 ? k.a1x : -k.a1x;
    if (y) f1 += y > 0 ? k.a1y : -k.a1y;
    if (z) f1 += z > 0 ? k.a1z : -k.a1z;
    C o = C(3) * f1;
    const double hxxy = (x * x - cs2) * y, hxyy = (y * y - cs2) * x;
    if (L::D == 2) {
        if (hxxy != 0.0) o += C(13.5 * hxxy) * k.xxy;
        if (hxyy != 0.0) o += C(13.5 * hxyy) * k.xyy;
    } else {
        const double hyzz = (z * z - cs2) * y, hxzz = (z * z - cs2) * x;
        const double hyyz = (y * y - cs2) * z, hxxz = (x * x - cs2) * z;
        const double p1 = hxxy + hyzz, m1 = hxxy - hyzz;
        const double p2 = hxzz + hxyy, m2 = hxzz - hxyy;
        const double p3 = hyyz + hxxz, m3 = hyyz - hxxz;
        if (p1 != 0.0) o += C(13.5 * p1) * (k.xxy + k.yzz);
        if (m1 != 0.0) o += C(4.5 * m1) * (k.xxy - k.yzz);
        if (p2 != 0.0) o += C(13.5 * p2) * (k.xzz + k.xyy);
        if (m2 != 0.0) o += C(4.5 * m2) * (k.xzz - k.xyy);
        if (p3 != 0.0) o += C(13.5 * p3) * (k.yyz + k.xxz);
        if (m3 != 0.0) o += C(4.5 * m3) * (k.yyz - k.xxz);
    }
    odd = o;
}

// Collision coefficients of one cell (bulk, sponge or velocity node)
template <class L, class C>
__device__ __forceinline__ Coef<C> cell_coefficients(const StepParams &p, const Mom<C> &m, int cx,
                                                     int cy, int cz, int inlet)
{
    const C om = C(p.omega);
    Coef<C> k{};
    if (inlet >= 0) {
        const C rho = C(1) + m.dr;
        const C inv = C(1) / rho;
        const Sym2<C> pn = pi_neq<C>(m, m.dr, rho, m.jx * inv, m.jy * inv, m.jz * inv, L::D);
        const int a = inlet >> 1;
        const int c[3] = {cx, cy, cz};
        const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
        const int64_t kf = c[t0] + (int64_t)p.n[t0] * c[t1];
        double ub[3];
        const double *prof = p.u_profile[inlet];
#pragma unroll
        for (int b = 0; b < 3; ++b) ub[b] = prof ? prof[3 * kf + b] : p.u_face[inlet][b];
        if (p.noise_amp > 0.0) {
            const double mag = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
            if (mag > 0.0) {
                const uint64_t base =
                    (p.noise_seed << 32) + ((uint64_t)p.step * (uint64_t)p.face_cells[inlet] + (uint64_t)kf) * 3u;
#pragma unroll
                for (int b = 0; b < L::D; ++b) ub[b] += p.noise_amp * mag * (2.0 * u01(base + b) - 1.0);
            }
        }
        const C ux = C(ub[0]), uy = C(ub[1]), uz = L::D == 3 ? C(ub[2]) : C(0);
        add_eq<C>(k, C(1), m.dr, rho, ux, uy, uz);
        add_neq<C>(k, om, ux, uy, uz, pn);
        return k;
    }
    C chi = C(0);
    if (p.any_sponge) {
        const int c[3] = {cx, cy, cz};
#pragma unroll
        for (int f = 0; f < 2 * L::D; ++f) {
            const int W = p.sponge_w[f];
            if (W > 0) {
                const int a = f >> 1;
                const int d = (f & 1) ? c[a] - (p.n[a] - W) : W - 1 - c[a];
                if (d >= 0) {
                    const C v = C(p.sponge_chi[f]) * sigma<C>(C(d), C(W));
                    chi = v > chi ? v : chi;
                }
            }
        }
    }
    if (chi > C(0)) {
        const C h = C(1) / (C(1) + C(0.5) * chi);
        const C rr = C(p.rho_ref);
        const C drs = (m.dr + C(0.5) * chi * C(p.rho_ref_m1)) * h;
        const C rs = C(1) + drs;
        const C inv = C(1) / rs;
        const C ux = (m.jx + C(0.5) * chi * rr * C(p.u_ref[0])) * h * inv;
        const C uy = (m.jy + C(0.5) * chi * rr * C(p.u_ref[1])) * h * inv;
        const C uz = L::D == 3 ? (m.jz + C(0.5) * chi * rr * C(p.u_ref[2])) * h * inv : C(0);
        const Sym2<C> pn = pi_neq<C>(m, drs, rs, ux, uy, uz, L::D);
        add_eq<C>(k, C(1) - chi, drs, rs, ux, uy, uz);
        add_eq<C>(k, chi, C(p.rho_ref_m1), rr, C(p.u_ref[0]), C(p.u_ref[1]), L::D == 3 ? C(p.u_ref[2]) : C(0));
        add_neq<C>(k, om, ux, uy, uz, pn);
        return k;
    }
    const C rho = C(1) + m.dr;
    const C inv = C(1) / rho;
    const C ux = m.jx * inv, uy = m.jy * inv, uz = L::D == 3 ? m.jz * inv : C(0);
    const Sym2<C> pn = pi_neq<C>(m, m.dr, rho, ux, uy, uz, L::D);
    add_eq<C>(k, C(1), m.dr, rho, ux, uy, uz);
    add_neq<C>(k, om, ux, uy, uz, pn);
    return k;
}

// ---------------------------------------------------------------------------
// The kernel.  Block = one warp-multiple of threads along one x row.
// Requires: no cell-type mask, nx % V == 0.
// ---------------------------------------------------------------------------
template <class L, class S, class C, int V>
__global__ void __launch_bounds__(256) k_stream_collide_vec(const __grid_constant__ StepParams p,
                                                             const S *__restrict__ fin,
                                                             S *__restrict__ fout)
{
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int lane = threadIdx.x & 31;
    const int x0raw = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool active = x0raw < nx;
    const int x0 = x0raw % nx;  // idle lanes load a wrapped, valid vector
    const int y = blockIdx.y, z = blockIdx.z;
    const int64_t N = p.ncell;
    const int64_t nxy = (int64_t)nx * ny;

    // rows streamed from (uniform per thread): inward neighbour on non-periodic y/z faces
    int sy = y, sz = z, inlet_row = -1;
    if (!p.periodic[1]) {
        if (y == 0) { sy = 1; if (p.kind[2] == BC_VELOCITY) inlet_row = 2; }
        if (y == ny - 1) { sy = ny - 2; if (p.kind[3] == BC_VELOCITY && inlet_row < 0) inlet_row = 3; }
    }
    if (L::D == 3 && !p.periodic[2]) {
        if (z == 0) { sz = 1; if (p.kind[4] == BC_VELOCITY && inlet_row < 0) inlet_row = 4; }
        if (z == nz - 1) { sz = nz - 2; if (p.kind[5] == BC_VELOCITY && inlet_row < 0) inlet_row = 5; }
    }
    const int ym = sy == 0 ? ny - 1 : sy - 1, yp = sy == ny - 1 ? 0 : sy + 1;
    const int zm = sz == 0 ? nz - 1 : sz - 1, zp = sz == nz - 1 ? 0 : sz + 1;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;        // cell left of the vector (wrapped)
    const int xr = x0 + V == nx ? 0 : x0 + V;        // cell right of the vector (wrapped)

    // ---- gather
    C g[L::Q][V];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
        const int Z = L::D == 2 ? 0 : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
        const S *row = fin + (int64_t)i * N + (int64_t)nx * Y + nxy * Z;
        C v[V];
        VecIO<S, V>::ld(row + x0, v);
        if (L::cx(i) == 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) g[i][k] = v[k];
        } else if (L::cx(i) > 0) {
            // f_i(x) = f*_i(x - 1): shift right, first element from the left neighbour
            C left = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
            if (lane == 0) left = Store<S>::ld(row + xl);
            g[i][0] = left;
#pragma unroll
            for (int k = 1; k < V; ++k) g[i][k] = v[k - 1];
        } else {
            C right = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (lane == 31) right = Store<S>::ld(row + xr);
#pragma unroll
            for (int k = 0; k < V - 1; ++k) g[i][k] = v[k + 1];
            g[i][V - 1] = right;
        }
    }
    if (!active) return;

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
    Coef<C> cf[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        C gk[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) gk[i] = g[i][k];
        const Mom<C> m = moments_pairs<L, C>(gk);
        int inlet = -1;
        if (k == 0 && xlo && p.kind[0] == BC_VELOCITY) inlet = 0;
        else if (k == V - 1 && xhi && p.kind[1] == BC_VELOCITY) inlet = 1;
        if (inlet < 0) inlet = inlet_row;
        cf[k] = cell_coefficients<L, C>(p, m, x0 + k, y, z, inlet);
    }

    // ---- rebuild and store, one direction pair at a time
    const int64_t base = (int64_t)nx * y + nxy * z + x0;
    {
        constexpr double cs2 = 1.0 / 3.0;
        C o[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            C f2 = C(-cs2) * (cf[k].xx + cf[k].yy);
            if (L::D == 3) f2 += C(-cs2) * cf[k].zz;
            o[k] = C(weight<L>(0)) * (cf[k].a0 + C(4.5) * f2);
        }
        VecIO<S, V>::st(fout + base, o);
    }
#pragma unroll
    for (int i = 1; i <= L::HALF; ++i) {
        C op[V], om[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            C e, o;
            rebuild_pair<L, C>(cf[k], i, e, o);
            op[k] = C(weight<L>(i)) * (e + o);
            om[k] = C(weight<L>(i)) * (e - o);
        }
        VecIO<S, V>::st(fout + (int64_t)i * N + base, op);
        VecIO<S, V>::st(fout + (int64_t)(i + L::HALF) * N + base, om);
    }
}

template <class L, class S, class C, int V>
cudaError_t launch_stream_collide_vec(const StepParams &p, const void *fin, void *fout, int block,
                                      cudaStream_t st)
{
    const int threads_per_row = (p.n[0] / V + 31) / 32 * 32;
    const int b = block < threads_per_row ? block : threads_per_row;
    dim3 bd(b, 1, 1);
    dim3 g((p.n[0] / V + b - 1) / b, p.n[1], p.n[2]);
    k_stream_collide_vec<L, S, C, V><<<g, bd, 0, st>>>(p, (const S *)fin, (S *)fout);
    return cudaGetLastError();
}

}  // namespace rr
