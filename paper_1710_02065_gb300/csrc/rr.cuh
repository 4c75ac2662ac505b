// rr.cuh -- lattice descriptors and the Hermite-regularized reconstruction
// shared by every kernel of liblbm (device code, sm_103a).
//
// Method: Brogi et al., arXiv:1710.02065, Sec. II.A.  A cell's populations
// are rebuilt from a small set of Hermite coefficients,
//     f_i = w_i [ a0 + xi_i . a1 / c_s^2 + H2_i : A2 / (2 c_s^4) + T3_i(A3) ]
// (Eq. HEeqAndNeq truncated to order 3, Eq. eqH + Eq. neqH), where
//   a0 = rho, a1 = rho u, A2 = rho u u (+ (1 - 1/tau) Pi^neq after collision),
//   A3 = rho u u u (Eq. recursive1) (+ (1 - 1/tau) a3_neq, Eq. recursive2).
// Populations are handled shifted, g_i = f_i - w_i (rho_0 = 1), so that
// a0 is replaced by rho - 1; sums of small numbers keep FP32 round-off low.
//
// Third order: on D2Q9 the supported components are xxy and xyy (H_xxx and
// H_yyy vanish on the lattice).  On D3Q19 the six a_aab components enter as
// the sum/difference pairs (xxy,yzz), (xzz,xyy), (yyz,xxz), each with the
// inverse of its lattice norm (2 c_s^6 for sums, 6 c_s^6 for differences), so
// the rebuilt populations carry exactly a_p + a_q and a_p - a_q.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rr {

// ---------------------------------------------------------------------------
// Lattices.  Direction 0 is the rest velocity; i and i + Q/2 (1 <= i <= Q/2)
// are opposite.  Weights by |xi|^2: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18,
// 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9, D = 2, HALF = 4;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[9] = {0, 1, 0, 1, -1, -1, 0, -1, 1};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3, HALF = 9;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[19] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[19] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int v[19] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
        return v[i];
    }
};

// The tensor product of D1Q3: the D3Q19 velocities plus the eight corners;
// every third-order Hermite polynomial but H_aaa is supported (H_xyz too).
struct D3Q27 {
    static constexpr int Q = 27, D = 3, HALF = 13;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[27] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 1, 1,
                               -1, 0, 0, -1, -1, -1, -1, 0, 0, -1, -1, -1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[27] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 1, 1, -1, -1,
                               0, -1, 0, -1, 1, 0, 0, -1, -1, -1, -1, 1, 1};
        return v[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int v[27] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1,
                               0, 0, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1};
        return v[i];
    }
};

// largest number of directions of a supported lattice (D3Q27)
constexpr int kMaxQ = 27;

// whether the lattice carries the complete third order (a_xyz as well)
template <class L>
__host__ __device__ constexpr bool full_third_order()
{
    return L::Q == 27;
}

template <class L>
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= L::HALF ? i + L::HALF : i - L::HALF);
}

template <class L>
__host__ __device__ constexpr double weight(int i)
{
    // |xi|^2 decides the weight class
    return L::Q == 27
               ? ((L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i)) == 0
                      ? 8.0 / 27.0
                      : ((L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i)) == 1
                             ? 2.0 / 27.0
                             : ((L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i)) == 2
                                    ? 1.0 / 54.0
                                    : 1.0 / 216.0)))
               : ((L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i)) == 0
                      ? (L::D == 2 ? 4.0 / 9.0 : 1.0 / 3.0)
                      : ((L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i)) == 1
                             ? (L::D == 2 ? 1.0 / 9.0 : 1.0 / 18.0)
                             : 1.0 / 36.0));
}

// ---------------------------------------------------------------------------
// Storage formats
// ---------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
    __device__ static double ld(const double *p) { return __ldg(p); }
    __device__ static void st(double *p, double v) { *p = v; }
    template <class C>
    __device__ static C to(double v) { return (C)v; }
    __device__ static double from(double v) { return v; }
    __device__ static double from(float v) { return (double)v; }
};
template <>
struct Store<float> {
    __device__ static float ld(const float *p) { return __ldg(p); }
    __device__ static void st(float *p, float v) { *p = v; }
    __device__ static float from(float v) { return v; }
    __device__ static float from(double v) { return (float)v; }
};
// 16-bit formats are moved as raw 16-bit words through the plain read-only
// load path and converted in registers (bf16 -> f32 is a 16-bit shift).
template <>
struct Store<__half> {
    __device__ static float ld(const __half *p)
    {
        const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p));
        return __half2float(__ushort_as_half(b));
    }
    __device__ static void st(__half *p, float v)
    {
        *reinterpret_cast<unsigned short *>(p) = __half_as_ushort(__float2half_rn(v));
    }
    __device__ static __half from(float v) { return __float2half_rn(v); }
    __device__ static __half from(double v) { return __double2half(v); }
};
template <>
struct Store<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16 *p)
    {
        const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p));
        return __uint_as_float((unsigned)b << 16);
    }
    __device__ static void st(__nv_bfloat16 *p, float v)
    {
        *reinterpret_cast<unsigned short *>(p) = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    __device__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    __device__ static __nv_bfloat16 from(double v) { return __double2bfloat16(v); }
};

// ---------------------------------------------------------------------------
// Fused multiply-add a * b + c with one rounding, written out so that every
// kernel performs the same operations in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

// Device cell-type byte: bits 0-1 the cell type (0 fluid, 1 solid wall,
// 2 fixed), bit 2 set when a lattice neighbour is a solid wall.
constexpr uint8_t MASK_TYPE = 3, MASK_SOLID = 1, MASK_NEAR_SOLID = 4;

// compute type a storage format is written from
template <class S>
struct StoreC {
    using C = float;
};
template <>
struct StoreC<double> {
    using C = double;
};

// ---------------------------------------------------------------------------
// Moments of shifted populations g_i = f_i - w_i:
//   dr = rho - 1, j = rho u, s_ab = Pi_ab - c_s^2 delta_ab   (Eq. moments)
// ---------------------------------------------------------------------------
template <class C>
struct Mom {
    C dr, jx, jy, jz, sxx, syy, szz, sxy, sxz, syz;
};

template <class L, class C>
__device__ __forceinline__ Mom<C> moments(const C (&g)[L::Q])
{
    Mom<C> m{};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
        m.dr += g[i];
        if (x) m.jx += x > 0 ? g[i] : -g[i];
        if (y) m.jy += y > 0 ? g[i] : -g[i];
        if (z) m.jz += z > 0 ? g[i] : -g[i];
        if (x) m.sxx += g[i];
        if (y) m.syy += g[i];
        if (z) m.szz += g[i];
        if (x && y) m.sxy += x * y > 0 ? g[i] : -g[i];
        if (x && z) m.sxz += x * z > 0 ? g[i] : -g[i];
        if (y && z) m.syz += y * z > 0 ? g[i] : -g[i];
    }
    return m;
}

// ---------------------------------------------------------------------------
// Hermite coefficients of a rebuilt cell (shifted form)
//   a0 = rho - 1, a1 = (jx, jy, jz), A2 (xx, yy, zz, xy, xz, yz),
//   A3 (xxy, xyy, xxz, xzz, yyz, yzz); the z ones are unused on D2Q9.
// ---------------------------------------------------------------------------
template <class C>
struct Coef {
    C a0, a1x, a1y, a1z;
    C xx, yy, zz, xy, xz, yz;
    C xxy, xyy, xxz, xzz, yyz, yzz;
    C xyz;   // D3Q27 only
    C xxyy;  // D2Q9 with the optional fourth order only
};

// Second-order symmetric tensor (xx, yy, zz, xy, xz, yz)
template <class C>
struct Sym2 {
    C xx, yy, zz, xy, xz, yz;
};

// Equilibrium coefficients of (rho, u), scaled by s: a0 += s (rho - 1),
// a1 += s rho u, A2 += s rho u u, A3 += s rho u u u.  dr = rho - 1 is passed
// separately so that it keeps its own precision.  O3 = false stops at second
// order: the quadratic equilibrium of the plain LBM-BGK (Eq. truncatedEq).
template <class C, int D = 3, bool O3 = true, bool XYZ = false>
__device__ __forceinline__ void add_eq(Coef<C> &k, C s, C dr, C rho, C ux, C uy, C uz, bool o4 = false)
{
    const C r = s * rho;
    k.a0 = fmac(s, dr, k.a0);
    const C rx = r * ux, ry = r * uy;
    k.a1x += rx;
    k.a1y += ry;
    k.xx = fmac(rx, ux, k.xx);
    k.yy = fmac(ry, uy, k.yy);
    k.xy = fmac(rx, uy, k.xy);
    const C rxx = rx * ux, ryy = ry * uy;
    if (O3) {
        k.xxy = fmac(rxx, uy, k.xxy);
        k.xyy = fmac(ryy, ux, k.xyy);
    }
    // optional fourth order on D2Q9: a4_xxyy = rho u_x^2 u_y^2 (Eq. recursive1)
    if (D == 2 && O3 && o4) k.xxyy = fmac(rxx, uy * uy, k.xxyy);
    if (D == 3) {
        const C rz = r * uz;
        k.a1z += rz;
        k.zz = fmac(rz, uz, k.zz);
        k.xz = fmac(rx, uz, k.xz);
        k.yz = fmac(ry, uz, k.yz);
        if (!O3) return;
        const C rzz = rz * uz;
        k.xxz = fmac(rxx, uz, k.xxz);
        k.xzz = fmac(rzz, ux, k.xzz);
        k.yyz = fmac(ryy, uz, k.yyz);
        k.yzz = fmac(rzz, uy, k.yzz);
        if (XYZ) k.xyz = fmac(rx * uy, uz, k.xyz);
    }
}

// Off-equilibrium coefficients scaled by s: A2 += s Pi^neq and
// A3 += s a3_neq, a3_neq,abc = u_a P_bc + u_b P_ac + u_c P_ab (Eq. recursive2, n = 3);
// O3 = false: A2 only.
template <class C, int D = 3, bool O3 = true, bool XYZ = false>
__device__ __forceinline__ void add_neq(Coef<C> &k, C s, C ux, C uy, C uz, const Sym2<C> &p, bool o4 = false)
{
    k.xx = fmac(s, p.xx, k.xx);
    k.yy = fmac(s, p.yy, k.yy);
    k.xy = fmac(s, p.xy, k.xy);
    if (!O3) {
        if (D == 3) {
            k.zz = fmac(s, p.zz, k.zz);
            k.xz = fmac(s, p.xz, k.xz);
            k.yz = fmac(s, p.yz, k.yz);
        }
        return;
    }
    const C ux2 = ux + ux, uy2 = uy + uy;
    k.xxy = fmac(s, fmac(ux2, p.xy, uy * p.xx), k.xxy);
    k.xyy = fmac(s, fmac(uy2, p.xy, ux * p.yy), k.xyy);
    // optional fourth order on D2Q9, Eq. recursive2 at n = 4 as the symmetric
    // sum over index pairs: a4_xxyy = u_x^2 P_yy + u_y^2 P_xx + 4 u_x u_y P_xy
    if (D == 2 && o4)
        k.xxyy = fmac(s, fmac(ux * ux, p.yy, fmac(uy * uy, p.xx, C(4) * ux * uy * p.xy)), k.xxyy);
    if (D == 3) {
        const C uz2 = uz + uz;
        k.zz = fmac(s, p.zz, k.zz);
        k.xz = fmac(s, p.xz, k.xz);
        k.yz = fmac(s, p.yz, k.yz);
        k.xxz = fmac(s, fmac(ux2, p.xz, uz * p.xx), k.xxz);
        k.xzz = fmac(s, fmac(uz2, p.xz, ux * p.zz), k.xzz);
        k.yyz = fmac(s, fmac(uy2, p.yz, uz * p.yy), k.yyz);
        k.yzz = fmac(s, fmac(uz2, p.yz, uy * p.zz), k.yzz);
        // a3_neq,xyz = u_x P_yz + u_y P_xz + u_z P_xy
        if (XYZ) k.xyz = fmac(s, fmac(ux, p.yz, fmac(uy, p.xz, uz * p.xy)), k.xyz);
    }
}

// g_i = w_i [ a0 + 3 xi.a1 + 4.5 H2_i:A2 + T3_i(A3) ]   (c_s^2 = 1/3)
template <class L, class C>
__device__ __forceinline__ C rebuild(const Coef<C> &k, int i)
{
    constexpr double cs2 = 1.0 / 3.0;
    const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
    C r = k.a0;
    // first order: xi . a1 / c_s^2
    C f1 = C(0);
    if (x) f1 += x > 0 ? k.a1x : -k.a1x;
    if (y) f1 += y > 0 ? k.a1y : -k.a1y;
    if (z) f1 += z > 0 ? k.a1z : -k.a1z;
    r += C(3) * f1;
    // second order: H2 : A2 / (2 c_s^4), H2_ab = xi_a xi_b - c_s^2 delta_ab
    C f2 = C(x * x - cs2) * k.xx + C(y * y - cs2) * k.yy;
    if (L::D == 3) f2 += C(z * z - cs2) * k.zz;
    if (x * y) f2 += C(2 * x * y) * k.xy;
    if (L::D == 3 && x * z) f2 += C(2 * x * z) * k.xz;
    if (L::D == 3 && y * z) f2 += C(2 * y * z) * k.yz;
    r += C(4.5) * f2;
    // third order, H_aab = xi_a^2 xi_b - c_s^2 xi_b
    const double hxxy = (x * x - cs2) * y, hxyy = (y * y - cs2) * x;
    if (L::D == 2) {
        // 1 / (2 c_s^6) = 13.5
        if (hxxy != 0.0) r += C(13.5 * hxxy) * k.xxy;
        if (hxyy != 0.0) r += C(13.5 * hxyy) * k.xyy;
        // optional fourth order: H_xxyy / (4 c_s^8) = 20.25 H_xxyy (zero coefficient otherwise)
        r += C(20.25 * (x * x - cs2) * (y * y - cs2)) * k.xxyy;
    } else if (full_third_order<L>()) {
        // every H_aab with 1 / (2 c_s^6) = 13.5, H_xyz with 1 / c_s^6 = 27
        const double hyzz = (z * z - cs2) * y, hxzz = (z * z - cs2) * x;
        const double hyyz = (y * y - cs2) * z, hxxz = (x * x - cs2) * z;
        if (hxxy != 0.0) r += C(13.5 * hxxy) * k.xxy;
        if (hxyy != 0.0) r += C(13.5 * hxyy) * k.xyy;
        if (hxxz != 0.0) r += C(13.5 * hxxz) * k.xxz;
        if (hxzz != 0.0) r += C(13.5 * hxzz) * k.xzz;
        if (hyyz != 0.0) r += C(13.5 * hyyz) * k.yyz;
        if (hyzz != 0.0) r += C(13.5 * hyzz) * k.yzz;
        if (x * y * z != 0) r += C(27.0 * x * y * z) * k.xyz;
    } else {
        const double hyzz = (z * z - cs2) * y, hxzz = (z * z - cs2) * x;
        const double hyyz = (y * y - cs2) * z, hxxz = (x * x - cs2) * z;
        // pairs (xxy, yzz), (xzz, xyy), (yyz, xxz); 1/(2 c_s^6) = 13.5, 1/(6 c_s^6) = 4.5
        const double p1 = hxxy + hyzz, m1 = hxxy - hyzz;
        const double p2 = hxzz + hxyy, m2 = hxzz - hxyy;
        const double p3 = hyyz + hxxz, m3 = hyyz - hxxz;
        if (p1 != 0.0) r += C(13.5 * p1) * (k.xxy + k.yzz);
        if (m1 != 0.0) r += C(4.5 * m1) * (k.xxy - k.yzz);
        if (p2 != 0.0) r += C(13.5 * p2) * (k.xzz + k.xyy);
        if (m2 != 0.0) r += C(4.5 * m2) * (k.xzz - k.xyy);
        if (p3 != 0.0) r += C(13.5 * p3) * (k.yyz + k.xxz);
        if (m3 != 0.0) r += C(4.5 * m3) * (k.yyz - k.xxz);
    }
    return C(weight<L>(i)) * r;
}

// Pi^neq about (rho, u) from shifted moments, dr = rho - 1:
//   s_ab - dr c_s^2 delta_ab - rho u_a u_b
template <class C>
__device__ __forceinline__ Sym2<C> pi_neq(const Mom<C> &m, C dr, C rho, C ux, C uy, C uz, int D)
{
    const C c = dr * C(1.0 / 3.0);
    const C rx = -(rho * ux), ry = -(rho * uy);
    Sym2<C> p;
    p.xx = fmac(rx, ux, m.sxx - c);
    p.yy = fmac(ry, uy, m.syy - c);
    p.xy = fmac(rx, uy, m.sxy);
    if (D == 3) {
        const C rz = -(rho * uz);
        p.zz = fmac(rz, uz, m.szz - c);
        p.xz = fmac(rx, uz, m.sxz);
        p.yz = fmac(ry, uz, m.syz);
    } else {
        p.zz = p.xz = p.yz = C(0);
    }
    return p;
}

// ---------------------------------------------------------------------------
// Moments from direction pairs: s = g_i + g_opp (even), d = g_i - g_opp (odd)
// (Eq. moments).  D2Q9 and D3Q19 are written out so that partial sums shared
// by several moments are formed once (the compiler may not reassociate
// floating-point sums); D3Q27 uses the generic loop over the pairs.
// ---------------------------------------------------------------------------
template <class L, class C>
__device__ __forceinline__ Mom<C> moments_pairs(const C *g)
{
    Mom<C> m;
    if constexpr (L::Q == 19) {
        // pairs 1 (1,0,0) 2 (0,1,0) 3 (0,0,1) 4 (1,1,0) 5 (1,-1,0)
        //       6 (1,0,1) 7 (1,0,-1) 8 (0,1,1) 9 (0,1,-1)
        C s[10], d[10];
#pragma unroll
        for (int i = 1; i <= 9; ++i) {
            s[i] = g[i] + g[i + 9];
            d[i] = g[i] - g[i + 9];
        }
        const C a = s[4] + s[5], b = s[6] + s[7], c = s[8] + s[9];
        m.dr = ((g[0] + s[1]) + (s[2] + s[3])) + ((a + b) + c);
        m.jx = (d[1] + (d[4] + d[5])) + (d[6] + d[7]);
        m.jy = (d[2] + (d[4] - d[5])) + (d[8] + d[9]);
        m.jz = (d[3] + (d[6] - d[7])) + (d[8] - d[9]);
        m.sxx = (s[1] + a) + b;
        m.syy = (s[2] + a) + c;
        m.szz = (s[3] + b) + c;
        m.sxy = s[4] - s[5];
        m.sxz = s[6] - s[7];
        m.syz = s[8] - s[9];
    } else if constexpr (L::Q == 9) {
        // pairs 1 (1,0) 2 (0,1) 3 (1,1) 4 (-1,1)
        const C s1 = g[1] + g[5], s2 = g[2] + g[6], s3 = g[3] + g[7], s4 = g[4] + g[8];
        const C d1 = g[1] - g[5], d2 = g[2] - g[6], d3 = g[3] - g[7], d4 = g[4] - g[8];
        const C a = s3 + s4;
        m.dr = (g[0] + s1) + (s2 + a);
        m.jx = d1 + (d3 - d4);
        m.jy = d2 + (d3 + d4);
        m.jz = C(0);
        m.sxx = s1 + a;
        m.syy = s2 + a;
        m.szz = C(0);
        m.sxy = s3 - s4;
        m.sxz = m.syz = C(0);
    } else {
        m = Mom<C>{};
        m.dr = g[0];
#pragma unroll
        for (int i = 1; i <= L::HALF; ++i) {
            const C s = g[i] + g[i + L::HALF], d = g[i] - g[i + L::HALF];
            const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
            m.dr += s;
            if (x) m.jx = x > 0 ? m.jx + d : m.jx - d;
            if (y) m.jy = y > 0 ? m.jy + d : m.jy - d;
            if (z) m.jz = z > 0 ? m.jz + d : m.jz - d;
            if (x) m.sxx += s;
            if (y) m.syy += s;
            if (z) m.szz += s;
            if (x && y) m.sxy = x * y > 0 ? m.sxy + s : m.sxy - s;
            if (x && z) m.sxz = x * z > 0 ? m.sxz + s : m.sxz - s;
            if (y && z) m.syz = y * z > 0 ? m.syz + s : m.syz - s;
        }
    }
    return m;
}

// ---------------------------------------------------------------------------
// Reconstruction g_i = w_i [a0 + 3 xi.a1 + 4.5 H2_i:A2 + T3_i(A3)] for the
// opposite pair (i, i + HALF): the even part E (a0 and second order) is
// shared, the odd part O (first and third order) changes sign, so
// g_i = w_i E + w_i O and g_opp = w_i E - w_i O, with w_i folded into the
// constants.  The second order uses the trace form
//   H2_i:A2 = sum_a xi_a^2 A_aa - tr(A2) / 3 + 2 sum_{a<b} xi_a xi_b A_ab
// (c_s^2 = 1/3), so a face direction needs A_aa - tr/3 and the two edge
// directions of a plane share A_aa + A_bb - tr/3.
// ---------------------------------------------------------------------------
template <class C>
struct RebuildPre {
    C tr3;             // tr(A2) / 3
    C wa1, wa2, wa3;   // w a0 for the directions with one / two / three non-zero components
    C bxy, bxz, byz;   // A_aa + A_bb - tr / 3 of the three coordinate planes
    C s1, d1, s2, d2, s3, d3;  // third-order pair sums / differences (D3Q19)
};

template <class L, class C>
__device__ __forceinline__ RebuildPre<C> rebuild_prep(const Coef<C> &k)
{
    // weight classes by |xi|^2 = 1 (direction 1 on every lattice), 2 and 3
    // (D3Q27 corners)
    RebuildPre<C> r;
    C tr = k.xx + k.yy;
    if (L::D == 3) tr += k.zz;
    r.tr3 = tr * C(1.0 / 3.0);
    r.wa1 = C(weight<L>(1)) * k.a0;
    r.wa2 = C(full_third_order<L>() ? 1.0 / 54.0 : 1.0 / 36.0) * k.a0;
    r.wa3 = full_third_order<L>() ? C(1.0 / 216.0) * k.a0 : C(0);
    r.bxy = (k.xx + k.yy) - r.tr3;
    if (L::D == 3) {
        r.bxz = (k.xx + k.zz) - r.tr3;
        r.byz = (k.yy + k.zz) - r.tr3;
        r.s1 = k.xxy + k.yzz; r.d1 = k.xxy - k.yzz;
        r.s2 = k.xzz + k.xyy; r.d2 = k.xzz - k.xyy;
        r.s3 = k.yyz + k.xxz; r.d3 = k.yyz - k.xxz;
    } else {
        r.bxz = r.byz = r.s1 = r.d1 = r.s2 = r.d2 = r.s3 = r.d3 = C(0);
    }
    return r;
}

// g_i (plus) and g_opp(i) (minus) of the pair of direction i (1 <= i <= HALF)
template <class L, class C>
__device__ __forceinline__ void rebuild_pair(const Coef<C> &k, const RebuildPre<C> &r, int i, C &plus, C &minus)
{
    constexpr double cs2 = 1.0 / 3.0;
    const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
    const double w = weight<L>(i);
    const int nnz = (x != 0) + (y != 0) + (z != 0);
    // second order
    C f2;
    if (nnz == 1) {
        f2 = (x ? k.xx : (y ? k.yy : k.zz)) - r.tr3;
    } else if (nnz == 2) {
        const C base = (x && y) ? r.bxy : ((x && z) ? r.bxz : r.byz);
        const C off = (x && y) ? k.xy : ((x && z) ? k.xz : k.yz);
        f2 = fmac(C(2 * x * y + 2 * x * z + 2 * y * z), off, base);
    } else {
        // corner (D3Q27): tr - tr/3 + 2 (xy A_xy + xz A_xz + yz A_yz)
        f2 = fmac(C(2 * x * y), k.xy, fmac(C(2 * x * z), k.xz, fmac(C(2 * y * z), k.yz, r.tr3 + r.tr3)));
    }
    C E = fmac(C(4.5 * w), f2, nnz == 1 ? r.wa1 : (nnz == 2 ? r.wa2 : r.wa3));
    // optional fourth order on D2Q9 (even): 20.25 w H_xxyy a4_xxyy; zero coefficient otherwise
    if (L::D == 2) E = fmac(C(20.25 * w * (x * x - cs2) * (y * y - cs2)), k.xxyy, E);
    // first order over the non-zero components
    C f1;
    if (x) f1 = x > 0 ? k.a1x : -k.a1x;
    if (y) f1 = x ? (y > 0 ? f1 + k.a1y : f1 - k.a1y) : (y > 0 ? k.a1y : -k.a1y);
    if (z) f1 = (x || y) ? (z > 0 ? f1 + k.a1z : f1 - k.a1z) : (z > 0 ? k.a1z : -k.a1z);
    C o = C(3.0 * w) * f1;
    // third order, H_aab = xi_a^2 xi_b - c_s^2 xi_b
    const double hxxy = (x * x - cs2) * y, hxyy = (y * y - cs2) * x;
    if (L::D == 2) {
        // 1 / (2 c_s^6) = 13.5
        if (hxxy != 0.0) o = fmac(C(13.5 * w * hxxy), k.xxy, o);
        if (hxyy != 0.0) o = fmac(C(13.5 * w * hxyy), k.xyy, o);
    } else if (full_third_order<L>()) {
        // D3Q27: every H_aab with 1/(2 c_s^6) = 13.5, H_xyz with 1/c_s^6 = 27
        const double hyzz = (z * z - cs2) * y, hxzz = (z * z - cs2) * x;
        const double hyyz = (y * y - cs2) * z, hxxz = (x * x - cs2) * z;
        if (hxxy != 0.0) o = fmac(C(13.5 * w * hxxy), k.xxy, o);
        if (hxyy != 0.0) o = fmac(C(13.5 * w * hxyy), k.xyy, o);
        if (hxxz != 0.0) o = fmac(C(13.5 * w * hxxz), k.xxz, o);
        if (hxzz != 0.0) o = fmac(C(13.5 * w * hxzz), k.xzz, o);
        if (hyyz != 0.0) o = fmac(C(13.5 * w * hyyz), k.yyz, o);
        if (hyzz != 0.0) o = fmac(C(13.5 * w * hyzz), k.yzz, o);
        if (x * y * z != 0) o = fmac(C(27.0 * w * x * y * z), k.xyz, o);
    } else {
        // pairs (xxy, yzz), (xzz, xyy), (yyz, xxz); 1/(2 c_s^6) = 13.5, 1/(6 c_s^6) = 4.5
        const double hyzz = (z * z - cs2) * y, hxzz = (z * z - cs2) * x;
        const double hyyz = (y * y - cs2) * z, hxxz = (x * x - cs2) * z;
        const double p1 = hxxy + hyzz, m1 = hxxy - hyzz;
        const double p2 = hxzz + hxyy, m2 = hxzz - hxyy;
        const double p3 = hyyz + hxxz, m3 = hyyz - hxxz;
        if (p1 != 0.0) o = fmac(C(13.5 * w * p1), r.s1, o);
        if (m1 != 0.0) o = fmac(C(4.5 * w * m1), r.d1, o);
        if (p2 != 0.0) o = fmac(C(13.5 * w * p2), r.s2, o);
        if (m2 != 0.0) o = fmac(C(4.5 * w * m2), r.d2, o);
        if (p3 != 0.0) o = fmac(C(13.5 * w * p3), r.s3, o);
        if (m3 != 0.0) o = fmac(C(4.5 * w * m3), r.d3, o);
    }
    plus = E + o;
    minus = E - o;
}

// Rest population: w_0 (a0 - c_s^2 tr(A2) / (2 c_s^4)) = w_0 a0 - 4.5 w_0 tr / 3
template <class L, class C>
__device__ __forceinline__ C rebuild_rest(const Coef<C> &k, const RebuildPre<C> &r)
{
    const C g0 = fmac(C(-4.5 * weight<L>(0)), r.tr3, C(weight<L>(0)) * k.a0);
    // optional fourth order on D2Q9: H_xxyy(0) = c_s^4 = 1/9
    return L::D == 2 ? fmac(C(20.25 * weight<L>(0) / 9.0), k.xxyy, g0) : g0;
}

// Reciprocal used for 1 / rho: the fast single-precision division intrinsic
// in FP32 (a few ulp; the FP32 path's tolerance is 1e-5), IEEE in FP64.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// ---------------------------------------------------------------------------
// All Q rebuilt populations of one cell, o[i] = w_i [a0 + 3 xi.a1 + 4.5 H2_i:A2
// + T3_i(A3)] in the lattice's direction order.  D2Q9 and D3Q19 are written
// out with the weights folded into the constants and the sums shared by an
// opposite pair (even part E, odd part O: o_i = E + O, o_opp = E - O) or by
// the two pairs of a coordinate plane formed once.  With the D3Q19 pairing
// of the third order (sums / differences of (xxy, yzz), (xzz, xyy),
// (yyz, xxz) over their lattice norms) the third-order part of a direction
// reduces to
//   face s e_a:            -9 w1 s T_a   (T_x = A_xyy + A_xzz,
//                                         T_y = A_xxy + A_yzz, T_z = A_xxz + A_yyz),
//   edge s_a e_a + s_b e_b:  9 w2 (s_b A_aab + s_a A_abb),
// which is what the pair sums and differences of rebuild_pair evaluate to.
// O4 = false drops the optional fourth-order D2Q9 term.  D3Q27 uses the
// generic pair rebuild.
// ---------------------------------------------------------------------------
template <class L, class C, bool O4 = true>
__device__ __forceinline__ void rebuild_all(const Coef<C> &k, C *o)
{
    if constexpr (L::Q == 19) {
        // w0 = 1/3, w1 = 1/18, w2 = 1/36; 4.5 w1 = 1/4, 4.5 w2 = 1/8, 9 w2 = 1/4
        const C tr = (k.xx + k.yy) + k.zz;
        const C tr3 = tr * C(1.0 / 3.0), t23 = tr - tr3;
        o[0] = fmac(C(-1.5), tr3, C(1.0 / 3.0) * k.a0);
        const C wa1 = C(1.0 / 18.0) * k.a0, wa2 = C(1.0 / 36.0) * k.a0;
        // faces: E = w1 a0 + (A_aa - tr/3) / 4, O = a1_a / 6 - T_a / 2
        {
            const C E = fmac(C(0.25), k.xx - tr3, wa1);
            const C O = fmac(C(-0.5), k.xzz + k.xyy, C(1.0 / 6.0) * k.a1x);
            o[1] = E + O;
            o[10] = E - O;
        }
        {
            const C E = fmac(C(0.25), k.yy - tr3, wa1);
            const C O = fmac(C(-0.5), k.xxy + k.yzz, C(1.0 / 6.0) * k.a1y);
            o[2] = E + O;
            o[11] = E - O;
        }
        {
            const C E = fmac(C(0.25), k.zz - tr3, wa1);
            const C O = fmac(C(-0.5), k.yyz + k.xxz, C(1.0 / 6.0) * k.a1z);
            o[3] = E + O;
            o[12] = E - O;
        }
        // edges: a1 / 12 shared by the three planes
        const C jx = C(1.0 / 12.0) * k.a1x, jy = C(1.0 / 12.0) * k.a1y, jz = C(1.0 / 12.0) * k.a1z;
        {  // xy plane: 4 (1,1,0) / 13, 5 (1,-1,0) / 14
            const C base = fmac(C(0.125), t23 - k.zz, wa2);
            const C Ep = fmac(C(0.25), k.xy, base), Em = fmac(C(-0.25), k.xy, base);
            const C Op = fmac(C(0.25), k.xxy + k.xyy, jx + jy);
            const C Om = fmac(C(0.25), k.xyy - k.xxy, jx - jy);
            o[4] = Ep + Op;
            o[13] = Ep - Op;
            o[5] = Em + Om;
            o[14] = Em - Om;
        }
        {  // xz plane: 6 (1,0,1) / 15, 7 (1,0,-1) / 16
            const C base = fmac(C(0.125), t23 - k.yy, wa2);
            const C Ep = fmac(C(0.25), k.xz, base), Em = fmac(C(-0.25), k.xz, base);
            const C Op = fmac(C(0.25), k.xzz + k.xxz, jx + jz);
            const C Om = fmac(C(0.25), k.xzz - k.xxz, jx - jz);
            o[6] = Ep + Op;
            o[15] = Ep - Op;
            o[7] = Em + Om;
            o[16] = Em - Om;
        }
        {  // yz plane: 8 (0,1,1) / 17, 9 (0,1,-1) / 18
            const C base = fmac(C(0.125), t23 - k.xx, wa2);
            const C Ep = fmac(C(0.25), k.yz, base), Em = fmac(C(-0.25), k.yz, base);
            const C Op = fmac(C(0.25), k.yzz + k.yyz, jy + jz);
            const C Om = fmac(C(0.25), k.yzz - k.yyz, jy - jz);
            o[8] = Ep + Op;
            o[17] = Ep - Op;
            o[9] = Em + Om;
            o[18] = Em - Om;
        }
    } else if constexpr (L::Q == 9) {
        // w0 = 4/9, w1 = 1/9, w2 = 1/36; H_xxyy / (4 c_s^8) weighted: rest 1,
        // faces -1/2, diagonals 1/4 (zero coefficient unless fourth order)
        const C tr = k.xx + k.yy;
        const C tr3 = tr * C(1.0 / 3.0);
        C g0 = fmac(C(-2.0), tr3, C(4.0 / 9.0) * k.a0);
        if (O4) g0 = g0 + k.xxyy;
        o[0] = g0;
        const C wa1 = C(1.0 / 9.0) * k.a0, wa2 = C(1.0 / 36.0) * k.a0;
        {  // 1 (1,0) / 5
            C E = fmac(C(0.5), k.xx - tr3, wa1);
            if (O4) E = fmac(C(-0.5), k.xxyy, E);
            const C O = fmac(C(-0.5), k.xyy, C(1.0 / 3.0) * k.a1x);
            o[1] = E + O;
            o[5] = E - O;
        }
        {  // 2 (0,1) / 6
            C E = fmac(C(0.5), k.yy - tr3, wa1);
            if (O4) E = fmac(C(-0.5), k.xxyy, E);
            const C O = fmac(C(-0.5), k.xxy, C(1.0 / 3.0) * k.a1y);
            o[2] = E + O;
            o[6] = E - O;
        }
        {  // 3 (1,1) / 7, 4 (-1,1) / 8
            C base = fmac(C(0.125), tr - tr3, wa2);
            if (O4) base = fmac(C(0.25), k.xxyy, base);
            const C jx = C(1.0 / 12.0) * k.a1x, jy = C(1.0 / 12.0) * k.a1y;
            const C Ep = fmac(C(0.25), k.xy, base), Em = fmac(C(-0.25), k.xy, base);
            const C Op = fmac(C(0.25), k.xxy + k.xyy, jx + jy);
            const C Om = fmac(C(0.25), k.xxy - k.xyy, jy - jx);
            o[3] = Ep + Op;
            o[7] = Ep - Op;
            o[4] = Em + Om;
            o[8] = Em - Om;
        }
    } else {
        const RebuildPre<C> r = rebuild_prep<L, C>(k);
        o[0] = rebuild_rest<L, C>(k, r);
#pragma unroll
        for (int i = 1; i <= L::HALF; ++i) rebuild_pair<L, C>(k, r, i, o[i], o[i + L::HALF]);
    }
}

// ---------------------------------------------------------------------------
// Collision coefficients of an interior cell (no boundary role) of the
// rrBGK update, Eq. optimizedLB: a0 = rho - 1, a1 = j, with
//   P_ab = j_a u_b (= rho u_a u_b),  Pi^neq_ab = s_ab - (rho - 1) c_s^2 d_ab - P_ab,
//   A2 = P + w Pi^neq (w = 1 - 1/tau),
//   A3_aab = a3_eq + w a3_neq = P_aa u_b + w (2 u_a Pi^neq_ab + u_b Pi^neq_aa)
//          = u_b A2_aa + 2 u_a (w Pi^neq_ab)                  (Eq. recursive1/2),
// and the optional fourth-order D2Q9 term a4 = P_xx u_y^2 + w (u_x^2 Pi_yy +
// u_y^2 Pi_xx + 4 u_x u_y Pi_xy).
// Sponge cells whose reference state is the rest state rho_ref = 1, u_ref = 0
// (Eq. spongeLB with Eq. dampingLBM, n = m = 1/2): the moments are damped,
// rho* - 1 = (rho - 1) h, j* = j h, h = 1 / (1 + chi / 2), the equilibrium part
// is scaled by 1 - chi and feqH(rho_ref, u_ref) is the rest state, zero in
// shifted form.  chi = 0 gives the bulk coefficients.
// ---------------------------------------------------------------------------
template <class L, class C, bool SPONGE>
__device__ __forceinline__ Coef<C> coef_interior(const Mom<C> &m, C om, C chi, bool o4 = false)
{
    Coef<C> k;
    C dr = m.dr, jx = m.jx, jy = m.jy, jz = m.jz, sc = C(1);
    if (SPONGE) {
        const C h = recip(fmac(C(0.5), chi, C(1)));
        dr = dr * h;
        jx = jx * h;
        jy = jy * h;
        jz = jz * h;
        sc = C(1) - chi;
    }
    const C inv = recip(C(1) + dr);
    const C ux = jx * inv, uy = jy * inv;
    const C c = dr * C(1.0 / 3.0);
    const C Pxx = jx * ux, Pyy = jy * uy, Pxy = jx * uy;
    const C nxx = (m.sxx - c) - Pxx, nyy = (m.syy - c) - Pyy;
    const C qxy = om * (m.sxy - Pxy);
    k.a0 = SPONGE ? sc * dr : dr;
    k.a1x = SPONGE ? sc * jx : jx;
    k.a1y = SPONGE ? sc * jy : jy;
    k.xx = fmac(om, nxx, SPONGE ? sc * Pxx : Pxx);
    k.yy = fmac(om, nyy, SPONGE ? sc * Pyy : Pyy);
    k.xy = fmac(SPONGE ? sc : C(1), Pxy, qxy);
    const C ux2 = ux + ux, uy2 = uy + uy;
    k.xxy = fmac(uy, k.xx, ux2 * qxy);
    k.xyy = fmac(ux, k.yy, uy2 * qxy);
    if constexpr (L::D == 3) {
        const C uz = jz * inv;
        const C Pzz = jz * uz, Pxz = jx * uz, Pyz = jy * uz;
        const C nzz = (m.szz - c) - Pzz;
        const C qxz = om * (m.sxz - Pxz), qyz = om * (m.syz - Pyz);
        k.a1z = SPONGE ? sc * jz : jz;
        k.zz = fmac(om, nzz, SPONGE ? sc * Pzz : Pzz);
        k.xz = fmac(SPONGE ? sc : C(1), Pxz, qxz);
        k.yz = fmac(SPONGE ? sc : C(1), Pyz, qyz);
        const C uz2 = uz + uz;
        k.xxz = fmac(uz, k.xx, ux2 * qxz);
        k.xzz = fmac(ux, k.zz, uz2 * qxz);
        k.yyz = fmac(uz, k.yy, uy2 * qyz);
        k.yzz = fmac(uy, k.zz, uz2 * qyz);
        if constexpr (full_third_order<L>()) {
            // A3_xyz = P_xy u_z (scaled) + w (u_x Pi_yz + u_y Pi_xz + u_z Pi_xy)
            //        = u_z A2_xy + u_x q_yz + u_y q_xz
            k.xyz = fmac(uz, k.xy, fmac(ux, qyz, uy * qxz));
        } else {
            k.xyz = C(0);
        }
        k.xxyy = C(0);
    } else {
        k.a1z = k.zz = k.xz = k.yz = C(0);
        k.xxz = k.xzz = k.yyz = k.yzz = k.xyz = C(0);
        k.xxyy = C(0);
        if (o4) {
            const C uxx = ux * ux, uyy = uy * uy;
            const C a4n = fmac(uxx, nyy, fmac(uyy, nxx, C(4) * ux * uy * (m.sxy - Pxy)));
            k.xxyy = fmac(om, a4n, (SPONGE ? sc * Pxx : Pxx) * uyy);
        }
    }
    return k;
}

// splitmix64 (Steele, Lea and Flood 2014): counter-based uniform in [0, 1)
__device__ __forceinline__ double u01(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// The same uniform in a collision precision: double as above, float from
// the leading 24 bits (u01 rounded down to a float)
template <class C>
__device__ __forceinline__ C u01c(uint64_t x);
template <>
__device__ __forceinline__ double u01c<double>(uint64_t x) { return u01(x); }
template <>
__device__ __forceinline__ float u01c<float>(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (float)(unsigned)(z >> 40) * (1.0f / 16777216.0f);
}

// Sponge profile (Sec. II.C): sigma(d) = 3125 (W - d) d^4 / (256 W^5), 0 <= d <= W
template <class C>
__device__ __forceinline__ C sigma(C d, C W)
{
    if (d < C(0) || d > W) return C(0);
    const C d2 = d * d, W2 = W * W;
    return C(3125) * (W - d) * d2 * d2 / (C(256) * W2 * W2 * W);
}

}  // namespace rr
