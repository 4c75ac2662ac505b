// refine.cuh -- 2:1 grid coupling kernels of a parent / child level pair (Sec. II.B, Eq. couplingCF,
// Eq. couplingFC), D2Q9, and D3Q19 / D3Q27 (the 3D kernels, templated on the
// lattice, are at the end of the file).
// Below, "coarse" is the parent level of a pair and "fine" its child; nested
// levels apply these kernels pair by pair.
//
// Layout (vertex based, dx_f = dx_c / 2, dt_f = dt_c / 2): the fine patch
// covers the coarse nodes X0..X0+Wc, Y0..Y0+Hc; fine node (i, j) sits at
// (X0 + i/2, Y0 + j/2).  The fine boundary ring is a fixed set of nodes
// rebuilt from coarse data after every fine substep; the first ring of
// covered coarse nodes is rebuilt from fine data after every coarse step;
// deeper covered coarse nodes are fixed and never read.
//
// Exchanged data are pre-collision moments (rho - 1, u, Pi^neq); a receiving
// node is rebuilt in post-collision form feqH(rho, u) + (1 - 1/tau) fneqH(u,
// alpha Pi^neq) with alpha = tau_f / (2 tau_c) coarse -> fine and
// 2 tau_c / tau_f fine -> coarse (leading-order Chapman-Enskog f^neq ~ tau
// dt grad u with dt_f = dt_c / 2).
//
//   k_line_moments : coarse moments on the four interface lines, extended by
//                    one node past each end (cubic stencils near corners)
//   k_fill_ring    : fine ring from line moments mixed in time ((1-a) M0 + a M1,
//                    a = 1/2 at the fine half step) and interpolated in space
//                    (copy at coincident nodes, (-1, 9, 9, -1)/16 at mid nodes)
//   k_restrict     : covered coarse ring from the coincident fine node's rho, u
//                    and its 3 x 3 full-weighted Pi^neq
#pragma once

#include "rr.cuh"

namespace rr {

struct RefineGeom {
    int X0, Y0, Wc, Hc;
    int nxc, nyc, nfx, nfy;
    // third axis of a 3D patch (zero / one for D2Q9)
    int Z0, Dc, nzc, nfz;
};

// number of line entries: two horizontal lines of Wc + 3, two vertical of Hc + 3
__host__ __device__ inline int line_count(const RefineGeom &g) { return 2 * (g.Wc + 3) + 2 * (g.Hc + 3); }

__device__ inline void line_coord(const RefineGeom &g, int e, int &x, int &y)
{
    const int nh = g.Wc + 3, nv = g.Hc + 3;
    if (e < nh) { x = g.X0 - 1 + e; y = g.Y0; }
    else if (e < 2 * nh) { x = g.X0 - 1 + (e - nh); y = g.Y0 + g.Hc; }
    else if (e < 2 * nh + nv) { x = g.X0; y = g.Y0 - 1 + (e - 2 * nh); }
    else { x = g.X0 + g.Wc; y = g.Y0 - 1 + (e - 2 * nh - nv); }
}

// entry of a coarse node on a horizontal line (top = 0/1) or vertical line (right = 0/1)
__device__ inline int entry_h(const RefineGeom &g, int x, int top) { return top * (g.Wc + 3) + (x - (g.X0 - 1)); }
__device__ inline int entry_v(const RefineGeom &g, int y, int right)
{
    return 2 * (g.Wc + 3) + right * (g.Hc + 3) + (y - (g.Y0 - 1));
}

// Arithmetic of the coupling runs in the storage format's compute type
// (FP32 for FP32/FP16/BF16 storage, FP64 for FP64); the interface moments
// are kept in FP64 arrays.
template <class S>
using CT = typename StoreC<S>::C;

// Pre-collision moments at node (x, y) of a 2D lattice: pull with periodic
// wrap and halfway bounce-back on mask == 1.  m = (rho - 1, ux, uy, Pxx, Pxy, Pyy).
template <class S>
__device__ void streamed_moments_2d(const S *__restrict__ f, const uint8_t *__restrict__ mask, int nx, int ny,
                                    int x, int y, CT<S> m[6])
{
    using C = CT<S>;
    const int64_t N = (int64_t)nx * ny;
    const int64_t cell = x + (int64_t)nx * y;
    C g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - D2Q9::cx(i), sy = y - D2Q9::cy(i);
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        const int64_t src = sx + (int64_t)nx * sy;
        if (mask && i != 0 && (mask[src] & MASK_TYPE) == MASK_SOLID)
            g[i] = Store<S>::ld(f + (int64_t)opp<D2Q9>(i) * N + cell);
        else
            g[i] = Store<S>::ld(f + (int64_t)i * N + src);
    }
    const Mom<C> mo = moments_pairs<D2Q9, C>(g);
    const C rho = C(1) + mo.dr;
    const C ux = mo.jx / rho, uy = mo.jy / rho;
    const Sym2<C> p = pi_neq<C>(mo, mo.dr, rho, ux, uy, C(0), 2);
    m[0] = mo.dr; m[1] = ux; m[2] = uy; m[3] = p.xx; m[4] = p.xy; m[5] = p.yy;
}

// Local (not streamed) moments of the stored populations at (x, y)
template <class S>
__device__ void local_moments_2d(const S *__restrict__ f, int nx, int ny, int x, int y, CT<S> m[6])
{
    using C = CT<S>;
    const int64_t N = (int64_t)nx * ny;
    const int64_t cell = x + (int64_t)nx * y;
    C g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = Store<S>::ld(f + (int64_t)i * N + cell);
    const Mom<C> mo = moments_pairs<D2Q9, C>(g);
    const C rho = C(1) + mo.dr;
    const C ux = mo.jx / rho, uy = mo.jy / rho;
    const Sym2<C> p = pi_neq<C>(mo, mo.dr, rho, ux, uy, C(0), 2);
    m[0] = mo.dr; m[1] = ux; m[2] = uy; m[3] = p.xx; m[4] = p.xy; m[5] = p.yy;
}

// Store feqH(rho, u) + omega fneqH(u, alpha Pi^neq) at a cell, omega = 1 - 1/tau
// (alpha and omega come from the host in the compute type)
template <class S>
__device__ void store_rebuilt_2d(S *__restrict__ f, int64_t N, int64_t cell, const CT<S> m[6], CT<S> alpha,
                                 CT<S> omega)
{
    using C = CT<S>;
    Coef<C> k{};
    const C rho = C(1) + m[0];
    add_eq<C, 2>(k, C(1), m[0], rho, m[1], m[2], C(0));
    Sym2<C> p;
    p.xx = alpha * m[3]; p.xy = alpha * m[4]; p.yy = alpha * m[5];
    p.zz = p.xz = p.yz = C(0);
    add_neq<C, 2>(k, omega, m[1], m[2], C(0), p);
    const RebuildPre<C> r = rebuild_prep<D2Q9, C>(k);
    Store<S>::st(f + cell, rebuild_rest<D2Q9, C>(k, r));
#pragma unroll
    for (int i = 1; i <= D2Q9::HALF; ++i) {
        C gp, gm;
        rebuild_pair<D2Q9, C>(k, r, i, gp, gm);
        Store<S>::st(f + (int64_t)i * N + cell, gp);
        Store<S>::st(f + (int64_t)(i + D2Q9::HALF) * N + cell, gm);
    }
}

template <class S>
__global__ void k_line_moments(RefineGeom g, const S *__restrict__ fc, const uint8_t *__restrict__ mask,
                               int streamed, CT<S> *__restrict__ M)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= line_count(g)) return;
    int x, y;
    line_coord(g, e, x, y);
    CT<S> m[6];
    if (streamed)
        streamed_moments_2d<S>(fc, mask, g.nxc, g.nyc, x, y, m);
    else
        local_moments_2d<S>(fc, g.nxc, g.nyc, x, y, m);
#pragma unroll
    for (int k = 0; k < 6; ++k) M[6 * e + k] = m[k];
}

template <class C>
__device__ inline void mix6(const C *__restrict__ M0, const C *__restrict__ M1, C a, int e, C out[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = (C(1) - a) * M0[6 * e + k] + a * M1[6 * e + k];
}

template <class S>
__global__ void k_fill_ring(RefineGeom g, const CT<S> *__restrict__ M0, const CT<S> *__restrict__ M1, CT<S> a,
                            CT<S> alpha, CT<S> omega, S *__restrict__ ff)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nfx = g.nfx, nfy = g.nfy;
    const int count = 2 * nfx + 2 * (nfy - 2);
    if (t >= count) return;
    int i, j;
    if (t < nfx) { i = t; j = 0; }
    else if (t < 2 * nfx) { i = t - nfx; j = nfy - 1; }
    else if (t < 2 * nfx + nfy - 2) { i = 0; j = 1 + t - 2 * nfx; }
    else { i = nfx - 1; j = 1 + t - 2 * nfx - (nfy - 2); }
    using C = CT<S>;
    const bool on_h = (j == 0 || j == nfy - 1);
    const C am = a;
    C m[6];
    if (on_h) {
        const int top = j == 0 ? 0 : 1;
        if ((i & 1) == 0) {
            mix6<C>(M0, M1, am, entry_h(g, g.X0 + i / 2, top), m);
        } else {
            const int xa = g.X0 + (i - 1) / 2;
            C t0[6], t1[6], t2[6], t3[6];
            mix6<C>(M0, M1, am, entry_h(g, xa - 1, top), t0);
            mix6<C>(M0, M1, am, entry_h(g, xa, top), t1);
            mix6<C>(M0, M1, am, entry_h(g, xa + 1, top), t2);
            mix6<C>(M0, M1, am, entry_h(g, xa + 2, top), t3);
#pragma unroll
            for (int k = 0; k < 6; ++k) m[k] = (-t0[k] + C(9) * t1[k] + C(9) * t2[k] - t3[k]) * C(0.0625);
        }
    } else {
        const int right = i == 0 ? 0 : 1;
        if ((j & 1) == 0) {
            mix6<C>(M0, M1, am, entry_v(g, g.Y0 + j / 2, right), m);
        } else {
            const int ya = g.Y0 + (j - 1) / 2;
            C t0[6], t1[6], t2[6], t3[6];
            mix6<C>(M0, M1, am, entry_v(g, ya - 1, right), t0);
            mix6<C>(M0, M1, am, entry_v(g, ya, right), t1);
            mix6<C>(M0, M1, am, entry_v(g, ya + 1, right), t2);
            mix6<C>(M0, M1, am, entry_v(g, ya + 2, right), t3);
#pragma unroll
            for (int k = 0; k < 6; ++k) m[k] = (-t0[k] + C(9) * t1[k] + C(9) * t2[k] - t3[k]) * C(0.0625);
        }
    }
    store_rebuilt_2d<S>(ff, (int64_t)nfx * nfy, i + (int64_t)nfx * j, m, alpha, omega);
}

template <class S>
__global__ void k_restrict(RefineGeom g, const S *__restrict__ ff_prev, const uint8_t *__restrict__ fmask,
                           CT<S> alpha, CT<S> omega, S *__restrict__ fc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = g.Wc - 1, h = g.Hc - 1;  // ring of the rectangle [X0+1, X0+Wc-1] x [Y0+1, Y0+Hc-1]
    const int count = 2 * w + 2 * (h - 2);
    if (t >= count) return;
    int x, y;
    if (t < w) { x = g.X0 + 1 + t; y = g.Y0 + 1; }
    else if (t < 2 * w) { x = g.X0 + 1 + (t - w); y = g.Y0 + g.Hc - 1; }
    else if (t < 2 * w + h - 2) { x = g.X0 + 1; y = g.Y0 + 2 + (t - 2 * w); }
    else { x = g.X0 + g.Wc - 1; y = g.Y0 + 2 + (t - 2 * w - (h - 2)); }
    using C = CT<S>;
    const int i = 2 * (x - g.X0), j = 2 * (y - g.Y0);
    const C w3[3] = {C(1), C(2), C(1)};
    C mc[6] = {C(0), C(0), C(0), C(0), C(0), C(0)}, m[6];
#pragma unroll
    for (int l = -1; l <= 1; ++l)
#pragma unroll
        for (int k = -1; k <= 1; ++k) {
            streamed_moments_2d<S>(ff_prev, fmask, g.nfx, g.nfy, i + k, j + l, m);
            const C wt = w3[k + 1] * w3[l + 1] * C(0.0625);
            mc[3] += wt * m[3];
            mc[4] += wt * m[4];
            mc[5] += wt * m[5];
            if (k == 0 && l == 0) { mc[0] = m[0]; mc[1] = m[1]; mc[2] = m[2]; }
        }
    store_rebuilt_2d<S>(fc, (int64_t)g.nxc * g.nyc, x + (int64_t)g.nxc * y, mc, alpha, omega);
}

// ===========================================================================
// D3Q19 and D3Q27 patches.  The fine patch covers the coarse nodes X0..X0+Wc,
// Y0..Y0+Hc, Z0..Z0+Dc; fine node (i, j, k) sits at (X0 + i/2, Y0 + j/2,
// Z0 + k/2).  The fine boundary shell is rebuilt from coarse data, the first
// shell of covered coarse nodes from fine data.  Interface moments m = (rho -
// 1, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz) of the coarse nodes on the six
// face planes of the patch box (extended by one node past every edge) are
// kept in a dense box array over [X0-1, X0+Wc+1] x [Y0-1, Y0+Hc+1] x
// [Z0-1, Z0+Dc+1] (10 values of the compute type per node; off-plane entries
// unused).
//   k_plane_moments3 : coarse moments on the six planes
//   k_fill_shell3    : fine shell from plane moments mixed in time and
//                      interpolated along every axis on which the fine node is
//                      odd by (-1, 9, 9, -1)/16 (tensor product on the planes)
//   k_restrict3      : covered coarse shell from the coincident fine node's
//                      rho, u and its (1,2,1)^3 / 64 full-weighted Pi^neq
// ===========================================================================
__host__ __device__ inline int64_t box3_entries(const RefineGeom &g)
{
    return (int64_t)(g.Wc + 3) * (g.Hc + 3) * (g.Dc + 3);
}
__device__ inline int64_t box3_index(const RefineGeom &g, int x, int y, int z)
{
    return (x - g.X0 + 1) + (int64_t)(g.Wc + 3) * ((y - g.Y0 + 1) + (int64_t)(g.Hc + 3) * (z - g.Z0 + 1));
}
// number of plane entries (edge nodes shared by two planes are listed twice)
__host__ __device__ inline int plane3_count(const RefineGeom &g)
{
    return 2 * (g.Hc + 3) * (g.Dc + 3) + 2 * (g.Wc + 3) * (g.Dc + 3) + 2 * (g.Wc + 3) * (g.Hc + 3);
}
__device__ inline void plane3_coord(const RefineGeom &g, int t, int &x, int &y, int &z)
{
    const int A = (g.Hc + 3) * (g.Dc + 3), B = (g.Wc + 3) * (g.Dc + 3);
    if (t < 2 * A) {
        const int side = t / A, r = t - side * A;
        x = g.X0 + side * g.Wc; y = g.Y0 - 1 + r % (g.Hc + 3); z = g.Z0 - 1 + r / (g.Hc + 3);
    } else if (t < 2 * A + 2 * B) {
        t -= 2 * A;
        const int side = t / B, r = t - side * B;
        y = g.Y0 + side * g.Hc; x = g.X0 - 1 + r % (g.Wc + 3); z = g.Z0 - 1 + r / (g.Wc + 3);
    } else {
        t -= 2 * A + 2 * B;
        const int Cn = (g.Wc + 3) * (g.Hc + 3);
        const int side = t / Cn, r = t - side * Cn;
        z = g.Z0 + side * g.Dc; x = g.X0 - 1 + r % (g.Wc + 3); y = g.Y0 - 1 + r / (g.Wc + 3);
    }
}

template <class C>
__device__ inline void pack_moments3(const Mom<C> &mo, C m[10])
{
    const C rho = C(1) + mo.dr;
    const C ux = mo.jx / rho, uy = mo.jy / rho, uz = mo.jz / rho;
    const Sym2<C> p = pi_neq<C>(mo, mo.dr, rho, ux, uy, uz, 3);
    m[0] = mo.dr; m[1] = ux; m[2] = uy; m[3] = uz;
    m[4] = p.xx; m[5] = p.xy; m[6] = p.xz; m[7] = p.yy; m[8] = p.yz; m[9] = p.zz;
}

// Pre-collision moments at (x, y, z) of a 3D lattice: pull with periodic
// wrap and halfway bounce-back on mask == 1.
template <class L, class S>
__device__ void streamed_moments_3d(const S *__restrict__ f, const uint8_t *__restrict__ mask, int nx, int ny,
                                    int nz, int x, int y, int z, CT<S> m[10])
{
    using C = CT<S>;
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
    C g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int sx = x - L::cx(i), sy = y - L::cy(i), sz = z - L::cz(i);
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
        const int64_t src = sx + (int64_t)nx * (sy + (int64_t)ny * sz);
        if (mask && i != 0 && (mask[src] & MASK_TYPE) == MASK_SOLID)
            g[i] = Store<S>::ld(f + (int64_t)opp<L>(i) * N + cell);
        else
            g[i] = Store<S>::ld(f + (int64_t)i * N + src);
    }
    pack_moments3<C>(moments_pairs<L, C>(g), m);
}

template <class L, class S>
__device__ void local_moments_3d(const S *__restrict__ f, int64_t N, int64_t cell, CT<S> m[10])
{
    using C = CT<S>;
    C g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) g[i] = Store<S>::ld(f + (int64_t)i * N + cell);
    pack_moments3<C>(moments_pairs<L, C>(g), m);
}

// Store feqH(rho, u) + omega fneqH(u, alpha Pi^neq) at a cell, omega = 1 - 1/tau
// (alpha and omega come from the host in the compute type: no FP64
// arithmetic on the device)
template <class L, class S>
__device__ void store_rebuilt_3d(S *__restrict__ f, int64_t N, int64_t cell, const CT<S> m[10], CT<S> alpha,
                                 CT<S> omega)
{
    using C = CT<S>;
    Coef<C> k{};
    const C rho = C(1) + m[0];
    add_eq<C, 3, true, full_third_order<L>()>(k, C(1), m[0], rho, m[1], m[2], m[3]);
    Sym2<C> p;
    p.xx = alpha * m[4]; p.xy = alpha * m[5]; p.xz = alpha * m[6];
    p.yy = alpha * m[7]; p.yz = alpha * m[8]; p.zz = alpha * m[9];
    add_neq<C, 3, true, full_third_order<L>()>(k, omega, m[1], m[2], m[3], p);
    const RebuildPre<C> r = rebuild_prep<L, C>(k);
    Store<S>::st(f + cell, rebuild_rest<L, C>(k, r));
#pragma unroll
    for (int i = 1; i <= L::HALF; ++i) {
        C gp, gm;
        rebuild_pair<L, C>(k, r, i, gp, gm);
        Store<S>::st(f + (int64_t)i * N + cell, gp);
        Store<S>::st(f + (int64_t)(i + L::HALF) * N + cell, gm);
    }
}

// Interface moments of the coarse plane nodes, stored in the compute type
// (10 per node: rho - 1, u, Pi^neq)
template <class L, class S>
__global__ void k_plane_moments3(RefineGeom g, const S *__restrict__ fc, const uint8_t *__restrict__ mask,
                                 int streamed, CT<S> *__restrict__ M)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane3_count(g)) return;
    int x, y, z;
    plane3_coord(g, t, x, y, z);
    CT<S> m[10];
    if (streamed)
        streamed_moments_3d<L, S>(fc, mask, g.nxc, g.nyc, g.nzc, x, y, z, m);
    else
        local_moments_3d<L, S>(fc, (int64_t)g.nxc * g.nyc * g.nzc, x + (int64_t)g.nxc * (y + (int64_t)g.nyc * z), m);
    const int64_t b = box3_index(g, x, y, z);
#pragma unroll
    for (int k = 0; k < 10; ++k) M[10 * b + k] = m[k];
}

// Point q of the 1D stencil of fine coordinate c on an axis with coarse
// origin o: the coincident node (even c, q = 0), or the centred cubic
// (-1, 9, 9, -1) / 16 between o + (c-1)/2 and o + (c+1)/2 (odd c, q = 0..3).
// No index arrays: a runtime index into a per-thread array would go through
// local memory.
template <class C>
__device__ inline void stencil_point(int c, int o, int q, int &idx, C &w)
{
    if ((c & 1) == 0) {
        idx = o + c / 2;
        w = C(1);
    } else {
        idx = o + (c - 1) / 2 - 1 + q;
        w = (q == 0 || q == 3) ? C(-0.0625) : C(0.5625);
    }
}

__host__ __device__ inline int shell3_count(int nx, int ny, int nz)
{
    return nx * ny * nz - (nx - 2) * (ny - 2) * (nz - 2);
}
// node t of the boundary shell of an nx x ny x nz box
__device__ inline void shell3_coord(int nx, int ny, int nz, int t, int &i, int &j, int &k)
{
    const int A = nx * ny, B = nx * (nz - 2);
    if (t < 2 * A) {
        const int side = t / A, r = t - side * A;
        k = side ? nz - 1 : 0; i = r % nx; j = r / nx;
    } else if (t < 2 * A + 2 * B) {
        t -= 2 * A;
        const int side = t / B, r = t - side * B;
        j = side ? ny - 1 : 0; i = r % nx; k = 1 + r / nx;
    } else {
        t -= 2 * A + 2 * B;
        const int Cn = (ny - 2) * (nz - 2);
        const int side = t / Cn, r = t - side * Cn;
        i = side ? nx - 1 : 0; j = 1 + r % (ny - 2); k = 1 + r / (ny - 2);
    }
}

// Fine shell node values at t + a (Sec. II.B, coarse to fine): the coarse
// plane moments interpolated linearly in time and by the tensor cubic in
// space, f^neq rescaled by alpha, rebuilt.  A shell node's stencil has 1, 4
// or 16 coarse points.  Four lanes take one node (lane r its points r, r + 4,
// r + 8, r + 12), the weighted moments are summed over the four by shuffles,
// and the node's first lane rebuilds and stores it: the loads are spread
// over more threads than one per node, while the rebuild is still shared by
// eight nodes per warp.
template <class L, class S>
__global__ void __launch_bounds__(256) k_fill_shell3(RefineGeom g, const CT<S> *__restrict__ M0,
                                                     const CT<S> *__restrict__ M1, CT<S> a, CT<S> alpha,
                                                     CT<S> omega, S *__restrict__ ff)
{
    using C = CT<S>;
    const int count = shell3_count(g.nfx, g.nfy, g.nfz);
    // block-strided over the nodes (every thread of a block takes the same
    // number of turns), so that a grid smaller than the work can leave room
    // on the SMs for a kernel running beside it
    for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x; b0 < 4 * (int64_t)count;
         b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gt = b0 + threadIdx.x;
        const int t = (int)(gt >> 2), r = (int)(gt & 3);
        const bool node = t < count;  // lanes past the last node still join the shuffles
        int i = 0, j = 0, k = 0;
        if (node) shell3_coord(g.nfx, g.nfy, g.nfz, t, i, j, k);
        // per axis: 1 point (even fine coordinate) or 4 (odd); lx = log2 of the count
        const int lx = (i & 1) << 1, ly = (j & 1) << 1, lz = (k & 1) << 1;
        const int npts = node ? 1 << (lx + ly + lz) : 0;
        const C am = a, bm = C(1) - a;
        C m[10];
#pragma unroll
        for (int e = 0; e < 10; ++e) m[e] = C(0);
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int q = r + 4 * s4;  // stencil point (qx, qy, qz) of the node's stencil
            if (q < npts) {
                const int qx = q & ((1 << lx) - 1), qy = (q >> lx) & ((1 << ly) - 1), qz = q >> (lx + ly);
                int cx, cy, cz;
                C wx, wy, wz;
                stencil_point<C>(i, g.X0, qx, cx, wx);
                stencil_point<C>(j, g.Y0, qy, cy, wy);
                stencil_point<C>(k, g.Z0, qz, cz, wz);
                const int64_t e0 = 10 * box3_index(g, cx, cy, cz);
                const C wt = wx * wy * wz;
                if (a == C(1)) {  // at t + 1 the moments at t do not enter (uniform: a kernel argument)
#pragma unroll
                    for (int e = 0; e < 10; ++e) m[e] = fmac(wt, M1[e0 + e], m[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < 10; ++e) m[e] = fmac(wt, bm * M0[e0 + e] + am * M1[e0 + e], m[e]);
                }
            }
        }
#pragma unroll
        for (int o = 2; o > 0; o >>= 1) {
#pragma unroll
            for (int e = 0; e < 10; ++e) m[e] += __shfl_xor_sync(0xffffffffu, m[e], o);
        }
        if (node && r == 0)
            store_rebuilt_3d<L, S>(ff, (int64_t)g.nfx * g.nfy * g.nfz, i + (int64_t)g.nfx * (j + (int64_t)g.nfy * k), m,
                                alpha, omega);
    }
}

// Covered coarse shell (Sec. II.B, fine to coarse): rho, u of the coincident
// fine node and the (1,2,1)^3 / 64 filtered Pi^neq of its 27 neighbours,
// rescaled by alpha, rebuilt.  One warp per coarse node: lane l < 27 pulls
// the streamed moments of stencil point l, the filtered sum is taken by
// shuffles, and the centre lane (13) supplies rho and u.
template <class L, class S>
__global__ void __launch_bounds__(256) k_restrict3(RefineGeom g, const S *__restrict__ ff_prev,
                                                   const uint8_t *__restrict__ fmask, CT<S> alpha, CT<S> omega,
                                                   S *__restrict__ fc)
{
    using C = CT<S>;
    const int w = g.Wc - 1, h = g.Hc - 1, d = g.Dc - 1;  // shell of [X0+1, X0+Wc-1] x ...
    const int count = shell3_count(w, h, d);
    // block-strided over the nodes, as k_fill_shell3
    for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x; b0 < 32 * (int64_t)count;
         b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gt = b0 + threadIdx.x;
        const int t = (int)(gt >> 5), l = (int)(gt & 31);
        const bool node = t < count;  // lanes past the last node still join the shuffles
        int a = 0, b = 0, c = 0;
        if (node) shell3_coord(w, h, d, t, a, b, c);
        const int x = g.X0 + 1 + a, y = g.Y0 + 1 + b, z = g.Z0 + 1 + c;
        const int i = 2 * (x - g.X0), j = 2 * (y - g.Y0), k = 2 * (z - g.Z0);
        C m[10];
#pragma unroll
        for (int e = 0; e < 10; ++e) m[e] = C(0);
        if (node && l < 27) {
            const int p = l % 3 - 1, q = (l / 3) % 3 - 1, r = l / 9 - 1;
            streamed_moments_3d<L, S>(ff_prev, fmask, g.nfx, g.nfy, g.nfz, i + p, j + q, k + r, m);
            const C wt = C((p ? 1 : 2) * (q ? 1 : 2) * (r ? 1 : 2)) * C(1.0 / 64.0);
#pragma unroll
            for (int e = 4; e < 10; ++e) m[e] *= wt;
        }
        C mc[10];
#pragma unroll
        for (int e = 0; e < 4; ++e) mc[e] = __shfl_sync(0xffffffffu, m[e], 13);
#pragma unroll
        for (int e = 4; e < 10; ++e) {
            C v = m[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            mc[e] = v;
        }
        if (node && l == 0)
            store_rebuilt_3d<L, S>(fc, (int64_t)g.nxc * g.nyc * g.nzc, x + (int64_t)g.nxc * (y + (int64_t)g.nyc * z), mc,
                                alpha, omega);
    }
}

}  // namespace rr
