// refine.cuh -- two-level 2:1 grid coupling kernels (Sec. II.B, Eq. couplingCF,
// Eq. couplingFC), D2Q9.
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
        if (mask && i != 0 && mask[src] == 1)
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

// Store feqH(rho, u) + (1 - 1/tau) fneqH(u, alpha Pi^neq) at a cell
template <class S>
__device__ void store_rebuilt_2d(S *__restrict__ f, int64_t N, int64_t cell, const CT<S> m[6], double alpha,
                                 double tau)
{
    using C = CT<S>;
    Coef<C> k{};
    const C rho = C(1) + m[0];
    add_eq<C, 2>(k, C(1), m[0], rho, m[1], m[2], C(0));
    Sym2<C> p;
    p.xx = C(alpha) * m[3]; p.xy = C(alpha) * m[4]; p.yy = C(alpha) * m[5];
    p.zz = p.xz = p.yz = C(0);
    add_neq<C, 2>(k, C(1.0 - 1.0 / tau), m[1], m[2], C(0), p);
    Store<S>::st(f + cell, rebuild_rest<D2Q9, C>(k));
#pragma unroll
    for (int i = 1; i <= D2Q9::HALF; ++i) {
        C e, o;
        rebuild_pair<D2Q9, C>(k, i, e, o);
        Store<S>::st(f + (int64_t)i * N + cell, C(weight<D2Q9>(i)) * (e + o));
        Store<S>::st(f + (int64_t)(i + D2Q9::HALF) * N + cell, C(weight<D2Q9>(i)) * (e - o));
    }
}

template <class S>
__global__ void k_line_moments(RefineGeom g, const S *__restrict__ fc, const uint8_t *__restrict__ mask,
                               int streamed, double *__restrict__ M)
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
    for (int k = 0; k < 6; ++k) M[6 * e + k] = (double)m[k];
}

template <class C>
__device__ inline void mix6(const double *__restrict__ M0, const double *__restrict__ M1, C a, int e, C out[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = (C(1) - a) * C(M0[6 * e + k]) + a * C(M1[6 * e + k]);
}

template <class S>
__global__ void k_fill_ring(RefineGeom g, const double *__restrict__ M0, const double *__restrict__ M1, double a,
                            double alpha, double tau_f, S *__restrict__ ff)
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
    const C am = C(a);
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
    store_rebuilt_2d<S>(ff, (int64_t)nfx * nfy, i + (int64_t)nfx * j, m, alpha, tau_f);
}

template <class S>
__global__ void k_restrict(RefineGeom g, const S *__restrict__ ff_prev, const uint8_t *__restrict__ fmask,
                           double alpha, double tau_c, S *__restrict__ fc)
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
    store_rebuilt_2d<S>(fc, (int64_t)g.nxc * g.nyc, x + (int64_t)g.nxc * y, mc, alpha, tau_c);
}

}  // namespace rr
