// step.cuh -- the fused stream + collide kernel (one time step of
// Eq. optimizedLB / Eq. spongeLB with the boundary rules of Sec. III).
//
// One thread updates one cell of a two-lattice pull scheme: it gathers the
// populations streamed into the cell, f_i(x) = f*_i(x - xi_i) (periodic wrap,
// halfway bounce-back on solid neighbours), takes the moments, rebuilds the
// Hermite-regularized populations, relaxes them and stores them in the
// other lattice.  Boundary roles come from coordinates, so a box without
// walls reads and writes exactly Q populations per cell (2 Q s bytes).
//
//   * velocity node (Sec. III, Dirichlet inflow): rho and Pi^neq of the
//     inward neighbour, prescribed u (+ seeded noise), f* = feqH(rho, u) +
//     (1 - 1/tau) fneqH(u, Pi^neq)
//   * free-slip node (Sec. III lateral walls): rho, u, Pi^neq of the inward
//     neighbour with zero normal velocity and zero normal-tangential Pi^neq
//   * constant-pressure node (Sec. IV outlet): u, Pi^neq of the inward
//     neighbour, imposed rho
//   * outflow node (zero gradient): collides the inward neighbour's streamed
//     populations
//   * sponge cell (Sec. II.C, Eq. spongeLB + Eq. dampingLBM, n = m = 1/2):
//     f* = (1 - chi) feqH(rho*, u*) + chi feqH(rho_ref, u_ref)
//          + (1 - 1/tau) fneqH(u*, Pi^neq about rho*, u*)
//   * bulk: f* = feqH(rho, u) + (1 - 1/tau) fneqH(u, Pi^neq)
//
// Populations are rebuilt by opposite pairs: the even Hermite part E = a0 +
// H2:A2 / (2 c_s^4) is shared and the odd part O = xi.a1 / c_s^2 + T3(A3)
// changes sign, f_i = w (E + O), f_opp = w (E - O).
#pragma once

#include <cmath>

#include "rr.cuh"

namespace rr {

enum { BC_PERIODIC = 0, BC_VELOCITY = 1, BC_OUTFLOW = 2, BC_FREESLIP = 3, BC_PRESSURE = 4 };

struct StepParams {
    int n[3];
    int periodic[3];
    int kind[6];
    int sponge_w[6];
    int any_sponge;
    int64_t ncell;
    int64_t face_cells[6];
    double u_face[6][3];
    double rho_face[6], rho_face_m1[6];  // density of a constant-pressure face (and minus 1)
    const double *u_profile[6];  // device, 3 doubles per face cell, or null
    double sponge_chi[6];
    // sponge strength of the face layers per axis coordinate, max over the two
    // faces of each axis: chi_x[0..nx), chi_y[nx..nx+ny), chi_z[nx+ny..);
    // device tables filled by the host in FP64 (and rounded to FP32)
    const float *chi_tab_f;
    const double *chi_tab_d;
    double radial[6];  // circular / spherical layer: centre (3), r0, width W, chi_max; W = 0: none
    double rho_ref, rho_ref_m1, u_ref[3];  // rho_ref_m1 = rho_ref - 1
    uint64_t noise_seed;
    double noise_amp;
    double omega;  // 1 - 1/tau
    const uint8_t *solid;  // device, or null
    int any_solid;         // the mask holds solid cells (else only fixed ones)
    int64_t step;
    // bulk box: cells with blo[a] <= c[a] < bhi[a] on every axis have no
    // boundary role and no sponge (filled by the host from faces and layers)
    int blo[3], bhi[3];
    // collision model: 0 rrBGK (Eq. optimizedLB), 1 plain BGK (Eq. standardLB;
    // general kernel only)
    int bgk;
    // round-jet similarity reference of the +x sponge layer (cells with
    // x >= jet_x_layer): yc, zc, U_J, B D, x0, a = (sqrt 2 - 1) / S^2;
    // jet_x_layer = INT_MAX when none
    int jet_x_layer;
    double jet_ref[6];
    // D2Q9: include the optional fourth-order H_xxyy term (rrBGK only)
    int order4;
    // per-direction base addresses of the lattice read (in) and written (out):
    // in[i] = f_in + i * ncell elements, i < Q <= kMaxQ; filled by the launchers
    const char *in[kMaxQ];
    char *out[kMaxQ];
    // device error word of the handle (or null): bit 0 a bounded wait of the
    // row-staged kernel gave up, bit 1 an index check of a checked build.
    // Kept after the base-address arrays: placed before them it shifted
    // their parameter offsets and cost the BF16 two-cell kernel 4% and the
    // FP32 one 2% (measured on GB300).
    unsigned *err;
    // every sponge layer relaxes to the rest state (rho_ref = 1, u_ref = 0,
    // no jet reference): the closed-form sponge coefficients apply
    int sponge_rest;
    // interior path of the vectorised kernel: byte offsets, from a cell's own
    // offset, of the cell its direction-i population is pulled from in the
    // lattice read (ld_off: direction i's array, row y - c_y, z - c_z) and of
    // direction i's array in the lattice written (st_off); valid when off32
    // (all directions of a lattice span fewer than 2^31 bytes)
    int off32;
    int ld_off[kMaxQ];
    int st_off[kMaxQ];
    int radial_on;  // the circular / spherical sponge layer is set (radial[4] > 0)
    // storage shift by a reference equilibrium: stored values are
    // f_i - feqH_i(1, u_s) instead of f_i - w_i; dsh[i] = feqH_i(1, u_s) - w_i is
    // added to a loaded value and subtracted before a store (general update
    // kernels only; 0 / unused when shifted = 0)
    int shifted;
    float dsh_f[kMaxQ];
    double dsh_d[kMaxQ];
};

template <class C>
__device__ __forceinline__ C dsh(const StepParams &p, int i);
template <>
__device__ __forceinline__ float dsh<float>(const StepParams &p, int i)
{
    return p.dsh_f[i];
}
template <>
__device__ __forceinline__ double dsh<double>(const StepParams &p, int i)
{
    return p.dsh_d[i];
}

// Bulk box of a lattice (host): on each axis the coordinates that are neither
// on a non-periodic face nor inside a sponge layer of that axis.
inline void set_bulk_box(StepParams &p)
{
    for (int a = 0; a < 3; ++a) {
        int lo = p.periodic[a] ? 0 : 1, hi = p.periodic[a] ? p.n[a] : p.n[a] - 1;
        if (p.any_sponge) {
            if (p.sponge_w[2 * a] > 0 && p.sponge_chi[2 * a] > 0.0 && p.sponge_w[2 * a] > lo) lo = p.sponge_w[2 * a];
            if (p.sponge_w[2 * a + 1] > 0 && p.sponge_chi[2 * a + 1] > 0.0 && p.n[a] - p.sponge_w[2 * a + 1] < hi)
                hi = p.n[a] - p.sponge_w[2 * a + 1];
        }
        if (p.any_sponge && p.radial[4] > 0.0 && a < (p.n[2] > 1 ? 3 : 2)) {
            // inside the cube inscribed in the circle (sphere) of radius r0
            const double half = p.radial[3] / std::sqrt(p.n[2] > 1 ? 3.0 : 2.0);
            const int rlo = (int)std::ceil(p.radial[a] - half), rhi = (int)std::floor(p.radial[a] + half) + 1;
            if (rlo > lo) lo = rlo;
            if (rhi < hi) hi = rhi;
        }
        p.blo[a] = lo;
        p.bhi[a] = hi > lo ? hi : lo;
    }
    p.radial_on = (p.any_sponge && p.radial[4] > 0.0) ? 1 : 0;
}

// Per-direction byte offsets of the vectorised kernel's interior path (host)
template <class L, class S>
inline void set_offsets(StepParams &p)
{
    const int64_t span = (int64_t)L::Q * p.ncell * (int64_t)sizeof(S);
    p.off32 = span < ((int64_t)1 << 31) ? 1 : 0;
    const int64_t nx = p.n[0], nxy = (int64_t)p.n[0] * p.n[1];
    for (int i = 0; i < kMaxQ; ++i) {
        p.ld_off[i] = p.st_off[i] = 0;
        if (!p.off32 || i >= L::Q) continue;
        p.st_off[i] = (int)(i * p.ncell * (int64_t)sizeof(S));
        p.ld_off[i] = (int)((i * p.ncell - L::cy(i) * nx - L::cz(i) * nxy) * (int64_t)sizeof(S));
    }
}

// Fill the per-direction base addresses for one launch (host)
template <class L, class S>
inline void set_bases(StepParams &p, const void *fin, void *fout)
{
    static_assert(L::Q <= kMaxQ, "StepParams holds kMaxQ direction bases");
    for (int i = 0; i < L::Q; ++i) {
        p.in[i] = (const char *)fin + (size_t)i * (size_t)p.ncell * sizeof(S);
        p.out[i] = (char *)fout + (size_t)i * (size_t)p.ncell * sizeof(S);
    }
    set_offsets<L, S>(p);
}

// ---------------------------------------------------------------------------
// Sponge strength chi = chi_max sigma(d), maximum over the layers (Sec. II.C).
// The face layers come from the per-axis tables (the y/z layers are uniform
// along a row; only the x layers vary along it); the circular layer is
// evaluated per cell.
// ---------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ C chi_tab(const StepParams &p, int k);
template <>
__device__ __forceinline__ float chi_tab<float>(const StepParams &p, int k)
{
    return __ldg(p.chi_tab_f + k);
}
template <>
__device__ __forceinline__ double chi_tab<double>(const StepParams &p, int k)
{
    return __ldg(p.chi_tab_d + k);
}

template <class L, class C>
__device__ __forceinline__ C chi_row(const StepParams &p, int y, int z)
{
    if (!p.any_sponge) return C(0);
    C chi = chi_tab<C>(p, p.n[0] + y);
    if (L::D == 3) {
        const C v = chi_tab<C>(p, p.n[0] + p.n[1] + z);
        chi = v > chi ? v : chi;
    }
    return chi;
}

template <class L, class C>
__device__ __forceinline__ C chi_cell(const StepParams &p, C row, int x, int y, int z)
{
    if (!p.any_sponge) return row;
    C v = chi_tab<C>(p, x);
    row = v > row ? v : row;
    if (p.radial_on) {
        // circular layer: the profile up to its maximum at r0 + 0.8 W, chi_max beyond
        const C dx = C(x) - C(p.radial[0]), dy = C(y) - C(p.radial[1]);
        C r2 = dx * dx + dy * dy;
        if (L::D == 3) {
            const C dz = C(z) - C(p.radial[2]);
            r2 += dz * dz;
        }
        const C d = sqrt(r2) - C(p.radial[3]), W = C(p.radial[4]);
        if (d >= C(0)) {
            v = C(p.radial[5]) * (d >= C(0.8) * W ? C(1) : sigma<C>(d, W));
            row = v > row ? v : row;
        }
    }
    return row;
}

// Velocity imposed at node (cx, cy, cz) of velocity face `inlet`: the face
// value or the per-cell profile, plus the seeded noise (counter-based
// splitmix64 keyed by seed, step, face cell and component) scaled by |u|,
// in the collision's precision (for float the uniform keeps its leading 24
// bits).  One component at a time keeps the 64-bit hash's registers short-lived.
template <class L, class C>
__device__ __forceinline__ void face_velocity(const StepParams &p, int inlet, int cx, int cy, int cz, C (&ub)[3])
{
    const int a = inlet >> 1;
    const int t0c = a == 0 ? cy : cx, t1c = a == 2 ? cy : cz;
    const int n0 = a == 0 ? p.n[1] : p.n[0];
    const int64_t kf = t0c + (int64_t)n0 * t1c;
    const double *prof = p.u_profile[inlet];
#pragma unroll
    for (int b = 0; b < 3; ++b) ub[b] = C(prof ? prof[3 * kf + b] : p.u_face[inlet][b]);
    if (p.noise_amp > 0.0) {
        const C mag = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
        if (mag > C(0)) {
            const uint64_t base =
                (p.noise_seed << 32) + ((uint64_t)p.step * (uint64_t)p.face_cells[inlet] + (uint64_t)kf) * 3u;
            const C amp = C(p.noise_amp) * mag;
#pragma unroll 1
            for (int b = 0; b < L::D; ++b) ub[b] += amp * (C(2) * u01c<C>(base + b) - C(1));
        }
    }
}

// Moments m' of a velocity / free-slip / pressure node such that the
// interior coefficients of m' (coef_interior) are the node's: density rho'
// and velocity u' as the rule imposes, and the off-equilibrium stress of the
// neighbour whose streamed moments m are given, Pi^neq about its own rho, u
// (zeroed normal-tangential components on a free-slip face):
//   dr' = rho' - 1,  j' = rho' u',  s' = Pi^neq' + dr' c_s^2 I + rho' u' u'.
template <class L, class C>
__device__ __forceinline__ Mom<C> face_moments(const StepParams &p, const Mom<C> &m, int inlet, int cx, int cy, int cz)
{
    const C rho = C(1) + m.dr;
    const C inv = recip(rho);
    C ux = m.jx * inv, uy = m.jy * inv, uz = L::D == 3 ? m.jz * inv : C(0);
    Sym2<C> pn = pi_neq<C>(m, m.dr, rho, ux, uy, uz, L::D);
    C dr = m.dr, r = rho;
    const int kind = p.kind[inlet];
    if (kind == BC_VELOCITY) {
        C ub[3];
        face_velocity<L, C>(p, inlet, cx, cy, cz, ub);
        ux = ub[0];
        uy = ub[1];
        uz = L::D == 3 ? ub[2] : C(0);
    } else if (kind == BC_PRESSURE) {
        dr = C(p.rho_face_m1[inlet]);
        r = C(p.rho_face[inlet]);
    } else {
        const int a = inlet >> 1;
        if (a == 0) { ux = C(0); pn.xy = C(0); pn.xz = C(0); }
        if (a == 1) { uy = C(0); pn.xy = C(0); pn.yz = C(0); }
        if (a == 2) { uz = C(0); pn.xz = C(0); pn.yz = C(0); }
    }
    Mom<C> o;
    const C c = dr * C(1.0 / 3.0);
    o.dr = dr;
    o.jx = r * ux;
    o.jy = r * uy;
    o.jz = r * uz;
    o.sxx = fmac(o.jx, ux, pn.xx + c);
    o.syy = fmac(o.jy, uy, pn.yy + c);
    o.szz = L::D == 3 ? fmac(o.jz, uz, pn.zz + c) : C(0);
    o.sxy = fmac(o.jx, uy, pn.xy);
    o.sxz = L::D == 3 ? fmac(o.jx, uz, pn.xz) : C(0);
    o.syz = L::D == 3 ? fmac(o.jy, uz, pn.yz) : C(0);
    return o;
}

// ---------------------------------------------------------------------------
// Collision coefficients of one cell: velocity node, sponge cell or bulk.
// BGK = true: the plain LBM-BGK (Eq. standardLB) -- boundary nodes rebuilt to
// second order, f^eq + (1 - 1/tau) f^neq_2; other cells get the quadratic
// equilibrium part (1 - 1/tau) f^eq (with the sponge's damping) and the
// caller adds (1 - 1/tau) g_i of the streamed populations.
// ---------------------------------------------------------------------------
template <class L, class C, bool BGK = false>
__device__ __forceinline__ Coef<C> cell_coefficients(const StepParams &p, const Mom<C> &m, C chi, int cx,
                                                     int cy, int cz, int inlet)
{
    constexpr bool O3 = !BGK;
    constexpr bool XYZ = !BGK && full_third_order<L>();
    const bool o4 = L::D == 2 && !BGK && p.order4;
    const C om = C(p.omega);
    Coef<C> k{};
    if (inlet >= 0 && p.kind[inlet] != BC_VELOCITY) {
        // free-slip or constant-pressure node: moments of the streamed neighbour
        const C rho = C(1) + m.dr;
        const C inv = recip(rho);
        C ux = m.jx * inv, uy = m.jy * inv, uz = L::D == 3 ? m.jz * inv : C(0);
        Sym2<C> pn = pi_neq<C>(m, m.dr, rho, ux, uy, uz, L::D);
        if (p.kind[inlet] == BC_PRESSURE) {
            add_eq<C, L::D, O3, XYZ>(k, C(1), C(p.rho_face_m1[inlet]), C(p.rho_face[inlet]), ux, uy, uz, o4);
        } else {
            const int a = inlet >> 1;
            if (a == 0) { ux = C(0); pn.xy = C(0); pn.xz = C(0); }
            if (a == 1) { uy = C(0); pn.xy = C(0); pn.yz = C(0); }
            if (a == 2) { uz = C(0); pn.xz = C(0); pn.yz = C(0); }
            add_eq<C, L::D, O3, XYZ>(k, C(1), m.dr, rho, ux, uy, uz, o4);
        }
        add_neq<C, L::D, O3, XYZ>(k, om, ux, uy, uz, pn, o4);
        return k;
    }
    if (inlet >= 0) {
        // velocity node: rho, Pi^neq from the streamed neighbour, prescribed u (+ noise)
        const C rho = C(1) + m.dr;
        const C inv = recip(rho);
        const Sym2<C> pn = pi_neq<C>(m, m.dr, rho, m.jx * inv, m.jy * inv, m.jz * inv, L::D);
        C ub[3];
        face_velocity<L, C>(p, inlet, cx, cy, cz, ub);
        const C ux = ub[0], uy = ub[1], uz = L::D == 3 ? ub[2] : C(0);
        add_eq<C, L::D, O3, XYZ>(k, C(1), m.dr, rho, ux, uy, uz, o4);
        add_neq<C, L::D, O3, XYZ>(k, om, ux, uy, uz, pn, o4);
        return k;
    }
    if (!BGK && chi > C(0) && p.sponge_rest) return coef_interior<L, C, true>(m, om, chi, o4);
    if (chi > C(0)) {
        // sponge: damped moments rho*, rho* u* (n = m = 1/2), then
        // f* = (1 - chi) feqH(rho*, u*) + chi feqH(rho_ref, u_ref) + (1 - 1/tau) fneqH
        const C h = recip(C(1) + C(0.5) * chi);
        const C rr = C(p.rho_ref);
        C urx = C(p.u_ref[0]), ury = C(p.u_ref[1]), urz = C(p.u_ref[2]);
        if (L::D == 3 && cx >= p.jet_x_layer) {
            // outflow layer: self-similar round jet, centreline min(U_J, B D U_J / xi),
            // profile (1 + a eta^2)^-2, eta = r / xi, xi = x - x0
            const C xi = C(cx) - C(p.jet_ref[4]);
            const C Uc = (xi > C(0) && C(p.jet_ref[3]) < xi) ? C(p.jet_ref[3]) * C(p.jet_ref[2]) / xi : C(p.jet_ref[2]);
            const C dy = C(cy) - C(p.jet_ref[0]), dz = C(cz) - C(p.jet_ref[1]);
            const C e2 = xi > C(0) ? (dy * dy + dz * dz) / (xi * xi) : C(0);
            const C q = C(1) + C(p.jet_ref[5]) * e2;
            urx = Uc / (q * q);
            ury = urz = C(0);
        }
        const C drs = (m.dr + C(0.5) * chi * C(p.rho_ref_m1)) * h;  // rho* - 1
        const C rs = C(1) + drs;
        const C inv = recip(rs);
        const C ux = (m.jx + C(0.5) * chi * rr * urx) * h * inv;
        const C uy = (m.jy + C(0.5) * chi * rr * ury) * h * inv;
        const C uz = L::D == 3 ? (m.jz + C(0.5) * chi * rr * urz) * h * inv : C(0);
        if (BGK) {
            // (1 - 1/tau - chi) f^eq(rho*, u*) + chi f^eq(ref); the caller adds (1 - 1/tau) g
            add_eq<C, L::D, O3, XYZ>(k, C(1) - om - chi, drs, rs, ux, uy, uz, o4);
            add_eq<C, L::D, O3, XYZ>(k, chi, C(p.rho_ref_m1), rr, urx, ury, L::D == 3 ? urz : C(0), o4);
            return k;
        }
        const Sym2<C> pn = pi_neq<C>(m, drs, rs, ux, uy, uz, L::D);
        add_eq<C, L::D, O3, XYZ>(k, C(1) - chi, drs, rs, ux, uy, uz, o4);
        add_eq<C, L::D, O3, XYZ>(k, chi, C(p.rho_ref_m1), rr, urx, ury, L::D == 3 ? urz : C(0), o4);
        add_neq<C, L::D, O3, XYZ>(k, om, ux, uy, uz, pn, o4);
        return k;
    }
    if (!BGK) return coef_interior<L, C, false>(m, om, C(0), o4);
    const C rho = C(1) + m.dr;
    const C inv = recip(rho);
    const C ux = m.jx * inv, uy = m.jy * inv, uz = L::D == 3 ? m.jz * inv : C(0);
    // (1 - 1/tau) f^eq; the caller adds (1 - 1/tau) g
    add_eq<C, L::D, O3, XYZ>(k, C(1) - om, m.dr, rho, ux, uy, uz, o4);
    return k;
}

// ---------------------------------------------------------------------------
// One cell's update (general form): pull with wrap and bounce-back, boundary
// role from coordinates, collision, store.  Shared by the single-lattice
// kernel below and the batched multi-domain kernel.
// ---------------------------------------------------------------------------
// Cell-type mask handling compiled into an update: none (no mask), skip
// (fixed cells are not updated; no solid cells, so no link tests), links
// (skip, plus halfway bounce-back at cells next to a solid).
enum { kMaskNone = 0, kMaskSkip = 1, kMaskLinks = 2 };

// Checked builds (-DLBM_BOUNDS_CHECK, `build(checked=True)`): every index an
// update reads or writes is tested against the lattice before any access; a
// cell whose indices fall outside is not updated and bit 1 of the handle's
// error word is set (reported by lbm_sync).  The substitute for a memory
// sanitizer on a pool where compute-sanitizer is closed; release builds
// compile the checks away.
constexpr unsigned kErrBounds = 2u;
__device__ __forceinline__ bool index_fault(const StepParams &p, bool bad)
{
#ifdef LBM_BOUNDS_CHECK
    if (bad && p.err) atomicOr(p.err, kErrBounds);
    return bad;
#else
    (void)p;
    (void)bad;
    return false;
#endif
}

template <class L, class S, class C, bool BGK = false, int MASK = kMaskLinks>
__device__ __forceinline__ void update_cell(const StepParams &p, const char *const *in, char *const *out,
                                            int x, int y, int z)
{
    // 32-bit cell offsets: a lattice holds fewer than 2^31 cells
    const unsigned nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const unsigned nxy = nx * ny;
    const unsigned cell = x + nx * y + nxy * z;
    if (index_fault(p, x < 0 || y < 0 || z < 0 || cell >= (unsigned)p.ncell)) return;
    // kMaskNone: compiled without any cell-type test (the lattice has no mask)
    const uint8_t *__restrict__ solid = MASK != kMaskNone ? p.solid : nullptr;
    if (solid && (solid[cell] & MASK_TYPE)) return;  // solid (1) and fixed (2) cells keep their populations

    // ---- boundary role and the node whose streamed populations are used
    unsigned sx = x, sy = y, sz = z;
    int inlet = -1;
    const bool bulk = x >= p.blo[0] && x < p.bhi[0] && y >= p.blo[1] && y < p.bhi[1] && z >= p.blo[2] &&
                      z < p.bhi[2];
    if (!bulk) {
    if (!p.periodic[0]) {
        if (x == 0) { sx = 1; if (p.kind[0] != BC_OUTFLOW) inlet = 0; }
        if (x == (int)nx - 1) { sx = nx - 2; if (p.kind[1] != BC_OUTFLOW && inlet < 0) inlet = 1; }
    }
    if (!p.periodic[1]) {
        if (y == 0) { sy = 1; if (p.kind[2] != BC_OUTFLOW && inlet < 0) inlet = 2; }
        if (y == (int)ny - 1) { sy = ny - 2; if (p.kind[3] != BC_OUTFLOW && inlet < 0) inlet = 3; }
    }
    if (L::D == 3 && !p.periodic[2]) {
        if (z == 0) { sz = 1; if (p.kind[4] != BC_OUTFLOW && inlet < 0) inlet = 4; }
        if (z == (int)nz - 1) { sz = nz - 2; if (p.kind[5] != BC_OUTFLOW && inlet < 0) inlet = 5; }
    }
    }
    // neighbour coordinates of s with wrap-around on periodic axes
    const unsigned xm = sx == 0 ? nx - 1 : sx - 1, xp = sx == nx - 1 ? 0 : sx + 1;
    const unsigned ym = sy == 0 ? ny - 1 : sy - 1, yp = sy == ny - 1 ? 0 : sy + 1;
    const unsigned zm = sz == 0 ? nz - 1 : sz - 1, zp = sz == nz - 1 ? 0 : sz + 1;
    const unsigned scell = sx + nx * sy + nxy * sz;
#ifdef LBM_BOUNDS_CHECK
    {
        bool bad = scell >= (unsigned)p.ncell;
        for (int i = 0; i < L::Q; ++i) {
            const unsigned X = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : sx);
            const unsigned Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
            const unsigned Z = L::D == 2 ? 0u : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
            bad = bad || X >= nx || Y >= ny || Z >= nz || X + nx * Y + nxy * Z >= (unsigned)p.ncell;
        }
        if (index_fault(p, bad)) return;
    }
#endif

    // ---- streaming (pull) with halfway bounce-back; only a node with a solid
    // neighbour tests its links
    const bool near = MASK == kMaskLinks && solid && (solid[scell] & MASK_NEAR_SOLID);
    C g[L::Q];
    // two gather loops, the link tests only in the one for cells next to a
    // solid: with the test inside a single loop the masked D2Q9 FP16 / BF16
    // update ran 30% slower on GB300 (1600 x 800 cylinder: 64 -> 92 G cell
    // updates/s with the split; FP32 83 -> 84)
    if (near) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const unsigned X = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : sx);
            const unsigned Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
            const unsigned Z = L::D == 2 ? 0u : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
            const unsigned src = X + nx * Y + nxy * Z;
            // a bounced population is stored in the opposite direction's array (and shift)
            const int k = (i != 0 && (solid[src] & MASK_TYPE) == MASK_SOLID) ? opp<L>(i) : i;
            g[i] = Store<S>::ld((const S *)in[k] + (k == i ? src : scell));
            if (p.shifted) g[i] += dsh<C>(p, k);
        }
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const unsigned X = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : sx);
            const unsigned Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : sy);
            const unsigned Z = L::D == 2 ? 0u : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : sz));
            g[i] = Store<S>::ld((const S *)in[i] + (X + nx * Y + nxy * Z));
        }
        if (p.shifted) {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) g[i] += dsh<C>(p, i);
        }
    }

    const Mom<C> m = moments_pairs<L, C>(g);
    const C chi = (bulk || inlet >= 0) ? C(0) : chi_cell<L, C>(p, chi_row<L, C>(p, y, z), x, y, z);
    const Coef<C> k = cell_coefficients<L, C, BGK>(p, m, chi, x, y, z, inlet);

    // ---- rebuild, relax and store (even/odd parts of each opposite pair);
    // plain BGK adds (1 - 1/tau) g of the streamed populations except at
    // rebuilt boundary nodes
    const C keep = (BGK && inlet < 0) ? C(p.omega) : C(0);
    C o[L::Q];
    if (L::D == 2 && p.order4)
        rebuild_all<L, C, true>(k, o);
    else
        rebuild_all<L, C, false>(k, o);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        if (BGK) o[i] = fmac(keep, g[i], o[i]);
    if (p.shifted) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) o[i] -= dsh<C>(p, i);
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Store<S>::st((S *)out[i] + cell, o[i]);
}

// ---------------------------------------------------------------------------
// In-place AA streaming: one lattice, two step types that alternate.
//   gather-push (LOC = false), from the standard layout P_i[x] = f*_i(x):
//     pull g_i = P_i[x - xi_i] (halfway bounce-back: P_opp(i)[x]), collide,
//     push o_i to P_opp(i)[x + xi_i] -- or back to P_i[x] when x + xi_i is a
//     solid cell or lies outside a non-periodic face;
//   local (LOC = true): g_i = P_opp(i)[x], which is where the push left the
//     population streamed into x (a bounce-back included), collide, o_i ->
//     P_i[x]: the standard layout again.
// Each cell writes exactly the slots it reads, so the lattice is updated in
// place without races.  A boundary node collides the populations streamed
// into its inward neighbour (the same rules as the pull update); to keep the
// reads and writes of those slots in one thread it is updated by the thread
// of that neighbour, and the threads of face nodes do nothing.  The
// arithmetic is the pull update's; only where the populations are read and
// written differs.
// ---------------------------------------------------------------------------
template <class L, class S, class C, bool BGK, int MASK, bool LOC>
__device__ __forceinline__ void update_cell_aa(const StepParams &p, char *const *f, int x, int y, int z)
{
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    if (!p.periodic[0] && (x == 0 || x == nx - 1)) return;
    if (!p.periodic[1] && (y == 0 || y == ny - 1)) return;
    if (L::D == 3 && !p.periodic[2] && (z == 0 || z == nz - 1)) return;
    const unsigned unx = nx, uny = ny, unz = nz, nxy = unx * uny;
    const unsigned cell = x + unx * y + nxy * z;
    if (index_fault(p, x < 0 || y < 0 || z < 0 || cell >= (unsigned)p.ncell)) return;
    const uint8_t *__restrict__ solid = MASK != kMaskNone ? p.solid : nullptr;
    // neighbours of the cell (it is not on a non-periodic face, so only
    // periodic axes wrap)
    const unsigned xm = x == 0 ? unx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const unsigned ym = y == 0 ? uny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const unsigned zm = z == 0 ? unz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;

    C g[L::Q];
    if (LOC) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = Store<S>::ld((const S *)f[opp<L>(i)] + cell);
    } else {
        const bool near = MASK == kMaskLinks && solid && (solid[cell] & MASK_NEAR_SOLID);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const unsigned X = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : (unsigned)x);
            const unsigned Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : (unsigned)y);
            const unsigned Z = L::D == 2 ? 0u : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : (unsigned)z));
            const unsigned src = X + unx * Y + nxy * Z;
            if (near && i != 0 && (solid[src] & MASK_TYPE) == MASK_SOLID)
                g[i] = Store<S>::ld((const S *)f[opp<L>(i)] + cell);
            else
                g[i] = Store<S>::ld((const S *)f[i] + src);
        }
    }
    const Mom<C> m = moments_pairs<L, C>(g);

    // this cell and the boundary nodes that take its populations
    int tx[3], ty[3], tz[3], ntx = 1, nty = 1, ntz = 1;
    tx[0] = x;
    ty[0] = y;
    tz[0] = z;
    if (!p.periodic[0]) {
        if (x == 1) tx[ntx++] = 0;
        if (x == nx - 2) tx[ntx++] = nx - 1;
    }
    if (!p.periodic[1]) {
        if (y == 1) ty[nty++] = 0;
        if (y == ny - 2) ty[nty++] = ny - 1;
    }
    if (L::D == 3 && !p.periodic[2]) {
        if (z == 1) tz[ntz++] = 0;
        if (z == nz - 2) tz[ntz++] = nz - 1;
    }
#pragma unroll 1
    for (int c = 0; c < ntz; ++c)
#pragma unroll 1
        for (int b = 0; b < nty; ++b)
#pragma unroll 1
            for (int a = 0; a < ntx; ++a) {
                const int X = tx[a], Y = ty[b], Z = tz[c];
                const unsigned t = X + unx * Y + nxy * Z;
                if (solid && (solid[t] & MASK_TYPE)) continue;  // solid and fixed cells keep their populations
                // boundary role of the target, as in update_cell
                int inlet = -1;
                if (!p.periodic[0]) {
                    if (X == 0 && p.kind[0] != BC_OUTFLOW) inlet = 0;
                    if (X == nx - 1 && p.kind[1] != BC_OUTFLOW && inlet < 0) inlet = 1;
                }
                if (!p.periodic[1]) {
                    if (Y == 0 && p.kind[2] != BC_OUTFLOW && inlet < 0) inlet = 2;
                    if (Y == ny - 1 && p.kind[3] != BC_OUTFLOW && inlet < 0) inlet = 3;
                }
                if (L::D == 3 && !p.periodic[2]) {
                    if (Z == 0 && p.kind[4] != BC_OUTFLOW && inlet < 0) inlet = 4;
                    if (Z == nz - 1 && p.kind[5] != BC_OUTFLOW && inlet < 0) inlet = 5;
                }
                const bool bulk = X >= p.blo[0] && X < p.bhi[0] && Y >= p.blo[1] && Y < p.bhi[1] &&
                                  Z >= p.blo[2] && Z < p.bhi[2];
                const C chi = (bulk || inlet >= 0) ? C(0) : chi_cell<L, C>(p, chi_row<L, C>(p, Y, Z), X, Y, Z);
                const Coef<C> k = cell_coefficients<L, C, BGK>(p, m, chi, X, Y, Z, inlet);
                const C keep = (BGK && inlet < 0) ? C(p.omega) : C(0);
                C o[L::Q];
                if (L::D == 2 && p.order4)
                    rebuild_all<L, C, true>(k, o);
                else
                    rebuild_all<L, C, false>(k, o);
                if (BGK) {
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) o[i] = fmac(keep, g[i], o[i]);
                }
                if (LOC) {
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) Store<S>::st((S *)f[i] + t, o[i]);
                } else {
                    const bool tnear = MASK == kMaskLinks && solid && (solid[t] & MASK_NEAR_SOLID);
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) {
                        int DX = X + L::cx(i), DY = Y + L::cy(i), DZ = Z + L::cz(i);
                        bool out = false;
                        if (DX < 0 || DX >= nx) {
                            if (p.periodic[0]) DX = DX < 0 ? nx - 1 : 0;
                            else out = true;
                        }
                        if (DY < 0 || DY >= ny) {
                            if (p.periodic[1]) DY = DY < 0 ? ny - 1 : 0;
                            else out = true;
                        }
                        if (L::D == 3 && (DZ < 0 || DZ >= nz)) {
                            if (p.periodic[2]) DZ = DZ < 0 ? nz - 1 : 0;
                            else out = true;
                        }
                        const unsigned dst = (unsigned)DX + unx * (unsigned)DY + nxy * (unsigned)(L::D == 2 ? 0 : DZ);
                        if (!out && tnear && i != 0 && (solid[dst] & MASK_TYPE) == MASK_SOLID) out = true;
                        if (out)
                            Store<S>::st((S *)f[i] + t, o[i]);
                        else
                            Store<S>::st((S *)f[opp<L>(i)] + dst, o[i]);
                    }
                }
            }
}

// The AA step kernels: one thread per cell, blocks along x (the face nodes'
// threads return at once)
template <class L, class S, class C, bool BGK, int MASK, bool LOC>
__global__ void __launch_bounds__(256) k_stream_collide_aa(const __grid_constant__ StepParams p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.n[0]) return;
    update_cell_aa<L, S, C, BGK, MASK, LOC>(p, p.out, x, blockIdx.y, blockIdx.z);
}

// Launch one AA step (loc: the local step, else gather-push) of the lattice f
template <class L, class S, class C>
cudaError_t launch_stream_collide_aa(const StepParams &p, void *f, int block, bool loc, cudaStream_t st)
{
    StepParams q = p;
    set_bases<L, S>(q, f, f);
    dim3 b(block, 1, 1);
    dim3 g((p.n[0] + block - 1) / block, p.n[1], p.n[2]);
    const bool links = p.solid != nullptr;  // user masks hold solid cells (no fixed cells without refinement)
    if (p.bgk) {
        if (loc)
            links ? k_stream_collide_aa<L, S, C, true, kMaskLinks, true><<<g, b, 0, st>>>(q)
                  : k_stream_collide_aa<L, S, C, true, kMaskNone, true><<<g, b, 0, st>>>(q);
        else
            links ? k_stream_collide_aa<L, S, C, true, kMaskLinks, false><<<g, b, 0, st>>>(q)
                  : k_stream_collide_aa<L, S, C, true, kMaskNone, false><<<g, b, 0, st>>>(q);
    } else {
        if (loc)
            links ? k_stream_collide_aa<L, S, C, false, kMaskLinks, true><<<g, b, 0, st>>>(q)
                  : k_stream_collide_aa<L, S, C, false, kMaskNone, true><<<g, b, 0, st>>>(q);
        else
            links ? k_stream_collide_aa<L, S, C, false, kMaskLinks, false><<<g, b, 0, st>>>(q)
                  : k_stream_collide_aa<L, S, C, false, kMaskNone, false><<<g, b, 0, st>>>(q);
    }
    return cudaGetLastError();
}

// In-place conversion of the AA push layout (left by a gather-push step)
// back to the standard layout: the pairs P_i[x] <-> P_opp(i)[x + xi_i]
// (i = 1..Q/2, x + xi_i inside the lattice with wrap-around on periodic axes,
// neither end solid) are swapped; each pair is visited once.
template <class L, class S>
__global__ void k_aa_unswap(StepParams p, S *f)
{
    const int64_t N = p.ncell;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < N;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if (p.solid && (p.solid[cell] & MASK_TYPE) == MASK_SOLID) continue;
        const int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((int64_t)nx * ny));
#pragma unroll
        for (int i = 1; i <= L::HALF; ++i) {
            int X = x + L::cx(i), Y = y + L::cy(i), Z = z + L::cz(i);
            if (X < 0 || X >= nx) {
                if (!p.periodic[0]) continue;
                X = X < 0 ? nx - 1 : 0;
            }
            if (Y < 0 || Y >= ny) {
                if (!p.periodic[1]) continue;
                Y = Y < 0 ? ny - 1 : 0;
            }
            if (Z < 0 || Z >= nz) {
                if (!p.periodic[2]) continue;
                Z = Z < 0 ? nz - 1 : 0;
            }
            const int64_t dst = X + (int64_t)nx * (Y + (int64_t)ny * Z);
            if (p.solid && (p.solid[dst] & MASK_TYPE) == MASK_SOLID) continue;
            S *a = f + (int64_t)i * N + cell, *b = f + (int64_t)opp<L>(i) * N + dst;
            const S t = *a;
            *a = *b;
            *b = t;
        }
    }
}

template <class L, class S>
cudaError_t launch_aa_unswap(const StepParams &p, void *f, cudaStream_t st)
{
    const int64_t blocks = (p.ncell + 255) / 256;
    k_aa_unswap<L, S><<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, st>>>(p, (S *)f);
    return cudaGetLastError();
}

// General kernel: one thread per cell; MASK: cell-type handling (above);
// BGK = true is the plain LBM-BGK collision (Eq. standardLB).
template <class L, class S, class C, bool BGK, int MASK>
__global__ void __launch_bounds__(256) k_stream_collide(const __grid_constant__ StepParams p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.n[0]) return;
    update_cell<L, S, C, BGK, MASK>(p, p.in, p.out, x, blockIdx.y, blockIdx.z);
}

// The same update with one thread per cell of the whole lattice, for rows
// whose length would leave many threads of their blocks idle (a 129-cell row
// in 128-thread blocks idles half of them); rrBGK only.
template <class L, class S, class C, int MASK>
__global__ void __launch_bounds__(256) k_stream_collide_lin(const __grid_constant__ StepParams p)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (unsigned)p.ncell) return;
    const unsigned nx = p.n[0], nxy = nx * (unsigned)p.n[1];
    const unsigned z = t / nxy, r = t - z * nxy, y = r / nx;
    update_cell<L, S, C, false, MASK>(p, p.in, p.out, (int)(r - y * nx), (int)y, (int)z);
}

// Launch wrapper: one thread per cell, blocks along x; p.bgk selects the
// collision model.
template <class L, class S, class C>
cudaError_t launch_stream_collide(const StepParams &p, const void *fin, void *fout, int block,
                                  cudaStream_t st)
{
    StepParams q = p;
    set_bases<L, S>(q, fin, fout);
    dim3 b(block, 1, 1);
    dim3 g((p.n[0] + block - 1) / block, p.n[1], p.n[2]);
    // rows that leave more than 1/8 of their threads idle: the whole-lattice
    // mapping
    const int64_t row_threads = (int64_t)g.x * block;
    const int mode = !p.solid ? kMaskNone : (p.any_solid ? kMaskLinks : kMaskSkip);
    if (!p.bgk && 8 * (row_threads - p.n[0]) > row_threads) {
        const dim3 gl((unsigned)((p.ncell + block - 1) / block), 1, 1);
        if (mode == kMaskLinks)
            k_stream_collide_lin<L, S, C, kMaskLinks><<<gl, b, 0, st>>>(q);
        else if (mode == kMaskSkip)
            k_stream_collide_lin<L, S, C, kMaskSkip><<<gl, b, 0, st>>>(q);
        else
            k_stream_collide_lin<L, S, C, kMaskNone><<<gl, b, 0, st>>>(q);
        return cudaGetLastError();
    }
    if (p.bgk) {
        if (p.solid)
            k_stream_collide<L, S, C, true, kMaskLinks><<<g, b, 0, st>>>(q);
        else
            k_stream_collide<L, S, C, true, kMaskNone><<<g, b, 0, st>>>(q);
    } else {
        if (mode == kMaskLinks)
            k_stream_collide<L, S, C, false, kMaskLinks><<<g, b, 0, st>>>(q);
        else if (mode == kMaskSkip)
            k_stream_collide<L, S, C, false, kMaskSkip><<<g, b, 0, st>>>(q);
        else
            k_stream_collide<L, S, C, false, kMaskNone><<<g, b, 0, st>>>(q);
    }
    return cudaGetLastError();
}

}  // namespace rr
