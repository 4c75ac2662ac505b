/*
 * FP64 CPU oracle for the recursive Hermite-regularized lattice Boltzmann
 * update (rrBGK) of Brogi, Malaspinas, Chopard and Bonadonna, arXiv:1710.02065.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  It is
 * compiled and called only by tests/, by __graft_entry__.smoke() and by the
 * CPU-baseline / reference legs of bench.py.  The product path never links,
 * loads or calls it, and it shares no code, header or table with the CUDA
 * sources: the lattice, the Hermite tensors and every boundary rule are
 * written out again here from the paper.
 *
 * Conventions
 *   - Populations are plain f_i (not shifted), one double per direction.
 *     A field is stored direction-major: f[i * ncell + cell], with
 *     cell = x + nx * (y + ny * z).
 *   - The stored state is the post-collision field f*(t).  One step pulls
 *     f_i(x) = f*_i(x - xi_i) (streaming, the left side of Eq. optimizedLB
 *     evaluated at x), applies the boundary rules, and collides.
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.
 *
 * Readings of the paper taken here (it is silent or garbled on these):
 *   R1  a^2 = Pi - rho c_s^2 I, a^2_eq = rho u u, a^2_neq = Pi^neq
 *       (the printed a^2 = P - rho(uu - delta) is a garbled form), Sec. II.A.
 *   R2  Eq. eqH is read with xi_i . u (the print drops the ". u"), and Eq. neqH
 *       without the spurious rho prefactor and index i on a^2_neq.
 *   R3  Third order on D3Q19: Sec. II.A defers to Malaspinas (2015).  The six
 *       a_aab components are kept as the sum/difference pairs (xxy,yzz),
 *       (xzz,xyy), (yyz,xxz), each projected with its own lattice norm, so that
 *       the regularized populations reproduce a_p + a_q and a_p - a_q exactly.
 *   R4  Sponge (Eq. spongeLB, Eq. dampingLBM): the modified moments use
 *       n = m = 1/2 and rho* u* = j + m sum_i F_i xi_i, which close to
 *       rho* = (rho + chi rho_ref / 2) / (1 + chi / 2) and
 *       rho* u* = (j + chi rho_ref u_ref / 2) / (1 + chi / 2).
 *       Pi^neq in a sponge cell is taken about rho*, u*.
 *   R5  Sponge strength chi(x) = chi_max * sigma(d) with the polynomial
 *       profile of Sec. II.C, sigma(d) = 3125 (W - d) d^4 / (256 W^5), where d
 *       is the distance of the cell from the inner edge of a layer of W cells
 *       (x0 = inner edge, L = x0 + W); overlapping layers take the maximum.
 *   R6  Velocity inflow (Dirichlet, scheme not given in Sec. III): the node
 *       takes rho and Pi^neq from its inward neighbour after streaming and
 *       rebuilds f = feqH(rho, u_in) + fneqH(u_in, Pi^neq) before colliding.
 *   R7  Outflow (zero gradient for all components, Sec. III): the node copies
 *       the streamed populations of its inward neighbour and collides them.
 *   R8  Walls: halfway bounce-back; a population that would stream out of a
 *       solid cell is replaced by the node's own post-collision population in
 *       the opposite direction.  Solid cells, and "fixed" cells whose
 *       populations are imposed from outside (grid coupling), are not updated.
 *   R9  Inlet noise: counter-based uniform numbers from splitmix64 (Steele,
 *       Lea and Flood 2014) keyed by (seed, step, face cell, component).
 *   R16 Free-slip wall (Sec. III, lateral boundaries: "zero-gradient for
 *       tangential velocity components"): the node takes rho, u and Pi^neq of
 *       its inward neighbour, sets the normal velocity and the normal-
 *       tangential Pi^neq components to zero (no flux, no shear), and is
 *       rebuilt as feqH(rho, u) + fneqH(u, Pi^neq) before colliding.
 *   R17 Constant-pressure outlet (Sec. IV, right boundary of the jet): the
 *       node takes u and Pi^neq of its inward neighbour (zero gradient) and
 *       the imposed density, p = c_s^2 rho_out, and is rebuilt likewise.
 *   R18 Circular sponge (Sec. III: circular layer, corners covered): chi =
 *       chi_max sigma(r - r0) for r - r0 < 0.8 W, chi_max beyond.
 *   R15 Forces on walls (lift, drag; not printed as a formula in the paper):
 *       momentum exchange over the bounce-back links.
 *   R23 D2Q9 fourth order (optional; Sec. II.A: D2Q9 supports an expansion
 *       beyond n = 3): the H_xxyy term with a4_eq = rho u_x^2 u_y^2 and
 *       Eq. recursive2 at n = 4 read as the symmetric sum over index pairs,
 *       a4_neq = u_x^2 P_yy + u_y^2 P_xx + 4 u_x u_y P_xy.
 *   R21 Jet outflow sponge reference (Sec. IV: the jet similarity solution of
 *       Pope 2000 as reference field of the outflow region): inside the +x
 *       layer the reference velocity is the self-similar round-jet mean
 *       axial profile (sponge_reference below); elsewhere the uniform u_ref.
 */
#include <pthread.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CS2 (1.0 / 3.0)

/* ------------------------------------------------------------------------ */
/* Lattices (velocities and weights are the textbook Gauss-Hermite sets; the */
/* paper only says they are specific to the lattice, Eq. truncatedEq).       */
/* ------------------------------------------------------------------------ */

#define QMAX 27 /* largest lattice: D3Q27 */

typedef struct {
    int d, q;
    int xi[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
} lattice_t;

static void build_lattice(int which, lattice_t *L)
{
    /* Directions 1..Q/2 are listed; Q/2+1..Q-1 are their negatives in the
     * same order, so that opp(i) = i +- Q/2.  Weight depends on |xi|^2. */
    static const int d2q9_half[4][3] = {
        {1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {-1, 1, 0}};
    static const int d3q19_half[9][3] = {
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
        {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
    /* D3Q27: the D3Q19 set plus the eight corners (tensor product of D1Q3) */
    static const int d3q27_half[13][3] = {
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
        {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1},
        {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
    const int (*half)[3];
    int h;
    double w0, w1, w2, w3 = 0.0;
    if (which == 0) {
        L->d = 2; L->q = 9; half = d2q9_half; h = 4;
        w0 = 4.0 / 9.0; w1 = 1.0 / 9.0; w2 = 1.0 / 36.0;
    } else if (which == 1) {
        L->d = 3; L->q = 19; half = d3q19_half; h = 9;
        w0 = 1.0 / 3.0; w1 = 1.0 / 18.0; w2 = 1.0 / 36.0;
    } else {
        L->d = 3; L->q = 27; half = d3q27_half; h = 13;
        w0 = 8.0 / 27.0; w1 = 2.0 / 27.0; w2 = 1.0 / 54.0; w3 = 1.0 / 216.0;
    }
    memset(L->xi, 0, sizeof L->xi);
    for (int i = 0; i < h; ++i)
        for (int a = 0; a < 3; ++a) {
            L->xi[1 + i][a] = half[i][a];
            L->xi[1 + h + i][a] = -half[i][a];
        }
    for (int i = 0; i < L->q; ++i) {
        int n2 = L->xi[i][0] * L->xi[i][0] + L->xi[i][1] * L->xi[i][1] +
                 L->xi[i][2] * L->xi[i][2];
        L->w[i] = n2 == 0 ? w0 : (n2 == 1 ? w1 : (n2 == 2 ? w2 : w3));
        for (int k = 0; k < L->q; ++k)
            if (L->xi[k][0] == -L->xi[i][0] && L->xi[k][1] == -L->xi[i][1] &&
                L->xi[k][2] == -L->xi[i][2])
                L->opp[i] = k;
    }
}

static const lattice_t *lattice(int which)
{
    static lattice_t lat[3];
    static int ready[3];
    if (!ready[which]) {
        build_lattice(which, &lat[which]);
        ready[which] = 1;
    }
    return &lat[which];
}

/* ------------------------------------------------------------------------ */
/* Hermite polynomials on the lattice (Sec. II.A, Eq. HE and Eq. HEeqAndNeq) */
/* ------------------------------------------------------------------------ */

static double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

/* H^(2)_{i,ab} = xi_a xi_b - c_s^2 delta_ab */
static double H2(const lattice_t *L, int i, int a, int b)
{
    return (double)L->xi[i][a] * L->xi[i][b] - CS2 * delta(a, b);
}

/* H^(3)_{i,abc} = xi_a xi_b xi_c - c_s^2 (xi_a d_bc + xi_b d_ac + xi_c d_ab) */
static double H3(const lattice_t *L, int i, int a, int b, int c)
{
    double xa = L->xi[i][a], xb = L->xi[i][b], xc = L->xi[i][c];
    return xa * xb * xc - CS2 * (xa * delta(b, c) + xb * delta(a, c) + xc * delta(a, b));
}

/* Third-order contribution T3_i(a) for a symmetric third-order tensor a,
 * given as a full 3x3x3 array.  Only components the lattice supports are
 * kept (reading R3 for D3Q19; on D2Q9 H_xxx = H_yyy = 0 and the surviving
 * terms xxy, xyy carry the full-contraction multiplicity 3/3! = 1/2). */
static double T3(const lattice_t *L, int i, double a[3][3][3])
{
    const double cs6 = CS2 * CS2 * CS2;
    enum { X = 0, Y = 1, Z = 2 };
    if (L->d == 2) {
        return (H3(L, i, X, X, Y) * a[X][X][Y] + H3(L, i, X, Y, Y) * a[X][Y][Y]) /
               (2.0 * cs6);
    }
    if (L->q == 27) {
        /* D3Q27 supports the full third order except H_aaa (xi^3 = xi on
         * {-1, 0, 1}): the six H_aab with multiplicity 3 and H_xyz with
         * multiplicity 6 in the contraction H3 : a3 / (3! c_s^6); all are
         * orthogonal on this tensor-product lattice with the continuous norms */
        static const int A[6][3] = {{X, X, Y}, {X, X, Z}, {Y, Y, X}, {Y, Y, Z}, {Z, Z, X}, {Z, Z, Y}};
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += H3(L, i, A[k][0], A[k][1], A[k][2]) * a[A[k][0]][A[k][1]][A[k][2]];
        return s / (2.0 * cs6) + H3(L, i, X, Y, Z) * a[X][Y][Z] / cs6;
    }
    /* pairs (p, q): (xxy, yzz), (xzz, xyy), (yyz, xxz) */
    static const int P[3][2][3] = {
        {{X, X, Y}, {Y, Z, Z}},
        {{X, Z, Z}, {X, Y, Y}},
        {{Y, Y, Z}, {X, X, Z}}};
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int *p = P[k][0], *q = P[k][1];
        double hp = H3(L, i, p[0], p[1], p[2]);
        double hq = H3(L, i, q[0], q[1], q[2]);
        double ap = a[p[0]][p[1]][p[2]];
        double aq = a[q[0]][q[1]][q[2]];
        s += (hp + hq) * (ap + aq) / (2.0 * cs6) + (hp - hq) * (ap - aq) / (6.0 * cs6);
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Moments, equilibrium and non-equilibrium parts                             */
/* ------------------------------------------------------------------------ */

/* Eq. moments plus the second moment Pi = sum_i f_i xi_i xi_i (Sec. II.A). */
static void moments(const lattice_t *L, const double *f, double *rho, double j[3],
                    double Pi[3][3])
{
    *rho = 0.0;
    for (int a = 0; a < 3; ++a) {
        j[a] = 0.0;
        for (int b = 0; b < 3; ++b) Pi[a][b] = 0.0;
    }
    for (int i = 0; i < L->q; ++i) {
        *rho += f[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += f[i] * L->xi[i][a];
            for (int b = 0; b < 3; ++b) Pi[a][b] += f[i] * L->xi[i][a] * L->xi[i][b];
        }
    }
}

/* Eq. eqH with a^0 = rho, a^1 = rho u and, from Eq. recursive1,
 * a^2_eq = rho u u, a^3_eq = rho u u u. */
static void feqH(const lattice_t *L, double rho, const double u[3], double *out)
{
    const double cs4 = CS2 * CS2;
    double a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) a3[a][b][c] = rho * u[a] * u[b] * u[c];
    for (int i = 0; i < L->q; ++i) {
        double xu = 0.0, h2 = 0.0;
        for (int a = 0; a < L->d; ++a) {
            xu += L->xi[i][a] * rho * u[a];
            for (int b = 0; b < L->d; ++b) h2 += H2(L, i, a, b) * rho * u[a] * u[b];
        }
        out[i] = L->w[i] * (rho + xu / CS2 + h2 / (2.0 * cs4) + T3(L, i, a3));
    }
}

/* Eq. neqH with a^2_neq = Pi^neq and a^3_neq from Eq. recursive2 at n = 3:
 * a^3_neq,abc = u_a Pi^neq_bc + u_b Pi^neq_ac + u_c Pi^neq_ab. */
static void fneqH(const lattice_t *L, const double u[3], double Pn[3][3], double *out)
{
    const double cs4 = CS2 * CS2;
    double a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
                a3[a][b][c] = u[a] * Pn[b][c] + u[b] * Pn[a][c] + u[c] * Pn[a][b];
    for (int i = 0; i < L->q; ++i) {
        double h2 = 0.0;
        for (int a = 0; a < L->d; ++a)
            for (int b = 0; b < L->d; ++b) h2 += H2(L, i, a, b) * Pn[a][b];
        out[i] = L->w[i] * (h2 / (2.0 * cs4) + T3(L, i, a3));
    }
}

/* Optional fourth order on D2Q9 (reading R23): H_xxyy = (xi_x^2 - c_s^2)
 * (xi_y^2 - c_s^2), supported by D2Q9 with the continuous norm 4 c_s^8; it
 * enters H4 : a4 / (4! c_s^8) with multiplicity 6, i.e. with 1 / (4 c_s^8).
 * Equilibrium a4_xxyy = rho u_x^2 u_y^2 (Eq. recursive1); off-equilibrium
 * from Eq. recursive2 at n = 4 read as the symmetric sum over the six index
 * pairs, a4_xxyy = u_x^2 P_yy + u_y^2 P_xx + 4 u_x u_y P_xy. */
static double H4xxyy(const lattice_t *L, int i)
{
    return ((double)L->xi[i][0] * L->xi[i][0] - CS2) * ((double)L->xi[i][1] * L->xi[i][1] - CS2);
}

static void add_fourth_eq(const lattice_t *L, double rho, const double u[3], double *f)
{
    const double a4 = rho * u[0] * u[0] * u[1] * u[1], c = 1.0 / (4.0 * CS2 * CS2 * CS2 * CS2);
    for (int i = 0; i < L->q; ++i) f[i] += L->w[i] * H4xxyy(L, i) * a4 * c;
}

static void add_fourth_neq(const lattice_t *L, const double u[3], double Pn[3][3], double *f)
{
    const double a4 = u[0] * u[0] * Pn[1][1] + u[1] * u[1] * Pn[0][0] + 4.0 * u[0] * u[1] * Pn[0][1];
    const double c = 1.0 / (4.0 * CS2 * CS2 * CS2 * CS2);
    for (int i = 0; i < L->q; ++i) f[i] += L->w[i] * H4xxyy(L, i) * a4 * c;
}

/* Pi^neq = Pi - rho c_s^2 I - rho u u (reading R1); components outside the
 * lattice's d dimensions are zero. */
static void pi_neq(int d, double rho, const double u[3], double Pi[3][3], double Pn[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Pn[a][b] = (a < d && b < d) ? Pi[a][b] - rho * CS2 * delta(a, b) - rho * u[a] * u[b] : 0.0;
}

/* One cell's collision: Eq. optimizedLB, or Eq. spongeLB with
 * Eq. dampingLBM when chi > 0 (reading R4).  g is a body force used only by
 * the oracle's own Poiseuille check (momentum source w_i rho xi_i.g / c_s^2). */
static void collide(const lattice_t *L, const double *f, double tau, double chi,
                    double rho_ref, const double u_ref[3], const double g[3], int o4, double *out)
{
    o4 = o4 && L->d == 2;
    double rho, j[3], Pi[3][3], u[3], Pn[3][3];
    double feq[QMAX], fneq[QMAX];
    moments(L, f, &rho, j, Pi);
    if (chi > 0.0) {
        double rs = (rho + 0.5 * chi * rho_ref) / (1.0 + 0.5 * chi);
        double fref[QMAX];
        for (int a = 0; a < 3; ++a)
            u[a] = (j[a] + 0.5 * chi * rho_ref * u_ref[a]) / (1.0 + 0.5 * chi) / rs;
        pi_neq(L->d, rs, u, Pi, Pn);
        feqH(L, rs, u, feq);
        fneqH(L, u, Pn, fneq);
        feqH(L, rho_ref, u_ref, fref);
        if (o4) {
            add_fourth_eq(L, rs, u, feq);
            add_fourth_neq(L, u, Pn, fneq);
            add_fourth_eq(L, rho_ref, u_ref, fref);
        }
        for (int i = 0; i < L->q; ++i)
            out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i] + chi * (fref[i] - feq[i]);
    } else {
        for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
        pi_neq(L->d, rho, u, Pi, Pn);
        feqH(L, rho, u, feq);
        fneqH(L, u, Pn, fneq);
        if (o4) {
            add_fourth_eq(L, rho, u, feq);
            add_fourth_neq(L, u, Pn, fneq);
        }
        for (int i = 0; i < L->q; ++i) out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i];
    }
    if (g && (g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0))
        for (int i = 0; i < L->q; ++i) {
            double xg = 0.0;
            for (int a = 0; a < 3; ++a) xg += L->xi[i][a] * g[a];
            out[i] += L->w[i] * rho * xg / CS2;
        }
}

/* Eq. truncatedEq: the quadratic equilibrium of the plain LBM-BGK,
 * w_i rho (1 + xi.u / c_s^2 + (xi.u)^2 / (2 c_s^4) - |u|^2 / (2 c_s^2)). */
static void feq_quadratic(const lattice_t *L, double rho, const double u[3], double *out)
{
    double uu = 0.0;
    for (int a = 0; a < L->d; ++a) uu += u[a] * u[a];
    for (int i = 0; i < L->q; ++i) {
        double xu = 0.0;
        for (int a = 0; a < L->d; ++a) xu += L->xi[i][a] * u[a];
        out[i] = L->w[i] * rho * (1.0 + xu / CS2 + xu * xu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Second-order Hermite part of f^neq, w_i H2_i : Pi^neq / (2 c_s^4): the
 * off-equilibrium part a boundary node is rebuilt with under plain BGK. */
static void fneq_second(const lattice_t *L, double Pn[3][3], double *out)
{
    for (int i = 0; i < L->q; ++i) {
        double h2 = 0.0;
        for (int a = 0; a < L->d; ++a)
            for (int b = 0; b < L->d; ++b) h2 += H2(L, i, a, b) * Pn[a][b];
        out[i] = L->w[i] * h2 / (2.0 * CS2 * CS2);
    }
}

/* Plain BGK collision (Eq. standardLB): f* = f - (f - f^eq) / tau with the
 * quadratic f^eq; in a sponge cell f^eq is taken at rho*, u* (reading R4) and
 * the damping term chi (f^eq(rho_ref, u_ref) - f^eq(rho*, u*)) is added. */
static void collide_bgk(const lattice_t *L, const double *f, double tau, double chi, double rho_ref,
                        const double u_ref[3], const double g[3], double *out)
{
    double rho, j[3], Pi[3][3], u[3], feq[QMAX];
    moments(L, f, &rho, j, Pi);
    double rs = rho;
    if (chi > 0.0) {
        rs = (rho + 0.5 * chi * rho_ref) / (1.0 + 0.5 * chi);
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * chi * rho_ref * u_ref[a]) / (1.0 + 0.5 * chi) / rs;
    } else {
        for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    }
    feq_quadratic(L, rs, u, feq);
    for (int i = 0; i < L->q; ++i) out[i] = f[i] - (f[i] - feq[i]) / tau;
    if (chi > 0.0) {
        double fref[QMAX];
        feq_quadratic(L, rho_ref, u_ref, fref);
        for (int i = 0; i < L->q; ++i) out[i] += chi * (fref[i] - feq[i]);
    }
    if (g && (g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0))
        for (int i = 0; i < L->q; ++i) {
            double xg = 0.0;
            for (int a = 0; a < 3; ++a) xg += L->xi[i][a] * g[a];
            out[i] += L->w[i] * rho * xg / CS2;
        }
}

/* Rebuilt boundary node: feqH(rho, u) + (1 - 1/tau) fneqH(u, Pi^neq) under
 * rrBGK; under plain BGK the node is rebuilt to second order, f^eq + f^neq_2,
 * and the BGK collision of that is f^eq + (1 - 1/tau) f^neq_2. */
static void rebuilt_node(int collision, double tau, const lattice_t *L, double rho, const double u[3],
                         double Pn[3][3], int o4, double *out)
{
    double feq[QMAX], fneq[QMAX];
    if (collision == 1) {
        feq_quadratic(L, rho, u, feq);
        fneq_second(L, Pn, fneq);
    } else {
        feqH(L, rho, u, feq);
        fneqH(L, u, Pn, fneq);
        if (o4 && L->d == 2) {
            add_fourth_eq(L, rho, u, feq);
            add_fourth_neq(L, u, Pn, fneq);
        }
    }
    for (int i = 0; i < L->q; ++i) out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i];
}

/* ------------------------------------------------------------------------ */
/* Counter-based uniform numbers (reading R9)                                 */
/* ------------------------------------------------------------------------ */

uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_u01(uint64_t counter)
{
    return (double)(orc_splitmix64(counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Problem description                                                       */
/* ------------------------------------------------------------------------ */

enum { BC_PERIODIC = 0, BC_VELOCITY = 1, BC_OUTFLOW = 2, BC_FREESLIP = 3, BC_PRESSURE = 4 };

typedef struct {
    int lattice;             /* 0 = D2Q9, 1 = D3Q19, 2 = D3Q27 */
    int n[3];                /* extents; n[2] = 1 for D2Q9 */
    double tau;
    int face_kind[6];        /* -x, +x, -y, +y, -z, +z */
    double u_face[6][3];     /* uniform velocity of a velocity face */
    double rho_face[6];      /* density of a constant-pressure face */
    const double *u_profile[6]; /* optional per-face-cell velocity, 3 per cell */
    uint64_t noise_seed;
    double noise_amp;        /* relative amplitude of inlet noise (0 = none) */
    int sponge_width[6];
    double sponge_chi[6];
    double rho_ref;
    double u_ref[3];
    double radial[6];        /* circular (spherical) layer: cx, cy, cz, r0, W, chi_max; W = 0: none */
    const uint8_t *solid;    /* optional per cell: 1 = solid wall, 2 = fixed */
    double g[3];             /* oracle-only body force */
    int collision;           /* 0 = rrBGK (Eq. optimizedLB), 1 = BGK (Eq. standardLB) */
    double jet_ref[7];       /* round-jet similarity reference of the +x sponge (reading R21):
                                yc, zc, U_J, D, x0, B, S; D = 0: none */
    int order4;              /* D2Q9: add the fourth-order H_xxyy term (reading R23) */
} orc_problem;

static int64_t ncell(const orc_problem *P) { return (int64_t)P->n[0] * P->n[1] * P->n[2]; }

/* Tangential index of a cell on a face (fastest tangential axis first). */
static int64_t face_index(const orc_problem *P, int face, const int c[3])
{
    int a = face / 2;
    int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
    return (int64_t)c[t0] + (int64_t)P->n[t0] * c[t1];
}

static int64_t face_cells(const orc_problem *P, int face)
{
    int a = face / 2;
    int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
    return (int64_t)P->n[t0] * P->n[t1];
}

/* Sponge profile of Sec. II.C for a layer of width W, d from the inner edge. */
double orc_sigma(double d, double W)
{
    if (d < 0.0 || d > W) return 0.0;
    return 3125.0 * (W - d) * d * d * d * d / (256.0 * W * W * W * W * W);
}

static double sponge_chi(const orc_problem *P, const int c[3])
{
    double chi = 0.0;
    if (P->radial[4] > 0.0) {
        /* circular layer (R18): d = r - r0; the polynomial profile up to its
         * maximum at d = 0.8 W, held at that maximum beyond (corners covered) */
        const lattice_t *L = lattice(P->lattice);
        double r2 = 0.0;
        for (int a = 0; a < L->d; ++a) r2 += (c[a] - P->radial[a]) * (c[a] - P->radial[a]);
        double d = sqrt(r2) - P->radial[3], W = P->radial[4];
        if (d >= 0.0) chi = P->radial[5] * (d >= 0.8 * W ? 1.0 : orc_sigma(d, W));
    }
    for (int face = 0; face < 6; ++face) {
        int W = P->sponge_width[face];
        if (W <= 0) continue;
        int a = face / 2;
        double d = (face % 2) ? (double)(c[a] - (P->n[a] - W)) : (double)(W - 1 - c[a]);
        double s = P->sponge_chi[face] * orc_sigma(d, (double)W);
        if (s > chi) chi = s;
    }
    return chi;
}

/* Sponge reference velocity of a cell (reading R21): the uniform u_ref, or,
 * inside the +x layer when a jet reference is set, the mean axial velocity of
 * the self-similar round jet (Sec. IV cites Pope 2000 for it): centreline
 * U_0 = min(U_J, B D U_J / (x - x0)), profile f(eta) = (1 + a eta^2)^-2 with
 * eta = r / (x - x0) and a = (sqrt 2 - 1) / S^2, so that u = U_0 / 2 at the
 * half-width r = S (x - x0); radial velocity not imposed. */
static void sponge_reference(const orc_problem *P, const int c[3], double u[3])
{
    for (int a = 0; a < 3; ++a) u[a] = P->u_ref[a];
    const double *J = P->jet_ref;
    if (!(J[3] > 0.0) || P->sponge_width[1] <= 0 || c[0] < P->n[0] - P->sponge_width[1]) return;
    const double xi = c[0] - J[4];
    const double Uc = xi > 0.0 && J[5] * J[3] / xi < 1.0 ? J[5] * J[3] * J[2] / xi : J[2];
    const double r = sqrt((c[1] - J[0]) * (c[1] - J[0]) + (c[2] - J[1]) * (c[2] - J[1]));
    const double eta = xi > 0.0 ? r / xi : 0.0;
    const double a = (sqrt(2.0) - 1.0) / (J[6] * J[6]);
    const double q = 1.0 + a * eta * eta;
    u[0] = Uc / (q * q);
    u[1] = u[2] = 0.0;
}

void orc_sponge_reference(const orc_problem *P, int x, int y, int z, double u[3])
{
    const int c[3] = {x, y, z};
    sponge_reference(P, c, u);
}

/* Post-collision populations of one cell at step `step` (the step that turns
 * f*(step) into f*(step+1)), read from the full field fin. */
void orc_update_cell(const orc_problem *P, const double *fin, int64_t cell, int64_t step,
                     double *out)
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    int c[3], s[3];
    c[0] = (int)(cell % P->n[0]);
    c[1] = (int)((cell / P->n[0]) % P->n[1]);
    c[2] = (int)(cell / ((int64_t)P->n[0] * P->n[1]));

    if (P->solid && P->solid[cell]) {
        for (int i = 0; i < L->q; ++i) out[i] = fin[(int64_t)i * N + cell];
        return;
    }

    /* Boundary role and the node whose streamed populations are used (R6, R7,
     * R16, R17): the first velocity, free-slip or pressure face the node lies
     * on decides how it is rebuilt. */
    int inlet = -1;
    for (int a = 0; a < 3; ++a) {
        s[a] = c[a];
        int lo = 2 * a, hi = 2 * a + 1;
        if (P->face_kind[lo] != BC_PERIODIC && c[a] == 0) {
            s[a] = 1;
            if (P->face_kind[lo] != BC_OUTFLOW && inlet < 0) inlet = lo;
        }
        if (P->face_kind[hi] != BC_PERIODIC && c[a] == P->n[a] - 1) {
            s[a] = P->n[a] - 2;
            if (P->face_kind[hi] != BC_OUTFLOW && inlet < 0) inlet = hi;
        }
    }
    int64_t scell = s[0] + (int64_t)P->n[0] * (s[1] + (int64_t)P->n[1] * s[2]);

    /* Streaming: pull f_i(s) = f*_i(s - xi_i), periodic wrap, bounce-back (R8). */
    double f[QMAX];
    for (int i = 0; i < L->q; ++i) {
        int src[3];
        for (int a = 0; a < 3; ++a) {
            src[a] = s[a] - L->xi[i][a];
            if (P->face_kind[2 * a] == BC_PERIODIC) src[a] = ((src[a] % P->n[a]) + P->n[a]) % P->n[a];
        }
        int64_t scl = src[0] + (int64_t)P->n[0] * (src[1] + (int64_t)P->n[1] * src[2]);
        if (P->solid && P->solid[scl] == 1)
            f[i] = fin[(int64_t)L->opp[i] * N + scell];
        else
            f[i] = fin[(int64_t)i * N + scl];
    }

    if (inlet >= 0 && P->face_kind[inlet] != BC_VELOCITY) {
        /* Free-slip (R16) or constant-pressure (R17) node. */
        double rho, j[3], Pi[3][3], us[3], Pn[3][3];
        moments(L, f, &rho, j, Pi);
        for (int a = 0; a < 3; ++a) us[a] = j[a] / rho;
        pi_neq(L->d, rho, us, Pi, Pn);
        if (P->face_kind[inlet] == BC_FREESLIP) {
            int an = inlet / 2;
            us[an] = 0.0;
            for (int b = 0; b < 3; ++b)
                if (b != an) Pn[an][b] = Pn[b][an] = 0.0;
        } else {
            rho = P->rho_face[inlet];
        }
        rebuilt_node(P->collision, P->tau, L, rho, us, Pn, P->order4, out);
        return;
    }

    if (inlet >= 0) {
        /* Velocity node (R6). */
        double rho, j[3], Pi[3][3], us[3], ub[3], Pn[3][3];
        moments(L, f, &rho, j, Pi);
        for (int a = 0; a < 3; ++a) us[a] = j[a] / rho;
        pi_neq(L->d, rho, us, Pi, Pn);
        int64_t k = face_index(P, inlet, c);
        for (int a = 0; a < 3; ++a)
            ub[a] = P->u_profile[inlet] ? P->u_profile[inlet][3 * k + a] : P->u_face[inlet][a];
        if (P->noise_amp > 0.0) {
            double mag = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
            if (mag > 0.0) {
                uint64_t base = (P->noise_seed << 32) +
                                ((uint64_t)step * (uint64_t)face_cells(P, inlet) + (uint64_t)k) * 3u;
                for (int a = 0; a < L->d; ++a)
                    ub[a] += P->noise_amp * mag * (2.0 * orc_u01(base + (uint64_t)a) - 1.0);
            }
        }
        rebuilt_node(P->collision, P->tau, L, rho, ub, Pn, P->order4, out);
        return;
    }

    double uref[3];
    sponge_reference(P, c, uref);
    if (P->collision == 1)
        collide_bgk(L, f, P->tau, sponge_chi(P, c), P->rho_ref, uref, P->g, out);
    else
        collide(L, f, P->tau, sponge_chi(P, c), P->rho_ref, uref, P->g, P->order4, out);
}

/* Post-collision populations of a list of cells (out: n x q, cell-major). */
void orc_update_cells(const orc_problem *P, const double *fin, int64_t n, const int64_t *cells,
                      int64_t step, double *out)
{
    const lattice_t *L = lattice(P->lattice);
    for (int64_t k = 0; k < n; ++k) orc_update_cell(P, fin, cells[k], step, out + k * L->q);
}

/* One full step: fout = update(fin).  Returns 0. */
int orc_step(const orc_problem *P, const double *fin, double *fout, int64_t step)
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    double out[QMAX];
    for (int64_t cell = 0; cell < N; ++cell) {
        orc_update_cell(P, fin, cell, step, out);
        for (int i = 0; i < L->q; ++i) fout[(int64_t)i * N + cell] = out[i];
    }
    return 0;
}

/* nsteps steps starting at step index step0, ping-ponging between f and work;
 * the result is left in f. */
int orc_run(const orc_problem *P, double *f, double *work, int64_t step0, int64_t nsteps)
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    double *a = f, *b = work;
    for (int64_t t = 0; t < nsteps; ++t) {
        orc_step(P, a, b, step0 + t);
        double *tmp = a; a = b; b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * (size_t)N * (size_t)L->q);
    return 0;
}

/* The same nsteps steps with the cells of each step split over nthreads host
 * threads (contiguous ranges, joined before the next step).  Every cell is
 * computed by orc_update_cell exactly as in orc_step, so the result is bitwise
 * that of orc_run; the threads only shorten long reference runs. */
typedef struct {
    const orc_problem *P;
    const double *fin;
    double *fout;
    int64_t c0, c1, step;
} orc_slice;

static void *orc_slice_run(void *arg)
{
    const orc_slice *s = (const orc_slice *)arg;
    const lattice_t *L = lattice(s->P->lattice);
    const int64_t N = ncell(s->P);
    double out[QMAX];
    for (int64_t cell = s->c0; cell < s->c1; ++cell) {
        orc_update_cell(s->P, s->fin, cell, s->step, out);
        for (int i = 0; i < L->q; ++i) s->fout[(int64_t)i * N + cell] = out[i];
    }
    return NULL;
}

int orc_run_threads(const orc_problem *P, double *f, double *work, int64_t step0, int64_t nsteps, int nthreads)
{
    enum { MAXT = 256 };
    if (nthreads <= 1) return orc_run(P, f, work, step0, nsteps);
    if (nthreads > MAXT) nthreads = MAXT;
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    double *a = f, *b = work;
    pthread_t th[MAXT];
    orc_slice sl[MAXT];
    for (int64_t t = 0; t < nsteps; ++t) {
        for (int k = 0; k < nthreads; ++k) {
            sl[k].P = P;
            sl[k].fin = a;
            sl[k].fout = b;
            sl[k].c0 = N * k / nthreads;
            sl[k].c1 = N * (k + 1) / nthreads;
            sl[k].step = step0 + t;
            if (pthread_create(&th[k], NULL, orc_slice_run, &sl[k]) != 0) return -1;
        }
        for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
        double *tmp = a; a = b; b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * (size_t)N * (size_t)L->q);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported single-cell pieces (for the oracle's own checks)                  */
/* ------------------------------------------------------------------------ */

int orc_lattice(int which, int *d, int *q, int *xi /* q*3 */, double *w, int *opp)
{
    if (which < 0 || which > 2) return -1;
    const lattice_t *L = lattice(which);
    *d = L->d;
    *q = L->q;
    for (int i = 0; i < L->q; ++i) {
        for (int a = 0; a < 3; ++a) xi[3 * i + a] = L->xi[i][a];
        w[i] = L->w[i];
        opp[i] = L->opp[i];
    }
    return 0;
}

void orc_feqH(int which, double rho, const double *u, double *out)
{
    feqH(lattice(which), rho, u, out);
}

void orc_fneqH(int which, const double *u, const double *Pn9, double *out)
{
    double Pn[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Pn[a][b] = Pn9[3 * a + b];
    fneqH(lattice(which), u, Pn, out);
}

void orc_collide(int which, const double *f, double tau, double chi, double rho_ref,
                 const double *u_ref, const double *g, int order4, double *out)
{
    collide(lattice(which), f, tau, chi, rho_ref, u_ref, g, order4, out);
}

/* Moments of a stored field: rho (N), u (3N, per cell xyz), Pi^neq (6N, per
 * cell xx,xy,xz,yy,yz,zz; in 2D only xx,xy,yy are meaningful). */
void orc_field_moments(const orc_problem *P, const double *fin, double *rho, double *u,
                       double *pn6)
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    for (int64_t cell = 0; cell < N; ++cell) {
        double f[QMAX], r, j[3], Pi[3][3], v[3], Pn[3][3];
        for (int i = 0; i < L->q; ++i) f[i] = fin[(int64_t)i * N + cell];
        moments(L, f, &r, j, Pi);
        for (int a = 0; a < 3; ++a) v[a] = j[a] / r;
        pi_neq(L->d, r, v, Pi, Pn);
        if (rho) rho[cell] = r;
        if (u)
            for (int a = 0; a < 3; ++a) u[3 * cell + a] = v[a];
        if (pn6) {
            pn6[6 * cell + 0] = Pn[0][0];
            pn6[6 * cell + 1] = Pn[0][1];
            pn6[6 * cell + 2] = Pn[0][2];
            pn6[6 * cell + 3] = Pn[1][1];
            pn6[6 * cell + 4] = Pn[1][2];
            pn6[6 * cell + 5] = Pn[2][2];
        }
    }
}

/* Initial state f = feqH(rho, u) per cell (rho: N, u: 3N). */
void orc_init_equilibrium(const orc_problem *P, const double *rho, const double *u, double *f)
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    for (int64_t cell = 0; cell < N; ++cell) {
        double out[QMAX];
        feqH(L, rho[cell], u + 3 * cell, out);
        if (P->order4 && L->d == 2) add_fourth_eq(L, rho[cell], u + 3 * cell, out);
        for (int i = 0; i < L->q; ++i) f[(int64_t)i * N + cell] = out[i];
    }
}

/* Force on the solid cells by momentum exchange over halfway bounce-back
 * links (reading R15): every fluid cell x and direction i with x + xi_i solid
 * hands the wall 2 xi_i f*_i(x) per step, f* the stored post-collision
 * field (the population leaves x towards the wall and comes back reversed). */
void orc_wall_force(const orc_problem *P, const double *fin, double F[3])
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    F[0] = F[1] = F[2] = 0.0;
    if (!P->solid) return;
    for (int64_t cell = 0; cell < N; ++cell) {
        if (P->solid[cell]) continue;
        int c[3];
        c[0] = (int)(cell % P->n[0]);
        c[1] = (int)((cell / P->n[0]) % P->n[1]);
        c[2] = (int)(cell / ((int64_t)P->n[0] * P->n[1]));
        for (int i = 1; i < L->q; ++i) {
            int d[3];
            int inside = 1;
            for (int a = 0; a < 3; ++a) {
                d[a] = c[a] + L->xi[i][a];
                if (P->face_kind[2 * a] == BC_PERIODIC) d[a] = ((d[a] % P->n[a]) + P->n[a]) % P->n[a];
                else if (d[a] < 0 || d[a] >= P->n[a]) inside = 0;
            }
            if (!inside) continue;
            int64_t nb = d[0] + (int64_t)P->n[0] * (d[1] + (int64_t)P->n[1] * d[2]);
            if (P->solid[nb] != 1) continue;
            double fi = fin[(int64_t)i * N + cell];
            for (int a = 0; a < 3; ++a) F[a] += 2.0 * L->xi[i][a] * fi;
        }
    }
}

double orc_chi_at(const orc_problem *P, int x, int y, int z)
{
    int c[3] = {x, y, z};
    return sponge_chi(P, c);
}

/* ------------------------------------------------------------------------ */
/* Two-level 2:1 grid refinement (Sec. II.B), 2D                             */
/* ------------------------------------------------------------------------ */
/*
 * Layout (reading R10; Fig. 1 of the paper is not available):
 *   - The fine patch covers the coarse nodes X0..X0+Wc, Y0..Y0+Hc (vertex
 *     based, dx_f = dx_c / 2): fine node (i, j), 0 <= i <= 2 Wc,
 *     0 <= j <= 2 Hc, sits at coarse coordinates (X0 + i/2, Y0 + j/2); even
 *     (i, j) coincide with coarse nodes.
 *   - The fine boundary ring (i or j on the patch edge) is not updated by the
 *     fine step; it is rebuilt from coarse data (Eq. couplingFC).
 *   - Coarse nodes strictly inside the patch are not updated by the coarse
 *     step; the first ring of them is rebuilt from fine data
 *     (Eq. couplingCF); deeper ones are never read.
 *   - Exchanged data are the pre-collision rho, u and Pi^neq of the sending
 *     grid; the receiving node is rebuilt as feqH(rho, u) + (1 - 1/tau)
 *     fneqH(u, alpha Pi^neq) in its own post-collision form, the regularized
 *     f^neq being a function of u and Pi^neq only (Eq. neqH, Eq. recursive2).
 *   - Scaling (reading R11): tau_f = 2 tau_c - 1/2 (Sec. II.B); alpha =
 *     tau_f / (2 tau_c) coarse -> fine and 2 tau_c / tau_f fine -> coarse,
 *     from the leading-order Chapman-Enskog f^neq ~ tau dt grad(u) with
 *     dt_f = dt_c / 2 (the printed alpha = 2 tau_f / tau_c is read as a misprint).
 *   - Coarse -> fine in space: copy at coincident nodes, 4-point centred cubic
 *     (-1, 9, 9, -1)/16 along the interface line at mid nodes; in time: the
 *     average of the coarse values at t and t + 1 for the fine half step
 *     (linear in time, Sec. II.B).
 *   - Fine -> coarse: rho and u of the coincident fine node, Pi^neq low-pass
 *     filtered with the 3 x 3 full-weighting kernel (1,2,1) x (1,2,1) / 16
 *     (reading R12: the filter is not specified).
 */
typedef struct {
    int X0, Y0, Wc, Hc;
} orc_patch;

/* Pre-collision moments at an interior node (pull with wrap and walls):
 * m = (rho, ux, uy, Pxx, Pxy, Pyy). */
static void streamed_moments(const orc_problem *P, const double *fin, int x, int y, double m[6])
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    const int64_t cell = x + (int64_t)P->n[0] * y;
    double f[QMAX], rho, j[3], Pi[3][3], u[3], Pn[3][3];
    for (int i = 0; i < L->q; ++i) {
        int sx = x - L->xi[i][0], sy = y - L->xi[i][1];
        sx = ((sx % P->n[0]) + P->n[0]) % P->n[0];
        sy = ((sy % P->n[1]) + P->n[1]) % P->n[1];
        int64_t scl = sx + (int64_t)P->n[0] * sy;
        if (P->solid && P->solid[scl] == 1)
            f[i] = fin[(int64_t)L->opp[i] * N + cell];
        else
            f[i] = fin[(int64_t)i * N + scl];
    }
    moments(L, f, &rho, j, Pi);
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    pi_neq(L->d, rho, u, Pi, Pn);
    m[0] = rho; m[1] = u[0]; m[2] = u[1];
    m[3] = Pn[0][0]; m[4] = Pn[0][1]; m[5] = Pn[1][1];
}

/* Post-collision populations rebuilt from (rho, u, alpha Pi^neq). */
static void rebuild_post(const lattice_t *L, const double m[6], double alpha, double tau, double *out)
{
    double u[3] = {m[1], m[2], 0.0};
    double Pn[3][3] = {{alpha * m[3], alpha * m[4], 0}, {alpha * m[4], alpha * m[5], 0}, {0, 0, 0}};
    double feq[QMAX], fneq[QMAX];
    feqH(L, m[0], u, feq);
    fneqH(L, u, Pn, fneq);
    for (int i = 0; i < L->q; ++i) out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i];
}

/* Coarse moments on the interface lines, extended by one node past each end:
 * stored per coarse cell (6 doubles), only line entries are written. */
static void coarse_line_moments(const orc_problem *Pc, const orc_patch *G, const double *fc, double *M)
{
    for (int x = G->X0 - 1; x <= G->X0 + G->Wc + 1; ++x) {
        streamed_moments(Pc, fc, x, G->Y0, M + 6 * (x + (int64_t)Pc->n[0] * G->Y0));
        streamed_moments(Pc, fc, x, G->Y0 + G->Hc, M + 6 * (x + (int64_t)Pc->n[0] * (G->Y0 + G->Hc)));
    }
    for (int y = G->Y0 - 1; y <= G->Y0 + G->Hc + 1; ++y) {
        streamed_moments(Pc, fc, G->X0, y, M + 6 * (G->X0 + (int64_t)Pc->n[0] * y));
        streamed_moments(Pc, fc, G->X0 + G->Wc, y, M + 6 * (G->X0 + G->Wc + (int64_t)Pc->n[0] * y));
    }
}

/* Time-weighted coarse moment at coarse node (x, y): (1 - a) M0 + a M1. */
static void mix(const double *M0, const double *M1, double a, int nxc, int x, int y, double out[6])
{
    const double *p = M0 + 6 * (x + (int64_t)nxc * y), *q = M1 + 6 * (x + (int64_t)nxc * y);
    for (int k = 0; k < 6; ++k) out[k] = (1.0 - a) * p[k] + a * q[k];
}

/* Rebuild the fine boundary ring from coarse line moments at time weight a. */
static void fill_fine_ring(const orc_problem *Pc, const orc_problem *Pf, const orc_patch *G,
                           const double *M0, const double *M1, double a, double *ff)
{
    const lattice_t *L = lattice(Pf->lattice);
    const int64_t Nf = ncell(Pf);
    const int nxc = Pc->n[0];
    const double tau_c = Pc->tau, tau_f = Pf->tau;
    const double alpha = tau_f / (2.0 * tau_c);
    const int nfx = 2 * G->Wc + 1, nfy = 2 * G->Hc + 1;
    for (int j = 0; j < nfy; ++j)
        for (int i = 0; i < nfx; ++i) {
            int on_h = (j == 0 || j == nfy - 1), on_v = (i == 0 || i == nfx - 1);
            if (!on_h && !on_v) continue;
            double m[6], t0[6], t1[6], t2[6], t3[6];
            if (i % 2 == 0 && j % 2 == 0) {
                mix(M0, M1, a, nxc, G->X0 + i / 2, G->Y0 + j / 2, m);
            } else if (on_h && i % 2 == 1) {
                int xa = G->X0 + (i - 1) / 2, yc = G->Y0 + j / 2;
                mix(M0, M1, a, nxc, xa - 1, yc, t0);
                mix(M0, M1, a, nxc, xa, yc, t1);
                mix(M0, M1, a, nxc, xa + 1, yc, t2);
                mix(M0, M1, a, nxc, xa + 2, yc, t3);
                for (int k = 0; k < 6; ++k) m[k] = (-t0[k] + 9.0 * t1[k] + 9.0 * t2[k] - t3[k]) / 16.0;
            } else {
                int xc = G->X0 + i / 2, ya = G->Y0 + (j - 1) / 2;
                mix(M0, M1, a, nxc, xc, ya - 1, t0);
                mix(M0, M1, a, nxc, xc, ya, t1);
                mix(M0, M1, a, nxc, xc, ya + 1, t2);
                mix(M0, M1, a, nxc, xc, ya + 2, t3);
                for (int k = 0; k < 6; ++k) m[k] = (-t0[k] + 9.0 * t1[k] + 9.0 * t2[k] - t3[k]) / 16.0;
            }
            double out[QMAX];
            rebuild_post(L, m, alpha, tau_f, out);
            int64_t cell = i + (int64_t)nfx * j;
            for (int q = 0; q < L->q; ++q) ff[(int64_t)q * Nf + cell] = out[q];
        }
}

/* Rebuild the first ring of covered coarse nodes from the fine grid
 * (Eq. couplingCF): rho, u at the coincident fine node, filtered Pi^neq. */
static void restrict_to_coarse(const orc_problem *Pc, const orc_problem *Pf, const orc_patch *G,
                               const double *ff_prev, double *fc)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t Nc = ncell(Pc);
    const double alpha = 2.0 * Pc->tau / Pf->tau;
    static const double w3[3] = {1.0, 2.0, 1.0};
    for (int y = G->Y0 + 1; y <= G->Y0 + G->Hc - 1; ++y)
        for (int x = G->X0 + 1; x <= G->X0 + G->Wc - 1; ++x) {
            int ring = (x == G->X0 + 1 || x == G->X0 + G->Wc - 1 || y == G->Y0 + 1 || y == G->Y0 + G->Hc - 1);
            if (!ring) continue;
            int i = 2 * (x - G->X0), j = 2 * (y - G->Y0);
            double m[6], mc[6] = {0, 0, 0, 0, 0, 0};
            for (int l = -1; l <= 1; ++l)
                for (int k = -1; k <= 1; ++k) {
                    streamed_moments(Pf, ff_prev, i + k, j + l, m);
                    double wgt = w3[k + 1] * w3[l + 1] / 16.0;
                    for (int c = 3; c < 6; ++c) mc[c] += wgt * m[c];
                    if (k == 0 && l == 0) { mc[0] = m[0]; mc[1] = m[1]; mc[2] = m[2]; }
                }
            double out[QMAX];
            rebuild_post(L, mc, alpha, Pc->tau, out);
            int64_t cell = x + (int64_t)Pc->n[0] * y;
            for (int q = 0; q < L->q; ++q) fc[(int64_t)q * Nc + cell] = out[q];
        }
}

/* Moments stored at t = 0 on the interface lines: local moments of the
 * stored populations (the initial state has no earlier step). */
void orc_refined_init_moments(const orc_problem *Pc, const orc_patch *G, const double *fc, double *M)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t N = ncell(Pc);
    for (int y = G->Y0 - 1; y <= G->Y0 + G->Hc + 1; ++y)
        for (int x = G->X0 - 1; x <= G->X0 + G->Wc + 1; ++x) {
            int64_t cell = x + (int64_t)Pc->n[0] * y;
            double f[QMAX], rho, j[3], Pi[3][3], u[3], Pn[3][3];
            for (int i = 0; i < L->q; ++i) f[i] = fc[(int64_t)i * N + cell];
            moments(L, f, &rho, j, Pi);
            for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
            pi_neq(L->d, rho, u, Pi, Pn);
            double *m = M + 6 * cell;
            m[0] = rho; m[1] = u[0]; m[2] = u[1];
            m[3] = Pn[0][0]; m[4] = Pn[0][1]; m[5] = Pn[1][1];
        }
}

/* One coarse step t -> t + 1 of the two-level grid:
 *   1. coarse step; coarse line moments at t + 1 from the pre-step field
 *   2. fine step t -> t + 1/2 (the ring holds t)
 *   3. fine ring <- coarse moments averaged between t and t + 1
 *   4. fine step t + 1/2 -> t + 1
 *   5. fine ring <- coarse moments at t + 1
 *   6. first covered coarse ring <- fine moments at t + 1
 * M0 holds the line moments at t on entry and at t + 1 on return. */
/* The three coupling operations of one parent / child pair, exported so that
 * a chain of nested patches can be stepped level by level (each level does
 * two steps per step of its parent, in the order of orc_refined_step). */
void orc_refine2_line_moments(const orc_problem *Pc, const orc_patch *G, const double *fc, double *M)
{
    coarse_line_moments(Pc, G, fc, M);
}

void orc_refine2_fill(const orc_problem *Pc, const orc_problem *Pf, const orc_patch *G, const double *M0,
                      const double *M1, double a, double *ff)
{
    fill_fine_ring(Pc, Pf, G, M0, M1, a, ff);
}

void orc_refine2_restrict(const orc_problem *Pc, const orc_problem *Pf, const orc_patch *G, const double *ff_half,
                          double *fc)
{
    restrict_to_coarse(Pc, Pf, G, ff_half, fc);
}

int orc_refined_step(const orc_problem *Pc, const orc_problem *Pf, const orc_patch *G,
                     double *fc, double *fc_work, double *ff, double *ff_work, double *M0,
                     double *M1, int64_t step)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t Nc = ncell(Pc), Nf = ncell(Pf);
    const size_t Mbytes = sizeof(double) * 6 * (size_t)Nc;
    coarse_line_moments(Pc, G, fc, M1);
    orc_step(Pc, fc, fc_work, step);
    orc_step(Pf, ff, ff_work, 2 * step);
    fill_fine_ring(Pc, Pf, G, M0, M1, 0.5, ff_work);
    orc_step(Pf, ff_work, ff, 2 * step + 1);
    fill_fine_ring(Pc, Pf, G, M0, M1, 1.0, ff);
    restrict_to_coarse(Pc, Pf, G, ff_work, fc_work);
    memcpy(fc, fc_work, sizeof(double) * (size_t)Nc * (size_t)L->q);
    memcpy(M0, M1, Mbytes);
    (void)Nf;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-level 2:1 grid refinement (Sec. II.B), 3D (D3Q19)                    */
/* ------------------------------------------------------------------------ */
/*
 * The 2D layout extended by one axis (readings R10-R12):
 *   - the fine patch covers the coarse nodes X0..X0+Wc, Y0..Y0+Hc,
 *     Z0..Z0+Dc; fine node (i, j, k) sits at (X0 + i/2, Y0 + j/2, Z0 + k/2);
 *   - the fine boundary shell (a coordinate on a face of the fine box) is
 *     rebuilt from coarse data after every fine substep; the first shell of
 *     covered coarse nodes is rebuilt from fine data after every coarse step;
 *     deeper covered coarse nodes are never read;
 *   - coarse -> fine in space: along every axis on which the fine node is
 *     odd, the 4-point centred cubic (-1, 9, 9, -1)/16; the tensor product of
 *     these on the interface planes (a node odd in both in-plane axes takes
 *     16 coarse nodes); linear in time as in 2D;
 *   - fine -> coarse: rho, u of the coincident fine node, Pi^neq filtered
 *     with the 3 x 3 x 3 full-weighting kernel (1,2,1)^3 / 64.
 * Interface moments m = (rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz) are
 * kept per coarse cell (10 doubles) on the six face planes of the patch
 * box, extended by one node past every edge.
 */
typedef struct {
    int X0, Y0, Z0, Wc, Hc, Dc;
} orc_patch3;

static void streamed_moments3(const orc_problem *P, const double *fin, int x, int y, int z, double m[10])
{
    const lattice_t *L = lattice(P->lattice);
    const int64_t N = ncell(P);
    const int64_t nx = P->n[0], ny = P->n[1], nz = P->n[2];
    const int64_t cell = x + nx * (y + ny * (int64_t)z);
    double f[QMAX], rho, j[3], Pi[3][3], u[3], Pn[3][3];
    for (int i = 0; i < L->q; ++i) {
        int64_t sx = ((x - L->xi[i][0]) % nx + nx) % nx;
        int64_t sy = ((y - L->xi[i][1]) % ny + ny) % ny;
        int64_t sz = ((z - L->xi[i][2]) % nz + nz) % nz;
        int64_t scl = sx + nx * (sy + ny * sz);
        if (P->solid && P->solid[scl] == 1)
            f[i] = fin[(int64_t)L->opp[i] * N + cell];
        else
            f[i] = fin[(int64_t)i * N + scl];
    }
    moments(L, f, &rho, j, Pi);
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    pi_neq(3, rho, u, Pi, Pn);
    m[0] = rho; m[1] = u[0]; m[2] = u[1]; m[3] = u[2];
    m[4] = Pn[0][0]; m[5] = Pn[0][1]; m[6] = Pn[0][2]; m[7] = Pn[1][1]; m[8] = Pn[1][2]; m[9] = Pn[2][2];
}

static void rebuild_post3(const lattice_t *L, const double m[10], double alpha, double tau, double *out)
{
    double u[3] = {m[1], m[2], m[3]};
    double Pn[3][3] = {{alpha * m[4], alpha * m[5], alpha * m[6]},
                       {alpha * m[5], alpha * m[7], alpha * m[8]},
                       {alpha * m[6], alpha * m[8], alpha * m[9]}};
    double feq[QMAX], fneq[QMAX];
    feqH(L, m[0], u, feq);
    fneqH(L, u, Pn, fneq);
    for (int i = 0; i < L->q; ++i) out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i];
}

/* Coarse node (x, y, z) lies on a face plane of the patch box, within the
 * box extended by one node along the in-plane axes. */
static int on_interface_plane3(const orc_patch3 *G, int x, int y, int z)
{
    const int ix = x - G->X0, iy = y - G->Y0, iz = z - G->Z0;
    if (ix < -1 || ix > G->Wc + 1 || iy < -1 || iy > G->Hc + 1 || iz < -1 || iz > G->Dc + 1) return 0;
    return ix == 0 || ix == G->Wc || iy == 0 || iy == G->Hc || iz == 0 || iz == G->Dc;
}

static void coarse_plane_moments3(const orc_problem *Pc, const orc_patch3 *G, const double *fc, double *M)
{
    const int64_t nx = Pc->n[0], ny = Pc->n[1];
    for (int z = G->Z0 - 1; z <= G->Z0 + G->Dc + 1; ++z)
        for (int y = G->Y0 - 1; y <= G->Y0 + G->Hc + 1; ++y)
            for (int x = G->X0 - 1; x <= G->X0 + G->Wc + 1; ++x)
                if (on_interface_plane3(G, x, y, z))
                    streamed_moments3(Pc, fc, x, y, z, M + 10 * (x + nx * (y + ny * (int64_t)z)));
}

/* 1D stencil of fine coordinate c along an axis: a coincident node (one
 * point, weight 1) or the centred cubic between coarse nodes (c-1)/2 and
 * (c+1)/2 (four points). */
static int stencil1(int c, int origin, int idx[4], double w[4])
{
    if (c % 2 == 0) {
        idx[0] = origin + c / 2;
        w[0] = 1.0;
        return 1;
    }
    const int a = origin + (c - 1) / 2;
    idx[0] = a - 1; idx[1] = a; idx[2] = a + 1; idx[3] = a + 2;
    w[0] = -1.0 / 16.0; w[1] = 9.0 / 16.0; w[2] = 9.0 / 16.0; w[3] = -1.0 / 16.0;
    return 4;
}

/* Interface moments at fine shell node (i, j, k): the time mix (1 - a) M0 +
 * a M1 of the coarse plane moments, interpolated by the tensor product of
 * the 1D stencils (exported for the pins as orc_refine3_interp). */
void orc_refine3_interp(const orc_problem *Pc, const orc_patch3 *G, const double *M0, const double *M1,
                        double a, int i, int j, int k, double m[10])
{
    const int64_t nxc = Pc->n[0], nyc = Pc->n[1];
    int ix[4], iy[4], iz[4];
    double wx[4], wy[4], wz[4];
    const int sx = stencil1(i, G->X0, ix, wx);
    const int sy = stencil1(j, G->Y0, iy, wy);
    const int sz = stencil1(k, G->Z0, iz, wz);
    for (int e = 0; e < 10; ++e) m[e] = 0.0;
    for (int c = 0; c < sz; ++c)
        for (int b = 0; b < sy; ++b)
            for (int q = 0; q < sx; ++q) {
                const int64_t cell = ix[q] + nxc * (iy[b] + nyc * (int64_t)iz[c]);
                const double wt = wx[q] * wy[b] * wz[c];
                for (int e = 0; e < 10; ++e)
                    m[e] += wt * ((1.0 - a) * M0[10 * cell + e] + a * M1[10 * cell + e]);
            }
}

static void fill_fine_shell3(const orc_problem *Pc, const orc_problem *Pf, const orc_patch3 *G,
                             const double *M0, const double *M1, double a, double *ff)
{
    const lattice_t *L = lattice(Pf->lattice);
    const int64_t Nf = ncell(Pf);
    const double alpha = Pf->tau / (2.0 * Pc->tau);
    const int nfx = 2 * G->Wc + 1, nfy = 2 * G->Hc + 1, nfz = 2 * G->Dc + 1;
    for (int k = 0; k < nfz; ++k)
        for (int j = 0; j < nfy; ++j)
            for (int i = 0; i < nfx; ++i) {
                if (!(i == 0 || j == 0 || k == 0 || i == nfx - 1 || j == nfy - 1 || k == nfz - 1)) continue;
                double m[10], out[QMAX];
                orc_refine3_interp(Pc, G, M0, M1, a, i, j, k, m);
                rebuild_post3(L, m, alpha, Pf->tau, out);
                const int64_t cell = i + (int64_t)nfx * (j + (int64_t)nfy * k);
                for (int q = 0; q < L->q; ++q) ff[(int64_t)q * Nf + cell] = out[q];
            }
}

/* Fine -> coarse moments from the 27 fine neighbours of the coincident node
 * (m27[10 * (a + 3 b + 9 c)], offsets a, b, c = 0, 1, 2 for -1, 0, +1):
 * rho, u of the centre, Pi^neq full-weighted by (1,2,1)^3 / 64 (exported
 * for the pins as orc_refine3_filter). */
void orc_refine3_filter(const double *m27, double mc[10])
{
    static const double w3[3] = {1.0, 2.0, 1.0};
    for (int e = 0; e < 10; ++e) mc[e] = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                const double *m = m27 + 10 * (a + 3 * b + 9 * c);
                const double wt = w3[a] * w3[b] * w3[c] / 64.0;
                for (int e = 4; e < 10; ++e) mc[e] += wt * m[e];
                if (a == 1 && b == 1 && c == 1)
                    for (int e = 0; e < 4; ++e) mc[e] = m[e];
            }
}

static void restrict_to_coarse3(const orc_problem *Pc, const orc_problem *Pf, const orc_patch3 *G,
                                const double *ff_prev, double *fc)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t Nc = ncell(Pc);
    const double alpha = 2.0 * Pc->tau / Pf->tau;
    for (int z = G->Z0 + 1; z <= G->Z0 + G->Dc - 1; ++z)
        for (int y = G->Y0 + 1; y <= G->Y0 + G->Hc - 1; ++y)
            for (int x = G->X0 + 1; x <= G->X0 + G->Wc - 1; ++x) {
                const int shell = x == G->X0 + 1 || x == G->X0 + G->Wc - 1 || y == G->Y0 + 1 ||
                                  y == G->Y0 + G->Hc - 1 || z == G->Z0 + 1 || z == G->Z0 + G->Dc - 1;
                if (!shell) continue;
                const int i = 2 * (x - G->X0), j = 2 * (y - G->Y0), k = 2 * (z - G->Z0);
                double m27[270], mc[10], out[QMAX];
                for (int c = 0; c < 3; ++c)
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a)
                            streamed_moments3(Pf, ff_prev, i + a - 1, j + b - 1, k + c - 1,
                                              m27 + 10 * (a + 3 * b + 9 * c));
                orc_refine3_filter(m27, mc);
                rebuild_post3(L, mc, alpha, Pc->tau, out);
                const int64_t cell = x + (int64_t)Pc->n[0] * (y + (int64_t)Pc->n[1] * z);
                for (int q = 0; q < L->q; ++q) fc[(int64_t)q * Nc + cell] = out[q];
            }
}

/* Interface moments at t = 0: local moments of the stored coarse populations. */
void orc_refined3_init_moments(const orc_problem *Pc, const orc_patch3 *G, const double *fc, double *M)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t N = ncell(Pc);
    const int64_t nx = Pc->n[0], ny = Pc->n[1];
    for (int z = G->Z0 - 1; z <= G->Z0 + G->Dc + 1; ++z)
        for (int y = G->Y0 - 1; y <= G->Y0 + G->Hc + 1; ++y)
            for (int x = G->X0 - 1; x <= G->X0 + G->Wc + 1; ++x) {
                if (!on_interface_plane3(G, x, y, z)) continue;
                const int64_t cell = x + nx * (y + ny * (int64_t)z);
                double f[QMAX], rho, j[3], Pi[3][3], u[3], Pn[3][3];
                for (int i = 0; i < L->q; ++i) f[i] = fc[(int64_t)i * N + cell];
                moments(L, f, &rho, j, Pi);
                for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
                pi_neq(3, rho, u, Pi, Pn);
                double *m = M + 10 * cell;
                m[0] = rho; m[1] = u[0]; m[2] = u[1]; m[3] = u[2];
                m[4] = Pn[0][0]; m[5] = Pn[0][1]; m[6] = Pn[0][2];
                m[7] = Pn[1][1]; m[8] = Pn[1][2]; m[9] = Pn[2][2];
            }
}

void orc_refine3_plane_moments(const orc_problem *Pc, const orc_patch3 *G, const double *fc, double *M)
{
    coarse_plane_moments3(Pc, G, fc, M);
}

void orc_refine3_fill(const orc_problem *Pc, const orc_problem *Pf, const orc_patch3 *G, const double *M0,
                      const double *M1, double a, double *ff)
{
    fill_fine_shell3(Pc, Pf, G, M0, M1, a, ff);
}

void orc_refine3_restrict(const orc_problem *Pc, const orc_problem *Pf, const orc_patch3 *G, const double *ff_half,
                          double *fc)
{
    restrict_to_coarse3(Pc, Pf, G, ff_half, fc);
}

/* One coarse step of the 3D two-level grid, in the order of the 2D one. */
int orc_refined3_step(const orc_problem *Pc, const orc_problem *Pf, const orc_patch3 *G,
                      double *fc, double *fc_work, double *ff, double *ff_work, double *M0,
                      double *M1, int64_t step)
{
    const lattice_t *L = lattice(Pc->lattice);
    const int64_t Nc = ncell(Pc);
    coarse_plane_moments3(Pc, G, fc, M1);
    orc_step(Pc, fc, fc_work, step);
    orc_step(Pf, ff, ff_work, 2 * step);
    fill_fine_shell3(Pc, Pf, G, M0, M1, 0.5, ff_work);
    orc_step(Pf, ff_work, ff, 2 * step + 1);
    fill_fine_shell3(Pc, Pf, G, M0, M1, 1.0, ff);
    restrict_to_coarse3(Pc, Pf, G, ff_work, fc_work);
    memcpy(fc, fc_work, sizeof(double) * (size_t)Nc * (size_t)L->q);
    memcpy(M0, M1, sizeof(double) * 10 * (size_t)Nc);
    return 0;
}
