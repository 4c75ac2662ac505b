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
//   * outflow node (zero gradient): collides the inward neighbour's streamed
//     populations
//   * sponge cell (Sec. II.C, Eq. spongeLB + Eq. dampingLBM, n = m = 1/2):
//     f* = (1 - chi) feqH(rho*, u*) + chi feqH(rho_ref, u_ref)
//          + (1 - 1/tau) fneqH(u*, Pi^neq about rho*, u*)
//   * bulk: f* = feqH(rho, u) + (1 - 1/tau) fneqH(u, Pi^neq)
#pragma once

#include "rr.cuh"

namespace rr {

enum { BC_PERIODIC = 0, BC_VELOCITY = 1, BC_OUTFLOW = 2 };

struct StepParams {
    int n[3];
    int periodic[3];
    int kind[6];
    int sponge_w[6];
    int any_sponge;
    int64_t ncell;
    int64_t face_cells[6];
    double u_face[6][3];
    const double *u_profile[6];  // device, 3 doubles per face cell, or null
    double sponge_chi[6];
    double rho_ref, rho_ref_m1, u_ref[3];  // rho_ref_m1 = rho_ref - 1
    uint64_t noise_seed;
    double noise_amp;
    double omega;  // 1 - 1/tau
    const uint8_t *solid;  // device, or null
    int64_t step;
};

template <class L, class S, class C>
__global__ void __launch_bounds__(256) k_stream_collide(const __grid_constant__ StepParams p,
                                                         const S *__restrict__ fin,
                                                         S *__restrict__ fout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    if (x >= nx) return;
    const int64_t N = p.ncell;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t cell = x + (int64_t)nx * y + nxy * z;
    const uint8_t *__restrict__ solid = p.solid;
    if (solid && solid[cell]) return;  // solid (1) and fixed (2) cells keep their populations

    // ---- boundary role and the node whose streamed populations are used
    int c[3] = {x, y, z};
    int s[3] = {x, y, z};
    int inlet = -1;
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        if (!p.periodic[a]) {
            if (c[a] == 0) {
                s[a] = 1;
                if (p.kind[2 * a] == BC_VELOCITY && inlet < 0) inlet = 2 * a;
            }
            if (c[a] == p.n[a] - 1) {
                s[a] = p.n[a] - 2;
                if (p.kind[2 * a + 1] == BC_VELOCITY && inlet < 0) inlet = 2 * a + 1;
            }
        }
    }
    // neighbour coordinates of s with wrap-around on periodic axes
    const int xm = s[0] == 0 ? nx - 1 : s[0] - 1, xp = s[0] == nx - 1 ? 0 : s[0] + 1;
    const int ym = s[1] == 0 ? ny - 1 : s[1] - 1, yp = s[1] == ny - 1 ? 0 : s[1] + 1;
    const int zm = s[2] == 0 ? nz - 1 : s[2] - 1, zp = s[2] == nz - 1 ? 0 : s[2] + 1;
    const int64_t scell = s[0] + (int64_t)nx * s[1] + nxy * s[2];

    // ---- streaming (pull) with halfway bounce-back
    C g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int X = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : s[0]);
        const int Y = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : s[1]);
        const int Z = L::D == 2 ? 0 : (L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : s[2]));
        const int64_t src = X + (int64_t)nx * Y + nxy * Z;
        if (solid && i != 0 && solid[src] == 1)
            g[i] = Store<S>::ld(fin + (int64_t)opp<L>(i) * N + scell);
        else
            g[i] = Store<S>::ld(fin + (int64_t)i * N + src);
    }

    const Mom<C> m = moments<L, C>(g);
    const C om = C(p.omega);
    Coef<C> k{};

    if (inlet >= 0) {
        // velocity node: rho, Pi^neq from the streamed neighbour, prescribed u
        const C rho = C(1) + m.dr;
        const C inv = C(1) / rho;
        const C vx = m.jx * inv, vy = m.jy * inv, vz = m.jz * inv;
        const Sym2<C> pn = pi_neq<C>(m, m.dr, rho, vx, vy, vz, L::D);
        const int a = inlet / 2;
        const int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
        const int64_t kf = c[t0] + (int64_t)p.n[t0] * c[t1];
        double ub[3];
        const double *prof = p.u_profile[inlet];
#pragma unroll
        for (int b = 0; b < 3; ++b) ub[b] = prof ? prof[3 * kf + b] : p.u_face[inlet][b];
        if (p.noise_amp > 0.0) {
            const double mag = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
            if (mag > 0.0) {
                const uint64_t base = (p.noise_seed << 32) +
                                      ((uint64_t)p.step * (uint64_t)p.face_cells[inlet] + (uint64_t)kf) * 3u;
#pragma unroll
                for (int b = 0; b < L::D; ++b) ub[b] += p.noise_amp * mag * (2.0 * u01(base + b) - 1.0);
            }
        }
        const C ux = C(ub[0]), uy = C(ub[1]), uz = L::D == 3 ? C(ub[2]) : C(0);
        add_eq<C>(k, C(1), m.dr, rho, ux, uy, uz);
        add_neq<C>(k, om, ux, uy, uz, pn);
    } else {
        C chi = C(0);
        if (p.any_sponge) {
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
            // sponge: damped moments rho*, rho* u* (n = m = 1/2)
            const C h = C(1) / (C(1) + C(0.5) * chi);
            const C rr = C(p.rho_ref);
            const C drs = (m.dr + C(0.5) * chi * C(p.rho_ref_m1)) * h;  // rho* - 1
            const C rs = C(1) + drs;
            const C jsx = (m.jx + C(0.5) * chi * rr * C(p.u_ref[0])) * h;
            const C jsy = (m.jy + C(0.5) * chi * rr * C(p.u_ref[1])) * h;
            const C jsz = (m.jz + C(0.5) * chi * rr * C(p.u_ref[2])) * h;
            const C inv = C(1) / rs;
            const C ux = jsx * inv, uy = jsy * inv, uz = L::D == 3 ? jsz * inv : C(0);
            const Sym2<C> pn = pi_neq<C>(m, drs, rs, ux, uy, uz, L::D);
            add_eq<C>(k, C(1) - chi, drs, rs, ux, uy, uz);
            add_eq<C>(k, chi, C(p.rho_ref_m1), rr, C(p.u_ref[0]), C(p.u_ref[1]), L::D == 3 ? C(p.u_ref[2]) : C(0));
            add_neq<C>(k, om, ux, uy, uz, pn);
        } else {
            const C rho = C(1) + m.dr;
            const C inv = C(1) / rho;
            const C ux = m.jx * inv, uy = m.jy * inv, uz = L::D == 3 ? m.jz * inv : C(0);
            const Sym2<C> pn = pi_neq<C>(m, m.dr, rho, ux, uy, uz, L::D);
            add_eq<C>(k, C(1), m.dr, rho, ux, uy, uz);
            add_neq<C>(k, om, ux, uy, uz, pn);
        }
    }

    // ---- rebuild, relax and store
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Store<S>::st(fout + (int64_t)i * N + cell, rebuild<L, C>(k, i));
}

// Launch wrapper: one thread per cell, blocks along x.
template <class L, class S, class C>
cudaError_t launch_stream_collide(const StepParams &p, const void *fin, void *fout, int block,
                                  cudaStream_t st)
{
    dim3 b(block, 1, 1);
    dim3 g((p.n[0] + block - 1) / block, p.n[1], p.n[2]);
    k_stream_collide<L, S, C><<<g, b, 0, st>>>(p, (const S *)fin, (S *)fout);
    return cudaGetLastError();
}

}  // namespace rr
