// serve.cuh -- batched multi-domain update for the serving engine.
//
// Many independent lattices advance in one launch: a tile list enumerates
// warp work items (domain, row, x segment); a persistent grid strides over
// them and every lane updates its cells with the same device functions as
// the single-lattice kernels (update_cell one cell per lane, update_vec V
// cells per lane, every row on its vector path since the domains are
// periodic), so a domain's arithmetic does not depend on what it is batched
// with.  Each domain carries its own step parameters, buffer pair
// (or one lattice with the in-place AA pattern), parity and remaining-step
// counter; k_batch_advance flips the parity and counts down after every
// step, and a domain whose counter reaches zero is skipped by later steps of
// the same captured round.
#pragma once

#include "step_vec.cuh"

namespace rr {

struct BatchDomain {
    StepParams p;
    void *f[2];
    char *base[2][kMaxQ];  // per-direction base addresses of the two lattices (the same lattice twice for AA)
    int cur;               // pull: the lattice holding the state; AA: 1 after a gather-push step
    int active;
    int aa;                // in-place AA streaming (one lattice)
    int64_t remaining;
};

// Work item of one warp: 32 * V consecutive cells of one row of one domain.
struct BatchTile {
    int domain;
    int row;   // y + ny z
    int xseg;  // cells [xseg * 32 V, (xseg + 1) * 32 V) of the row
    int pad;
};

// Resident 256-thread blocks per SM asked of the compiler: as the
// single-lattice kernel, 16-bit storage with two cells per lane is latency-
// bound and gets 64 registers (32 resident warps per SM) on D2Q9 / D3Q19;
// the other groups keep the registers they need.
template <class L, class S, int V>
struct BatchMinBlocks {
    static constexpr int value = (sizeof(S) == 2 && V == 2 && L::Q <= 19) ? 4 : 0;
};

template <class L, class S, class C, int V>
__global__ void __launch_bounds__(256, (BatchMinBlocks<L, S, V>::value))
    k_batched(const BatchDomain *__restrict__ doms, const BatchTile *__restrict__ tiles, int ntiles)
{
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = blockIdx.x * wpb + warp; t < ntiles; t += gridDim.x * wpb) {
        const BatchTile tl = tiles[t];
        const BatchDomain &d = doms[tl.domain];
        if (!d.active) continue;  // uniform across the warp
        const int ny = d.p.n[1];
        const int y = tl.row % ny, z = tl.row / ny;
        const int x0 = (tl.xseg * 32 + lane) * V;
        if (d.aa) {  // uniform across the warp: one domain per tile
            if constexpr (V == 1) {
                if (x0 < d.p.n[0]) {
                    if (d.cur)
                        update_cell_aa<L, S, C, false, kMaskNone, true>(d.p, d.base[0], x0, y, z);
                    else
                        update_cell_aa<L, S, C, false, kMaskNone, false>(d.p, d.base[0], x0, y, z);
                }
            } else {
                if (d.cur)
                    update_vec<L, S, C, V, V, kAALocal, 1>(d.p, d.base[0], d.base[0], x0, y, z);
                else
                    update_vec<L, S, C, V, V, kAAPush, 1>(d.p, d.base[0], d.base[0], x0, y, z);
            }
        } else if constexpr (V == 1) {
            if (x0 < d.p.n[0]) update_cell<L, S, C, false, kMaskNone>(d.p, d.base[d.cur], d.base[1 - d.cur], x0, y, z);
        } else {
            update_vec<L, S, C, V, V, kPull, 1>(d.p, d.base[d.cur], d.base[1 - d.cur], x0, y, z);
        }
    }
}

__global__ void k_batch_advance(BatchDomain *__restrict__ doms, int ndom)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ndom) return;
    BatchDomain &d = doms[k];
    if (!d.active) return;
    d.cur = 1 - d.cur;
    d.p.step += 1;
    d.remaining -= 1;
    if (d.remaining <= 0) d.active = 0;
}

}  // namespace rr
