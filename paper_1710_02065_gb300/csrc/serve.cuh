// serve.cuh -- batched multi-domain update for the serving engine.
//
// Many independent lattices advance in one launch: a tile list enumerates
// (domain, first row, rows) work items; a persistent grid strides over the
// tiles and every thread updates cells with the same update_cell() as the
// single-lattice kernel, so a domain's arithmetic does not depend on what it
// is batched with.  Each domain carries its own step parameters, buffer pair,
// parity and remaining-step counter; k_batch_advance flips the parity and
// counts down after every step, and a domain whose counter reaches zero is
// skipped by later steps of the same captured round.
#pragma once

#include "step.cuh"

namespace rr {

struct BatchDomain {
    StepParams p;
    void *f[2];
    char *base[2][19];  // per-direction base addresses of the two lattices
    int cur;
    int active;
    int64_t remaining;
};

struct BatchTile {
    int domain;
    int row0;   // first row (y + ny z)
    int rows;   // number of consecutive rows
    int pad;
};

template <class L, class S, class C>
__global__ void __launch_bounds__(128) k_batched(const BatchDomain *__restrict__ doms,
                                                  const BatchTile *__restrict__ tiles, int ntiles)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        const BatchDomain &d = doms[tl.domain];
        if (!d.active) continue;
        const int nx = d.p.n[0], ny = d.p.n[1];
        const char *const *in = d.base[d.cur];
        char *const *out = d.base[1 - d.cur];
        const int cells = tl.rows * nx;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int r = tl.row0 + i / nx;
            update_cell<L, S, C>(d.p, in, out, i % nx, r % ny, r / ny);
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
