// lbm_api.cu -- host runtime behind include/lbm.h: handle, validation,
// device memory, launches.  Every numerical step runs in the kernels of
// step.cuh / aux_kernels.cuh; this file only moves arguments.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "aux_kernels.cuh"
#include "dispatch.h"
#include "refine.cuh"
#include "step.cuh"

using namespace rr;

// A refined level (Sec. II.B): level k + 1 covers a box of level k's nodes
// at half the spacing; levels nest, each inside the previous one.
struct FineLevel {
    int n[3] = {1, 1, 1};
    int64_t ncell = 0;
    double tau = 0.0;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *mask_d = nullptr;           // ring fixed + user solids
    bool has_solid = false;              // the mask holds solid cells
    std::vector<uint8_t> user_mask;      // user solids (host copy)
    RefineGeom geom{};                   // position in the parent level's nodes
    double *M[2] = {nullptr, nullptr};   // parent-side interface moments at t and t + 1 (compute type; sized for FP64)
    int mcur = 0;
};

struct lbm_ctx {
    int lattice = 0, q = 0, d = 0, prec = 0;
    int n[3] = {1, 1, 1};
    int64_t ncell = 0;
    size_t elem = 0;
    double tau = 0.0, Ma_ref = 0.0;
    cudaStream_t stream = nullptr;
    // refined levels beneath level 0 run on a second stream of higher
    // priority, concurrent with the level-0 update (fork / join events)
    int level_overlap = 1;
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int sms = 0;  // SMs of the device (set with the second stream)
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *solid_d = nullptr;
    bool has_solid = false;  // level 0's mask holds solid cells (else only fixed ones)
    double *prof_d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int kind[6] = {0, 0, 0, 0, 0, 0};
    double u_face[6][3] = {};
    double rho_face[6] = {1, 1, 1, 1, 1, 1};
    int sponge_w[6] = {0, 0, 0, 0, 0, 0};
    double sponge_chi[6] = {0, 0, 0, 0, 0, 0};
    double radial[6] = {0, 0, 0, 0, 0, 0};
    float *chi_tab_f = nullptr;   // per-axis face-layer strength (nx + ny + nz), FP32
    double *chi_tab_d = nullptr;  // the same in FP64
    bool ref_set = false;
    double rho_ref = 1.0, u_ref[3] = {0, 0, 0};
    uint64_t noise_seed = 0;
    double noise_amp = 0.0;
    int64_t step = 0, launches = 0;
    int block = 0;  // 0: automatic
    int vec = 0;    // cells per thread; 0: automatic, 1: scalar kernel
    int staging = -1;     // row-staged kernel: -1 default (off), 0 off, 1 on where eligible
    int stages = 0;       // its shared-memory stages (0: 2)
    int rows_block = 0;   // its threads per CTA (0: automatic)
    unsigned *err_d = nullptr;  // device error word of the row-staged kernel (bounded waits)
    uint64_t rows_wait_ns = 2000000000ull;  // limit of each of its waits for a tile's copies
    int collision = LBM_COLLISION_RR;
    // streaming pattern of level 0: LBM_STREAM_PULL (two lattices) or
    // LBM_STREAM_AA (one lattice in place, f[1] aliases f[0]); aa_odd: the
    // lattice holds the push layout a gather-push step left (the next step is
    // a local one), else the standard layout
    int pattern = LBM_STREAM_PULL;
    int aa_odd = 0;
    // storage shift by the equilibrium at (1, shift_u): dsh[i] = feqH_i(1, u) - w_i
    // (host in FP64, device table dsh_d of q doubles); shifted = false: w_i
    bool shifted = false;
    double shift_u[3] = {0, 0, 0};
    double dsh[27] = {};
    double *dsh_d = nullptr;
    double jet_ref[7] = {0, 0, 0, 0, 0, 0, 0};  // yc, zc, U_J, D, x0, B, S; D = 0: none
    int order4 = 0;             // D2Q9: optional fourth-order H_xxyy term
    double *rho_acc = nullptr;  // running sum of rho per cell (temporal mean of p), or null
    int64_t rho_count = 0;
    double *red_d = nullptr;  // reduction partials + result
    // bounded device staging of host transfers (set/get state, populations,
    // moments), allocated on first use, at most kStageBytes; bad_d: lowest
    // index of an invalid cell found by the state upload
    double *stage_d = nullptr;
    size_t stage_bytes = 0;
    size_t stage_max = size_t(256) << 20;
    unsigned long long *bad_d = nullptr;
    int red_blocks = 0;
    std::vector<uint8_t> user_mask;  // caller's cell types (host copy); empty: none
    std::vector<FineLevel *> levels;  // refined levels 1, 2, ... (each inside the previous one)
    // graphs of 1, 2, 4, 8 or 16 step pairs (the parity period) replayed by
    // lbm_step, per lattice parity; valid for one configuration version
    int64_t cfg_version = 0;
    struct StepGraph {
        uint64_t sig;  // lattice parities the graph was captured at
        int pairs;     // step pairs it holds
        cudaGraphExec_t exec;
        int64_t launches;  // kernel launches per replay
    };
    std::vector<StepGraph> graphs;
    int64_t graphs_version = -1;
    std::string err;
};

// Device shift table of a level's storage (null: the w_i shift); only the
// single level carries one (a shift is not combined with refinement patches)
struct GridRef;
static const double *shift_of(const lbm_ctx *h, const GridRef &g);

// View of one level's storage, so state and diagnostics work on either level
struct GridRef {
    int n[3];
    int64_t ncell;
    void **f;
    int *cur;
    const uint8_t *mask;
};

static const double *shift_of(const lbm_ctx *h, const GridRef &g)
{
    return (h->shifted && g.f == h->f) ? h->dsh_d : nullptr;
}

static GridRef coarse_ref(lbm_ctx *h)
{
    return GridRef{{h->n[0], h->n[1], h->n[2]}, h->ncell, h->f, &h->cur, h->solid_d};
}
static int nlevels(const lbm_ctx *h) { return 1 + (int)h->levels.size(); }
static FineLevel *fine_level(lbm_ctx *h, int k) { return h->levels[(size_t)k - 1]; }  // k >= 1
static GridRef level_grid(lbm_ctx *h, int k)
{
    if (k == 0) return coarse_ref(h);
    FineLevel *F = fine_level(h, k);
    return GridRef{{F->n[0], F->n[1], F->n[2]}, F->ncell, F->f, &F->cur, F->mask_d};
}
static double level_tau(lbm_ctx *h, int k) { return k == 0 ? h->tau : fine_level(h, k)->tau; }
// Bytes of one interface-moment buffer of a refined level (sized for FP64)
static size_t moment_bytes(bool three, const RefineGeom &g)
{
    return three ? sizeof(double) * 10 * (size_t)box3_entries(g) : sizeof(double) * 6 * (size_t)line_count(g);
}
// The mask the interface kernels test for bounce-back links: null when the
// level holds no solid cells (its fixed cells need no test there)
static const uint8_t *links_mask(lbm_ctx *h, int k)
{
    return (k == 0 ? h->has_solid : fine_level(h, k)->has_solid) ? level_grid(h, k).mask : nullptr;
}

static thread_local std::string g_create_err;

void rr::rr_set_global_error(const char *msg) { g_create_err = msg; }

static int fail(lbm_ctx *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_err = buf;
    return code;
}

#define CUDA_TRY(h, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(h, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

#define CHECK_HANDLE(h)                                                                           \
    do {                                                                                          \
        if (!(h)) return fail(nullptr, LBM_EINVAL, "null handle");                              \
    } while (0)

// ---------------------------------------------------------------------------
// Typed dispatch of the auxiliary kernels
// ---------------------------------------------------------------------------
template <template <class, class> class Fn, class... A>
static cudaError_t dispatch(int lattice, int prec, A... args)
{
    if (lattice == LBM_D2Q9) {
        switch (prec) {
        case LBM_FP64: return Fn<D2Q9, double>::run(args...);
        case LBM_FP32: return Fn<D2Q9, float>::run(args...);
        case LBM_FP16_SHIFTED: return Fn<D2Q9, __half>::run(args...);
        case LBM_BF16_SHIFTED: return Fn<D2Q9, __nv_bfloat16>::run(args...);
        }
    } else if (lattice == LBM_D3Q27) {
        switch (prec) {
        case LBM_FP64: return Fn<D3Q27, double>::run(args...);
        case LBM_FP32: return Fn<D3Q27, float>::run(args...);
        case LBM_FP16_SHIFTED: return Fn<D3Q27, __half>::run(args...);
        case LBM_BF16_SHIFTED: return Fn<D3Q27, __nv_bfloat16>::run(args...);
        }
    } else {
        switch (prec) {
        case LBM_FP64: return Fn<D3Q19, double>::run(args...);
        case LBM_FP32: return Fn<D3Q19, float>::run(args...);
        case LBM_FP16_SHIFTED: return Fn<D3Q19, __half>::run(args...);
        case LBM_BF16_SHIFTED: return Fn<D3Q19, __nv_bfloat16>::run(args...);
        }
    }
    return cudaErrorInvalidValue;
}

static unsigned grid1(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class L, class S>
struct InitEq {
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, const double *rho, const double *u,
                           void *f0, void *f1, int order4, unsigned long long *bad, const double *dsh)
    {
        k_init_eq<L, S><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, rho, u, (S *)f0, (S *)f1, order4, bad, dsh);
        return cudaGetLastError();
    }
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, const float *rho, const float *u,
                           void *f0, void *f1, int order4, unsigned long long *bad, const double *dsh)
    {
        k_init_eq<L, S, float><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, rho, u, (S *)f0, (S *)f1, order4, bad, dsh);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct SetDir {
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, int i, const double *src, void *f0,
                           void *f1, const double *dsh)
    {
        k_set_dir<L, S><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, i, src, (S *)f0, (S *)f1, dsh);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct GetDir {
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, int i, const void *f, double *dst,
                           const double *dsh)
    {
        k_get_dir<L, S><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, i, (const S *)f, dst, dsh);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Moments {
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, const void *f, double *rho,
                           double *u, double *pn, const double *dsh)
    {
        k_moments<L, S><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, (const S *)f, rho, u, pn, dsh);
        return cudaGetLastError();
    }
    static cudaError_t run(cudaStream_t st, int64_t N, int64_t c0, int64_t n, const void *f, float *rho,
                           float *u, float *pn, const double *dsh)
    {
        k_moments<L, S, float><<<grid1(n, 256), 256, 0, st>>>(N, c0, n, (const S *)f, rho, u, pn, dsh);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Reduce {
    static cudaError_t run(cudaStream_t st, int64_t N, const void *f, const uint8_t *solid,
                           double *partial, int nblocks, const double *dsh)
    {
        k_reduce<L, S><<<nblocks, RED_BLOCK, 0, st>>>(N, (const S *)f, solid, partial, dsh);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, 32 * RED_FIELDS, 0, st>>>(nblocks, partial, partial + (int64_t)nblocks * RED_FIELDS);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Force {
    static cudaError_t run(cudaStream_t st, const int *n, const int *per, const void *f, const uint8_t *mask,
                           double *partial, int nblocks, const double *dsh)
    {
        k_force<L, S><<<nblocks, RED_BLOCK, 0, st>>>(n[0], n[1], n[2], per[0], per[1], per[2], (const S *)f, mask,
                                                      partial, dsh);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, 32 * RED_FIELDS, 0, st>>>(nblocks, partial, partial + (int64_t)nblocks * RED_FIELDS);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct ShiftValues {
    static cudaError_t run(cudaStream_t st, int64_t N, int i, void *f, double delta)
    {
        k_shift_values<S><<<grid1(N, 256), 256, 0, st>>>(N, (S *)f + (int64_t)i * N, delta);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct ShiftTable {
    // dsh[i] = feqH_i(1, u) - w_i: the w_i-shifted equilibrium of one cell at rho = 1, in FP64
    static cudaError_t run(cudaStream_t st, const double *one_u, double *dsh)
    {
        k_init_eq<L, double><<<1, 1, 0, st>>>(1, 0, 1, one_u, one_u + 1, dsh, dsh, 0, nullptr);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Probe {
    static cudaError_t run(cudaStream_t st, int n, const int64_t *cells, int64_t N, const void *f,
                           double *rho, int pressure, double rho_ref)
    {
        k_probe<L, S><<<grid1(n, 128), 128, 0, st>>>(n, cells, N, (const S *)f, rho, pressure, rho_ref);
        return cudaGetLastError();
    }
};

template <class L, class S>
struct RhoAccumulate {
    static cudaError_t run(cudaStream_t st, int64_t N, const void *f, double *acc)
    {
        k_rho_accumulate<L, S><<<grid1(N, 256), 256, 0, st>>>(N, (const S *)f, acc);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct PressureFluct {
    static cudaError_t run(cudaStream_t st, int64_t N, const void *f, const double *acc, double count, double *dp,
                           double *dp_mean)
    {
        k_pressure_fluct<L, S><<<grid1(N, 256), 256, 0, st>>>(N, (const S *)f, acc, count, dp, dp_mean);
        return cudaGetLastError();
    }
};

// ---------------------------------------------------------------------------
// Lattice table (host)
// ---------------------------------------------------------------------------
template <class L>
static void table(int *q, int *d, int *xi, double *w)
{
    if (q) *q = L::Q;
    if (d) *d = L::D;
    for (int i = 0; i < L::Q; ++i) {
        if (xi) {
            xi[3 * i] = L::cx(i);
            xi[3 * i + 1] = L::cy(i);
            xi[3 * i + 2] = L::cz(i);
        }
        if (w) w[i] = weight<L>(i);
    }
}

extern "C" int lbm_lattice_table(int lattice, int *q, int *d, int *xi, double *w)
{
    if (lattice == LBM_D2Q9)
        table<D2Q9>(q, d, xi, w);
    else if (lattice == LBM_D3Q19)
        table<D3Q19>(q, d, xi, w);
    else if (lattice == LBM_D3Q27)
        table<D3Q27>(q, d, xi, w);
    else
        return fail(nullptr, LBM_EINVAL, "unknown lattice %d", lattice);
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Lifetime
// ---------------------------------------------------------------------------
static size_t prec_bytes(int prec)
{
    switch (prec) {
    case LBM_FP64: return 8;
    case LBM_FP32: return 4;
    case LBM_FP16_SHIFTED:
    case LBM_BF16_SHIFTED: return 2;
    }
    return 0;
}

// Per-axis sponge strength of the face layers (Sec. II.C): for each
// coordinate c of axis a, the max over the axis's two faces of
// chi_max sigma(d), d = depth of c inside the layer (0 at its inner edge),
// sigma(d) = 3125 (W - d) d^4 / (256 W^5).  Computed in FP64 on the host and
// copied, in stream order, to the FP64 and FP32 device tables the kernels
// read (so launches already queued keep their own values).
static int upload_sponge_tables(lbm_ctx *h)
{
    const int total = h->n[0] + h->n[1] + h->n[2];
    if (!h->chi_tab_d) {
        if (cudaMalloc(&h->chi_tab_d, sizeof(double) * (size_t)total) != cudaSuccess ||
            cudaMalloc(&h->chi_tab_f, sizeof(float) * (size_t)total) != cudaSuccess)
            return LBM_ENOMEM;
    }
    std::vector<double> td((size_t)total, 0.0);
    std::vector<float> tf((size_t)total, 0.0f);
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < h->n[a]; ++c) {
            double v = 0.0;
            for (int f = 2 * a; f <= 2 * a + 1; ++f) {
                const int W = h->sponge_w[f];
                if (W <= 0 || !(h->sponge_chi[f] > 0.0)) continue;
                const int d = (f & 1) ? c - (h->n[a] - W) : W - 1 - c;
                if (d < 0) continue;
                const double dd = d, WW = W;
                const double sig = 3125.0 * (WW - dd) * dd * dd * dd * dd / (256.0 * WW * WW * WW * WW * WW);
                const double chi = h->sponge_chi[f] * sig;
                if (chi > v) v = chi;
            }
            td[(size_t)(off + c)] = v;
            tf[(size_t)(off + c)] = (float)v;
        }
        off += h->n[a];
    }
    if (cudaMemcpyAsync(h->chi_tab_d, td.data(), sizeof(double) * td.size(), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(h->chi_tab_f, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess)
        return LBM_ECUDA;
    // pageable sources: the copies are staged before the calls return, but
    // make the host buffers' lifetime independent of that
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static void release(lbm_ctx *h)
{
    if (!h) return;
    if (h->f[0]) cudaFree(h->f[0]);
    if (h->f[1] && h->f[1] != h->f[0]) cudaFree(h->f[1]);
    if (h->dsh_d) cudaFree(h->dsh_d);
    if (h->solid_d) cudaFree(h->solid_d);
    for (int k = 0; k < 6; ++k)
        if (h->prof_d[k]) cudaFree(h->prof_d[k]);
    if (h->red_d) cudaFree(h->red_d);
    if (h->err_d) cudaFree(h->err_d);
    if (h->chi_tab_f) cudaFree(h->chi_tab_f);
    if (h->stage_d) cudaFree(h->stage_d);
    if (h->bad_d) cudaFree(h->bad_d);
    if (h->chi_tab_d) cudaFree(h->chi_tab_d);
    if (h->rho_acc) cudaFree(h->rho_acc);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    for (FineLevel *F : h->levels) {
        for (int k = 0; k < 2; ++k) {
            if (F->f[k]) cudaFree(F->f[k]);
            if (F->M[k]) cudaFree(F->M[k]);
        }
        if (F->mask_d) cudaFree(F->mask_d);
        delete F;
    }
    delete h;
}

extern "C" int lbm_create(lbm_handle *out, int lattice, const int extents[3], double tau_or_nu,
                          int value_is_nu, double Ma_ref, int precision, void *cuda_stream)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is null");
    *out = nullptr;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q27)
        return fail(nullptr, LBM_EINVAL, "unknown lattice %d", lattice);
    if (!prec_bytes(precision)) return fail(nullptr, LBM_EINVAL, "unknown precision %d", precision);
    if (!extents) return fail(nullptr, LBM_EINVAL, "extents is null");
    for (int a = 0; a < 3; ++a)
        if (extents[a] < 1) return fail(nullptr, LBM_EINVAL, "extent %d is %d (< 1)", a, extents[a]);
    if (lattice == LBM_D2Q9 && extents[2] != 1)
        return fail(nullptr, LBM_EINVAL, "D2Q9 needs extents[2] == 1");
    if (extents[1] > 65535 || extents[2] > 65535)
        return fail(nullptr, LBM_EINVAL, "extents[1] and extents[2] must be <= 65535");
    if ((int64_t)extents[0] * extents[1] * extents[2] > 2147483647LL)
        return fail(nullptr, LBM_EINVAL, "a lattice holds at most 2^31 - 1 cells");
    double tau = value_is_nu ? tau_or_nu * 3.0 + 0.5 : tau_or_nu;
    if (!(tau > 0.5) || !std::isfinite(tau))
        return fail(nullptr, LBM_EINVAL, "tau = %g must be > 1/2 (nu > 0)", tau);
    if (!(Ma_ref >= 0.0 && Ma_ref <= 0.6))
        return fail(nullptr, LBM_EINVAL, "Ma_ref = %g outside [0, 0.6]", Ma_ref);

    lbm_ctx *h = new lbm_ctx();
    h->lattice = lattice;
    h->q = lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q19 ? 19 : 27);
    h->d = lattice == LBM_D2Q9 ? 2 : 3;
    h->prec = precision;
    h->elem = prec_bytes(precision);
    for (int a = 0; a < 3; ++a) h->n[a] = extents[a];
    h->ncell = (int64_t)extents[0] * extents[1] * extents[2];
    h->tau = tau;
    h->Ma_ref = Ma_ref;
    h->stream = (cudaStream_t)cuda_stream;

    const size_t bytes = (size_t)h->q * (size_t)h->ncell * h->elem;
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(&h->f[k], bytes);
        if (e != cudaSuccess) {
            int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
            fail(nullptr, code, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
            cudaGetLastError();
            release(h);
            return code;
        }
    }
    h->red_blocks = 4 * 152;
    if (cudaMalloc(&h->red_d, sizeof(double) * (size_t)(h->red_blocks + 1) * RED_FIELDS) != cudaSuccess) {
        cudaGetLastError();
        release(h);
        return fail(nullptr, LBM_ENOMEM, "cudaMalloc of reduction scratch failed");
    }
    if (cudaMalloc(&h->err_d, sizeof(unsigned)) != cudaSuccess ||
        cudaMemsetAsync(h->err_d, 0, sizeof(unsigned), h->stream) != cudaSuccess) {
        cudaGetLastError();
        release(h);
        return fail(nullptr, LBM_ENOMEM, "cudaMalloc of the error word failed");
    }
    if (upload_sponge_tables(h) != LBM_OK) {
        cudaGetLastError();
        release(h);
        return fail(nullptr, LBM_ENOMEM, "allocating the sponge tables failed");
    }
    // rest state: rho = 1, u = 0 is g = f - w = 0 in every storage format
    for (int k = 0; k < 2; ++k)
        if (cudaMemsetAsync(h->f[k], 0, bytes, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            fail(nullptr, LBM_ECUDA, "clearing the populations failed: %s", cudaGetErrorString(cudaGetLastError()));
            release(h);
            return LBM_ECUDA;
        }
    *out = h;
    return LBM_OK;
}

extern "C" void lbm_destroy(lbm_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
}

extern "C" const char *lbm_last_error(lbm_handle h)
{
    return h ? h->err.c_str() : g_create_err.c_str();
}

// ---------------------------------------------------------------------------
// Configuration
// ---------------------------------------------------------------------------
// Device cell-type byte: bits 0-1 the type (fluid 0, solid 1, fixed 2); bit 2
// (MASK_NEAR_SOLID) set when some lattice neighbour x - xi_i (with wrap-around
// on every axis, as the kernels pull) is solid, so that cells away from walls
// skip the per-direction bounce-back tests.
template <class L>
static void add_near_solid_bits(std::vector<uint8_t> &m, const int n[3])
{
    // a cell c has the solid neighbour s = c - xi_i exactly when c = s + xi_i:
    // mark the neighbours of every solid cell
    const int64_t nx = n[0], ny = n[1], nz = n[2];
    std::vector<int64_t> solids;
    for (size_t c = 0; c < m.size(); ++c)
        if ((m[c] & 3) == LBM_CELL_SOLID) solids.push_back((int64_t)c);
    for (const int64_t c : solids) {
        const int64_t x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
        for (int i = 1; i < L::Q; ++i) {
            const int64_t X = (x + L::cx(i) + nx) % nx, Y = (y + L::cy(i) + ny) % ny, Z = (z + L::cz(i) + nz) % nz;
            m[X + nx * (Y + ny * Z)] |= MASK_NEAR_SOLID;
        }
    }
}

static void add_near_solid(lbm_ctx *h, std::vector<uint8_t> &m, const int n[3])
{
    if (h->lattice == LBM_D2Q9)
        add_near_solid_bits<D2Q9>(m, n);
    else if (h->lattice == LBM_D3Q19)
        add_near_solid_bits<D3Q19>(m, n);
    else
        add_near_solid_bits<D3Q27>(m, n);
}

// Upload the cell types of level k: the caller's types; on a refined level
// its boundary ring (2D) / shell (3D), rebuilt from the parent, as fixed
// cells; on a level with a child the child's covered interior (strictly
// inside the child's box on every axis) as fixed cells; plus the near-solid
// bits.  Level 0 without types and without a child has no mask.
static int upload_level_mask(lbm_ctx *h, int k)
{
    const bool has_child = k < (int)h->levels.size();
    GridRef g = level_grid(h, k);
    const std::vector<uint8_t> &user = k == 0 ? h->user_mask : fine_level(h, k)->user_mask;
    if (k == 0 && user.empty() && !has_child) {
        if (h->solid_d) cudaFree(h->solid_d);
        h->solid_d = nullptr;
        h->has_solid = false;
        return LBM_OK;
    }
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    std::vector<uint8_t> m(user);
    if (m.empty()) m.assign((size_t)g.ncell, (uint8_t)LBM_CELL_FLUID);
    auto at = [&](int x, int y, int z) -> uint8_t & { return m[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)]; };
    const bool three = h->d == 3;
    if (k >= 1)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x)
                    if (x == 0 || y == 0 || x == nx - 1 || y == ny - 1 || (three && (z == 0 || z == nz - 1)))
                        at(x, y, z) = LBM_CELL_FIXED;
    if (has_child) {
        const RefineGeom &c = fine_level(h, k + 1)->geom;
        const int z0 = three ? c.Z0 + 1 : 0, z1 = three ? c.Z0 + c.Dc : 1;
        for (int z = z0; z < z1; ++z)
            for (int y = c.Y0 + 1; y < c.Y0 + c.Hc; ++y)
                for (int x = c.X0 + 1; x < c.X0 + c.Wc; ++x) at(x, y, z) = LBM_CELL_FIXED;
    }
    add_near_solid(h, m, g.n);
    bool any = false;
    for (const uint8_t v : m) any = any || (v & MASK_TYPE) == MASK_SOLID;
    (k == 0 ? h->has_solid : fine_level(h, k)->has_solid) = any;
    uint8_t *&dst = k == 0 ? h->solid_d : fine_level(h, k)->mask_d;
    if (!dst) CUDA_TRY(h, cudaMalloc(&dst, (size_t)g.ncell));
    CUDA_TRY(h, cudaMemcpyAsync(dst, m.data(), (size_t)g.ncell, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

static int check_cell_types(lbm_ctx *h, const uint8_t *t, int64_t n)
{
    for (int64_t c = 0; c < n; ++c)
        if (t[c] > LBM_CELL_FIXED)
            return fail(h, LBM_EINVAL, "cell_type[%lld] = %d is not a cell type", (long long)c, t[c]);
    return LBM_OK;
}

extern "C" int lbm_set_geometry(lbm_handle h, const uint8_t *cell_type)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (cell_type) {
        int rc = check_cell_types(h, cell_type, h->ncell);
        if (rc != LBM_OK) return rc;
        h->user_mask.assign(cell_type, cell_type + h->ncell);
    } else {
        h->user_mask.clear();
    }
    return upload_level_mask(h, 0);
}

static int64_t face_cells(const lbm_ctx *h, int face)
{
    int a = face / 2;
    int t0 = a == 0 ? 1 : 0, t1 = a == 2 ? 1 : 2;
    return (int64_t)h->n[t0] * h->n[t1];
}

extern "C" int lbm_set_boundary(lbm_handle h, int face, int kind, const double u_in[3],
                                const double *u_profile)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (face < 0 || face > 5) return fail(h, LBM_EINVAL, "face %d out of range", face);
    if (kind < LBM_BC_PERIODIC || kind > LBM_BC_PRESSURE) return fail(h, LBM_EINVAL, "unknown boundary kind %d", kind);
    if (h->d == 2 && face >= 4 && kind != LBM_BC_PERIODIC)
        return fail(h, LBM_EINVAL, "2D lattice: z faces are periodic");
    if (kind == LBM_BC_VELOCITY && !u_in && !u_profile)
        return fail(h, LBM_EINVAL, "velocity face needs u_in or u_profile");
    if (h->prof_d[face]) {
        cudaFree(h->prof_d[face]);
        h->prof_d[face] = nullptr;
    }
    h->kind[face] = kind;
    for (int a = 0; a < 3; ++a) h->u_face[face][a] = (kind == LBM_BC_VELOCITY && u_in) ? u_in[a] : 0.0;
    if (h->d == 2 && h->u_face[face][2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_z must be 0");
    if (kind == LBM_BC_VELOCITY && u_profile) {
        const int64_t nf = face_cells(h, face);
        if (h->d == 2)
            for (int64_t k = 0; k < nf; ++k)
                if (u_profile[3 * k + 2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: profile u_z must be 0");
        CUDA_TRY(h, cudaMalloc(&h->prof_d[face], sizeof(double) * 3 * (size_t)nf));
        CUDA_TRY(h, cudaMemcpyAsync(h->prof_d[face], u_profile, sizeof(double) * 3 * (size_t)nf,
                                    cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

extern "C" int lbm_set_pressure(lbm_handle h, int face, double rho_out)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (!(rho_out > 0.0) || !std::isfinite(rho_out))
        return fail(h, LBM_EINVAL, "rho_out = %g must be finite and > 0", rho_out);
    int rc = lbm_set_boundary(h, face, LBM_BC_PRESSURE, nullptr, nullptr);
    if (rc != LBM_OK) return rc;
    h->rho_face[face] = rho_out;
    return LBM_OK;
}

extern "C" int lbm_set_inlet_noise(lbm_handle h, uint64_t seed, double amplitude)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (!(amplitude >= 0.0) || !std::isfinite(amplitude))
        return fail(h, LBM_EINVAL, "noise amplitude %g must be finite and >= 0", amplitude);
    if (seed >= (1ull << 32)) return fail(h, LBM_EINVAL, "noise seed must be < 2^32");
    h->noise_seed = seed;
    h->noise_amp = amplitude;
    return LBM_OK;
}

extern "C" int lbm_set_sponge(lbm_handle h, int face, int width, double chi_max, double rho_ref,
                              const double u_ref[3])
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (face < 0 || face > 5) return fail(h, LBM_EINVAL, "face %d out of range", face);
    if (h->d == 2 && face >= 4 && width != 0) return fail(h, LBM_EINVAL, "2D lattice: no z sponge");
    if (width < 0 || width > h->n[face / 2])
        return fail(h, LBM_EINVAL, "sponge width %d outside [0, %d]", width, h->n[face / 2]);
    if (width == 0) {
        h->sponge_w[face] = 0;
        h->sponge_chi[face] = 0.0;
        return upload_sponge_tables(h) == LBM_OK ? LBM_OK
                                                 : fail(h, LBM_ECUDA, "uploading the sponge tables failed");
    }
    if (!(chi_max >= 0.0) || !(chi_max < 4.0 * h->tau))
        return fail(h, LBM_EINVAL, "chi_max = %g must be in [0, 4 tau = %g) for stability", chi_max, 4.0 * h->tau);
    double ur[3] = {0, 0, 0};
    if (u_ref)
        for (int a = 0; a < 3; ++a) ur[a] = u_ref[a];
    if (h->d == 2 && ur[2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_ref z must be 0");
    if (!(rho_ref > 0.0)) return fail(h, LBM_EINVAL, "rho_ref = %g must be > 0", rho_ref);
    bool other = h->radial[4] > 0.0;
    for (int f = 0; f < 6; ++f)
        if (f != face && h->sponge_w[f] > 0) other = true;
    if (other && h->ref_set &&
        (rho_ref != h->rho_ref || ur[0] != h->u_ref[0] || ur[1] != h->u_ref[1] || ur[2] != h->u_ref[2]))
        return fail(h, LBM_EINVAL, "all sponge layers share one reference state");
    h->sponge_w[face] = width;
    h->sponge_chi[face] = chi_max;
    h->rho_ref = rho_ref;
    for (int a = 0; a < 3; ++a) h->u_ref[a] = ur[a];
    h->ref_set = true;
    if (upload_sponge_tables(h) != LBM_OK) return fail(h, LBM_ECUDA, "uploading the sponge tables failed");
    return LBM_OK;
}

extern "C" int lbm_set_radial_sponge(lbm_handle h, const double center[3], double r0, double width,
                                     double chi_max, double rho_ref, const double u_ref[3])
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (width == 0.0) {
        for (int k = 0; k < 6; ++k) h->radial[k] = 0.0;
        return LBM_OK;
    }
    if (!center) return fail(h, LBM_EINVAL, "center is null");
    if (!(r0 >= 0.0) || !(width > 0.0) || !std::isfinite(r0) || !std::isfinite(width))
        return fail(h, LBM_EINVAL, "r0 must be >= 0 and width > 0");
    if (!(chi_max >= 0.0) || !(chi_max < 4.0 * h->tau))
        return fail(h, LBM_EINVAL, "chi_max = %g must be in [0, 4 tau = %g) for stability", chi_max, 4.0 * h->tau);
    double ur[3] = {0, 0, 0};
    if (u_ref)
        for (int a = 0; a < 3; ++a) ur[a] = u_ref[a];
    if (h->d == 2 && ur[2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_ref z must be 0");
    if (!(rho_ref > 0.0)) return fail(h, LBM_EINVAL, "rho_ref = %g must be > 0", rho_ref);
    bool other = false;
    for (int f = 0; f < 6; ++f) other = other || h->sponge_w[f] > 0;
    if (other && h->ref_set &&
        (rho_ref != h->rho_ref || ur[0] != h->u_ref[0] || ur[1] != h->u_ref[1] || ur[2] != h->u_ref[2]))
        return fail(h, LBM_EINVAL, "all sponge layers share one reference state");
    for (int a = 0; a < 3; ++a) h->radial[a] = (a < h->d) ? center[a] : 0.0;
    h->radial[3] = r0;
    h->radial[4] = width;
    h->radial[5] = chi_max;
    h->rho_ref = rho_ref;
    for (int a = 0; a < 3; ++a) h->u_ref[a] = ur[a];
    h->ref_set = true;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// State
// ---------------------------------------------------------------------------
// Host transfers go through one device staging buffer per handle, in chunks
// of whole cells, so that moving a field in or out never allocates more than
// h->stage_max (nor the size of the field) on the device.  Chunks reuse the
// buffer in stream order; the call synchronises once at the end.
static int stage(lbm_ctx *h, int64_t N, size_t bytes_per_cell, int64_t &chunk)
{
    const size_t want = std::min(h->stage_max, (size_t)N * bytes_per_cell);
    if (h->stage_bytes < want || h->stage_bytes > h->stage_max) {
        if (h->stage_d) {
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            cudaFree(h->stage_d);
            h->stage_d = nullptr;
            h->stage_bytes = 0;
        }
        const cudaError_t e = cudaMalloc(&h->stage_d, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->stage_d = nullptr;
            return fail(h, LBM_ENOMEM, "cudaMalloc of %zu bytes of transfer staging: %s", want, cudaGetErrorString(e));
        }
        h->stage_bytes = want;
    }
    chunk = (int64_t)(h->stage_bytes / bytes_per_cell);
    if (chunk > N) chunk = N;
    return LBM_OK;
}

extern "C" int lbm_set_transfer_staging(lbm_handle h, size_t max_bytes)
{
    CHECK_HANDLE(h);
    if (max_bytes < 1024) return fail(h, LBM_EINVAL, "max_bytes = %zu must be >= 1024", max_bytes);
    h->stage_max = max_bytes;
    return LBM_OK;
}

// Cells per thread the vector kernels provide for the handle: D3Q27 has the
// two-cell form only (other requests run the one-cell-per-thread kernels)
static bool vec_available(const lbm_ctx *h, int vec)
{
    return vec_supported(h->prec, vec) && (h->lattice != LBM_D3Q27 || vec == 2);
}

static int aa_normalize(lbm_ctx *h);

// Device address of a page-locked host buffer the device can reach (allocated
// by cudaHostAlloc / cudaMallocHost or registered by cudaHostRegister, which
// unified addressing maps into the device's address space), or null for
// pageable memory.  Transfers of such buffers skip the staging copies: the
// kernels read or write them over the host link directly.
template <class T>
static T *mapped_host(T *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, (const void *)p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? (T *)a.devicePointer : nullptr;
}

template <class T>
static int set_state_grid(lbm_ctx *h, const GridRef &g, const T *rho, const T *u)
{
    if (!rho || !u) return fail(h, LBM_EINVAL, "rho and u are required");
    const int64_t N = g.ncell;
    const T *rho_m = mapped_host(rho), *u_m = mapped_host(u);
    const bool direct = rho_m && u_m;
    int64_t chunk = N;
    if (!direct) {
        const int rc = stage(h, N, 4 * sizeof(T), chunk);
        if (rc != LBM_OK) return rc;
    }
    if (!h->bad_d) CUDA_TRY(h, cudaMalloc(&h->bad_d, sizeof(unsigned long long)));
    // the values are checked on the device while the field is written
    cudaError_t e = cudaMemsetAsync(h->bad_d, 0xff, sizeof(unsigned long long), h->stream);
    if (direct && e == cudaSuccess) {
        // one pass, the kernel reading the page-locked host arrays
        e = dispatch<InitEq>(h->lattice, h->prec, h->stream, N, (int64_t)0, N, rho_m, u_m, g.f[0], g.f[1],
                             h->order4, h->bad_d, shift_of(h, g));
        h->launches += 1;
    }
    T *rd = direct ? nullptr : (T *)h->stage_d, *ud = direct ? nullptr : (T *)h->stage_d + chunk;
    for (int64_t c0 = 0; !direct && c0 < N && e == cudaSuccess; c0 += chunk) {
        const int64_t n = std::min(chunk, N - c0);
        e = cudaMemcpyAsync(rd, rho + c0, sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ud, u + 3 * c0, sizeof(T) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = dispatch<InitEq>(h->lattice, h->prec, h->stream, N, c0, n, (const T *)rd, (const T *)ud,
                                 g.f[0], g.f[1], h->order4, h->bad_d, shift_of(h, g));
        h->launches += 1;
    }
    unsigned long long bad = ~0ull;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, h->bad_d, sizeof bad, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "set state: %s", cudaGetErrorString(e));
    *g.cur = 0;
    if (g.f == h->f) h->aa_odd = 0;
    if (bad != ~0ull) {
        const int64_t c = (int64_t)bad;
        if (!(rho[c] > T(0)) || !std::isfinite((double)rho[c]))
            return fail(h, LBM_EINVAL, "rho[%lld] = %g must be finite and > 0 (the field is unspecified until set again)",
                        (long long)c, (double)rho[c]);
        return fail(h, LBM_EINVAL, "2D lattice: u_z must be 0 (cell %lld; the field is unspecified until set again)",
                    (long long)c);
    }
    return LBM_OK;
}

static int set_pops_grid(lbm_ctx *h, const GridRef &g, const double *f)
{
    if (!f) return fail(h, LBM_EINVAL, "f is null");
    const int64_t N = g.ncell;
    int64_t chunk = 0;
    int rc = stage(h, N, sizeof(double), chunk);
    if (rc != LBM_OK) return rc;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->q && e == cudaSuccess; ++i) {
        for (int64_t c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
            const int64_t n = std::min(chunk, N - c0);
            e = cudaMemcpyAsync(h->stage_d, f + (size_t)i * N + c0, sizeof(double) * (size_t)n,
                                cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = dispatch<SetDir>(h->lattice, h->prec, h->stream, N, c0, n, i, (const double *)h->stage_d,
                                     g.f[0], g.f[1], shift_of(h, g));
            h->launches += 1;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "set populations: %s", cudaGetErrorString(e));
    *g.cur = 0;
    if (g.f == h->f) h->aa_odd = 0;
    return LBM_OK;
}

static int get_pops_grid(lbm_ctx *h, const GridRef &g, double *f)
{
    if (g.f == h->f) {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!f) return fail(h, LBM_EINVAL, "f is null");
    const int64_t N = g.ncell;
    int64_t chunk = 0;
    int rc = stage(h, N, sizeof(double), chunk);
    if (rc != LBM_OK) return rc;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->q && e == cudaSuccess; ++i) {
        for (int64_t c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
            const int64_t n = std::min(chunk, N - c0);
            e = dispatch<GetDir>(h->lattice, h->prec, h->stream, N, c0, n, i, (const void *)g.f[*g.cur], h->stage_d,
                                 shift_of(h, g));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(f + (size_t)i * N + c0, h->stage_d, sizeof(double) * (size_t)n,
                                    cudaMemcpyDeviceToHost, h->stream);
            h->launches += 1;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "get populations: %s", cudaGetErrorString(e));
    return LBM_OK;
}

static int refresh_after_set(lbm_ctx *h, int k);
static int level_ref(lbm_ctx *h, int level, GridRef &g);
template <class T>
static int moments_grid(lbm_ctx *h, const GridRef &g, T *rho, T *u, T *pi_neq);

extern "C" int lbm_set_state(lbm_handle h, const double *rho, const double *u)
{
    CHECK_HANDLE(h);
    int rc = set_state_grid(h, coarse_ref(h), rho, u);
    if (rc != LBM_OK) return rc;
    h->step = 0;
    return refresh_after_set(h, 0);
}

extern "C" int lbm_set_state_f32(lbm_handle h, const float *rho, const float *u)
{
    CHECK_HANDLE(h);
    int rc = set_state_grid(h, coarse_ref(h), rho, u);
    if (rc != LBM_OK) return rc;
    h->step = 0;
    return refresh_after_set(h, 0);
}

extern "C" int lbm_set_populations(lbm_handle h, const double *f)
{
    CHECK_HANDLE(h);
    int rc = set_pops_grid(h, coarse_ref(h), f);
    if (rc != LBM_OK) return rc;
    h->step = 0;
    return refresh_after_set(h, 0);
}

extern "C" int lbm_get_populations(lbm_handle h, double *f)
{
    CHECK_HANDLE(h);
    return get_pops_grid(h, coarse_ref(h), f);
}

// ---------------------------------------------------------------------------
// Time stepping
// ---------------------------------------------------------------------------
static int build_params(lbm_ctx *h, StepParams &p)
{
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) {
        p.n[a] = h->n[a];
        const bool plo = h->kind[2 * a] == LBM_BC_PERIODIC, phi = h->kind[2 * a + 1] == LBM_BC_PERIODIC;
        if (plo != phi)
            return fail(h, LBM_EINVAL, "axis %d: both faces must be periodic or neither", a);
        p.periodic[a] = plo ? 1 : 0;
        if (!plo && h->n[a] < 3) return fail(h, LBM_EINVAL, "axis %d: a non-periodic axis needs >= 3 cells", a);
    }
    p.ncell = h->ncell;
    for (int f = 0; f < 6; ++f) {
        p.kind[f] = h->kind[f];
        p.sponge_w[f] = h->sponge_w[f];
        p.sponge_chi[f] = h->sponge_chi[f];
        if (h->sponge_w[f] > 0 && h->sponge_chi[f] > 0.0) p.any_sponge = 1;
        p.radial[f] = h->radial[f];
        p.face_cells[f] = face_cells(h, f);
        p.rho_face[f] = h->rho_face[f];
        p.rho_face_m1[f] = h->rho_face[f] - 1.0;
        for (int a = 0; a < 3; ++a) p.u_face[f][a] = h->u_face[f][a];
        p.u_profile[f] = h->prof_d[f];
    }
    if (h->radial[4] > 0.0 && h->radial[5] > 0.0) p.any_sponge = 1;
    p.chi_tab_f = h->chi_tab_f;
    p.chi_tab_d = h->chi_tab_d;
    p.rho_ref = h->rho_ref;
    p.rho_ref_m1 = h->rho_ref - 1.0;
    for (int a = 0; a < 3; ++a) p.u_ref[a] = h->u_ref[a];
    p.noise_seed = h->noise_seed;
    p.noise_amp = h->noise_amp;
    p.omega = 1.0 - 1.0 / h->tau;
    p.solid = h->solid_d;
    p.any_solid = h->has_solid ? 1 : 0;
    p.err = h->err_d;
    p.bgk = h->collision == LBM_COLLISION_BGK ? 1 : 0;
    p.order4 = h->order4;
    p.jet_x_layer = INT_MAX;
    if (h->jet_ref[3] > 0.0 && h->sponge_w[1] > 0 && h->sponge_chi[1] > 0.0) {
        p.jet_x_layer = h->n[0] - h->sponge_w[1];
        p.jet_ref[0] = h->jet_ref[0];
        p.jet_ref[1] = h->jet_ref[1];
        p.jet_ref[2] = h->jet_ref[2];
        p.jet_ref[3] = h->jet_ref[5] * h->jet_ref[3];  // B D
        p.jet_ref[4] = h->jet_ref[4];
        p.jet_ref[5] = (std::sqrt(2.0) - 1.0) / (h->jet_ref[6] * h->jet_ref[6]);
    }
    p.shifted = h->shifted ? 1 : 0;
    for (int i = 0; i < h->q && h->shifted; ++i) {
        p.dsh_d[i] = h->dsh[i];
        p.dsh_f[i] = (float)h->dsh[i];
    }
    p.sponge_rest = (h->rho_ref == 1.0 && h->u_ref[0] == 0.0 && h->u_ref[1] == 0.0 && h->u_ref[2] == 0.0 &&
                     p.jet_x_layer == INT_MAX)
                        ? 1
                        : 0;
    set_bulk_box(p);
    return LBM_OK;
}

// Whether the row-staged kernel is asked for (it still runs only where eligible)
static bool staging_wanted(const lbm_ctx *h)
{
    if (h->staging == 0 || h->pattern == LBM_STREAM_AA || h->shifted) return false;
    // default: off -- measured on GB300 for the D3Q19 jet (384 x 256 x 256) the
    // register kernels are faster (FP32 43.3 vs 25.9 GLUPS, FP16 48.9 vs 34.9)
    return h->staging == 1;
}

// Whether the vectorised kernel can update a grid: no cell-type mask, the
// rrBGK collision, the default storage shift, and sponge layers (if any)
// relaxing to the rest state through face layers only (its closed form)
static bool vec_eligible(const StepParams &p)
{
    return !p.solid && !p.bgk && !p.shifted && (!p.any_sponge || (p.sponge_rest && !p.radial_on));
}

// Launch one update of a grid: the row-staged kernel where it is wanted and
// eligible; else the vectorised kernel when there is no mask and the row
// length allows it; else the general kernel.
static cudaError_t step_general(lbm_ctx *h, const StepParams &p, const void *fin, void *fout, int block)
{
    switch (h->lattice) {
    case LBM_D2Q9: return step_d2q9(h->prec, p, fin, fout, block, h->stream);
    case LBM_D3Q19: return step_d3q19(h->prec, p, fin, fout, block, h->stream);
    default: return step_d3q27(h->prec, p, fin, fout, block, h->stream);
    }
}

static cudaError_t launch_update(lbm_ctx *h, const StepParams &p, const void *fin, void *fout)
{
    if (p.bgk) {
        // plain BGK: the general kernel only
        h->launches += 1;
        return step_general(h, p, fin, fout, h->block > 0 ? h->block : block_default(1));
    }
    if (staging_wanted(h) && h->lattice != LBM_D3Q27) {
        const cudaError_t e = h->lattice == LBM_D2Q9
                                  ? rows_d2q9(h->prec, p, fin, fout, h->rows_block, h->stages, h->err_d,
                                              h->rows_wait_ns, h->stream)
                                  : rows_d3q19(h->prec, p, fin, fout, h->rows_block, h->stages, h->err_d,
                                               h->rows_wait_ns, h->stream);
        if (e != cudaErrorNotSupported) {
            h->launches += 1;
            return e;
        }
    }
    int vec = h->vec == 0 ? vec_default(h->lattice, h->prec) : h->vec;
    if (!vec_eligible(p) || vec == 1 || !vec_available(h, vec) || p.n[0] % vec != 0) vec = 1;
    const int block = h->block > 0 ? h->block : block_default(vec);
    h->launches += 1;
    if (vec == 1) return step_general(h, p, fin, fout, block);
    switch (h->lattice) {
    case LBM_D2Q9: return stepvec_d2q9(h->prec, vec, p, fin, fout, block, h->stream);
    case LBM_D3Q19: return stepvec_d3q19(h->prec, vec, p, fin, fout, block, h->stream);
    default: return stepvec_d3q27(h->prec, vec, p, fin, fout, block, h->stream);
    }
}

// Step parameters of refined level k >= 1: periodic box, ring fixed, no sponge/inflow
static void fine_params(lbm_ctx *h, int k, StepParams &p)
{
    FineLevel *F = fine_level(h, k);
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) {
        p.n[a] = F->n[a];
        p.periodic[a] = 1;
    }
    p.ncell = F->ncell;
    for (int f = 0; f < 6; ++f) p.face_cells[f] = 1;
    p.rho_ref = 1.0;
    p.omega = 1.0 - 1.0 / F->tau;
    p.jet_x_layer = INT_MAX;
    p.solid = F->mask_d;
    p.any_solid = F->has_solid ? 1 : 0;
    p.err = h->err_d;
    set_bulk_box(p);
}

// 256-thread blocks per SM of the 3D fill and restriction when they run
// beside the level-0 update
constexpr int kInterfaceBlocksPerSm = 2;

// 3D patch (D3Q19 or D3Q27): plane moments, fine shell, covered coarse shell
template <class L, class S>
static cudaError_t refine_kernels3(lbm_ctx *h, int k, int stage, int a_half)
{
    FineLevel *F = fine_level(h, k);
    const GridRef P = level_grid(h, k - 1);  // the parent level
    const double tau_p = level_tau(h, k - 1);
    const RefineGeom &g = F->geom;
    cudaStream_t st = h->stream;
    // Beside the level-0 update (second stream) the fill and restriction run
    // on a bounded grid, so that their blocks, of the higher-priority stream,
    // leave SMs to the HBM-bound update (two-level jet: 0.7675 -> 0.7628 ms per
    // coarse step; 1 to 8 blocks per SM measured the same).
    auto side_cap = [&](unsigned grid) {
        const unsigned cap = (unsigned)(h->sms * kInterfaceBlocksPerSm);
        return h->side && st == h->side && cap > 0 && grid > cap ? cap : grid;
    };
    switch (stage) {
    case 0:  // coarse plane moments at t + 1 from the pre-step coarse field
    case 3: {  // plane moments at t = 0: local moments of the stored coarse field
        const int n = plane3_count(g);
        // the moment buffers (sized for FP64) hold the compute type
        CT<S> *M = (CT<S> *)(stage == 0 ? F->M[1 - F->mcur] : F->M[F->mcur]);
        k_plane_moments3<L, S><<<grid1(n, 128), 128, 0, st>>>(g, (const S *)P.f[*P.cur], links_mask(h, k - 1),
                                                            stage == 0 ? 1 : 0, M);
        break;
    }
    case 1: {  // fine shell at t + 1/2 (a_half = 1) or t + 1 (a_half = 0)
        const int n = shell3_count(g.nfx, g.nfy, g.nfz);
        // 4 threads per shell node
        k_fill_shell3<L, S><<<side_cap(grid1(4 * (int64_t)n, 256)), 256, 0, st>>>(
            g, (const CT<S> *)F->M[F->mcur], (const CT<S> *)F->M[1 - F->mcur], CT<S>(a_half ? 0.5 : 1.0),
            CT<S>(F->tau / (2.0 * tau_p)), CT<S>(1.0 - 1.0 / F->tau), (S *)F->f[F->cur]);
        break;
    }
    case 2: {  // covered coarse shell from the fine field; fine moments pulled from f(t + 1/2)
        const int n = shell3_count(g.Wc - 1, g.Hc - 1, g.Dc - 1);
        // one warp per covered coarse node (one lane per filter point)
        k_restrict3<L, S><<<side_cap(grid1(32 * (int64_t)n, 256)), 256, 0, st>>>(
            g, (const S *)F->f[1 - F->cur], links_mask(h, k), CT<S>(2.0 * tau_p / F->tau), CT<S>(1.0 - 1.0 / tau_p),
            (S *)P.f[*P.cur]);
        break;
    }
    }
    h->launches += 1;
    return cudaGetLastError();
}

// Coupling of refined level k >= 1 with its parent k - 1:
//   stage 0: parent-side interface moments at t + 1 from the pre-step parent field
//   stage 1: level k's ring / shell at t + 1/2 (a_half = 1) or t + 1 (a_half = 0)
//   stage 2: the parent's covered ring / shell from level k at t + 1/2
//   stage 3: interface moments at t = 0 (local moments of the stored parent field)
template <class S>
static cudaError_t refine_kernels(lbm_ctx *h, int k, int stage, int a_half)
{
    if (h->lattice == LBM_D3Q27) return refine_kernels3<D3Q27, S>(h, k, stage, a_half);
    if (h->d == 3) return refine_kernels3<D3Q19, S>(h, k, stage, a_half);
    FineLevel *F = fine_level(h, k);
    const GridRef P = level_grid(h, k - 1);
    const double tau_p = level_tau(h, k - 1);
    const RefineGeom &g = F->geom;
    cudaStream_t st = h->stream;
    switch (stage) {
    case 0: {  // coarse line moments at t + 1 from the pre-step coarse field
        const int n = line_count(g);
        k_line_moments<S><<<grid1(n, 128), 128, 0, st>>>(g, (const S *)P.f[*P.cur], links_mask(h, k - 1), 1,
                                                          (CT<S> *)F->M[1 - F->mcur]);
        break;
    }
    case 1: {  // fine ring at t + 1/2 (a_half = 1) or t + 1 (a_half = 0)
        const int n = 2 * g.nfx + 2 * (g.nfy - 2);
        k_fill_ring<S><<<grid1(n, 128), 128, 0, st>>>(
            g, (const CT<S> *)F->M[F->mcur], (const CT<S> *)F->M[1 - F->mcur], CT<S>(a_half ? 0.5 : 1.0),
            CT<S>(F->tau / (2.0 * tau_p)), CT<S>(1.0 - 1.0 / F->tau), (S *)F->f[F->cur]);
        break;
    }
    case 2: {  // covered coarse ring from the fine field; pre-collision fine moments pulled from f(t + 1/2)
        const int n = 2 * (g.Wc - 1) + 2 * (g.Hc - 3);
        k_restrict<S><<<grid1(n, 128), 128, 0, st>>>(g, (const S *)F->f[1 - F->cur], links_mask(h, k),
                                                      CT<S>(2.0 * tau_p / F->tau), CT<S>(1.0 - 1.0 / tau_p),
                                                      (S *)P.f[*P.cur]);
        break;
    }
    case 3: {  // line moments at t = 0: local moments of the stored coarse field
        const int n = line_count(g);
        k_line_moments<S><<<grid1(n, 128), 128, 0, st>>>(g, (const S *)P.f[*P.cur], links_mask(h, k - 1), 0,
                                                          (CT<S> *)F->M[F->mcur]);
        break;
    }
    }
    h->launches += 1;
    return cudaGetLastError();
}

static cudaError_t refine_stage(lbm_ctx *h, int k, int stage, int a_half = 0)
{
    switch (h->prec) {
    case LBM_FP64: return refine_kernels<double>(h, k, stage, a_half);
    case LBM_FP32: return refine_kernels<float>(h, k, stage, a_half);
    case LBM_FP16_SHIFTED: return refine_kernels<__half>(h, k, stage, a_half);
    case LBM_BF16_SHIFTED: return refine_kernels<__nv_bfloat16>(h, k, stage, a_half);
    }
    return cudaErrorInvalidValue;
}

// Interface moments at t = 0 of the pair (k - 1, k), k >= 1
static int init_pair_moments(lbm_ctx *h, int k)
{
    cudaError_t e = refine_stage(h, k, 3);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "interface moments: %s", cudaGetErrorString(e));
    return LBM_OK;
}

// After level k's state was set: refresh the interface moments it is the parent of
static int refresh_after_set(lbm_ctx *h, int k)
{
    return k < (int)h->levels.size() ? init_pair_moments(h, k + 1) : LBM_OK;
}

// One in-place AA step of level 0: gather-push from the standard layout or
// the local step from the push layout (which restores the standard one)
static cudaError_t aa_step(lbm_ctx *h, const StepParams &p)
{
    const bool loc = h->aa_odd != 0;
    int vec = h->vec == 0 ? vec_default(h->lattice, h->prec) : h->vec;
    if (!vec_eligible(p) || vec == 1 || !vec_available(h, vec) || p.n[0] % vec != 0) vec = 1;
    const int block = h->block > 0 ? h->block : block_default(vec);
    h->launches += 1;
    h->aa_odd ^= 1;
    if (vec > 1) {
        const int sp = loc ? 2 : 1;
        switch (h->lattice) {
        case LBM_D2Q9: return stepvec_d2q9(h->prec, vec, p, h->f[0], h->f[0], block, h->stream, sp);
        case LBM_D3Q19: return stepvec_d3q19(h->prec, vec, p, h->f[0], h->f[0], block, h->stream, sp);
        default: return stepvec_d3q27(h->prec, vec, p, h->f[0], h->f[0], block, h->stream, sp);
        }
    }
    switch (h->lattice) {
    case LBM_D2Q9: return step_aa_d2q9(h->prec, p, h->f[0], block, loc, h->stream);
    case LBM_D3Q19: return step_aa_d3q19(h->prec, p, h->f[0], block, loc, h->stream);
    default: return step_aa_d3q27(h->prec, p, h->f[0], block, loc, h->stream);
    }
}

// Bring an AA lattice left in the push layout back to the standard layout
// (in place, stream-ordered) before its populations are read as f*_i(x)
static int aa_normalize(lbm_ctx *h)
{
    if (h->pattern != LBM_STREAM_AA || !h->aa_odd) return LBM_OK;
    StepParams p;
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) {
        p.n[a] = h->n[a];
        p.periodic[a] = h->kind[2 * a] == LBM_BC_PERIODIC ? 1 : 0;
    }
    p.ncell = h->ncell;
    p.solid = h->solid_d;
    cudaError_t e;
    switch (h->lattice) {
    case LBM_D2Q9: e = aa_unswap_d2q9(h->prec, p, h->f[0], h->stream); break;
    case LBM_D3Q19: e = aa_unswap_d3q19(h->prec, p, h->f[0], h->stream); break;
    default: e = aa_unswap_d3q27(h->prec, p, h->f[0], h->stream); break;
    }
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "AA layout conversion: %s", cudaGetErrorString(e));
    h->aa_odd = 0;
    return LBM_OK;
}

// The second stream and the fork / join events of the level overlap
static cudaError_t ensure_side_stream(lbm_ctx *h)
{
    if (h->side) return cudaSuccess;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

static cudaError_t advance_level(lbm_ctx *h, std::vector<StepParams> &params, int k, int64_t step);

// The child's part of a step of level k: two steps of level k + 1 with its
// ring refilled at t + 1/2 and t + 1, and the covered ring of level k rebuilt
// from the child at t + 1/2.
static cudaError_t advance_child(lbm_ctx *h, std::vector<StepParams> &params, int k, int64_t step)
{
    cudaError_t e = advance_level(h, params, k + 1, 2 * step);
    if (e == cudaSuccess) e = refine_stage(h, k + 1, 1, 1);
    if (e == cudaSuccess) e = advance_level(h, params, k + 1, 2 * step + 1);
    if (e == cudaSuccess) e = refine_stage(h, k + 1, 1, 0);
    if (e == cudaSuccess) e = refine_stage(h, k + 1, 2);
    FineLevel *F = fine_level(h, k + 1);
    F->mcur = 1 - F->mcur;
    return e;
}

// One step of level k (Sec. II.B applied level by level): the interface
// moments of its child at t + 1 from the pre-step field, its own update, and
// the child's part (advance_child).  The child's part reads the interface
// moments, not level k's update: it touches level k only to write the
// covered ring of level k's new field, whose cells level k's update skips
// (fixed cells) and does not read (it pulls from the old field).  So below
// level 0 it runs on a second stream of the highest priority, concurrently
// with the level-0 update, which is HBM-bound while the child's interface
// kernels are latency-bound; the level-0 stream waits for it before the next
// step.  The result is bitwise that of running the two in order.
static cudaError_t advance_level(lbm_ctx *h, std::vector<StepParams> &params, int k, int64_t step)
{
    const bool child = k < (int)h->levels.size();
    cudaError_t e = cudaSuccess;
    if (child) e = refine_stage(h, k + 1, 0);
    GridRef g = level_grid(h, k);
    params[k].step = step;
    const bool aa = k == 0 && h->pattern == LBM_STREAM_AA;  // (never with refined levels)
    if (e == cudaSuccess && child && k == 0 && h->level_overlap && !aa) {
        const void *fin = g.f[*g.cur];
        void *fout = g.f[1 - *g.cur];
        *g.cur = 1 - *g.cur;  // the child's restriction writes the new field
        e = ensure_side_stream(h);
        if (e == cudaSuccess) e = cudaEventRecord(h->fork_ev, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->fork_ev, 0);
        if (e == cudaSuccess) {
            const cudaStream_t main = h->stream;
            h->stream = h->side;
            e = advance_child(h, params, k, step);
            h->stream = main;
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->join_ev, h->side);
        if (e == cudaSuccess) e = launch_update(h, params[k], fin, fout);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->join_ev, 0);
        return e;
    }
    if (e == cudaSuccess) e = aa ? aa_step(h, params[k]) : launch_update(h, params[k], g.f[*g.cur], g.f[1 - *g.cur]);
    if (e != cudaSuccess) return e;
    if (!aa) *g.cur = 1 - *g.cur;
    if (!child) return cudaSuccess;
    return advance_child(h, params, k, step);
}

// Enqueue n steps of level 0 (each with all refined levels beneath it).
static int enqueue_steps(lbm_ctx *h, std::vector<StepParams> &params, int64_t n)
{
    for (int64_t t = 0; t < n; ++t) {
        const cudaError_t e = advance_level(h, params, 0, h->step);
        if (e != cudaSuccess) return fail(h, LBM_ECUDA, "step launch: %s", cudaGetErrorString(e));
        h->step += 1;
    }
    return LBM_OK;
}

// Lattice parities of all levels and interface-moment buffers (the state a
// captured pair of steps depends on)
static uint64_t parity_signature(const lbm_ctx *h)
{
    uint64_t sig = (uint64_t)h->cur | ((uint64_t)h->aa_odd << 63);
    int bit = 1;
    for (const FineLevel *F : h->levels) {
        sig |= (uint64_t)F->cur << bit++;
        sig |= (uint64_t)F->mcur << bit++;
    }
    return sig;
}

// Capture npairs step pairs into a graph for the current configuration and
// parity, appended to the handle's graphs.  The host-side counters advanced
// by the capture are restored: the captured work runs only when the graph is
// launched.
static int capture_pairs(lbm_ctx *h, std::vector<StepParams> &params, int npairs)
{
    const int cur = h->cur, aa_odd = h->aa_odd;
    std::vector<int> fcur, mcur;
    for (FineLevel *F : h->levels) {
        fcur.push_back(F->cur);
        mcur.push_back(F->mcur);
    }
    const uint64_t sig = parity_signature(h);
    const int64_t step = h->step, launches = h->launches;
    cudaGraph_t g = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_steps(h, params, 2 * (int64_t)npairs);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    const int64_t per_graph = h->launches - launches;
    h->cur = cur;
    h->aa_odd = aa_odd;
    h->step = step;
    h->launches = launches;
    for (size_t k = 0; k < h->levels.size(); ++k) {
        h->levels[k]->cur = fcur[k];
        h->levels[k]->mcur = mcur[k];
    }
    if (rc != LBM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != LBM_OK ? rc : fail(h, LBM_ECUDA, "capturing steps: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "instantiating steps: %s", cudaGetErrorString(e));
    h->graphs.push_back(lbm_ctx::StepGraph{sig, npairs, exec, per_graph});
    return LBM_OK;
}

static void drop_graphs(lbm_ctx *h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

extern "C" int lbm_step(lbm_handle h, int64_t n)
{
    CHECK_HANDLE(h);
    if (n < 0) return fail(h, LBM_EINVAL, "n = %lld < 0", (long long)n);
    if (n == 0) return LBM_OK;
    std::vector<StepParams> params((size_t)nlevels(h));
    int rc = build_params(h, params[0]);
    if (rc != LBM_OK) return rc;
    for (int k = 1; k < nlevels(h); ++k) fine_params(h, k, params[(size_t)k]);
    // Without inlet noise every step of a pair has the same parameters, so
    // pairs of steps are replayed from captured graphs (needs a stream other
    // than the legacy default one).  Every refined level returns to the same
    // lattice parity after two coarse steps.  The n / 2 pairs of a call run
    // as replays of a 16-pair graph and at most one graph each of 8, 4, 2
    // and 1 pairs (the binary digits of the rest), each captured once per
    // configuration and parity and kept, so calls of varying n reuse them;
    // only an odd last step runs as direct launches.
    constexpr int kGraphPairs = 16;
    if (h->stream && h->noise_amp == 0.0 && n >= 2) {
        if (h->graphs_version != h->cfg_version || h->graphs.size() > 20) {
            drop_graphs(h);
            h->graphs_version = h->cfg_version;
        }
        const uint64_t sig = parity_signature(h);
        int64_t pairs_left = n / 2;
        for (int size = kGraphPairs; size >= 1 && pairs_left > 0; size >>= 1) {
            const int64_t reps = size == kGraphPairs ? pairs_left / size : (pairs_left >= size ? 1 : 0);
            if (reps == 0) continue;
            const lbm_ctx::StepGraph *G = nullptr;
            for (const auto &g : h->graphs)
                if (g.sig == sig && g.pairs == size) G = &g;
            if (!G) {
                rc = capture_pairs(h, params, size);
                if (rc != LBM_OK) return rc;
                G = &h->graphs.back();
            }
            for (int64_t k = 0; k < reps; ++k) {
                cudaError_t e = cudaGraphLaunch(G->exec, h->stream);
                if (e != cudaSuccess) return fail(h, LBM_ECUDA, "graph launch: %s", cudaGetErrorString(e));
            }
            h->step += 2 * (int64_t)size * reps;
            h->launches += G->launches * reps;
            pairs_left -= (int64_t)size * reps;
            n -= 2 * (int64_t)size * reps;
        }
    }
    return enqueue_steps(h, params, n);
}

// ---------------------------------------------------------------------------
// Refined levels
// ---------------------------------------------------------------------------
extern "C" int lbm_add_refinement_patch(lbm_handle h, const int origin[3], const int extent[3])
{
    CHECK_HANDLE(h);
    if (h->pattern == LBM_STREAM_AA)
        return fail(h, LBM_EINVAL, "refinement patches need the two-lattice pull pattern (lbm_set_streaming)");
    if (h->shifted) return fail(h, LBM_EINVAL, "refinement patches need the default storage shift");
    h->cfg_version++;
    if (h->collision != LBM_COLLISION_RR)
        return fail(h, LBM_EINVAL, "refinement patches couple rrBGK levels; select LBM_COLLISION_RR first");
    if (h->order4) return fail(h, LBM_EINVAL, "refinement patches couple order-3 levels; set order 3 first");
    if (!origin || !extent) return fail(h, LBM_EINVAL, "origin and extent are required");
    if (h->levels.size() >= LBM_MAX_LEVELS - 1)
        return fail(h, LBM_EINVAL, "at most %d levels", LBM_MAX_LEVELS);
    const int parent = nlevels(h) - 1;  // the new patch nests inside the finest level
    const GridRef P = level_grid(h, parent);
    const bool three = h->d == 3;
    const int X0 = origin[0], Y0 = origin[1], Wc = extent[0], Hc = extent[1];
    const int Z0 = three ? origin[2] : 0, Dc = three ? extent[2] : 0;
    if (Wc < 4 || Hc < 4 || (three && Dc < 4))
        return fail(h, LBM_EINVAL, "patch extent must be >= 4 parent cells per axis");
    if (X0 < 2 || Y0 < 2 || X0 + Wc > P.n[0] - 3 || Y0 + Hc > P.n[1] - 3 ||
        (three && (Z0 < 2 || Z0 + Dc > P.n[2] - 3)))
        return fail(h, LBM_EINVAL, "patch must keep 2 cells from every face of level %d", parent);
    if ((int64_t)(2 * Wc + 1) * (2 * Hc + 1) * (three ? 2 * Dc + 1 : 1) > 2147483647LL)
        return fail(h, LBM_EINVAL, "the new level would hold more than 2^31 - 1 cells");
    FineLevel *F = new FineLevel();
    F->n[0] = 2 * Wc + 1;
    F->n[1] = 2 * Hc + 1;
    F->n[2] = three ? 2 * Dc + 1 : 1;
    F->ncell = (int64_t)F->n[0] * F->n[1] * F->n[2];
    F->tau = 2.0 * level_tau(h, parent) - 0.5;
    F->geom = RefineGeom{X0, Y0, Wc, Hc, P.n[0], P.n[1], F->n[0], F->n[1], Z0, Dc, P.n[2], F->n[2]};
    const size_t bytes = (size_t)h->q * (size_t)F->ncell * h->elem;
    const size_t mbytes = moment_bytes(three, F->geom);
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k)
        ok = cudaMalloc(&F->f[k], bytes) == cudaSuccess && cudaMalloc(&F->M[k], mbytes) == cudaSuccess &&
             cudaMemsetAsync(F->f[k], 0, bytes, h->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (int k = 0; k < 2; ++k) {
            if (F->f[k]) cudaFree(F->f[k]);
            if (F->M[k]) cudaFree(F->M[k]);
        }
        delete F;
        return fail(h, LBM_ENOMEM, "allocating level %d failed", parent + 1);
    }
    h->levels.push_back(F);
    const int k = parent + 1;
    int rc = upload_level_mask(h, k);
    if (rc == LBM_OK) rc = upload_level_mask(h, parent);
    if (rc == LBM_OK) rc = init_pair_moments(h, k);
    return rc;
}

static int level_ref(lbm_ctx *h, int level, GridRef &g)
{
    if (level < 0 || level >= nlevels(h)) return fail(h, LBM_EINVAL, "no level %d", level);
    g = level_grid(h, level);
    return LBM_OK;
}

extern "C" int lbm_force(lbm_handle h, int level, double F[3])
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!F) return fail(h, LBM_EINVAL, "F is null");
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    F[0] = F[1] = F[2] = 0.0;
    if (!g.mask) return LBM_OK;
    int per[3] = {1, 1, 1};
    if (level == 0)
        for (int a = 0; a < 3; ++a) per[a] = h->kind[2 * a] == LBM_BC_PERIODIC ? 1 : 0;
    double out[RED_FIELDS];
    cudaError_t e = dispatch<Force>(h->lattice, h->prec, h->stream, (const int *)g.n, (const int *)per,
                                    (const void *)g.f[*g.cur], g.mask, h->red_d, h->red_blocks, shift_of(h, g));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, h->red_d + (size_t)h->red_blocks * RED_FIELDS, sizeof out, cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 2;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_force: %s", cudaGetErrorString(e));
    for (int a = 0; a < 3; ++a) F[a] = out[a];
    return LBM_OK;
}

extern "C" int lbm_force_async(lbm_handle h, int level, double *F_dev)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!F_dev) return fail(h, LBM_EINVAL, "F_dev is null");
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    cudaError_t e;
    if (!g.mask) {
        e = cudaMemsetAsync(F_dev, 0, 3 * sizeof(double), h->stream);
    } else {
        int per[3] = {1, 1, 1};
        if (level == 0)
            for (int a = 0; a < 3; ++a) per[a] = h->kind[2 * a] == LBM_BC_PERIODIC ? 1 : 0;
        e = dispatch<Force>(h->lattice, h->prec, h->stream, (const int *)g.n, (const int *)per,
                            (const void *)g.f[*g.cur], g.mask, h->red_d, h->red_blocks, shift_of(h, g));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(F_dev, h->red_d + (size_t)h->red_blocks * RED_FIELDS, 3 * sizeof(double),
                                cudaMemcpyDeviceToDevice, h->stream);
        h->launches += 2;
    }
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_force_async: %s", cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" int lbm_level_info(lbm_handle h, int level, int extents[3], double *tau)
{
    CHECK_HANDLE(h);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    if (extents)
        for (int a = 0; a < 3; ++a) extents[a] = g.n[a];
    if (tau) *tau = level_tau(h, level);
    return LBM_OK;
}

extern "C" int lbm_set_geometry_level(lbm_handle h, int level, const uint8_t *cell_type)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (level == 0) return lbm_set_geometry(h, cell_type);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    FineLevel *F = fine_level(h, level);
    if (cell_type) {
        rc = check_cell_types(h, cell_type, F->ncell);
        if (rc != LBM_OK) return rc;
        F->user_mask.assign(cell_type, cell_type + F->ncell);
    } else {
        F->user_mask.clear();
    }
    return upload_level_mask(h, level);
}

extern "C" int lbm_set_state_level(lbm_handle h, int level, const double *rho, const double *u)
{
    CHECK_HANDLE(h);
    if (level == 0) return lbm_set_state(h, rho, u);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    h->step = 0;
    rc = set_state_grid(h, g, rho, u);
    return rc == LBM_OK ? refresh_after_set(h, level) : rc;
}

extern "C" int lbm_set_populations_level(lbm_handle h, int level, const double *f)
{
    CHECK_HANDLE(h);
    if (level == 0) return lbm_set_populations(h, f);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    h->step = 0;
    rc = set_pops_grid(h, g, f);
    return rc == LBM_OK ? refresh_after_set(h, level) : rc;
}

extern "C" int lbm_get_populations_level(lbm_handle h, int level, double *f)
{
    CHECK_HANDLE(h);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    return get_pops_grid(h, g, f);
}

extern "C" int lbm_moments_level(lbm_handle h, int level, double *rho, double *u, double *pi_neq)
{
    CHECK_HANDLE(h);
    GridRef g;
    int rc = level_ref(h, level, g);
    if (rc != LBM_OK) return rc;
    return moments_grid(h, g, rho, u, pi_neq);
}

extern "C" int lbm_set_level_streams(lbm_handle h, int concurrent)
{
    CHECK_HANDLE(h);
    if (concurrent != 0 && concurrent != 1) return fail(h, LBM_EINVAL, "concurrent must be 0 or 1");
    h->cfg_version++;
    h->level_overlap = concurrent;
    return LBM_OK;
}

extern "C" int lbm_set_launch(lbm_handle h, int block, int cells_per_thread)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (block != 0 && (block < 32 || block > 256 || block % 32 != 0))
        return fail(h, LBM_EINVAL, "block = %d must be 0 or a multiple of 32 in [32, 256]", block);
    if (cells_per_thread != 0 && cells_per_thread != 1 && !vec_supported(h->prec, cells_per_thread))
        return fail(h, LBM_EINVAL, "cells_per_thread = %d is not supported for this precision", cells_per_thread);
    h->block = block;
    h->vec = cells_per_thread;
    return LBM_OK;
}

extern "C" int lbm_get_launch(lbm_handle h, int *block, int *cells_per_thread)
{
    CHECK_HANDLE(h);
    int vec = h->vec == 0 ? vec_default(h->lattice, h->prec) : h->vec;
    if (h->solid_d || vec == 1 || !vec_available(h, vec) || h->n[0] % vec != 0) vec = 1;
    if (block) *block = h->block > 0 ? h->block : block_default(vec);  // level 0
    if (cells_per_thread) *cells_per_thread = vec;
    return LBM_OK;
}

extern "C" int lbm_set_hermite_order(lbm_handle h, int order)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (order != 3 && order != 4) return fail(h, LBM_EINVAL, "order = %d must be 3 or 4", order);
    if (order == 4 && h->lattice != LBM_D2Q9) return fail(h, LBM_EINVAL, "order 4 exists for D2Q9 only");
    if (order == 4 && !h->levels.empty()) return fail(h, LBM_EINVAL, "order 4 is not available with refinement");
    h->order4 = order == 4 ? 1 : 0;
    return LBM_OK;
}

extern "C" int lbm_set_collision(lbm_handle h, int model)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (model != LBM_COLLISION_RR && model != LBM_COLLISION_BGK)
        return fail(h, LBM_EINVAL, "collision model %d is not LBM_COLLISION_RR or LBM_COLLISION_BGK", model);
    if (model == LBM_COLLISION_BGK && !h->levels.empty())
        return fail(h, LBM_EINVAL, "plain BGK is not available with a refinement patch");
    h->collision = model;
    return LBM_OK;
}

extern "C" int lbm_set_sponge_jet_reference(lbm_handle h, double yc, double zc, double U_jet, double D, double x0,
                                            double B, double S)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (h->d != 3) return fail(h, LBM_EINVAL, "the round-jet reference needs a 3D lattice");
    if (D == 0.0) {
        for (double &v : h->jet_ref) v = 0.0;
        return LBM_OK;
    }
    if (!(D > 0.0) || !(U_jet >= 0.0) || !(B > 0.0) || !(S > 0.0) || !std::isfinite(x0) || !std::isfinite(yc) ||
        !std::isfinite(zc) || !std::isfinite(U_jet * B * D / S))
        return fail(h, LBM_EINVAL, "jet reference needs D > 0, U_jet >= 0, B > 0, S > 0, finite values");
    const double v[7] = {yc, zc, U_jet, D, x0, B, S};
    for (int k = 0; k < 7; ++k) h->jet_ref[k] = v[k];
    return LBM_OK;
}

extern "C" int lbm_pressure_mean(lbm_handle h, int op)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (op != LBM_MEAN_RESET && op != LBM_MEAN_ACCUMULATE)
        return fail(h, LBM_EINVAL, "op = %d is not LBM_MEAN_RESET or LBM_MEAN_ACCUMULATE", op);
    const size_t bytes = sizeof(double) * (size_t)h->ncell;
    if (op == LBM_MEAN_RESET) {
        if (h->rho_acc) CUDA_TRY(h, cudaMemsetAsync(h->rho_acc, 0, bytes, h->stream));
        h->rho_count = 0;
        return LBM_OK;
    }
    if (!h->rho_acc) {
        if (cudaMalloc(&h->rho_acc, bytes) != cudaSuccess) {
            cudaGetLastError();
            h->rho_acc = nullptr;
            return fail(h, LBM_ENOMEM, "cudaMalloc of the mean-pressure accumulator (%zu bytes) failed", bytes);
        }
        CUDA_TRY(h, cudaMemsetAsync(h->rho_acc, 0, bytes, h->stream));
        h->rho_count = 0;
    }
    CUDA_TRY(h, dispatch<RhoAccumulate>(h->lattice, h->prec, h->stream, h->ncell, (const void *)h->f[h->cur],
                                        h->rho_acc));
    h->launches += 1;
    h->rho_count += 1;
    return LBM_OK;
}

extern "C" int lbm_pressure_fluctuation(lbm_handle h, double *dp_tilde, double *dp_mean)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!dp_tilde && !dp_mean) return LBM_OK;
    if (!h->rho_acc || h->rho_count == 0)
        return fail(h, LBM_EINVAL, "no accumulated samples: call lbm_pressure_mean(h, LBM_MEAN_ACCUMULATE) first");
    const int64_t N = h->ncell;
    double *buf = nullptr;
    CUDA_TRY(h, cudaMalloc(&buf, sizeof(double) * 2 * (size_t)N));
    cudaError_t e = dispatch<PressureFluct>(h->lattice, h->prec, h->stream, N, (const void *)h->f[h->cur],
                                            (const double *)h->rho_acc, (double)h->rho_count, buf,
                                            dp_mean ? buf + N : (double *)nullptr);
    if (e == cudaSuccess && dp_tilde)
        e = cudaMemcpyAsync(dp_tilde, buf, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && dp_mean)
        e = cudaMemcpyAsync(dp_mean, buf + N, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_pressure_fluctuation: %s", cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" int lbm_set_staging(lbm_handle h, int mode, int stages, int block)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    if (mode < -1 || mode > 1) return fail(h, LBM_EINVAL, "mode = %d must be -1, 0 or 1", mode);
    if (stages != 0 && (stages < 2 || stages > 8)) return fail(h, LBM_EINVAL, "stages = %d must be 0 or in [2, 8]", stages);
    if (block != 0 && (block < 32 || block > 384 || block % 32 != 0))
        return fail(h, LBM_EINVAL, "block = %d must be 0 or a multiple of 32 in [32, 384]", block);
    h->staging = mode;
    h->stages = stages;
    h->rows_block = block;
    return LBM_OK;
}

extern "C" int lbm_set_storage_shift(lbm_handle h, const double u_s[3])
{
    CHECK_HANDLE(h);
    const double u[3] = {u_s ? u_s[0] : 0.0, u_s ? u_s[1] : 0.0, (u_s && h->d == 3) ? u_s[2] : 0.0};
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(u[a])) return fail(h, LBM_EINVAL, "u_s[%d] is not finite", a);
    if (u_s && h->d == 2 && u_s[2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_s[2] must be 0");
    if (u[0] * u[0] + u[1] * u[1] + u[2] * u[2] >= 1.0 / 3.0)
        return fail(h, LBM_EINVAL, "|u_s| must be below the lattice sound speed");
    const bool on = u[0] != 0.0 || u[1] != 0.0 || u[2] != 0.0;
    if (on && h->pattern == LBM_STREAM_AA)
        return fail(h, LBM_EINVAL, "a reference-equilibrium storage shift needs the pull pattern");
    if (on && !h->levels.empty()) return fail(h, LBM_EINVAL, "a storage shift is not combined with refinement");
    // the new table, from the device's own equilibrium (one cell, rho = 1, u_s)
    double newd[27] = {};
    if (on) {
        if (!h->dsh_d) CUDA_TRY(h, cudaMalloc(&h->dsh_d, sizeof(double) * 27));
        double *tmp = nullptr;
        CUDA_TRY(h, cudaMalloc(&tmp, sizeof(double) * (4 + 27)));
        const double one_u[4] = {1.0, u[0], u[1], u[2]};
        cudaError_t e = cudaMemcpyAsync(tmp, one_u, sizeof one_u, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = dispatch<ShiftTable>(h->lattice, h->prec, h->stream, (const double *)tmp, tmp + 4);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(newd, tmp + 4, sizeof(double) * h->q, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return fail(h, LBM_ECUDA, "storage shift table: %s", cudaGetErrorString(e));
    }
    // re-express the stored field (both lattices) in the new shift
    for (int i = 0; i < h->q; ++i) {
        const double delta = h->dsh[i] - newd[i];
        if (delta == 0.0) continue;
        for (int b = 0; b < 2; ++b) {
            if (b == 1 && h->f[1] == h->f[0]) break;
            CUDA_TRY(h, dispatch<ShiftValues>(h->lattice, h->prec, h->stream, h->ncell, i, h->f[b], delta));
            h->launches += 1;
        }
    }
    for (int i = 0; i < 27; ++i) h->dsh[i] = newd[i];
    for (int a = 0; a < 3; ++a) h->shift_u[a] = u[a];
    h->shifted = on;
    if (on) CUDA_TRY(h, cudaMemcpyAsync(h->dsh_d, h->dsh, sizeof(double) * 27, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->cfg_version++;
    return LBM_OK;
}

extern "C" int lbm_set_streaming(lbm_handle h, int pattern)
{
    CHECK_HANDLE(h);
    if (pattern != LBM_STREAM_PULL && pattern != LBM_STREAM_AA)
        return fail(h, LBM_EINVAL, "pattern = %d must be LBM_STREAM_PULL or LBM_STREAM_AA", pattern);
    if (pattern == h->pattern) return LBM_OK;
    const size_t bytes = (size_t)h->q * (size_t)h->ncell * h->elem;
    if (pattern == LBM_STREAM_AA) {
        if (!h->levels.empty())
            return fail(h, LBM_EINVAL, "the AA pattern is not available with refinement patches");
        if (h->shifted)
            return fail(h, LBM_EINVAL, "the AA pattern is not available with a reference-equilibrium storage shift");
        // keep the current lattice, release the other one
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        if (h->cur == 1) std::swap(h->f[0], h->f[1]);
        CUDA_TRY(h, cudaFree(h->f[1]));
        h->f[1] = h->f[0];
        h->cur = 0;
        h->aa_odd = 0;
    } else {
        int rc = aa_normalize(h);
        if (rc != LBM_OK) return rc;
        void *f1 = nullptr;
        cudaError_t e = cudaMalloc(&f1, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LBM_ENOMEM, "second lattice of %zu bytes: %s", bytes, cudaGetErrorString(e));
        }
        // both lattices hold the state (solid cells are never rewritten by the pull update)
        e = cudaMemcpyAsync(f1, h->f[0], bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            cudaFree(f1);
            return fail(h, LBM_ECUDA, "copying the lattice: %s", cudaGetErrorString(e));
        }
        h->f[1] = f1;
        h->cur = 0;
    }
    h->pattern = pattern;
    h->cfg_version++;
    return LBM_OK;
}

extern "C" int lbm_get_streaming(lbm_handle h, int *pattern)
{
    CHECK_HANDLE(h);
    if (pattern) *pattern = h->pattern;
    return LBM_OK;
}

extern "C" int lbm_set_staging_wait(lbm_handle h, uint64_t limit_ns)
{
    CHECK_HANDLE(h);
    h->cfg_version++;
    h->rows_wait_ns = limit_ns;
    return LBM_OK;
}

extern "C" int lbm_get_staging(lbm_handle h, int *active, int *stages, int *block, int *rows_per_tile,
                               int *grid)
{
    CHECK_HANDLE(h);
    RowsPlan pl{};
    bool on = false;
    if (staging_wanted(h) && h->lattice != LBM_D3Q27) {
        StepParams p;
        int rc = build_params(h, p);
        if (rc != LBM_OK) return rc;
        const void *fin = h->f[h->cur];
        const void *fout = h->f[1 - h->cur];
        const cudaError_t e = h->lattice == LBM_D2Q9
                                  ? rows_plan_d2q9(h->prec, p, fin, fout, h->rows_block, h->stages, pl)
                                  : rows_plan_d3q19(h->prec, p, fin, fout, h->rows_block, h->stages, pl);
        if (e != cudaSuccess && e != cudaErrorNotSupported) {
            cudaGetLastError();
            return fail(h, LBM_ECUDA, "row-staged kernel plan: %s", cudaGetErrorString(e));
        }
        on = e == cudaSuccess;
    }
    if (active) *active = on ? 1 : 0;
    if (stages) *stages = on ? pl.stages : 0;
    if (block) *block = on ? pl.block : 0;
    if (rows_per_tile) *rows_per_tile = on ? pl.R : 0;
    if (grid) *grid = on ? pl.grid : 0;
    return LBM_OK;
}

extern "C" int lbm_sync(lbm_handle h)
{
    CHECK_HANDLE(h);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaGetLastError());
    unsigned err = 0;
    CUDA_TRY(h, cudaMemcpy(&err, h->err_d, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CUDA_TRY(h, cudaMemset(h->err_d, 0, sizeof err));
        if (err & kErrBounds)
            return fail(h, LBM_ECUDA, "checked build: an update computed an index outside its lattice (error word %u)",
                        err);
        return fail(h, LBM_ECUDA, "row-staged kernel: a bulk copy did not arrive within 2 s (error word %u)", err);
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------
template <class T>
static int moments_grid(lbm_ctx *h, const GridRef &g, T *rho, T *u, T *pi_neq)
{
    if (g.f == h->f) {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!rho && !u && !pi_neq) return LBM_OK;
    const int64_t N = g.ncell;
    {
        // page-locked outputs: one pass, the kernel writing them over the host link
        T *rm = mapped_host(rho), *um = mapped_host(u), *pm = mapped_host(pi_neq);
        if ((!rho || rm) && (!u || um) && (!pi_neq || pm)) {
            cudaError_t e = dispatch<Moments>(h->lattice, h->prec, h->stream, N, (int64_t)0, N,
                                              (const void *)g.f[*g.cur], rm, um, pm, shift_of(h, g));
            h->launches += 1;
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return fail(h, LBM_ECUDA, "moments: %s", cudaGetErrorString(e));
            return LBM_OK;
        }
    }
    const size_t per = sizeof(T) * ((rho ? 1 : 0) + (u ? 3 : 0) + (pi_neq ? 6 : 0));
    int64_t chunk = 0;
    int rc = stage(h, N, per, chunk);
    if (rc != LBM_OK) return rc;
    T *sd = (T *)h->stage_d;
    T *rd = rho ? sd : nullptr;
    T *ud = u ? sd + (rho ? chunk : 0) : nullptr;
    T *pd = pi_neq ? sd + (rho ? chunk : 0) + (u ? 3 * chunk : 0) : nullptr;
    cudaError_t e = cudaSuccess;
    for (int64_t c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
        const int64_t n = std::min(chunk, N - c0);
        e = dispatch<Moments>(h->lattice, h->prec, h->stream, N, c0, n, (const void *)g.f[*g.cur], rd, ud, pd,
                              shift_of(h, g));
        if (e == cudaSuccess && rho)
            e = cudaMemcpyAsync(rho + c0, rd, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && u)
            e = cudaMemcpyAsync(u + 3 * c0, ud, sizeof(T) * 3 * (size_t)n, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && pi_neq)
            e = cudaMemcpyAsync(pi_neq + 6 * c0, pd, sizeof(T) * 6 * (size_t)n, cudaMemcpyDeviceToHost,
                                h->stream);
        h->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "moments: %s", cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" int lbm_moments(lbm_handle h, double *rho, double *u, double *pi_neq)
{
    CHECK_HANDLE(h);
    return moments_grid(h, coarse_ref(h), rho, u, pi_neq);
}

extern "C" int lbm_moments_f32(lbm_handle h, float *rho, float *u, float *pi_neq)
{
    CHECK_HANDLE(h);
    return moments_grid(h, coarse_ref(h), rho, u, pi_neq);
}

extern "C" int lbm_reduce(lbm_handle h, double *mass, double momentum[3])
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    double out[RED_FIELDS];
    cudaError_t e = dispatch<Reduce>(h->lattice, h->prec, h->stream, h->ncell, (const void *)h->f[h->cur],
                                     (const uint8_t *)h->solid_d, h->red_d, h->red_blocks, (const double *)h->dsh_d);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, h->red_d + (size_t)h->red_blocks * RED_FIELDS, sizeof out,
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 2;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_reduce: %s", cudaGetErrorString(e));
    // sum rho = (fluid cells) + sum (rho - 1)
    if (mass) *mass = out[4] + out[0];
    if (momentum) {
        momentum[0] = out[1];
        momentum[1] = out[2];
        momentum[2] = out[3];
    }
    if (out[5] > 0.0)
        return fail(h, LBM_EUNSTABLE, "%.0f cells are unstable (non-finite, rho <= 0 or |u| >= c_s)", out[5]);
    return LBM_OK;
}

extern "C" int lbm_probe(lbm_handle h, int n, const int64_t *cells, double *p_prime)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (n < 0) return fail(h, LBM_EINVAL, "n < 0");
    if (n == 0) return LBM_OK;
    if (!cells || !p_prime) return fail(h, LBM_EINVAL, "cells and p_prime are required");
    for (int k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= h->ncell)
            return fail(h, LBM_EINVAL, "probe cell %lld out of range", (long long)cells[k]);
    int64_t *cd = nullptr;
    CUDA_TRY(h, cudaMalloc(&cd, sizeof(int64_t) * (size_t)n + sizeof(double) * (size_t)n));
    double *rd = (double *)(cd + n);
    cudaError_t e = cudaMemcpyAsync(cd, cells, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = dispatch<Probe>(h->lattice, h->prec, h->stream, n, (const int64_t *)cd, h->ncell,
                            (const void *)h->f[h->cur], rd, 0, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p_prime, rd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(cd);
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_probe: %s", cudaGetErrorString(e));
    for (int k = 0; k < n; ++k) p_prime[k] = (p_prime[k] - h->rho_ref) / 3.0;
    return LBM_OK;
}

extern "C" int lbm_probe_async(lbm_handle h, int n, const int64_t *cells_dev, double *p_dev)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (n < 0) return fail(h, LBM_EINVAL, "n < 0");
    if (n == 0) return LBM_OK;
    if (!cells_dev || !p_dev) return fail(h, LBM_EINVAL, "cells_dev and p_dev are required");
    const cudaError_t e = dispatch<Probe>(h->lattice, h->prec, h->stream, n, cells_dev, h->ncell,
                                          (const void *)h->f[h->cur], p_dev, 1, h->rho_ref);
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_probe_async: %s", cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" int lbm_info(lbm_handle h, int64_t *step, int64_t *launches, double *bytes_per_cell, double *tau)
{
    CHECK_HANDLE(h);
    if (step) *step = h->step;
    if (launches) *launches = h->launches;
    if (bytes_per_cell) *bytes_per_cell = 2.0 * h->q * (double)h->elem + (h->solid_d ? 1.0 : 0.0);
    if (tau) *tau = h->tau;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint
// ---------------------------------------------------------------------------
// Checkpoint file: header, then per level (0 = coarse / single) its extents
// and current field in the storage format; per refined level its interface
// moments at the current time; the pressure-mean accumulator if sampled.
struct FileHeader {
    char magic[8];
    int32_t lattice, prec, n[3], nlevels;
    int64_t step;
    int64_t rho_count;
    double shift_u[3];  // storage shift of the stored values (0: w_i); from version 3
};

static bool write_all(FILE *fp, const void *p, size_t n) { return std::fwrite(p, 1, n, fp) == n; }
static bool read_all(FILE *fp, void *p, size_t n) { return std::fread(p, 1, n, fp) == n; }

extern "C" int lbm_save(lbm_handle h, const char *path)
{
    CHECK_HANDLE(h);
    {
        const int rc0 = aa_normalize(h);
        if (rc0 != LBM_OK) return rc0;
    }
    if (!path) return fail(h, LBM_EINVAL, "path is null");
    FileHeader hd{};
    std::memcpy(hd.magic, "LBMRRv03", 8);
    for (int a = 0; a < 3; ++a) hd.shift_u[a] = h->shift_u[a];
    hd.lattice = h->lattice;
    hd.prec = h->prec;
    for (int a = 0; a < 3; ++a) hd.n[a] = h->n[a];
    hd.nlevels = nlevels(h);
    hd.step = h->step;
    hd.rho_count = h->rho_acc ? h->rho_count : 0;
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(h, LBM_EIO, "cannot open %s for writing", path);
    bool ok = write_all(fp, &hd, sizeof hd);
    std::vector<char> host;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < hd.nlevels && ok && e == cudaSuccess; ++k) {
        const GridRef g = level_grid(h, k);
        const int32_t ext[4] = {g.n[0], g.n[1], g.n[2], 0};
        const size_t bytes = (size_t)h->q * (size_t)g.ncell * h->elem;
        host.resize(bytes);
        e = cudaMemcpyAsync(host.data(), g.f[*g.cur], bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        ok = e == cudaSuccess && write_all(fp, ext, sizeof ext) && write_all(fp, host.data(), bytes);
    }
    for (int k = 1; k < hd.nlevels && ok && e == cudaSuccess; ++k) {
        FineLevel *F = fine_level(h, k);
        const size_t mb = moment_bytes(h->d == 3, F->geom);
        host.resize(mb);
        e = cudaMemcpyAsync(host.data(), F->M[F->mcur], mb, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        ok = e == cudaSuccess && write_all(fp, host.data(), mb);
    }
    if (ok && e == cudaSuccess && hd.rho_count > 0) {
        const size_t rb = sizeof(double) * (size_t)h->ncell;
        host.resize(rb);
        e = cudaMemcpyAsync(host.data(), h->rho_acc, rb, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        ok = e == cudaSuccess && write_all(fp, host.data(), rb);
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_save: %s", cudaGetErrorString(e));
    if (!ok) return fail(h, LBM_EIO, "short write to %s", path);
    return LBM_OK;
}

extern "C" int lbm_load(lbm_handle h, const char *path)
{
    CHECK_HANDLE(h);
    if (!path) return fail(h, LBM_EINVAL, "path is null");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(h, LBM_EIO, "cannot open %s", path);
    FileHeader hd{};
    if (!read_all(fp, &hd, sizeof hd) || std::memcmp(hd.magic, "LBMRRv03", 8) != 0) {
        std::fclose(fp);
        return fail(h, LBM_EIO, "%s is not a checkpoint", path);
    }
    if (hd.shift_u[0] != h->shift_u[0] || hd.shift_u[1] != h->shift_u[1] || hd.shift_u[2] != h->shift_u[2]) {
        std::fclose(fp);
        return fail(h, LBM_EINVAL, "checkpoint stored with storage shift (%g, %g, %g); set it (lbm_set_storage_shift) "
                                   "before loading",
                    hd.shift_u[0], hd.shift_u[1], hd.shift_u[2]);
    }
    if (hd.lattice != h->lattice || hd.prec != h->prec || hd.n[0] != h->n[0] || hd.n[1] != h->n[1] ||
        hd.n[2] != h->n[2] || hd.nlevels != nlevels(h)) {
        std::fclose(fp);
        return fail(h, LBM_EINVAL, "checkpoint lattice/precision/extents/levels differ from the handle's");
    }
    // read everything before touching the device state
    std::vector<std::vector<char>> fields((size_t)hd.nlevels), moms((size_t)hd.nlevels);
    bool ok = true;
    for (int k = 0; k < hd.nlevels && ok; ++k) {
        const GridRef g = level_grid(h, k);
        int32_t ext[4];
        ok = read_all(fp, ext, sizeof ext);
        if (ok && (ext[0] != g.n[0] || ext[1] != g.n[1] || ext[2] != g.n[2])) {
            std::fclose(fp);
            return fail(h, LBM_EINVAL, "checkpoint level %d extents differ from the handle's", k);
        }
        fields[(size_t)k].resize((size_t)h->q * (size_t)g.ncell * h->elem);
        ok = ok && read_all(fp, fields[(size_t)k].data(), fields[(size_t)k].size());
    }
    for (int k = 1; k < hd.nlevels && ok; ++k) {
        moms[(size_t)k].resize(moment_bytes(h->d == 3, fine_level(h, k)->geom));
        ok = read_all(fp, moms[(size_t)k].data(), moms[(size_t)k].size());
    }
    std::vector<double> racc;
    if (ok && hd.rho_count > 0) {
        racc.resize((size_t)h->ncell);
        ok = read_all(fp, racc.data(), sizeof(double) * racc.size());
    }
    std::fclose(fp);
    if (!ok) return fail(h, LBM_EIO, "short read from %s", path);
    for (int k = 0; k < hd.nlevels; ++k) {
        const GridRef g = level_grid(h, k);
        const std::vector<char> &fk = fields[(size_t)k];
        CUDA_TRY(h, cudaMemcpyAsync(g.f[0], fk.data(), fk.size(), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaMemcpyAsync(g.f[1], fk.data(), fk.size(), cudaMemcpyHostToDevice, h->stream));
        *g.cur = 0;
        if (g.f == h->f) h->aa_odd = 0;
    }
    for (int k = 1; k < hd.nlevels; ++k) {
        FineLevel *F = fine_level(h, k);
        CUDA_TRY(h, cudaMemcpyAsync(F->M[0], moms[(size_t)k].data(), moms[(size_t)k].size(), cudaMemcpyHostToDevice,
                                    h->stream));
        F->mcur = 0;
    }
    if (hd.rho_count > 0) {
        const size_t rb = sizeof(double) * (size_t)h->ncell;
        if (!h->rho_acc) CUDA_TRY(h, cudaMalloc(&h->rho_acc, rb));
        CUDA_TRY(h, cudaMemcpyAsync(h->rho_acc, racc.data(), rb, cudaMemcpyHostToDevice, h->stream));
    }
    h->rho_count = hd.rho_count;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->step = hd.step;
    h->cfg_version++;  // level parities changed: recapture the step graph
    return LBM_OK;
}
