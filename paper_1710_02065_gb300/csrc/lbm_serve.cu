// lbm_serve.cu -- continuous-batching solve server behind lbm_server_* in
// include/lbm.h.
//
// Requests (independent periodic lattices with their own lattice, size, tau,
// step count and storage precision) are queued by lbm_server_submit.  Each
// lbm_server_run call is one round: queued requests are admitted first-fit
// while their population lattices (two, or one with the in-place AA pattern)
// fit in the HBM budget and a slot is free; all active domains then advance
// together for up to `steps` steps in one CUDA-graph replay of [batched
// update per (lattice, precision) group + per-domain advance] x steps;
// domains that reach their step count stop inside the round and are retired
// behind it (moments copied to pinned host memory, device memory returned),
// which frees budget and slots for the next round.
//
// Nothing in a round waits for the GPU: which domains finish is known on the
// host from the step counts (the device counters follow the same
// arithmetic), admissions and retirements are enqueued in stream order
// around the round's graph, and a retired request becomes DONE when the
// event behind its result copy has completed (lbm_server_poll).  At most two
// rounds are in flight, so the host stays at most one round ahead.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <climits>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "lbm.h"
#include "aux_kernels.cuh"
#include "dispatch.h"
#include "serve.cuh"

using namespace rr;

namespace {

struct Request {
    int64_t id = 0;
    int lattice = 0, prec = 0, q = 0;
    int n[3] = {1, 1, 1};
    int64_t ncell = 0;
    double tau = 0.0;
    int64_t steps = 0, done = 0;
    size_t bytes = 0;
    int state = LBM_REQ_QUEUED;
    int slot = -1;
    std::vector<double> rho, u;      // initial state, then the result
    void *f[2] = {nullptr, nullptr};
    bool aa = false;                 // one lattice, in-place AA steps
    double *res_h = nullptr;         // pinned result: rho (ncell), then u (3 ncell)
    cudaEvent_t res_ev = nullptr;    // recorded behind the result copy
    bool retiring = false;           // result copy enqueued, not yet finalised
};

// groups: lattice (3) x precision (4) x cells per lane (1, 2)
constexpr int NGROUPS = 24;
constexpr int NKINDS = 12;  // (lattice, precision) pairs
// Default launch shape of every group: two cells per lane (the vector path,
// every row of a periodic domain on it) and two warps per block, the shape
// the serving stream's tuning picked for D2Q9 / D3Q19 at FP32 and FP16
// (GB300: D2Q9 FP32 87 vs 38 G cell updates/s with one cell per lane, D3Q19
// FP16 52 vs 32).  A row of odd length takes one cell per lane.
inline int lanes_default(int prec)
{
    (void)prec;
    return 2;
}
constexpr int kWarpsDefault = 2;
inline int kind_of(int lattice, int prec) { return lattice * 4 + prec; }
inline int group_of(int lattice, int prec, int v) { return kind_of(lattice, prec) * 2 + (v == 2 ? 1 : 0); }

size_t elem_bytes(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2); }

template <class L, class S, int V>
cudaError_t launch_batched(const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, int wpb,
                           cudaStream_t st)
{
    using C = typename StoreC<S>::C;
    k_batched<L, S, C, V><<<grid, 32 * wpb, 0, st>>>(doms, tiles, ntiles);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t launch_v(int v, const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, int wpb,
                     cudaStream_t st)
{
    return v == 2 ? launch_batched<L, S, 2>(doms, tiles, ntiles, grid, wpb, st)
                  : launch_batched<L, S, 1>(doms, tiles, ntiles, grid, wpb, st);
}

// One persistent launch of group g: `grid` blocks of `wpb` warps
cudaError_t launch_group(int g, const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, int wpb,
                         cudaStream_t st)
{
    const int v = (g & 1) ? 2 : 1;
    switch (g >> 1) {
    case 0: return launch_v<D2Q9, double>(v, doms, tiles, ntiles, grid, wpb, st);
    case 1: return launch_v<D2Q9, float>(v, doms, tiles, ntiles, grid, wpb, st);
    case 2: return launch_v<D2Q9, __half>(v, doms, tiles, ntiles, grid, wpb, st);
    case 3: return launch_v<D2Q9, __nv_bfloat16>(v, doms, tiles, ntiles, grid, wpb, st);
    case 4: return launch_v<D3Q19, double>(v, doms, tiles, ntiles, grid, wpb, st);
    case 5: return launch_v<D3Q19, float>(v, doms, tiles, ntiles, grid, wpb, st);
    case 6: return launch_v<D3Q19, __half>(v, doms, tiles, ntiles, grid, wpb, st);
    case 7: return launch_v<D3Q19, __nv_bfloat16>(v, doms, tiles, ntiles, grid, wpb, st);
    case 8: return launch_v<D3Q27, double>(v, doms, tiles, ntiles, grid, wpb, st);
    case 9: return launch_v<D3Q27, float>(v, doms, tiles, ntiles, grid, wpb, st);
    case 10: return launch_v<D3Q27, __half>(v, doms, tiles, ntiles, grid, wpb, st);
    case 11: return launch_v<D3Q27, __nv_bfloat16>(v, doms, tiles, ntiles, grid, wpb, st);
    }
    return cudaErrorInvalidValue;
}

template <class L, class S>
cudaError_t init_eq(const Request &r, const double *rho, const double *u, cudaStream_t st)
{
    const int64_t N = r.ncell;
    k_init_eq<L, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, 0, N, rho, u, (S *)r.f[0], (S *)r.f[1], 0,
                                                                 nullptr);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t moments(const Request &r, int cur, double *rho, double *u, cudaStream_t st)
{
    const int64_t N = r.ncell;
    k_moments<L, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, 0, N, (const S *)r.f[cur], rho, u, (double *)nullptr);
    return cudaGetLastError();
}

// Per-direction offsets of the vectorised interior path for a domain
template <class L, class S>
cudaError_t domain_offsets(StepParams &p)
{
    set_offsets<L, S>(p);
    return cudaSuccess;
}

#define TYPED_L(fn, L, prec, ...)                                                                   \
    ((prec) == LBM_FP64 ? fn<L, double>(__VA_ARGS__)                                                \
                        : (prec) == LBM_FP32 ? fn<L, float>(__VA_ARGS__)                            \
                                             : (prec) == LBM_FP16_SHIFTED ? fn<L, __half>(__VA_ARGS__) \
                                                                          : fn<L, __nv_bfloat16>(__VA_ARGS__))
#define TYPED(fn, lat, prec, ...)                                                                   \
    ((lat) == LBM_D2Q9 ? TYPED_L(fn, D2Q9, prec, __VA_ARGS__)                                       \
                       : (lat) == LBM_D3Q19 ? TYPED_L(fn, D3Q19, prec, __VA_ARGS__)                 \
                                            : TYPED_L(fn, D3Q27, prec, __VA_ARGS__))

}  // namespace

struct lbm_server {
    size_t budget = 0, used = 0;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t next_id = 1;
    std::deque<Request *> queue;
    std::map<int64_t, Request *> reqs;
    std::vector<int64_t> slot_req;       // request id per slot, 0 = free
    std::vector<BatchDomain> doms_h;
    BatchDomain *doms_d = nullptr;
    std::vector<BatchTile> tiles_h[NGROUPS];
    BatchTile *tiles_d[NGROUPS] = {};
    size_t tiles_cap[NGROUPS] = {};
    bool dirty = true;                   // composition changed since the graph was captured
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;
    int sms = 152;
    // launch shape per (lattice, precision): cells per lane (0: the default
    // rule) and warps per block
    int lanes[NKINDS] = {};
    int wpb[NKINDS] = {kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault,
                       kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault, kWarpsDefault};
    int64_t cell_updates = 0;
    int pattern = LBM_STREAM_PULL;       // streaming pattern of requests admitted from now on
    std::vector<int64_t> remaining;      // host copy of each slot's remaining steps
    cudaEvent_t round_ev[2] = {nullptr, nullptr};
    bool round_rec[2] = {false, false};
    // device time of the rounds' graphs: events around each launch, summed
    // once the round has completed
    cudaEvent_t gpu_t0[2] = {nullptr, nullptr}, gpu_t1[2] = {nullptr, nullptr};
    bool gpu_rec[2] = {false, false};
    double gpu_ms = 0.0;
    int64_t rounds = 0;
    std::vector<Request *> retiring;     // results in flight
    std::string err;
};

static int sfail(lbm_server *s, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else rr_set_global_error(buf);
    return code;
}

#define SCUDA(s, call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return sfail(s, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" int lbm_server_create(lbm_server_handle *out, size_t hbm_budget_bytes, int max_slots, void *cuda_stream)
{
    if (!out) return sfail(nullptr, LBM_EINVAL, "out is null");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 65536) return sfail(nullptr, LBM_EINVAL, "max_slots must be in [1, 65536]");
    if (hbm_budget_bytes == 0) return sfail(nullptr, LBM_EINVAL, "hbm budget must be > 0");
    lbm_server *s = new lbm_server();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->stream = (cudaStream_t)cuda_stream;
    if (!s->stream) {  // stream capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return sfail(nullptr, LBM_ECUDA, "creating the server stream failed");
        }
        s->own_stream = true;
    }
    s->slot_req.assign((size_t)max_slots, 0);
    s->remaining.assign((size_t)max_slots, 0);
    s->doms_h.assign((size_t)max_slots, BatchDomain{});
    for (int k = 0; k < 2; ++k)
        if (cudaEventCreateWithFlags(&s->round_ev[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&s->gpu_t0[k]) != cudaSuccess || cudaEventCreate(&s->gpu_t1[k]) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return sfail(nullptr, LBM_ECUDA, "creating the round events failed");
        }
    if (cudaMalloc(&s->doms_d, sizeof(BatchDomain) * (size_t)max_slots) != cudaSuccess ||
        cudaMemset(s->doms_d, 0, sizeof(BatchDomain) * (size_t)max_slots) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(nullptr, LBM_ENOMEM, "allocating the domain table failed");
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (sms > 0) s->sms = sms;
    *out = s;
    return LBM_OK;
}

static void free_request_memory(lbm_server *s, Request *r)
{
    if (r->f[0]) cudaFreeAsync(r->f[0], s->stream);
    if (r->f[1] && r->f[1] != r->f[0]) cudaFreeAsync(r->f[1], s->stream);
    r->f[0] = r->f[1] = nullptr;
}

static void free_request_host(Request *r)
{
    if (r->res_h) cudaFreeHost(r->res_h);
    if (r->res_ev) cudaEventDestroy(r->res_ev);
    r->res_h = nullptr;
    r->res_ev = nullptr;
}

extern "C" void lbm_server_destroy(lbm_server_handle s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->reqs) {
        free_request_memory(s, kv.second);
        free_request_host(kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 2; ++k) {
        if (s->round_ev[k]) cudaEventDestroy(s->round_ev[k]);
        if (s->gpu_t0[k]) cudaEventDestroy(s->gpu_t0[k]);
        if (s->gpu_t1[k]) cudaEventDestroy(s->gpu_t1[k]);
    }
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (int g = 0; g < NGROUPS; ++g)
        if (s->tiles_d[g]) cudaFree(s->tiles_d[g]);
    if (s->doms_d) cudaFree(s->doms_d);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" const char *lbm_server_last_error(lbm_server_handle s) { return s ? s->err.c_str() : lbm_last_error(nullptr); }

extern "C" int lbm_server_submit(lbm_server_handle s, const lbm_request *req, int64_t *id)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (!req || !id) return sfail(s, LBM_EINVAL, "req and id are required");
    if (req->lattice != LBM_D2Q9 && req->lattice != LBM_D3Q19 && req->lattice != LBM_D3Q27)
        return sfail(s, LBM_EINVAL, "unknown lattice");
    if (req->precision < LBM_FP64 || req->precision > LBM_BF16_SHIFTED) return sfail(s, LBM_EINVAL, "unknown precision");
    if (!(req->tau > 0.5) || !std::isfinite(req->tau)) return sfail(s, LBM_EINVAL, "tau must be > 1/2");
    if (req->steps < 0) return sfail(s, LBM_EINVAL, "steps must be >= 0");
    for (int a = 0; a < 3; ++a)
        if (req->extents[a] < 1 || req->extents[a] > 65535) return sfail(s, LBM_EINVAL, "extents must be in [1, 65535]");
    if ((int64_t)req->extents[0] * req->extents[1] * req->extents[2] > 2147483647LL)
        return sfail(s, LBM_EINVAL, "a lattice holds at most 2^31 - 1 cells");
    if (req->lattice == LBM_D2Q9 && req->extents[2] != 1) return sfail(s, LBM_EINVAL, "D2Q9 needs extents[2] == 1");
    Request *r = new Request();
    r->lattice = req->lattice;
    r->prec = req->precision;
    r->q = req->lattice == LBM_D2Q9 ? 9 : (req->lattice == LBM_D3Q19 ? 19 : 27);
    for (int a = 0; a < 3; ++a) r->n[a] = req->extents[a];
    r->ncell = (int64_t)r->n[0] * r->n[1] * r->n[2];
    r->tau = req->tau;
    r->steps = req->steps;
    r->aa = s->pattern == LBM_STREAM_AA;
    r->bytes = (r->aa ? 1 : 2) * (size_t)r->q * (size_t)r->ncell * elem_bytes(r->prec);
    if (r->bytes > s->budget) {
        const size_t need = r->bytes;
        delete r;
        return sfail(s, LBM_EINVAL, "request needs %zu bytes, more than the whole budget (%zu)", need, s->budget);
    }
    r->rho.assign((size_t)r->ncell, 1.0);
    r->u.assign((size_t)r->ncell * 3, 0.0);
    if (req->rho) std::memcpy(r->rho.data(), req->rho, sizeof(double) * (size_t)r->ncell);
    if (req->u) std::memcpy(r->u.data(), req->u, sizeof(double) * 3 * (size_t)r->ncell);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *id = r->id;
    return LBM_OK;
}

// Admission: first fit in arrival order while budget and slots allow.  The
// allocation, the initial state's upload, the equilibrium kernel and the
// domain-table entry are enqueued on the server stream (pageable host data
// are staged by the copy calls themselves, so nothing is awaited here).
static int admit(lbm_server *s)
{
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request *r = *it;
        int slot = -1;
        for (int k = 0; k < s->max_slots; ++k)
            if (s->slot_req[k] == 0) {
                slot = k;
                break;
            }
        if (slot < 0) break;
        if (s->used + r->bytes > s->budget) {
            ++it;
            continue;
        }
        const size_t lat = (size_t)r->q * (size_t)r->ncell * elem_bytes(r->prec);
        cudaError_t e = cudaMallocAsync(&r->f[0], lat, s->stream);
        if (e == cudaSuccess) {
            if (r->aa)
                r->f[1] = r->f[0];
            else
                e = cudaMallocAsync(&r->f[1], lat, s->stream);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_request_memory(s, r);
            ++it;  // device memory short of the budget: try again next round
            continue;
        }
        double *buf = nullptr;
        e = cudaMallocAsync((void **)&buf, sizeof(double) * 4 * (size_t)r->ncell, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf, r->rho.data(), sizeof(double) * (size_t)r->ncell, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf + r->ncell, r->u.data(), sizeof(double) * 3 * (size_t)r->ncell,
                                cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = TYPED(init_eq, r->lattice, r->prec, *r, buf, buf + r->ncell, s->stream);
        if (buf) cudaFreeAsync(buf, s->stream);
        if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "admitting request %lld: %s", (long long)r->id, cudaGetErrorString(e));
        std::vector<double>().swap(r->rho);
        std::vector<double>().swap(r->u);
        BatchDomain d{};
        std::memset(&d, 0, sizeof d);
        for (int a = 0; a < 3; ++a) {
            d.p.n[a] = r->n[a];
            d.p.periodic[a] = 1;
        }
        d.p.ncell = r->ncell;
        for (int f = 0; f < 6; ++f) d.p.face_cells[f] = 1;
        d.p.rho_ref = 1.0;
        d.p.sponge_rest = 1;
        d.p.omega = 1.0 - 1.0 / r->tau;
        d.p.jet_x_layer = INT_MAX;
        set_bulk_box(d.p);
        TYPED(domain_offsets, r->lattice, r->prec, d.p);
        d.f[0] = r->f[0];
        d.f[1] = r->f[1];
        for (int b = 0; b < 2; ++b)
            for (int i = 0; i < r->q; ++i)
                d.base[b][i] = (char *)r->f[b] + (size_t)i * (size_t)r->ncell * elem_bytes(r->prec);
        d.cur = 0;
        d.active = r->steps > 0 ? 1 : 0;
        d.aa = r->aa ? 1 : 0;
        d.remaining = r->steps;
        // the host table entry of a slot changes only when the slot is
        // admitted again, after this copy was staged
        s->doms_h[slot] = d;
        e = cudaMemcpyAsync(s->doms_d + slot, &s->doms_h[slot], sizeof(BatchDomain), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "domain table upload: %s", cudaGetErrorString(e));
        s->slot_req[slot] = r->id;
        s->remaining[slot] = r->steps;
        r->slot = slot;
        r->state = LBM_REQ_RUNNING;
        s->used += r->bytes;
        s->dirty = true;
        it = s->queue.erase(it);
    }
    return LBM_OK;
}

// Cells per lane of a request: the chosen (or default) value; one for a row
// of odd length or a lattice whose direction arrays span 2 GB or more (the
// vector path addresses them with 32-bit offsets)
static int lanes_of(const lbm_server *s, const Request *r)
{
    const int k = kind_of(r->lattice, r->prec);
    const int v = s->lanes[k] ? s->lanes[k] : lanes_default(r->prec);
    const bool off32 = (int64_t)r->q * r->ncell * (int64_t)elem_bytes(r->prec) < ((int64_t)1 << 31);
    return (v == 2 && r->n[0] % 2 == 0 && off32) ? 2 : 1;
}

// Warp tile lists per group: 32 x V consecutive cells of a row each.
static int build_tiles(lbm_server *s)
{
    for (int g = 0; g < NGROUPS; ++g) s->tiles_h[g].clear();
    for (int k = 0; k < s->max_slots; ++k) {
        if (!s->slot_req[k] || s->remaining[k] <= 0) continue;
        Request *r = s->reqs[s->slot_req[k]];
        const int v = lanes_of(s, r);
        const int rows = r->n[1] * r->n[2];
        const int segs = (r->n[0] + 32 * v - 1) / (32 * v);
        std::vector<BatchTile> &list = s->tiles_h[group_of(r->lattice, r->prec, v)];
        for (int row = 0; row < rows; ++row)
            for (int xs = 0; xs < segs; ++xs) list.push_back(BatchTile{k, row, xs, 0});
    }
    for (int g = 0; g < NGROUPS; ++g) {
        const size_t n = s->tiles_h[g].size();
        if (n == 0) continue;
        if (n > s->tiles_cap[g]) {
            // a larger list: the old one may still be read by a round in flight
            SCUDA(s, cudaStreamSynchronize(s->stream));
            if (s->tiles_d[g]) cudaFree(s->tiles_d[g]);
            s->tiles_d[g] = nullptr;
            SCUDA(s, cudaMalloc(&s->tiles_d[g], sizeof(BatchTile) * n * 2));
            s->tiles_cap[g] = n * 2;
        }
        // staged by the copy (pageable): the host list may change afterwards
        SCUDA(s, cudaMemcpyAsync(s->tiles_d[g], s->tiles_h[g].data(), sizeof(BatchTile) * n, cudaMemcpyHostToDevice,
                                 s->stream));
    }
    return LBM_OK;
}

static cudaError_t enqueue_steps(lbm_server *s, int64_t steps)
{
    for (int64_t t = 0; t < steps; ++t) {
        for (int g = 0; g < NGROUPS; ++g) {
            const int n = (int)s->tiles_h[g].size();
            if (n == 0) continue;
            // persistent grid: at most 32 resident warps per SM asked for
            const int wpb = s->wpb[g >> 1];
            const int blocks = (n + wpb - 1) / wpb, cap = s->sms * (32 / wpb);
            cudaError_t e = launch_group(g, s->doms_d, s->tiles_d[g], n, blocks < cap ? blocks : cap, wpb, s->stream);
            if (e != cudaSuccess) return e;
        }
        k_batch_advance<<<(s->max_slots + 127) / 128, 128, 0, s->stream>>>(s->doms_d, s->max_slots);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Standard layout of a retiring AA domain left after a gather-push step
template <class L, class S>
cudaError_t unswap(const Request &r, const StepParams &p, cudaStream_t st)
{
    return launch_aa_unswap<L, S>(p, r.f[0], st);
}

// Enqueue the retirement of the request in slot k, whose last step ran in
// the work already enqueued: its moments into pinned host memory (an event
// behind the copy), its device memory and slot returned.
static int retire_slot(lbm_server *s, int k)
{
    Request *r = s->reqs[s->slot_req[k]];
    const int par = (int)(r->steps & 1);  // lattice (pull) / layout (AA) after the last step
    cudaError_t e = cudaSuccess;
    if (r->aa && par) e = TYPED(unswap, r->lattice, r->prec, *r, s->doms_h[k].p, s->stream);
    double *buf = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&buf, sizeof(double) * 4 * (size_t)r->ncell, s->stream);
    if (e == cudaSuccess) e = TYPED(moments, r->lattice, r->prec, *r, r->aa ? 0 : par, buf, buf + r->ncell, s->stream);
    if (e == cudaSuccess && !r->res_h)
        e = cudaHostAlloc((void **)&r->res_h, sizeof(double) * 4 * (size_t)r->ncell, cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->res_h, buf, sizeof(double) * 4 * (size_t)r->ncell, cudaMemcpyDeviceToHost, s->stream);
    if (buf) cudaFreeAsync(buf, s->stream);
    if (e == cudaSuccess && !r->res_ev) e = cudaEventCreateWithFlags(&r->res_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->res_ev, s->stream);
    if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "retiring request %lld: %s", (long long)r->id, cudaGetErrorString(e));
    free_request_memory(s, r);
    s->used -= r->bytes;
    s->slot_req[k] = 0;
    r->slot = -1;
    r->done = r->steps;
    r->retiring = true;
    s->retiring.push_back(r);
    s->dirty = true;
    return LBM_OK;
}

// A retiring request whose result copy has completed: DONE, or FAILED when
// the result is not finite.  wait: block until the copy has completed.
static int finalize(lbm_server *s, Request *r, bool wait, bool *finished)
{
    *finished = false;
    if (!r->retiring) return LBM_OK;
    const cudaError_t q = wait ? cudaEventSynchronize(r->res_ev) : cudaEventQuery(r->res_ev);
    if (q == cudaErrorNotReady) return LBM_OK;
    if (q != cudaSuccess) return sfail(s, LBM_ECUDA, "result of request %lld: %s", (long long)r->id, cudaGetErrorString(q));
    bool finite = true;
    for (int64_t c = 0; c < r->ncell; ++c) finite = finite && std::isfinite(r->res_h[c]);
    r->state = finite ? LBM_REQ_DONE : LBM_REQ_FAILED;
    r->retiring = false;
    s->retiring.erase(std::find(s->retiring.begin(), s->retiring.end(), r));
    *finished = true;
    return LBM_OK;
}

static int finalize_ready(lbm_server *s, int *completed)
{
    std::vector<Request *> now = s->retiring;
    for (Request *r : now) {
        bool fin = false;
        const int rc = finalize(s, r, false, &fin);
        if (rc != LBM_OK) return rc;
        if (fin && completed) ++*completed;
    }
    return LBM_OK;
}

extern "C" int lbm_server_set_streaming(lbm_server_handle s, int pattern)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (pattern != LBM_STREAM_PULL && pattern != LBM_STREAM_AA)
        return sfail(s, LBM_EINVAL, "pattern must be LBM_STREAM_PULL or LBM_STREAM_AA");
    s->pattern = pattern;
    return LBM_OK;
}

extern "C" int lbm_server_set_launch(lbm_server_handle s, int lattice, int precision, int cells_per_lane,
                                     int warps_per_block)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return sfail(s, LBM_EINVAL, "unknown lattice");
    if (precision < LBM_FP64 || precision > LBM_BF16_SHIFTED) return sfail(s, LBM_EINVAL, "unknown precision");
    if (cells_per_lane < 0 || cells_per_lane > 2) return sfail(s, LBM_EINVAL, "cells_per_lane must be 0, 1 or 2");
    if (warps_per_block != 0 && warps_per_block != 1 && warps_per_block != 2 && warps_per_block != 4 &&
        warps_per_block != 8)
        return sfail(s, LBM_EINVAL, "warps_per_block must be 0, 1, 2, 4 or 8");
    const int k = kind_of(lattice, precision);
    s->lanes[k] = cells_per_lane;
    s->wpb[k] = warps_per_block ? warps_per_block : kWarpsDefault;
    s->dirty = true;  // new tile lists and a new graph at the next round
    return LBM_OK;
}

extern "C" int lbm_server_get_launch(lbm_server_handle s, int lattice, int precision, int *cells_per_lane,
                                     int *warps_per_block)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return sfail(s, LBM_EINVAL, "unknown lattice");
    if (precision < LBM_FP64 || precision > LBM_BF16_SHIFTED) return sfail(s, LBM_EINVAL, "unknown precision");
    const int k = kind_of(lattice, precision);
    if (cells_per_lane) *cells_per_lane = s->lanes[k] ? s->lanes[k] : lanes_default(precision);
    if (warps_per_block) *warps_per_block = s->wpb[k];
    return LBM_OK;
}

extern "C" int lbm_server_run(lbm_server_handle s, int64_t steps, int *completed)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (steps < 1) return sfail(s, LBM_EINVAL, "steps must be >= 1");
    if (completed) *completed = 0;
    // at most two rounds in flight: wait for the one before the previous
    const int slot_ev = (int)(s->rounds & 1);
    if (s->round_rec[slot_ev]) SCUDA(s, cudaEventSynchronize(s->round_ev[slot_ev]));
    if (s->gpu_rec[slot_ev]) {
        float ms = 0.0f;
        SCUDA(s, cudaEventElapsedTime(&ms, s->gpu_t0[slot_ev], s->gpu_t1[slot_ev]));
        s->gpu_ms += ms;
        s->gpu_rec[slot_ev] = false;
    }
    int rc = finalize_ready(s, completed);
    if (rc != LBM_OK) return rc;
    rc = admit(s);
    if (rc != LBM_OK) return rc;
    // requests with zero steps finish at admission
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slot_req[k] && s->remaining[k] <= 0) {
            rc = retire_slot(s, k);
            if (rc != LBM_OK) return rc;
        }
    bool any = false;
    for (int k = 0; k < s->max_slots; ++k) any = any || s->slot_req[k] != 0;
    if (any) {
        if (s->dirty || s->graph_steps != steps) {
            rc = build_tiles(s);
            if (rc != LBM_OK) return rc;
            if (s->graph) {
                cudaGraphExecDestroy(s->graph);
                s->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            SCUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_steps(s, steps);
            cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return sfail(s, LBM_ECUDA, "capturing the batched round: %s",
                             cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&s->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "instantiating the batched round: %s", cudaGetErrorString(e));
            s->graph_steps = steps;
            s->dirty = false;
        }
        SCUDA(s, cudaEventRecord(s->gpu_t0[slot_ev], s->stream));
        SCUDA(s, cudaGraphLaunch(s->graph, s->stream));
        SCUDA(s, cudaEventRecord(s->gpu_t1[slot_ev], s->stream));
        s->gpu_rec[slot_ev] = true;
        // the device counters advance as the host's: domains that finish in
        // this round are retired behind it
        for (int k = 0; k < s->max_slots; ++k) {
            if (!s->slot_req[k]) continue;
            Request *r = s->reqs[s->slot_req[k]];
            const int64_t adv = s->remaining[k] < steps ? s->remaining[k] : steps;
            s->cell_updates += r->ncell * adv;
            s->remaining[k] -= adv;
            r->done = r->steps - s->remaining[k];
            if (s->remaining[k] <= 0) {
                rc = retire_slot(s, k);
                if (rc != LBM_OK) return rc;
            }
        }
    }
    SCUDA(s, cudaEventRecord(s->round_ev[slot_ev], s->stream));
    s->round_rec[slot_ev] = true;
    s->rounds += 1;
    return finalize_ready(s, completed);
}

extern "C" int lbm_server_poll(lbm_server_handle s, int64_t id, int *state, int64_t *steps_done)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_EINVAL, "unknown request %lld", (long long)id);
    bool fin = false;
    const int rc = finalize(s, it->second, false, &fin);
    if (rc != LBM_OK) return rc;
    if (state) *state = it->second->state;
    if (steps_done) *steps_done = it->second->done;
    return LBM_OK;
}

extern "C" int lbm_server_result(lbm_server_handle s, int64_t id, double *rho, double *u)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_EINVAL, "unknown request %lld", (long long)id);
    Request *r = it->second;
    bool fin = false;
    const int rc0 = finalize(s, r, true, &fin);
    if (rc0 != LBM_OK) return rc0;
    if (r->state != LBM_REQ_DONE && r->state != LBM_REQ_FAILED)
        return sfail(s, LBM_EINVAL, "request %lld has not finished", (long long)id);
    if (rho) std::memcpy(rho, r->res_h, sizeof(double) * (size_t)r->ncell);
    if (u) std::memcpy(u, r->res_h + r->ncell, sizeof(double) * 3 * (size_t)r->ncell);
    const int st = r->state;
    free_request_host(r);
    s->reqs.erase(it);
    delete r;
    return st == LBM_REQ_DONE ? LBM_OK : sfail(s, LBM_EUNSTABLE, "request %lld produced non-finite values", (long long)id);
}

extern "C" int lbm_server_gpu_time(lbm_server_handle s, double *ms)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    SCUDA(s, cudaStreamSynchronize(s->stream));
    for (int k = 0; k < 2; ++k)
        if (s->gpu_rec[k]) {
            float m = 0.0f;
            SCUDA(s, cudaEventElapsedTime(&m, s->gpu_t0[k], s->gpu_t1[k]));
            s->gpu_ms += m;
            s->gpu_rec[k] = false;
        }
    if (ms) *ms = s->gpu_ms;
    return LBM_OK;
}

extern "C" int lbm_server_stats(lbm_server_handle s, int *queued, int *running, size_t *bytes_in_use,
                                int64_t *cell_updates)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    int run = 0;
    for (int k = 0; k < s->max_slots; ++k) run += s->slot_req[k] != 0;
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = run;
    if (bytes_in_use) *bytes_in_use = s->used;
    if (cell_updates) *cell_updates = s->cell_updates;
    return LBM_OK;
}
