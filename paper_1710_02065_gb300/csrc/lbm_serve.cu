// lbm_serve.cu -- continuous-batching solve server behind lbm_server_* in
// include/lbm.h.
//
// Requests (independent periodic lattices with their own lattice, size, tau,
// step count and storage precision) are queued by lbm_server_submit.  Each
// lbm_server_run call is one round: queued requests are admitted first-fit
// while their two population lattices fit in the HBM budget and a slot is
// free; all active domains then advance together for up to `steps` steps in
// one CUDA-graph replay of [batched update per (lattice, precision) group +
// per-domain advance] x steps; domains that reach their step count stop
// inside the round and are retired at its end (moments copied to the host,
// memory returned), which frees budget and slots for the next round.
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
};

// groups: lattice (3) x precision (4) x cells per lane (1, 2)
constexpr int NGROUPS = 24;
// Cells per lane: two except for FP32 (in the batched kernel a warp item is
// 32 x V cells of a row, and larger items amortise the per-item work; one
// cell per lane for every D2Q9 request measured slower on the serving stream:
// 33.2 vs 35.0 G cell updates/s saturated)
inline int lanes_v(int lattice, int prec, int nx)
{
    (void)lattice;
    return (prec != LBM_FP32 && nx % 2 == 0) ? 2 : 1;
}
inline int group_of(int lattice, int prec, int v) { return (lattice * 4 + prec) * 2 + (v == 2 ? 1 : 0); }

size_t elem_bytes(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2); }

template <class L, class S, int V>
cudaError_t launch_batched(const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, cudaStream_t st)
{
    using C = typename StoreC<S>::C;
    k_batched<L, S, C, V><<<grid, 128, 0, st>>>(doms, tiles, ntiles);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t launch_v(int v, const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, cudaStream_t st)
{
    return v == 2 ? launch_batched<L, S, 2>(doms, tiles, ntiles, grid, st)
                  : launch_batched<L, S, 1>(doms, tiles, ntiles, grid, st);
}

cudaError_t launch_group(int g, const BatchDomain *doms, const BatchTile *tiles, int ntiles, int grid, cudaStream_t st)
{
    const int v = (g & 1) ? 2 : 1;
    switch (g >> 1) {
    case 0: return launch_v<D2Q9, double>(v, doms, tiles, ntiles, grid, st);
    case 1: return launch_v<D2Q9, float>(v, doms, tiles, ntiles, grid, st);
    case 2: return launch_v<D2Q9, __half>(v, doms, tiles, ntiles, grid, st);
    case 3: return launch_v<D2Q9, __nv_bfloat16>(v, doms, tiles, ntiles, grid, st);
    case 4: return launch_v<D3Q19, double>(v, doms, tiles, ntiles, grid, st);
    case 5: return launch_v<D3Q19, float>(v, doms, tiles, ntiles, grid, st);
    case 6: return launch_v<D3Q19, __half>(v, doms, tiles, ntiles, grid, st);
    case 7: return launch_v<D3Q19, __nv_bfloat16>(v, doms, tiles, ntiles, grid, st);
    case 8: return launch_v<D3Q27, double>(v, doms, tiles, ntiles, grid, st);
    case 9: return launch_v<D3Q27, float>(v, doms, tiles, ntiles, grid, st);
    case 10: return launch_v<D3Q27, __half>(v, doms, tiles, ntiles, grid, st);
    case 11: return launch_v<D3Q27, __nv_bfloat16>(v, doms, tiles, ntiles, grid, st);
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
    k_moments<L, S><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, 0, N, (const S *)r.f[cur], rho, u, nullptr);
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
    int grid = 0;
    int64_t cell_updates = 0;
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
    s->doms_h.assign((size_t)max_slots, BatchDomain{});
    if (cudaMalloc(&s->doms_d, sizeof(BatchDomain) * (size_t)max_slots) != cudaSuccess ||
        cudaMemset(s->doms_d, 0, sizeof(BatchDomain) * (size_t)max_slots) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(nullptr, LBM_ENOMEM, "allocating the domain table failed");
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    s->grid = (sms > 0 ? sms : 152) * 8;
    *out = s;
    return LBM_OK;
}

static void free_request_memory(lbm_server *s, Request *r)
{
    for (int k = 0; k < 2; ++k)
        if (r->f[k]) {
            cudaFreeAsync(r->f[k], s->stream);
            r->f[k] = nullptr;
        }
}

extern "C" void lbm_server_destroy(lbm_server_handle s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->reqs) {
        free_request_memory(s, kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(s->stream);
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
    r->bytes = 2 * (size_t)r->q * (size_t)r->ncell * elem_bytes(r->prec);
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

// Admission: first fit in arrival order while budget and slots allow.
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
        const size_t half = r->bytes / 2;
        cudaError_t e = cudaMallocAsync(&r->f[0], half, s->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&r->f[1], half, s->stream);
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
        d.remaining = r->steps;
        s->doms_h[slot] = d;
        e = cudaMemcpyAsync(s->doms_d + slot, &s->doms_h[slot], sizeof(BatchDomain), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "domain table upload: %s", cudaGetErrorString(e));
        // the host copy must stay valid until the copy ran
        SCUDA(s, cudaStreamSynchronize(s->stream));
        s->slot_req[slot] = r->id;
        r->slot = slot;
        r->state = LBM_REQ_RUNNING;
        s->used += r->bytes;
        s->dirty = true;
        it = s->queue.erase(it);
    }
    return LBM_OK;
}

// Warp tile lists per group: 32 x V consecutive cells of a row each.
static int build_tiles(lbm_server *s)
{
    for (int g = 0; g < NGROUPS; ++g) s->tiles_h[g].clear();
    for (int k = 0; k < s->max_slots; ++k) {
        if (!s->slot_req[k]) continue;
        Request *r = s->reqs[s->slot_req[k]];
        if (r->state != LBM_REQ_RUNNING) continue;
        const int v = lanes_v(r->lattice, r->prec, r->n[0]);
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
            if (s->tiles_d[g]) cudaFree(s->tiles_d[g]);
            s->tiles_d[g] = nullptr;
            SCUDA(s, cudaMalloc(&s->tiles_d[g], sizeof(BatchTile) * n));
            s->tiles_cap[g] = n;
        }
        SCUDA(s, cudaMemcpyAsync(s->tiles_d[g], s->tiles_h[g].data(), sizeof(BatchTile) * n, cudaMemcpyHostToDevice,
                                 s->stream));
    }
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

static cudaError_t enqueue_steps(lbm_server *s, int64_t steps)
{
    for (int64_t t = 0; t < steps; ++t) {
        for (int g = 0; g < NGROUPS; ++g) {
            const int n = (int)s->tiles_h[g].size();
            if (n == 0) continue;
            const int blocks = (n + 3) / 4;  // 4 warps per block
            cudaError_t e = launch_group(g, s->doms_d, s->tiles_d[g], n, blocks < s->grid ? blocks : s->grid, s->stream);
            if (e != cudaSuccess) return e;
        }
        k_batch_advance<<<(s->max_slots + 127) / 128, 128, 0, s->stream>>>(s->doms_d, s->max_slots);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Retire domains that finished: moments to the host, memory back to the budget.
static int retire(lbm_server *s, int *completed)
{
    std::vector<BatchDomain> now((size_t)s->max_slots);
    SCUDA(s, cudaMemcpyAsync(now.data(), s->doms_d, sizeof(BatchDomain) * (size_t)s->max_slots, cudaMemcpyDeviceToHost,
                             s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    for (int k = 0; k < s->max_slots; ++k) {
        if (!s->slot_req[k]) continue;
        Request *r = s->reqs[s->slot_req[k]];
        r->done = r->steps - now[k].remaining;
        if (now[k].active) continue;
        double *buf = nullptr;
        SCUDA(s, cudaMallocAsync((void **)&buf, sizeof(double) * 4 * (size_t)r->ncell, s->stream));
        cudaError_t e = TYPED(moments, r->lattice, r->prec, *r, now[k].cur, buf, buf + r->ncell, s->stream);
        r->rho.resize((size_t)r->ncell);
        r->u.resize((size_t)r->ncell * 3);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->rho.data(), buf, sizeof(double) * (size_t)r->ncell, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->u.data(), buf + r->ncell, sizeof(double) * 3 * (size_t)r->ncell,
                                cudaMemcpyDeviceToHost, s->stream);
        cudaFreeAsync(buf, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return sfail(s, LBM_ECUDA, "retiring request %lld: %s", (long long)r->id, cudaGetErrorString(e));
        bool finite = true;
        for (double v : r->rho) finite = finite && std::isfinite(v);
        free_request_memory(s, r);
        s->used -= r->bytes;
        s->slot_req[k] = 0;
        r->slot = -1;
        r->state = finite ? LBM_REQ_DONE : LBM_REQ_FAILED;
        s->dirty = true;
        if (completed) ++*completed;
    }
    return LBM_OK;
}

extern "C" int lbm_server_run(lbm_server_handle s, int64_t steps, int *completed)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    if (steps < 1) return sfail(s, LBM_EINVAL, "steps must be >= 1");
    if (completed) *completed = 0;
    int rc = admit(s);
    if (rc != LBM_OK) return rc;
    // requests with zero steps finish at admission
    rc = retire(s, completed);
    if (rc != LBM_OK) return rc;
    bool any = false;
    for (int k = 0; k < s->max_slots; ++k) any = any || s->slot_req[k] != 0;
    if (!any) return LBM_OK;
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
    // cell updates this round, counted on the host from the remaining steps
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slot_req[k]) {
            Request *r = s->reqs[s->slot_req[k]];
            const int64_t left = r->steps - r->done;
            s->cell_updates += r->ncell * (left < steps ? left : steps);
        }
    SCUDA(s, cudaGraphLaunch(s->graph, s->stream));
    return retire(s, completed);
}

extern "C" int lbm_server_poll(lbm_server_handle s, int64_t id, int *state, int64_t *steps_done)
{
    if (!s) return sfail(nullptr, LBM_EINVAL, "null server");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_EINVAL, "unknown request %lld", (long long)id);
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
    if (r->state != LBM_REQ_DONE && r->state != LBM_REQ_FAILED)
        return sfail(s, LBM_EINVAL, "request %lld has not finished", (long long)id);
    if (rho) std::memcpy(rho, r->rho.data(), sizeof(double) * (size_t)r->ncell);
    if (u) std::memcpy(u, r->u.data(), sizeof(double) * 3 * (size_t)r->ncell);
    const int st = r->state;
    s->reqs.erase(it);
    delete r;
    return st == LBM_REQ_DONE ? LBM_OK : sfail(s, LBM_EUNSTABLE, "request %lld produced non-finite values", (long long)id);
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
