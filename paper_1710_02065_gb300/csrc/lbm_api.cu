// lbm_api.cu -- host runtime behind include/lbm.h: handle, validation,
// device memory, launches.  Every numerical step runs in the kernels of
// step.cuh / aux_kernels.cuh; this file only moves arguments.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "aux_kernels.cuh"
#include "dispatch.h"
#include "step.cuh"

using namespace rr;

struct lbm_ctx {
    int lattice = 0, q = 0, d = 0, prec = 0;
    int n[3] = {1, 1, 1};
    int64_t ncell = 0;
    size_t elem = 0;
    double tau = 0.0, Ma_ref = 0.0;
    cudaStream_t stream = nullptr;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *solid_d = nullptr;
    double *prof_d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int kind[6] = {0, 0, 0, 0, 0, 0};
    double u_face[6][3] = {};
    int sponge_w[6] = {0, 0, 0, 0, 0, 0};
    double sponge_chi[6] = {0, 0, 0, 0, 0, 0};
    bool ref_set = false;
    double rho_ref = 1.0, u_ref[3] = {0, 0, 0};
    uint64_t noise_seed = 0;
    double noise_amp = 0.0;
    int64_t step = 0, launches = 0;
    int block = 0;  // 0: automatic
    int vec = 0;    // cells per thread; 0: automatic, 1: scalar kernel
    double *red_d = nullptr;  // reduction partials + result
    int red_blocks = 0;
    std::string err;
};

static thread_local std::string g_create_err;

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
    static cudaError_t run(cudaStream_t st, int64_t N, const double *rho, const double *u, void *f0,
                           void *f1)
    {
        k_init_eq<L, S><<<grid1(N, 256), 256, 0, st>>>(N, rho, u, (S *)f0, (S *)f1);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct SetDir {
    static cudaError_t run(cudaStream_t st, int64_t N, int i, const double *src, void *f0, void *f1)
    {
        k_set_dir<L, S><<<grid1(N, 256), 256, 0, st>>>(N, i, src, (S *)f0, (S *)f1);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct GetDir {
    static cudaError_t run(cudaStream_t st, int64_t N, int i, const void *f, double *dst)
    {
        k_get_dir<L, S><<<grid1(N, 256), 256, 0, st>>>(N, i, (const S *)f, dst);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Moments {
    static cudaError_t run(cudaStream_t st, int64_t N, const void *f, double *rho, double *u, double *pn)
    {
        k_moments<L, S><<<grid1(N, 256), 256, 0, st>>>(N, (const S *)f, rho, u, pn);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Reduce {
    static cudaError_t run(cudaStream_t st, int64_t N, const void *f, const uint8_t *solid,
                           double *partial, int nblocks)
    {
        k_reduce<L, S><<<nblocks, RED_BLOCK, 0, st>>>(N, (const S *)f, solid, partial);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, 32 * RED_FIELDS, 0, st>>>(nblocks, partial, partial + (int64_t)nblocks * RED_FIELDS);
        return cudaGetLastError();
    }
};
template <class L, class S>
struct Probe {
    static cudaError_t run(cudaStream_t st, int n, const int64_t *cells, int64_t N, const void *f,
                           double *rho)
    {
        k_probe<L, S><<<grid1(n, 128), 128, 0, st>>>(n, cells, N, (const S *)f, rho);
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

static void release(lbm_ctx *h)
{
    if (!h) return;
    for (int k = 0; k < 2; ++k)
        if (h->f[k]) cudaFree(h->f[k]);
    if (h->solid_d) cudaFree(h->solid_d);
    for (int k = 0; k < 6; ++k)
        if (h->prof_d[k]) cudaFree(h->prof_d[k]);
    if (h->red_d) cudaFree(h->red_d);
    delete h;
}

extern "C" int lbm_create(lbm_handle *out, int lattice, const int extents[3], double tau_or_nu,
                          int value_is_nu, double Ma_ref, int precision, void *cuda_stream)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is null");
    *out = nullptr;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19)
        return fail(nullptr, LBM_EINVAL, "unknown lattice %d", lattice);
    if (!prec_bytes(precision)) return fail(nullptr, LBM_EINVAL, "unknown precision %d", precision);
    if (!extents) return fail(nullptr, LBM_EINVAL, "extents is null");
    for (int a = 0; a < 3; ++a)
        if (extents[a] < 1) return fail(nullptr, LBM_EINVAL, "extent %d is %d (< 1)", a, extents[a]);
    if (lattice == LBM_D2Q9 && extents[2] != 1)
        return fail(nullptr, LBM_EINVAL, "D2Q9 needs extents[2] == 1");
    if (extents[1] > 65535 || extents[2] > 65535)
        return fail(nullptr, LBM_EINVAL, "extents[1] and extents[2] must be <= 65535");
    double tau = value_is_nu ? tau_or_nu * 3.0 + 0.5 : tau_or_nu;
    if (!(tau > 0.5) || !std::isfinite(tau))
        return fail(nullptr, LBM_EINVAL, "tau = %g must be > 1/2 (nu > 0)", tau);
    if (!(Ma_ref >= 0.0 && Ma_ref <= 0.6))
        return fail(nullptr, LBM_EINVAL, "Ma_ref = %g outside [0, 0.6]", Ma_ref);

    lbm_ctx *h = new lbm_ctx();
    h->lattice = lattice;
    h->q = lattice == LBM_D2Q9 ? 9 : 19;
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
extern "C" int lbm_set_geometry(lbm_handle h, const uint8_t *cell_type)
{
    CHECK_HANDLE(h);
    if (!cell_type) {
        if (h->solid_d) cudaFree(h->solid_d);
        h->solid_d = nullptr;
        return LBM_OK;
    }
    for (int64_t c = 0; c < h->ncell; ++c)
        if (cell_type[c] > LBM_CELL_FIXED)
            return fail(h, LBM_EINVAL, "cell_type[%lld] = %d is not a cell type", (long long)c, cell_type[c]);
    if (!h->solid_d) CUDA_TRY(h, cudaMalloc(&h->solid_d, (size_t)h->ncell));
    CUDA_TRY(h, cudaMemcpyAsync(h->solid_d, cell_type, (size_t)h->ncell, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
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
    if (face < 0 || face > 5) return fail(h, LBM_EINVAL, "face %d out of range", face);
    if (kind < LBM_BC_PERIODIC || kind > LBM_BC_OUTFLOW) return fail(h, LBM_EINVAL, "unknown boundary kind %d", kind);
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

extern "C" int lbm_set_inlet_noise(lbm_handle h, uint64_t seed, double amplitude)
{
    CHECK_HANDLE(h);
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
    if (face < 0 || face > 5) return fail(h, LBM_EINVAL, "face %d out of range", face);
    if (h->d == 2 && face >= 4 && width != 0) return fail(h, LBM_EINVAL, "2D lattice: no z sponge");
    if (width < 0 || width > h->n[face / 2])
        return fail(h, LBM_EINVAL, "sponge width %d outside [0, %d]", width, h->n[face / 2]);
    if (width == 0) {
        h->sponge_w[face] = 0;
        h->sponge_chi[face] = 0.0;
        return LBM_OK;
    }
    if (!(chi_max >= 0.0) || !(chi_max < 4.0 * h->tau))
        return fail(h, LBM_EINVAL, "chi_max = %g must be in [0, 4 tau = %g) for stability", chi_max, 4.0 * h->tau);
    double ur[3] = {0, 0, 0};
    if (u_ref)
        for (int a = 0; a < 3; ++a) ur[a] = u_ref[a];
    if (h->d == 2 && ur[2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_ref z must be 0");
    if (!(rho_ref > 0.0)) return fail(h, LBM_EINVAL, "rho_ref = %g must be > 0", rho_ref);
    bool other = false;
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
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// State
// ---------------------------------------------------------------------------
extern "C" int lbm_set_state(lbm_handle h, const double *rho, const double *u)
{
    CHECK_HANDLE(h);
    if (!rho || !u) return fail(h, LBM_EINVAL, "rho and u are required");
    const int64_t N = h->ncell;
    for (int64_t c = 0; c < N; ++c) {
        if (!(rho[c] > 0.0) || !std::isfinite(rho[c]))
            return fail(h, LBM_EINVAL, "rho[%lld] = %g must be finite and > 0", (long long)c, rho[c]);
        if (h->d == 2 && u[3 * c + 2] != 0.0) return fail(h, LBM_EINVAL, "2D lattice: u_z must be 0");
    }
    double *buf = nullptr;
    CUDA_TRY(h, cudaMalloc(&buf, sizeof(double) * 4 * (size_t)N));
    cudaError_t e = cudaMemcpyAsync(buf, rho, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf + N, u, sizeof(double) * 3 * (size_t)N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = dispatch<InitEq>(h->lattice, h->prec, h->stream, N, buf, buf + N, h->f[0], h->f[1]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_set_state: %s", cudaGetErrorString(e));
    h->launches += 1;
    h->cur = 0;
    h->step = 0;
    return LBM_OK;
}

extern "C" int lbm_set_populations(lbm_handle h, const double *f)
{
    CHECK_HANDLE(h);
    if (!f) return fail(h, LBM_EINVAL, "f is null");
    const int64_t N = h->ncell;
    double *buf = nullptr;
    CUDA_TRY(h, cudaMalloc(&buf, sizeof(double) * (size_t)N));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->q && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync(buf, f + (size_t)i * N, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = dispatch<SetDir>(h->lattice, h->prec, h->stream, N, i, (const double *)buf, h->f[0], h->f[1]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        h->launches += 1;
    }
    cudaFree(buf);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_set_populations: %s", cudaGetErrorString(e));
    h->cur = 0;
    h->step = 0;
    return LBM_OK;
}

extern "C" int lbm_get_populations(lbm_handle h, double *f)
{
    CHECK_HANDLE(h);
    if (!f) return fail(h, LBM_EINVAL, "f is null");
    const int64_t N = h->ncell;
    double *buf = nullptr;
    CUDA_TRY(h, cudaMalloc(&buf, sizeof(double) * (size_t)N));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->q && e == cudaSuccess; ++i) {
        e = dispatch<GetDir>(h->lattice, h->prec, h->stream, N, i, (const void *)h->f[h->cur], buf);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f + (size_t)i * N, buf, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        h->launches += 1;
    }
    cudaFree(buf);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_get_populations: %s", cudaGetErrorString(e));
    return LBM_OK;
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
        p.face_cells[f] = face_cells(h, f);
        for (int a = 0; a < 3; ++a) p.u_face[f][a] = h->u_face[f][a];
        p.u_profile[f] = h->prof_d[f];
    }
    p.rho_ref = h->rho_ref;
    p.rho_ref_m1 = h->rho_ref - 1.0;
    for (int a = 0; a < 3; ++a) p.u_ref[a] = h->u_ref[a];
    p.noise_seed = h->noise_seed;
    p.noise_amp = h->noise_amp;
    p.omega = 1.0 - 1.0 / h->tau;
    p.solid = h->solid_d;
    return LBM_OK;
}

extern "C" int lbm_step(lbm_handle h, int64_t n)
{
    CHECK_HANDLE(h);
    if (n < 0) return fail(h, LBM_EINVAL, "n = %lld < 0", (long long)n);
    if (n == 0) return LBM_OK;
    StepParams p;
    int rc = build_params(h, p);
    if (rc != LBM_OK) return rc;
    int vec = h->vec == 0 ? vec_default(h->prec) : h->vec;
    if (h->solid_d || vec == 1 || !vec_supported(h->prec, vec) || h->n[0] % vec != 0) vec = 1;
    const int block = h->block > 0 ? h->block : (vec == 1 ? 128 : 128);
    for (int64_t t = 0; t < n; ++t) {
        p.step = h->step;
        cudaError_t e;
        if (vec == 1)
            e = h->lattice == LBM_D2Q9 ? step_d2q9(h->prec, p, h->f[h->cur], h->f[1 - h->cur], block, h->stream)
                                       : step_d3q19(h->prec, p, h->f[h->cur], h->f[1 - h->cur], block, h->stream);
        else
            e = h->lattice == LBM_D2Q9
                    ? stepvec_d2q9(h->prec, vec, p, h->f[h->cur], h->f[1 - h->cur], block, h->stream)
                    : stepvec_d3q19(h->prec, vec, p, h->f[h->cur], h->f[1 - h->cur], block, h->stream);
        if (e != cudaSuccess) return fail(h, LBM_ECUDA, "stream-collide launch: %s", cudaGetErrorString(e));
        h->cur = 1 - h->cur;
        h->step += 1;
        h->launches += 1;
    }
    return LBM_OK;
}

extern "C" int lbm_set_launch(lbm_handle h, int block, int cells_per_thread)
{
    CHECK_HANDLE(h);
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
    int vec = h->vec == 0 ? vec_default(h->prec) : h->vec;
    if (h->solid_d || vec == 1 || !vec_supported(h->prec, vec) || h->n[0] % vec != 0) vec = 1;
    if (block) *block = h->block > 0 ? h->block : 128;
    if (cells_per_thread) *cells_per_thread = vec;
    return LBM_OK;
}

extern "C" int lbm_sync(lbm_handle h)
{
    CHECK_HANDLE(h);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaGetLastError());
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------
extern "C" int lbm_moments(lbm_handle h, double *rho, double *u, double *pi_neq)
{
    CHECK_HANDLE(h);
    if (!rho && !u && !pi_neq) return LBM_OK;
    const int64_t N = h->ncell;
    double *buf = nullptr;
    CUDA_TRY(h, cudaMalloc(&buf, sizeof(double) * 10 * (size_t)N));
    double *rd = buf, *ud = buf + N, *pd = buf + 4 * N;
    cudaError_t e = dispatch<Moments>(h->lattice, h->prec, h->stream, N, (const void *)h->f[h->cur],
                                      rho ? rd : nullptr, u ? ud : nullptr, pi_neq ? pd : nullptr);
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, rd, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u)
        e = cudaMemcpyAsync(u, ud, sizeof(double) * 3 * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && pi_neq)
        e = cudaMemcpyAsync(pi_neq, pd, sizeof(double) * 6 * (size_t)N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_moments: %s", cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" int lbm_reduce(lbm_handle h, double *mass, double momentum[3])
{
    CHECK_HANDLE(h);
    double out[RED_FIELDS];
    cudaError_t e = dispatch<Reduce>(h->lattice, h->prec, h->stream, h->ncell, (const void *)h->f[h->cur],
                                     (const uint8_t *)h->solid_d, h->red_d, h->red_blocks);
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
    if (out[5] > 0.0) return fail(h, LBM_EUNSTABLE, "%.0f cells hold non-finite populations", out[5]);
    return LBM_OK;
}

extern "C" int lbm_probe(lbm_handle h, int n, const int64_t *cells, double *p_prime)
{
    CHECK_HANDLE(h);
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
                            (const void *)h->f[h->cur], rd);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p_prime, rd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(cd);
    h->launches += 1;
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "lbm_probe: %s", cudaGetErrorString(e));
    for (int k = 0; k < n; ++k) p_prime[k] = (p_prime[k] - h->rho_ref) / 3.0;
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
struct FileHeader {
    char magic[8];
    int32_t lattice, prec, n[3], pad;
    int64_t step;
};

extern "C" int lbm_save(lbm_handle h, const char *path)
{
    CHECK_HANDLE(h);
    if (!path) return fail(h, LBM_EINVAL, "path is null");
    const size_t bytes = (size_t)h->q * (size_t)h->ncell * h->elem;
    std::vector<char> host(bytes);
    CUDA_TRY(h, cudaMemcpyAsync(host.data(), h->f[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    FileHeader hd{};
    std::memcpy(hd.magic, "LBMRRv01", 8);
    hd.lattice = h->lattice;
    hd.prec = h->prec;
    for (int a = 0; a < 3; ++a) hd.n[a] = h->n[a];
    hd.step = h->step;
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(h, LBM_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 && std::fwrite(host.data(), 1, bytes, fp) == bytes;
    ok = (std::fclose(fp) == 0) && ok;
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
    if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, "LBMRRv01", 8) != 0) {
        std::fclose(fp);
        return fail(h, LBM_EIO, "%s is not a checkpoint", path);
    }
    if (hd.lattice != h->lattice || hd.prec != h->prec || hd.n[0] != h->n[0] || hd.n[1] != h->n[1] ||
        hd.n[2] != h->n[2]) {
        std::fclose(fp);
        return fail(h, LBM_EINVAL, "checkpoint lattice/precision/extents differ from the handle's");
    }
    const size_t bytes = (size_t)h->q * (size_t)h->ncell * h->elem;
    std::vector<char> host(bytes);
    bool ok = std::fread(host.data(), 1, bytes, fp) == bytes;
    std::fclose(fp);
    if (!ok) return fail(h, LBM_EIO, "short read from %s", path);
    CUDA_TRY(h, cudaMemcpyAsync(h->f[0], host.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->f[1], host.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->step = hd.step;
    return LBM_OK;
}
