// C ABI of the CSPH-TVD + Exner solver (declared in include/swe.h).
// Host-side orchestration only: argument checks, device memory, uploads,
// CUDA-graph capture of step sequences, and status read-back.  Every step of
// the method runs in the kernels of swe_kernels.cuh.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "swe_internal.h"
#include "swe_trace.h"

using namespace swe_impl;

namespace swe_impl {
// Fixed-order final reduction of the diagnostics partials (one block).
__global__ void diag_final_kernel(SweBufs B, int nblocks, double *out3) {
    __shared__ double r[3][256];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 256) {
        a += B.partials[3 * i]; b += B.partials[3 * i + 1]; c += B.partials[3 * i + 2];
    }
    r[0][threadIdx.x] = a; r[1][threadIdx.x] = b; r[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 3; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) { out3[0] = r[0][0]; out3[1] = r[1][0]; out3[2] = r[2][0]; }
}

__global__ void set_tend_kernel(SweDev *d, double t_end) {
    d->t_end = t_end;
    d->done = 0;
}
__global__ void set_time_kernel(SweDev *d, double t) { d->t = t; }
}  // namespace swe_impl

struct swe_handle {
    swe_params p{};
    SweConst c{};
    SweBufs b{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int bw = 256;
    size_t cell_bytes = 16;
    bool state_set = false;
    bool tend_active = false;
    SweDev *h_dev = nullptr;      // pinned read-back copy of the device bookkeeping
    double *h_diag = nullptr;     // pinned read-back of the diagnostics sums
    double *d_diag = nullptr;
    int diag_blocks = 0;
    void *allocs[32] = {};
    int nalloc = 0;
    cudaGraphExec_t graph = nullptr;    // the graph in use (one of gcache)
    cudaGraphExec_t gcache[2][2] = {};  // by sediment_on, by launch (dense, sparse)
    int graph_steps = 0;
    int sparse_grid = 0;                // CUDA blocks of a sparse step (about one wave)
    int *h_hint = nullptr;              // pinned: blocks computed by the last step of the last replay
    bool stepped = false;               // a step ran since the state was set (active_last is current)
    std::string err;
};

static swe_status fail(swe_handle *h, swe_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

#define CU(h, call)                                                                               \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail((h), SWE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

static bool is_f32(const swe_handle *h) { return h->p.precision == SWE_FP32; }

static cudaError_t dev_alloc(swe_handle *h, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess && h->nalloc < 32) h->allocs[h->nalloc++] = *p;
    return e;
}

static void dev_free(swe_handle *h, void *p) {
    if (!p) return;
    for (int i = 0; i < h->nalloc; ++i)
        if (h->allocs[i] == p) { h->allocs[i] = h->allocs[--h->nalloc]; break; }
    cudaFree(p);
}

// ---------------------------------------------------------------- launchers

static cudaError_t L_step(swe_handle *h, int grid, bool list) {
    return is_f32(h) ? launch_step<float>(h->c, h->b, h->bw, h->stream, grid, list)
                     : launch_step<double>(h->c, h->b, h->bw, h->stream, grid, list);
}
static cudaError_t L_between_compact(swe_handle *h) {
    return is_f32(h) ? launch_between_compact<float>(h->c, h->b, h->stream)
                     : launch_between_compact<double>(h->c, h->b, h->stream);
}
static cudaError_t L_between(swe_handle *h, int commit) {
    return is_f32(h) ? launch_between<float>(h->c, h->b, commit, h->stream)
                     : launch_between<double>(h->c, h->b, commit, h->stream);
}
static cudaError_t L_init(swe_handle *h) {
    return is_f32(h) ? launch_init<float>(h->c, h->b, h->stream) : launch_init<double>(h->c, h->b, h->stream);
}
static cudaError_t L_bed(swe_handle *h) {
    return is_f32(h) ? launch_bed_source<float>(h->c, h->b, h->stream) : launch_bed_source<double>(h->c, h->b, h->stream);
}
// grid: 0 for a dense step, > 0 for a sparse one (see launch_step)
// One step: (the work list), the step, the bed source, then the commit and
// the next step's work list in one launch.  list = false only for a step that
// directly follows another one on the stream (inside a graph).
static cudaError_t L_one_step(swe_handle *h, int grid = 0, bool list = true) {
    cudaError_t e = L_step(h, grid, list);
    if (e == cudaSuccess && h->c.has_qb) e = L_bed(h);
    if (e == cudaSuccess) e = L_between_compact(h);
    return e;
}

// ---------------------------------------------------------------- create

extern "C" swe_status swe_params_default(swe_params *p, int nx, int ny, double dx) {
    if (!p) return SWE_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->nx = nx; p->ny = ny; p->dx = dx;
    p->g = 9.81; p->cfl_K = 0.4; p->eps_wet = 1e-4; p->dt_max = 1.0; p->psi = 0.4;
    p->sediment_on = 1; p->aj_mode = 0; p->A_J = 0.001; p->m_exp = 2.0; p->C_J = 2.0;
    p->d50 = 5e-4; p->s_rel = 2.65; p->C_Sh = 5.0; p->dt_literal_D = 0;
    p->precision = SWE_FP32; p->hgs_skip = 1; p->tile_rows = 0; p->block_cols = 0;
    p->neg_tol = -1.0;  // resolved per precision at create
    return SWE_OK;
}

static float float_floor_of(double e) {
    float f = (float)e;
    if ((double)f > e) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}

static swe_status upload_manning(swe_handle *h, const std::vector<double> &n, int shift, int w);

extern "C" swe_status swe_create(const swe_params *pp, void *cuda_stream, swe_handle **out) {
    if (!pp || !out) return SWE_EINVAL;
    *out = nullptr;
    const swe_params &p = *pp;
    if (p.nx < 1 || p.ny < 1 || (long long)p.nx * p.ny > (1ll << 31) - 1) return SWE_EINVAL;
    if (!(p.dx > 0) || !(p.g > 0) || !(p.cfl_K > 0 && p.cfl_K < 1) || !(p.eps_wet > 0) || !(p.dt_max > 0) ||
        !(p.psi >= 0 && p.psi < 1) || !(p.A_J >= 0) || !(p.m_exp >= 0) || !(p.C_J >= 0) || !(p.d50 > 0) ||
        !(p.s_rel > 1) || !(p.C_Sh >= 0) || (p.precision != SWE_FP32 && p.precision != SWE_FP64) ||
        (p.aj_mode != 0 && p.aj_mode != 1) || p.tile_rows < 0 || (p.tile_rows % 8) != 0 ||
        (p.block_cols != 0 && p.block_cols != 128 && p.block_cols != 256))
        return SWE_EINVAL;
    for (int q = 0; q < 4; ++q)
        if (p.bc[q] != SWE_BC_WALL && p.bc[q] != SWE_BC_OPEN) return SWE_EINVAL;
    swe_handle *h = new swe_handle();
    h->p = p;
    if (!(h->p.neg_tol >= 0)) h->p.neg_tol = p.precision == SWE_FP32 ? 1e-4 : 1e-10;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return SWE_ECUDA; }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return SWE_ECUDA; }
        h->own_stream = true;
    }
    h->cell_bytes = is_f32(h) ? 16 : 32;
    // block shape: BW threads = columns (BW-8 written), th rows per strip.
    // Default width, measured on GB300 (FP32, half-wet terrain): 128 columns
    // from 2^25 cells (six blocks per SM: 16384^2 59.2 against 58.3 Gcell/s,
    // 8192^2 53.8 against 52.5), 256 below (4096^2 and 2048^2 have fewer
    // 128-column blocks than resident slots), 128 on grids of at most 120
    // columns
    long long ncell = (long long)p.nx * p.ny;
    h->bw = p.block_cols ? p.block_cols : ((p.nx <= 120 || ncell >= (1ll << 25)) ? 128 : 256);
    int th = p.tile_rows;
    // default strip height, measured on GB300 (FP32, half-wet terrain): 256
    // rows from 2^28 cells, 128 from 2^25 (8192^2: 53.8 Gcell/s against 51.9
    // at 256), 64 from 2^22, 32 below
    if (th == 0) th = ncell >= (1ll << 28) ? 256 : (ncell >= (1ll << 25) ? 128 : (ncell >= (1ll << 22) ? 64 : 32));
    SweConst &c = h->c;
    c.nx = p.nx; c.ny = p.ny;
    c.tw = h->bw - 8; c.th = th;
    c.tiles_x = (p.nx + c.tw - 1) / c.tw;
    c.tiles_y = (p.ny + c.th - 1) / c.th;
    c.sediment_on = p.sediment_on ? 1 : 0;
    c.aj_mode = p.aj_mode;
    c.m_is_2 = p.m_exp == 2.0 ? 1 : 0;
    c.hgs = p.hgs_skip ? 1 : 0;
    c.literal_D = p.dt_literal_D ? 1 : 0;
    c.nk = 0; c.has_qb = 0; c.nsrc = 0; c.has_rain = 0; c.has_beta = 0;
    for (int q = 0; q < 4; ++q) c.bc[q] = p.bc[q];
    c.g = p.g; c.dx = p.dx; c.eps = p.eps_wet;
    c.coef = p.g / (2.0 * p.dx);
    c.cjh = (0.5 * p.C_J) / p.dx;
    c.ksh = std::pow(p.C_Sh, 6.0) * (p.d50 * p.d50);
    c.A_J = p.A_J; c.m_exp = p.m_exp; c.sm1 = p.s_rel - 1.0; c.d50 = p.d50; c.C_J = p.C_J;
    c.psi = p.psi; c.K = p.cfl_K; c.dt_max = p.dt_max; c.neg_tol = h->p.neg_tol;
    c.eps_f = float_floor_of(p.eps_wet);
    swe_fill_f32(c);
    swe_set_regions(c);

    SweBufs &b = h->b;
    size_t ntiles = (size_t)c.tiles_x * c.tiles_y;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = dev_alloc(h, &b.buf[q], (size_t)ncell * h->cell_bytes);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = dev_alloc(h, (void **)&b.census[q], ntiles * sizeof(int));
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&b.skipped, ntiles);
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&b.work, (ntiles + 2) * sizeof(int));
    const size_t nreg = (size_t)c.regions_x * c.regions_y;
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&b.rcen, nreg * sizeof(int));
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = dev_alloc(h, (void **)&b.rneed[q], nreg);
    {   // a sparse step launches about one wave of the step kernel (two blocks per SM)
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        h->sparse_grid = 2 * (sms > 0 ? sms : 1);
    }
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&b.dev, sizeof(SweDev));
    h->diag_blocks = (int)std::min<long long>(1024, (ncell + 255) / 256);
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&b.partials, sizeof(double) * 3 * h->diag_blocks);
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&h->d_diag, sizeof(double) * 4);
    int *rowptr = nullptr;
    if (e == cudaSuccess) e = dev_alloc(h, (void **)&rowptr, sizeof(int) * (p.ny + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(rowptr, 0, sizeof(int) * (p.ny + 1), h->stream);
    b.src_rowptr = rowptr;
    b.src_x = nullptr;
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_dev, sizeof(SweDev));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_hint, sizeof(int));
    if (e == cudaSuccess) *h->h_hint = (int)ntiles;
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_diag, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.dev, 0, sizeof(SweDev), h->stream);
    if (e != cudaSuccess) {
        swe_status s = (e == cudaErrorMemoryAllocation) ? SWE_ENOMEM : SWE_ECUDA;
        swe_destroy(h);
        return s;
    }
    std::vector<double> n0(1, 0.03);
    swe_status s = upload_manning(h, n0, 30, 1);
    if (s != SWE_OK) { swe_destroy(h); return s; }
    *out = h;
    return SWE_OK;
}

// Step graphs are captured per coupling mode (Exner on / off) and dropped
// whenever anything they bake in (parameters, buffers, tiling) changes.
static void drop_graphs(swe_handle *h) {
    for (auto &gs : h->gcache)
        for (cudaGraphExec_t &g : gs)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    h->graph = nullptr;
}

extern "C" swe_status swe_destroy(swe_handle *h) {
    if (!h) return SWE_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (int i = 0; i < h->nalloc; ++i) cudaFree(h->allocs[i]);
    if (h->h_dev) cudaFreeHost(h->h_dev);
    if (h->h_hint) cudaFreeHost(h->h_hint);
    if (h->h_diag) cudaFreeHost(h->h_diag);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return SWE_OK;
}

// ---------------------------------------------------------------- inputs

template <typename T>
static std::vector<unsigned char> pack(const std::vector<double> &v) {
    std::vector<unsigned char> out(v.size() * sizeof(T));
    for (size_t i = 0; i < v.size(); ++i) { T x = (T)v[i]; std::memcpy(&out[i * sizeof(T)], &x, sizeof(T)); }
    return out;
}

static swe_status upload_manning(swe_handle *h, const std::vector<double> &n, int shift, int w) {
    std::vector<double> gn2(n.size()), ajn(n.size());
    for (size_t i = 0; i < n.size(); ++i) {
        gn2[i] = (h->p.g * n[i]) * n[i];
        ajn[i] = 0.05 * n[i] * n[i] * n[i];
    }
    std::vector<unsigned char> a = is_f32(h) ? pack<float>(gn2) : pack<double>(gn2);
    std::vector<unsigned char> bb = is_f32(h) ? pack<float>(ajn) : pack<double>(ajn);
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, (void *)h->b.gn2);
    dev_free(h, (void *)h->b.ajn);
    h->b.gn2 = nullptr; h->b.ajn = nullptr;
    void *pa = nullptr, *pb = nullptr;
    CU(h, dev_alloc(h, &pa, a.size()));
    CU(h, dev_alloc(h, &pb, bb.size()));
    CU(h, cudaMemcpy(pa, a.data(), a.size(), cudaMemcpyHostToDevice));
    CU(h, cudaMemcpy(pb, bb.data(), bb.size(), cudaMemcpyHostToDevice));
    h->b.gn2 = pa; h->b.ajn = pb;
    h->c.man_shift = shift; h->c.man_w = w;
    drop_graphs(h);
    return SWE_OK;
}

extern "C" swe_status swe_set_manning(swe_handle *h, const double *n, int block) {
    if (!h || !n || block < 0) return fail(h, SWE_EINVAL, "swe_set_manning: bad argument");
    int shift = 0, w = h->c.nx, rows = h->c.ny;
    if (block > 1) {
        if (block & (block - 1)) return fail(h, SWE_EINVAL, "swe_set_manning: block must be a power of two");
        while ((1 << shift) < block) ++shift;
        w = (h->c.nx + block - 1) / block;
        rows = (h->c.ny + block - 1) / block;
    }
    std::vector<double> v(n, n + (size_t)w * rows);
    for (double x : v)
        if (!(x >= 0) || !std::isfinite(x)) return fail(h, SWE_EINVAL, "swe_set_manning: n must be finite and >= 0");
    return upload_manning(h, v, shift, w);
}

extern "C" swe_status swe_set_sources(swe_handle *h, const uint8_t *mask, const double *t, const double *Q, int nk) {
    if (!h) return SWE_EINVAL;
    if (mask && nk > 0 && (!t || !Q)) return fail(h, SWE_EINVAL, "swe_set_sources: t and Q required");
    for (int k = 1; mask && k < nk; ++k)
        if (!(t[k] > t[k - 1])) return fail(h, SWE_EINVAL, "swe_set_sources: t must be increasing");
    std::vector<int> rowptr(h->c.ny + 1, 0), xs;
    if (mask && nk > 0) {
        for (int y = 0; y < h->c.ny; ++y) {
            for (int x = 0; x < h->c.nx; ++x)
                if (mask[(size_t)y * h->c.nx + x]) xs.push_back(x);
            rowptr[y + 1] = (int)xs.size();
        }
    }
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, (void *)h->b.src_x);
    dev_free(h, (void *)h->b.hyd_t);
    dev_free(h, (void *)h->b.hyd_q);
    h->b.src_x = nullptr; h->b.hyd_t = nullptr; h->b.hyd_q = nullptr;
    void *px = nullptr, *pt = nullptr, *pq = nullptr;
    CU(h, dev_alloc(h, &px, sizeof(int) * std::max<size_t>(1, xs.size())));
    if (!xs.empty()) CU(h, cudaMemcpy(px, xs.data(), sizeof(int) * xs.size(), cudaMemcpyHostToDevice));
    CU(h, cudaMemcpy((void *)h->b.src_rowptr, rowptr.data(), sizeof(int) * rowptr.size(), cudaMemcpyHostToDevice));
    int nkk = (mask && nk > 0 && !xs.empty()) ? nk : 0;
    CU(h, dev_alloc(h, &pt, sizeof(double) * std::max(1, nkk)));
    CU(h, dev_alloc(h, &pq, sizeof(double) * std::max(1, nkk)));
    if (nkk) {
        CU(h, cudaMemcpy(pt, t, sizeof(double) * nkk, cudaMemcpyHostToDevice));
        CU(h, cudaMemcpy(pq, Q, sizeof(double) * nkk, cudaMemcpyHostToDevice));
    }
    h->b.src_x = (const int *)px; h->b.hyd_t = (const double *)pt; h->b.hyd_q = (const double *)pq;
    h->c.nk = nkk;
    h->c.nsrc = nkk ? (int)xs.size() : 0;
    drop_graphs(h);
    h->state_set = false;  // census and dt depend on the sources: set the state again
    return SWE_OK;
}

extern "C" swe_status swe_set_bed_source(swe_handle *h, const double *q) {
    if (!h) return SWE_EINVAL;
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, (void *)h->b.qb);
    h->b.qb = nullptr;
    h->c.has_qb = 0;
    if (q) {
        size_t N = (size_t)h->c.nx * h->c.ny;
        std::vector<double> v(q, q + N);
        std::vector<unsigned char> a = is_f32(h) ? pack<float>(v) : pack<double>(v);
        void *p = nullptr;
        CU(h, dev_alloc(h, &p, a.size()));
        CU(h, cudaMemcpy(p, a.data(), a.size(), cudaMemcpyHostToDevice));
        h->b.qb = p;
        h->c.has_qb = 1;
    }
    // a bed source or rain changes dry blocks too: no skipping while either is set
    h->c.hgs = (h->p.hgs_skip && !h->c.has_qb && !h->c.has_rain) ? 1 : 0;
    drop_graphs(h);
    return SWE_OK;
}

extern "C" swe_status swe_set_infiltration(swe_handle *h, const double *beta) {
    if (!h) return SWE_EINVAL;
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, (void *)h->b.beta);
    h->b.beta = nullptr;
    h->c.has_beta = 0;
    if (beta) {
        size_t N = (size_t)h->c.nx * h->c.ny;
        std::vector<double> v(beta, beta + N);
        for (double x : v)
            if (!(x >= 0.0) || !std::isfinite(x)) return fail(h, SWE_EINVAL, "swe_set_infiltration: rate must be >= 0");
        std::vector<unsigned char> a = is_f32(h) ? pack<float>(v) : pack<double>(v);
        void *p = nullptr;
        CU(h, dev_alloc(h, &p, a.size()));
        CU(h, cudaMemcpy(p, a.data(), a.size(), cudaMemcpyHostToDevice));
        h->b.beta = p;
        h->c.has_beta = 1;
    }
    drop_graphs(h);
    return SWE_OK;
}

extern "C" swe_status swe_set_rain(swe_handle *h, const double *sigma) {
    if (!h) return SWE_EINVAL;
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, (void *)h->b.rain);
    h->b.rain = nullptr;
    h->c.has_rain = 0;
    if (sigma) {
        size_t N = (size_t)h->c.nx * h->c.ny;
        std::vector<double> v(sigma, sigma + N);
        for (double x : v)
            if (!std::isfinite(x)) return fail(h, SWE_EINVAL, "swe_set_rain: non-finite source");
        std::vector<unsigned char> a = is_f32(h) ? pack<float>(v) : pack<double>(v);
        void *p = nullptr;
        CU(h, dev_alloc(h, &p, a.size()));
        CU(h, cudaMemcpy(p, a.data(), a.size(), cudaMemcpyHostToDevice));
        h->b.rain = p;
        h->c.has_rain = 1;
    }
    h->c.hgs = (h->p.hgs_skip && !h->c.has_qb && !h->c.has_rain) ? 1 : 0;
    drop_graphs(h);
    return SWE_OK;
}

// ---------------------------------------------------------------- state

static swe_status read_dev(swe_handle *h) {
    CU(h, cudaMemcpyAsync(h->h_dev, h->b.dev, sizeof(SweDev), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (h->stepped && h->h_hint) *h->h_hint = h->h_dev->active_last;   // the launch hint, exact here
    return SWE_OK;
}

static swe_status check_status(swe_handle *h) {
    if (h->h_dev->status) {
        char msg[128];
        const unsigned s = h->h_dev->status;
        std::snprintf(msg, sizeof msg, "step failure (status 0x%x): %s", s,
                      (s & 8u) ? "an index outside its buffer (checked build)"
                               : ((s & 1u) ? "non-finite value" : "depth below -neg_tol"));
        return fail(h, SWE_ENUMERIC, msg);
    }
    return SWE_OK;
}

extern "C" swe_status swe_set_state_ex(swe_handle *h, const void *H, const void *Hu, const void *Hv, const void *bb,
                                       int dtype, int where) {
    const SweRange range_("swe_set_state");
    if (!h || !H || !Hu || !Hv || !bb || (dtype != SWE_FP64 && dtype != SWE_FP32) ||
        (where != SWE_HOST && where != SWE_DEVICE))
        return fail(h, SWE_EINVAL, "swe_set_state: bad argument");
    const size_t N = (size_t)h->c.nx * h->c.ny;
    const size_t es = dtype == SWE_FP64 ? 8 : 4;
    CU(h, cudaSetDevice(h->device));
    const void *src[4] = {H, Hu, Hv, bb};
    void *stage = nullptr;
    if (where == SWE_HOST) {
        CU(h, cudaMallocAsync(&stage, 4 * N * es, h->stream));
        for (int q = 0; q < 4; ++q) {
            cudaError_t e = cudaMemcpyAsync((char *)stage + q * N * es, src[q], N * es, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) { cudaFreeAsync(stage, h->stream); return fail(h, SWE_ECUDA, cudaGetErrorString(e)); }
            src[q] = (char *)stage + q * N * es;
        }
    }
    // the state is placed in buf[0] and the bookkeeping restarts at n = 0, t = 0
    SweDev init{};
    init.t_end = INFINITY;
    CU(h, cudaMemcpyAsync(h->b.dev, &init, sizeof(SweDev), cudaMemcpyHostToDevice, h->stream));
    cudaError_t e = is_f32(h) ? launch_convert_in<float>(h->c, h->b.buf[0], src[0], src[1], src[2], src[3], dtype == SWE_FP64, h->stream)
                              : launch_convert_in<double>(h->c, h->b.buf[0], src[0], src[1], src[2], src[3], dtype == SWE_FP64, h->stream);
    if (stage) cudaFreeAsync(stage, h->stream);
    if (e != cudaSuccess) return fail(h, SWE_ECUDA, cudaGetErrorString(e));
    CU(h, L_init(h));
    CU(h, L_between(h, 2));
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    h->state_set = true;
    h->stepped = false;
    *h->h_hint = h->c.tiles_x * h->c.tiles_y;   // unknown activity: dense launches until a step tells
    h->tend_active = false;
    return check_status(h);
}

extern "C" swe_status swe_set_state(swe_handle *h, const double *H, const double *Hu, const double *Hv, const double *b) {
    return swe_set_state_ex(h, H, Hu, Hv, b, SWE_FP64, SWE_HOST);
}

extern "C" swe_status swe_get_state_ex(swe_handle *h, void *H, void *Hu, void *Hv, void *bb, int dtype, int where) {
    const SweRange range_("swe_get_state");
    if (!h || (dtype != SWE_FP64 && dtype != SWE_FP32) || (where != SWE_HOST && where != SWE_DEVICE))
        return fail(h, SWE_EINVAL, "swe_get_state: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_get_state before swe_set_state");
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    const size_t N = (size_t)h->c.nx * h->c.ny;
    const size_t es = dtype == SWE_FP64 ? 8 : 4;
    const void *cur = h->b.buf[h->h_dev->n & 1];
    void *dst[4] = {H, Hu, Hv, bb};
    void *stage = nullptr;
    if (where == SWE_HOST) {
        CU(h, cudaMallocAsync(&stage, 4 * N * es, h->stream));
        for (int q = 0; q < 4; ++q) dst[q] = dst[q] ? (char *)stage + q * N * es : nullptr;
    }
    cudaError_t e = is_f32(h) ? launch_convert_out<float>(h->c, cur, dst[0], dst[1], dst[2], dst[3], dtype == SWE_FP64, h->stream)
                              : launch_convert_out<double>(h->c, cur, dst[0], dst[1], dst[2], dst[3], dtype == SWE_FP64, h->stream);
    if (e == cudaSuccess && where == SWE_HOST) {
        void *outs[4] = {H, Hu, Hv, bb};
        for (int q = 0; q < 4 && e == cudaSuccess; ++q)
            if (outs[q]) e = cudaMemcpyAsync(outs[q], dst[q], N * es, cudaMemcpyDeviceToHost, h->stream);
    }
    if (stage) cudaFreeAsync(stage, h->stream);
    if (e != cudaSuccess) return fail(h, SWE_ECUDA, cudaGetErrorString(e));
    CU(h, cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

extern "C" swe_status swe_get_state(swe_handle *h, double *H, double *Hu, double *Hv, double *b) {
    return swe_get_state_ex(h, H, Hu, Hv, b, SWE_FP64, SWE_HOST);
}

// ---------------------------------------------------------------- stepping

// Re-prepares the next dt for free stepping (no t_end clip) if an advance
// left a clipped one behind.
static swe_status free_stepping(swe_handle *h) {
    if (!h->tend_active) return SWE_OK;
    set_tend_kernel<<<1, 1, 0, h->stream>>>(h->b.dev, INFINITY);
    CU(h, cudaGetLastError());
    CU(h, L_between(h, 0));
    h->tend_active = false;
    return SWE_OK;
}

// Launch of the next steps: sparse (a wave of CUDA blocks walking the block
// list) while the blocks computed by the last known step fit in it, dense
// (one CUDA block per grid block) otherwise.  Results are the same either
// way; only the launch differs.
static int step_grid(const swe_handle *h, int active) {
    return (h->c.hgs && active >= 0 && active <= h->sparse_grid) ? h->sparse_grid : 0;
}

// The step graph of the current coupling and launch kind; each replay ends by
// copying the blocks computed by its last step into the pinned hint.
static swe_status ensure_graph(swe_handle *h, bool sparse) {
    cudaGraphExec_t &slot = h->gcache[h->c.sediment_on ? 1 : 0][sparse ? 1 : 0];
    h->graph = slot;
    if (h->graph) return SWE_OK;
    long long ncell = (long long)h->c.nx * h->c.ny;
    int m = ncell >= (1ll << 24) ? 8 : (ncell >= (1ll << 20) ? 32 : 128);
    cudaGraph_t g;
    CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < m && e == cudaSuccess; ++i) e = L_one_step(h, sparse ? h->sparse_grid : 0, i == 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_hint, &h->b.dev->active_last, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(h, SWE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(h, SWE_ECUDA, std::string("capture end: ") + cudaGetErrorString(e2));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->graph = nullptr; return fail(h, SWE_ECUDA, cudaGetErrorString(e)); }
    slot = h->graph;
    h->graph_steps = m;
    return SWE_OK;
}

extern "C" swe_status swe_step(swe_handle *h, double *dt_taken) {
    const SweRange range_("swe_step");
    if (!h) return SWE_EINVAL;
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_step before swe_set_state");
    swe_status s = free_stepping(h);
    if (s != SWE_OK) return s;
    CU(h, L_one_step(h, step_grid(h, *h->h_hint)));
    h->stepped = true;
    s = read_dev(h);
    if (s != SWE_OK) return s;
    if (dt_taken) *dt_taken = h->h_dev->dt_last;
    return check_status(h);
}

extern "C" swe_status swe_run_steps(swe_handle *h, int64_t nsteps) {
    const SweRange range_("swe_run_steps");
    if (!h || nsteps < 0) return fail(h, SWE_EINVAL, "swe_run_steps: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_run_steps before swe_set_state");
    swe_status s = free_stepping(h);
    if (s != SWE_OK) return s;
    // the hint is what the last replay left in pinned memory (possibly an older
    // replay's if the last one is still running), or the last step's count
    // read back: it only picks the launch, per replay
    int64_t left = nsteps;
    for (;;) {
        const int grid = step_grid(h, *h->h_hint);
        s = ensure_graph(h, grid > 0);
        if (s != SWE_OK) return s;
        if (left < h->graph_steps) {
            for (; left > 0; --left) CU(h, L_one_step(h, grid));
            break;
        }
        CU(h, cudaGraphLaunch(h->graph, h->stream));
        h->stepped = true;
        left -= h->graph_steps;
    }
    if (nsteps > 0) h->stepped = true;
    return SWE_OK;
}

extern "C" swe_status swe_advance(swe_handle *h, double t_end, int64_t *steps_taken) {
    const SweRange range_("swe_advance");
    if (!h || !std::isfinite(t_end)) return fail(h, SWE_EINVAL, "swe_advance: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_advance before swe_set_state");
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    const long long n0 = h->h_dev->n;
    set_tend_kernel<<<1, 1, 0, h->stream>>>(h->b.dev, t_end);
    CU(h, cudaGetLastError());
    CU(h, L_between(h, 0));
    h->tend_active = true;
    for (;;) {
        s = read_dev(h);
        if (s != SWE_OK) return s;
        if (h->h_dev->status) break;
        if (h->h_dev->done || !h->h_dev->scheduled) break;
        s = ensure_graph(h, step_grid(h, *h->h_hint) > 0);
        if (s != SWE_OK) return s;
        CU(h, cudaGraphLaunch(h->graph, h->stream));
        h->stepped = true;
    }
    if (steps_taken) *steps_taken = h->h_dev->n - n0;
    return check_status(h);
}

extern "C" swe_status swe_sync(swe_handle *h) {
    if (!h) return SWE_EINVAL;
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    return check_status(h);
}

extern "C" swe_status swe_get_time(swe_handle *h, double *t) {
    if (!h || !t) return fail(h, SWE_EINVAL, "swe_get_time: bad argument");
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    *t = h->h_dev->t;
    return SWE_OK;
}

extern "C" swe_status swe_set_time(swe_handle *h, double t) {
    if (!h || !std::isfinite(t)) return fail(h, SWE_EINVAL, "swe_set_time: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_set_time before swe_set_state");
    set_time_kernel<<<1, 1, 0, h->stream>>>(h->b.dev, t);
    CU(h, cudaGetLastError());
    CU(h, L_between(h, 0));  // the source increment depends on t
    return read_dev(h);
}

extern "C" swe_status swe_set_sediment(swe_handle *h, int on) {
    if (!h) return SWE_EINVAL;
    h->c.sediment_on = on ? 1 : 0;
    h->p.sediment_on = h->c.sediment_on;
    h->graph = nullptr;   // ensure_graph picks the cached graph of this coupling
    if (!h->state_set) return SWE_OK;
    // the Eq. 7 maxima depend on the coupling: gather them again for the current state
    CU(h, L_init(h));
    CU(h, L_between(h, 2));
    return read_dev(h);
}

extern "C" swe_status swe_get_diag(swe_handle *h, swe_diag *out) {
    if (!h || !out) return fail(h, SWE_EINVAL, "swe_get_diag: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_get_diag before swe_set_state");
    cudaError_t e = is_f32(h) ? launch_diag<float>(h->c, h->b, h->diag_blocks, h->stream)
                              : launch_diag<double>(h->c, h->b, h->diag_blocks, h->stream);
    if (e != cudaSuccess) return fail(h, SWE_ECUDA, cudaGetErrorString(e));
    diag_final_kernel<<<1, 256, 0, h->stream>>>(h->b, h->diag_blocks, h->d_diag);
    CU(h, cudaGetLastError());
    CU(h, cudaMemcpyAsync(h->h_diag, h->d_diag, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream));
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    const SweDev &d = *h->h_dev;
    const double a = h->c.dx * h->c.dx;
    out->t = d.t;
    out->dt_last = d.dt_last;
    out->dt_next = d.dt_unclipped;
    out->binding = d.binding_last;
    out->water_volume = h->h_diag[0] * a;
    out->sediment_volume = h->h_diag[1] * a;
    out->inflow_volume = d.inflow_total;
    out->steps = d.n;
    out->wet_cells = (int64_t)h->h_diag[2];
    out->active_tiles = d.active_last;
    out->total_tiles = h->c.tiles_x * h->c.tiles_y;
    out->tile_x = h->c.tw;
    out->tile_y = h->c.th;
    out->status = d.status;
    out->cells_computed = d.cells_computed;
    out->cells_copied = d.cells_copied;
    return SWE_OK;
}

extern "C" swe_status swe_get_census(swe_handle *h, int32_t *out, int *tiles_x, int *tiles_y) {
    if (!h) return SWE_EINVAL;
    if (tiles_x) *tiles_x = h->c.tiles_x;
    if (tiles_y) *tiles_y = h->c.tiles_y;
    if (!out) return SWE_OK;
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_get_census before swe_set_state");
    swe_status s = read_dev(h);
    if (s != SWE_OK) return s;
    CU(h, cudaMemcpyAsync(out, h->b.census[h->h_dev->n & 1], sizeof(int) * h->c.tiles_x * h->c.tiles_y,
                          cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

extern "C" const char *swe_last_error(const swe_handle *h) { return h ? h->err.c_str() : "null handle"; }

// ---------------------------------------------------------------- internal hooks

namespace swe_impl {
bool handle_view(swe_handle *h, SweConst **c, SweBufs **b, cudaStream_t *s, int *bw, int *precision, bool *state_set) {
    if (!h) return false;
    if (c) *c = &h->c;
    if (b) *b = &h->b;
    if (s) *s = h->stream;
    if (bw) *bw = h->bw;
    if (precision) *precision = h->p.precision;
    if (state_set) *state_set = h->state_set;
    return true;
}

int handle_free_stepping(swe_handle *h) { return (int)free_stepping(h); }

void *handle_current_state(swe_handle *h) {
    if (!h || !h->state_set || read_dev(h) != SWE_OK) return nullptr;
    return h->b.buf[h->h_dev->n & 1];
}

int handle_state_changed(swe_handle *h) {
    if (!h) return SWE_EINVAL;
    const size_t nt = (size_t)h->c.tiles_x * h->c.tiles_y;
    // every block's buffers may differ, and the region census is stale (the
    // next compaction rebuilds it: rescan's low byte set, the others are 0)
    if (cudaMemsetAsync(h->b.skipped, 0, nt, h->stream) != cudaSuccess ||
        cudaMemsetAsync(&h->b.dev->rescan, 1, 1, h->stream) != cudaSuccess)
        return SWE_ECUDA;
    *h->h_hint = (int)nt;
    h->stepped = false;
    return SWE_OK;
}

int handle_regions_stale(swe_handle *h) {
    if (!h) return SWE_EINVAL;
    return cudaMemsetAsync(&h->b.dev->rescan, 1, 1, h->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

int handle_retile(swe_handle *h, int bw, int th) {
    if (!h || (bw != 128 && bw != 256) || th < 8 || (th % 8) != 0) return SWE_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SWE_ECUDA;
    SweConst &c = h->c;
    const int tw = bw - 8;
    const int tx = (c.nx + tw - 1) / tw, ty = (c.ny + th - 1) / th;
    const size_t nt = (size_t)tx * ty;
    const size_t nreg = (size_t)((tx + SWE_REGION - 1) / SWE_REGION) * ((ty + SWE_REGION - 1) / SWE_REGION);
    void *cen0 = nullptr, *cen1 = nullptr, *skp = nullptr, *wrk = nullptr;
    void *rc0 = nullptr, *rn0 = nullptr, *rn1 = nullptr;
    if (dev_alloc(h, &cen0, nt * sizeof(int)) != cudaSuccess || dev_alloc(h, &cen1, nt * sizeof(int)) != cudaSuccess ||
        dev_alloc(h, &skp, nt) != cudaSuccess || dev_alloc(h, &wrk, (nt + 2) * sizeof(int)) != cudaSuccess ||
        dev_alloc(h, &rc0, nreg * sizeof(int)) != cudaSuccess ||
        dev_alloc(h, &rn0, nreg) != cudaSuccess || dev_alloc(h, &rn1, nreg) != cudaSuccess) {
        dev_free(h, cen0); dev_free(h, cen1); dev_free(h, skp); dev_free(h, wrk);
        dev_free(h, rc0); dev_free(h, rn0); dev_free(h, rn1);
        return SWE_ENOMEM;
    }
    dev_free(h, h->b.census[0]); dev_free(h, h->b.census[1]); dev_free(h, h->b.skipped); dev_free(h, h->b.work);
    dev_free(h, h->b.rcen); dev_free(h, h->b.rneed[0]); dev_free(h, h->b.rneed[1]);
    h->b.census[0] = (int *)cen0; h->b.census[1] = (int *)cen1; h->b.skipped = (unsigned char *)skp;
    h->b.work = (int *)wrk;
    h->b.rcen = (int *)rc0;
    h->b.rneed[0] = (unsigned char *)rn0; h->b.rneed[1] = (unsigned char *)rn1;
    h->bw = bw;
    c.tw = tw; c.th = th; c.tiles_x = tx; c.tiles_y = ty;
    swe_set_regions(c);
    *h->h_hint = (int)nt;
    h->stepped = false;
    drop_graphs(h);
    if (!h->state_set) return SWE_OK;
    // census of the current state (its buffer is buf[n & 1]); the maxima the
    // census kernel gathers are those of the same state, so dt is unchanged
    if (read_dev(h) != SWE_OK) return SWE_ECUDA;
    if (L_init(h) != cudaSuccess) return SWE_ECUDA;
    // the init kernel restarted the accumulation: re-take the maxima
    if (L_between(h, 2) != cudaSuccess) return SWE_ECUDA;
    return (int)read_dev(h);
}
}  // namespace swe_impl

extern "C" swe_status swe_autotune(swe_handle *h, int trial_steps, int *block_cols, int *tile_rows) {
    const SweRange range_("swe_autotune");
    if (!h || trial_steps < 1) return fail(h, SWE_EINVAL, "swe_autotune: bad argument");
    if (!h->state_set) return fail(h, SWE_ESTATE, "swe_autotune before swe_set_state");
    const bool f32 = is_f32(h);
    const size_t N = (size_t)h->c.nx * h->c.ny, es = f32 ? 4 : 8;
    const int dt = f32 ? SWE_FP32 : SWE_FP64;
    void *copy = nullptr;
    if (dev_alloc(h, &copy, 4 * N * es) != cudaSuccess) return fail(h, SWE_ENOMEM, "swe_autotune: state copy");
    char *q = (char *)copy;
    double t0 = 0;
    swe_status s = swe_get_state_ex(h, q, q + N * es, q + 2 * N * es, q + 3 * N * es, dt, SWE_DEVICE);
    if (s == SWE_OK) s = swe_get_time(h, &t0);
    auto restore = [&]() -> swe_status {
        swe_status r = swe_set_state_ex(h, q, q + N * es, q + 2 * N * es, q + 3 * N * es, dt, SWE_DEVICE);
        return r == SWE_OK ? swe_set_time(h, t0) : r;
    };
    const int bw0 = h->bw, th0 = h->c.th;
    int best_bw = bw0, best_th = th0;
    float best = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == SWE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) s = SWE_ECUDA;
    const int cand_th[8] = {16, 32, 64, 96, 128, 160, 192, 256};
    for (int bw : {128, 256}) {
        if (s != SWE_OK) break;
        if (bw == 256 && h->c.nx <= 120) continue;
        for (int th : cand_th) {
            if (th > 16 && th >= h->c.ny + 8) break;   // one strip already covers the grid
            if ((s = (swe_status)swe_impl::handle_retile(h, bw, th)) != SWE_OK || (s = restore()) != SWE_OK ||
                (s = swe_run_steps(h, 1)) != SWE_OK || (s = restore()) != SWE_OK || (s = swe_run_steps(h, 1)) != SWE_OK)
                break;   // untimed: builds the step graph and warms up
            cudaEventRecord(e0, h->stream);
            if ((s = swe_run_steps(h, trial_steps)) != SWE_OK) break;
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { s = SWE_ECUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if ((s = swe_sync(h)) != SWE_OK) break;
            if (ms < best) { best = ms; best_bw = bw; best_th = th; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // the chosen shape (the original one if a trial failed), the saved state and time
    const swe_status rt = (swe_status)swe_impl::handle_retile(h, s == SWE_OK ? best_bw : bw0, s == SWE_OK ? best_th : th0);
    const swe_status rs = restore();
    dev_free(h, copy);
    if (s == SWE_OK) s = rt != SWE_OK ? rt : rs;
    if (s != SWE_OK) return fail(h, s, "swe_autotune failed");
    if (block_cols) *block_cols = h->bw;
    if (tile_rows) *tile_rows = h->c.th;
    return SWE_OK;
}

