// Batched ensembles of independent flood scenarios (grids of uneven sizes and
// parameters) advanced together by ONE persistent launch per run call,
// captured in a CUDA graph.
//
// Each scenario is an ordinary solver handle (swe_create): its state, Manning
// field, sources and diagnostics are set and read with the usual calls.  The
// persistent kernel schedules (step, block) work items by dataflow, with no
// grid-wide barrier:
//   * the launch's blocks are split into one group per scenario, sized on the
//     host so that the scenarios' steps take about as long (each further block
//     goes to the scenario with the most grid blocks per launch block);
//   * a block draws the (step, block) items of its group's scenario in order
//     from the scenario's counter, step-major, while that scenario's next item
//     belongs to a step already open; otherwise (the scenario's current step
//     is all drawn, or all its steps are) it draws an open item of another
//     scenario, the one with the most items left per block of its group, so
//     that no block idles while any scenario has work it could start;
//   * an item of step n waits (bounded) until its scenario has completed n
//     steps in this launch -- other scenarios never hold it up, since each
//     keeps its own dt (its own K3) and time;
//   * each item runs the same per-block step as the single-grid kernel (K1
//     skip, K2-K8, census and Eq. 7 maxima) and counts itself done; the block
//     that completes the scenario's step commits it and forms the next dt,
//     then publishes the step count.
// An item's scenario is the same for the whole block, so the scenario's
// constants and buffer pointers are read from the launch parameters (the
// scenario table travels in them, about 29 KB for 64 scenarios) at an offset
// that is the same for the whole block: the sweep gets them as it gets the
// single-grid kernel's constants, and fits the register budget of three
// blocks per SM.
// Items are drawn in increasing order within a scenario and an item only
// waits for items of its scenario drawn before it, which running blocks hold,
// so the schedule cannot deadlock.  Every wait polls %globaltimer with a time
// limit; on expiry the kernel sets a status bit, every block returns, the
// host reads SWE_ETIMEOUT, and the context stays usable.
//
// An autotuner (swe_ensemble_autotune) times each candidate block shape on
// the ensemble's own states and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/swe.h"
#include "swe_kernels.cuh"
#include "swe_trace.h"

using namespace swe_impl;

namespace swe_impl {

struct EnsScen {
    SweConst c;
    SweBufs B;
};

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Layout of the launch's synchronisation words (zeroed before every launch):
// [2] status, then per scenario k: ENS_SYNC + 3k its (step, block) counter,
// + 1 the items of its current step completed, + 2 the steps completed in
// this launch.
#define ENS_SYNC 4
#define ENS_WORDS(n) (ENS_SYNC + 3 * (size_t)(n))

// The launch parameters: the scenario table and the block groups (scenario k
// owns blocks pre[k] .. pre[k + 1] - 1).
struct EnsParams {
    EnsScen scen[SWE_ENSEMBLE_MAX];
    int pre[SWE_ENSEMBLE_MAX + 1];
    int n, nsteps;
    unsigned extra;   // completions each scenario step waits for beyond its items (> 0 only in a test)
    unsigned *sync;
    unsigned long long timeout_ns;
};
static_assert(sizeof(EnsParams) <= 32000, "the scenario table must fit the kernel parameters");

// GEN: compile the general transport laws (A_J from Eq. 4, m != 2) in; FLD:
// the rain and infiltration fields; the inflow is always compiled in
// (scenarios carry inflow); 24 warps per SM (three 256-thread or six
// 128-thread blocks).
template <int BW, bool GEN, bool FLD>
__global__ void __launch_bounds__(BW, BW == 128 ? 6 : 3) ensemble_kernel(const __grid_constant__ EnsParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<float, BW> &S = *reinterpret_cast<StepSmem<float, BW> *>(smem_raw);
    __shared__ unsigned s_g;
    __shared__ int s_k, s_stop;
    if ((int)blockIdx.x >= P.pre[P.n]) return;
    int own = 0;   // the block's group
    while (own + 1 < P.n && (int)blockIdx.x >= P.pre[own + 1]) ++own;
    volatile unsigned *vsync = P.sync;
    for (;;) {
        __syncthreads();
        if (threadIdx.x < 32) {
            // Warp 0 draws the block's next item: one of its own scenario
            // while that scenario's next item belongs to a step already open;
            // otherwise an open item of the scenario with the most items left
            // per block of its group (the lanes examine the scenarios together,
            // two each, and agree on the largest key); with no open item
            // anywhere, its own scenario's next item (waited for below), or,
            // once its own items are all drawn, that scenario's.  So blocks do
            // not idle at the end of their scenario's steps, nor once their
            // scenario has finished.
            const int lane = (int)threadIdx.x;
            int kk = -1;
            unsigned gg = 0;
            for (int tries = 0; tries <= P.n && kk < 0 && !(vsync[2] & SWE_STATUS_TIMEOUT); ++tries) {
                const unsigned ntk = (unsigned)(P.scen[own].c.tiles_x * P.scen[own].c.tiles_y);
                const unsigned ck = vsync[ENS_SYNC + 3 * own];
                const bool own_left = ck < ntk * (unsigned)P.nsteps;
                const bool own_open = own_left && vsync[ENS_SYNC + 3 * own + 2] >= ck / ntk;
                int pick = own;
                if (!own_open) {
                    // key: open (bit 63) | valid (bit 62) | items left per group block << 6 | scenario
                    unsigned long long key = 0;
                    for (int j = lane; j < P.n; j += 32) {
                        const unsigned nt = (unsigned)(P.scen[j].c.tiles_x * P.scen[j].c.tiles_y);
                        const unsigned tot = nt * (unsigned)P.nsteps;
                        const unsigned c0 = vsync[ENS_SYNC + 3 * j];
                        if (c0 >= tot) continue;
                        const bool open = vsync[ENS_SYNC + 3 * j + 2] >= c0 / nt;
                        const unsigned long long rem =
                            ((unsigned long long)(tot - c0) << 16) / (unsigned)(P.pre[j + 1] - P.pre[j]);
                        const unsigned long long kj =
                            ((unsigned long long)open << 63) | (1ull << 62) | (rem << 6) | (unsigned long long)j;
                        key = kj > key ? kj : key;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
                        key = y > key ? y : key;
                    }
                    if (key == 0) break;   // every scenario's items are drawn
                    if ((key >> 63) || !own_left) pick = (int)(key & 63ull);
                }
                const unsigned ntp = (unsigned)(P.scen[pick].c.tiles_x * P.scen[pick].c.tiles_y);
                unsigned v = 0;
                if (lane == 0) v = atomicAdd(P.sync + ENS_SYNC + 3 * pick, 1u);
                gg = __shfl_sync(0xffffffffu, v, 0);
                if (gg < ntp * (unsigned)P.nsteps) kk = pick;
            }
            if (lane == 0) {
                s_k = kk;
                s_g = gg;
                s_stop = 0;
            }
        }
        __syncthreads();
        const int k = s_k;   // the item's scenario
        if (k < 0) return;
        const EnsScen &sc = P.scen[k];
        const unsigned ntile = (unsigned)(sc.c.tiles_x * sc.c.tiles_y);
        unsigned *cnt = P.sync + ENS_SYNC + 3 * k;
        const unsigned g = s_g;
        // wait until the scenario has completed the item's step count
        if (threadIdx.x == 0) {
            const unsigned step = g / ntile;
            volatile unsigned *done_steps = vsync + ENS_SYNC + 3 * k + 2;
            if (*done_steps < step) {
                const unsigned long long t0 = global_ns();
                while (*done_steps < step) {
                    if ((vsync[2] & SWE_STATUS_TIMEOUT) || global_ns() - t0 > P.timeout_ns) {
                        atomicOr(P.sync + 2, SWE_STATUS_TIMEOUT);
                        s_stop = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        __syncthreads();
        if (s_stop) return;
        const unsigned tile = g % ntile;
        step_tile<float, BW, true, SWE_SRC_INFLOW | (FLD ? SWE_SRC_FIELDS : 0), GEN>(
            sc.c, sc.B, (int)(tile % (unsigned)sc.c.tiles_x), (int)(tile / (unsigned)sc.c.tiles_x), S);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned step = g / ntile;
            __threadfence();   // this item's state, census and maxima before its count
            if (atomicAdd(cnt + 1, 1u) + 1u == ntile + P.extra) {
                // the scenario's step is complete: commit it, form its next dt
                atomicExch(cnt + 1, 0u);
                __threadfence();
                between_body<float>(sc.c, sc.B, 1);
                __threadfence();
                atomicExch(cnt + 2, step + 1);
            }
        }
    }
}

}  // namespace swe_impl

struct swe_ensemble {
    std::vector<swe_handle *> members;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int bw = 256, th = 64;
    EnsParams P;                 // the launch parameters of the next run (nsteps set per launch)
    unsigned *d_sync = nullptr;  // ENS_WORDS(n) words: status, per-scenario counters
    unsigned long long timeout_ns = 2000000000ull;
    int extra = 0;            // test hook: completions each scenario step waits for beyond its items
    std::map<long long, cudaGraphExec_t> graphs;   // per step count, for the parameters in graph_P
    EnsParams graph_P;        // the parameters (nsteps aside) the cached graphs were captured with
    int max_tiles = 0;        // grid blocks of the largest scenario
    int resident = 0;         // co-resident blocks of the persistent kernel variant resident_key
    int resident_key = -1;
    bool gen = false;        // some scenario uses the general transport laws
    bool fld = false;        // some scenario has a rain or infiltration field
    bool graph_ok = true;    // false if this driver cannot capture the persistent launch
};

namespace {

template <int BW, bool GEN, bool FLD> int resident_blocks() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = sizeof(StepSmem<float, BW>);
    cudaFuncSetAttribute(ensemble_kernel<BW, GEN, FLD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ensemble_kernel<BW, GEN, FLD>, BW, smem);
    return std::max(1, per) * sms;
}

void clear_graphs(swe_ensemble *e) {
    for (auto &g : e->graphs) cudaGraphExecDestroy(g.second);
    e->graphs.clear();
}

int resident_for(const swe_ensemble *e);

// Block groups: every scenario one block, then each further block to the
// scenario with the most grid blocks per launch block (ties: the larger
// scenario), up to the resident blocks or every grid block its own.
void split_blocks(const std::vector<int> &tiles, int resident, int *pre) {
    const int n = (int)tiles.size();
    std::vector<int> b(n, 1);
    int used = n;
    auto load = [&](int k) { return (tiles[k] + b[k] - 1) / b[k]; };
    while (used < resident) {
        int best = -1;
        for (int k = 0; k < n; ++k) {
            if (b[k] >= tiles[k]) continue;
            if (best < 0 || load(k) > load(best) || (load(k) == load(best) && tiles[k] > tiles[best])) best = k;
        }
        if (best < 0) break;
        ++b[best];
        ++used;
    }
    pre[0] = 0;
    for (int k = 0; k < n; ++k) pre[k + 1] = pre[k] + b[k];
}

// Gathers the scenario table and the block groups into the launch
// parameters; the cached graphs are dropped when they change.
swe_status upload(swe_ensemble *e) {
    const int n = (int)e->members.size();
    EnsParams &P = e->P;
    std::memset(&P, 0, sizeof(P));
    std::vector<int> tiles(n);
    bool fld = false;
    for (int k = 0; k < n; ++k) {
        SweConst *c = nullptr;
        SweBufs *b = nullptr;
        bool set = false;
        handle_view(e->members[k], &c, &b, nullptr, nullptr, nullptr, &set);
        if (!set) return SWE_ESTATE;
        if (handle_free_stepping(e->members[k]) != SWE_OK) return SWE_ECUDA;
        P.scen[k].c = *c;
        P.scen[k].B = *b;
        fld = fld || c->has_rain || c->has_beta;
        tiles[k] = c->tiles_x * c->tiles_y;
    }
    e->fld = fld;
    const int key = (e->bw == 128 ? 4 : 0) | (e->gen ? 2 : 0) | (e->fld ? 1 : 0);
    if (key != e->resident_key) {
        e->resident = resident_for(e);
        e->resident_key = key;
    }
    split_blocks(tiles, std::max(e->resident, n), P.pre);
    P.n = n;
    P.extra = (unsigned)e->extra;
    P.sync = e->d_sync;
    P.timeout_ns = e->timeout_ns;
    e->max_tiles = *std::max_element(tiles.begin(), tiles.end());
    if (std::memcmp(&P, &e->graph_P, sizeof(P)) != 0) {
        clear_graphs(e);
        e->graph_P = P;
    }
    return SWE_OK;
}

template <int BW, bool GEN, bool FLD> cudaError_t launch_persistent(swe_ensemble *e, int nsteps) {
    const size_t smem = sizeof(StepSmem<float, BW>);
    cudaError_t err = cudaMemsetAsync(e->d_sync, 0, ENS_WORDS(e->members.size()) * sizeof(unsigned), e->stream);
    if (err != cudaSuccess) return err;
    e->P.nsteps = nsteps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e->P.pre[e->P.n]);
    cfg.blockDim = dim3(BW);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = e->stream;
    cfg.numAttrs = 0;   // no grid barrier: blocks need not be co-resident
    return cudaLaunchKernelEx(&cfg, ensemble_kernel<BW, GEN, FLD>, e->P);
}

int resident_for(const swe_ensemble *e) {
    const int v = (e->bw == 128 ? 4 : 0) | (e->gen ? 2 : 0) | (e->fld ? 1 : 0);
    switch (v) {
    case 0: return resident_blocks<256, false, false>();
    case 1: return resident_blocks<256, false, true>();
    case 2: return resident_blocks<256, true, false>();
    case 3: return resident_blocks<256, true, true>();
    case 4: return resident_blocks<128, false, false>();
    case 5: return resident_blocks<128, false, true>();
    case 6: return resident_blocks<128, true, false>();
    default: return resident_blocks<128, true, true>();
    }
}

cudaError_t launch_any(swe_ensemble *e, int nsteps) {
    const int v = (e->bw == 128 ? 4 : 0) | (e->gen ? 2 : 0) | (e->fld ? 1 : 0);
    switch (v) {
    case 0: return launch_persistent<256, false, false>(e, nsteps);
    case 1: return launch_persistent<256, false, true>(e, nsteps);
    case 2: return launch_persistent<256, true, false>(e, nsteps);
    case 3: return launch_persistent<256, true, true>(e, nsteps);
    case 4: return launch_persistent<128, false, false>(e, nsteps);
    case 5: return launch_persistent<128, false, true>(e, nsteps);
    case 6: return launch_persistent<128, true, false>(e, nsteps);
    default: return launch_persistent<128, true, true>(e, nsteps);
    }
}

// The graph of one persistent launch of `nsteps` steps (cached per count).
swe_status graph_for(swe_ensemble *e, int nsteps, cudaGraphExec_t *out) {
    auto f = e->graphs.find(nsteps);
    if (f != e->graphs.end()) { *out = f->second; return SWE_OK; }
    cudaGraph_t g;
    if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SWE_ECUDA;
    cudaError_t le = launch_any(e, nsteps);
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        cudaGetLastError();
        e->graph_ok = false;   // run the same single persistent launch without a graph
        return SWE_ECUDA;
    }
    cudaGraphExec_t ge;
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return SWE_ECUDA;
    e->graphs[nsteps] = ge;
    *out = ge;
    return SWE_OK;
}

swe_status check(swe_ensemble *e) {
    unsigned st = 0;
    if (cudaMemcpyAsync(&st, e->d_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream) != cudaSuccess ||
        cudaStreamSynchronize(e->stream) != cudaSuccess)
        return SWE_ECUDA;
    if (st & SWE_STATUS_TIMEOUT) {
        // clear the bit so the ensemble can be used again once the cause is fixed
        cudaMemsetAsync(e->d_sync, 0, ENS_WORDS(e->members.size()) * sizeof(unsigned), e->stream);
        cudaStreamSynchronize(e->stream);
        return SWE_ETIMEOUT;
    }
    for (swe_handle *h : e->members) {
        swe_status s = swe_sync(h);
        if (s != SWE_OK) return s;
    }
    return SWE_OK;
}

}  // namespace

extern "C" swe_status swe_ensemble_create(int n, const swe_params *params, void *cuda_stream, swe_ensemble **out) {
    if (n < 1 || n > SWE_ENSEMBLE_MAX || !params || !out) return SWE_EINVAL;
    *out = nullptr;
    for (int k = 0; k < n; ++k)
        if (params[k].precision != SWE_FP32 || params[k].block_cols != params[0].block_cols ||
            params[k].tile_rows != params[0].tile_rows)
            return SWE_EINVAL;
    swe_ensemble *e = new swe_ensemble();
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) { delete e; return SWE_ECUDA; }
        e->own_stream = true;
    }
    e->bw = params[0].block_cols ? params[0].block_cols : 256;
    e->th = params[0].tile_rows ? params[0].tile_rows : 64;
    for (int k = 0; k < n; ++k) {
        swe_params p = params[k];
        if (p.aj_mode == 1 || p.m_exp != 2.0) e->gen = true;
        p.block_cols = e->bw;
        p.tile_rows = e->th;
        swe_handle *h = nullptr;
        swe_status s = swe_create(&p, e->stream, &h);
        if (s != SWE_OK) { swe_ensemble_destroy(e); return s; }
        e->members.push_back(h);
    }
    if (cudaMalloc(&e->d_sync, ENS_WORDS(n) * sizeof(unsigned)) != cudaSuccess ||
        cudaMemsetAsync(e->d_sync, 0, ENS_WORDS(n) * sizeof(unsigned), e->stream) != cudaSuccess) {
        swe_ensemble_destroy(e);
        return SWE_ENOMEM;
    }
    *out = e;
    return SWE_OK;
}

extern "C" swe_status swe_ensemble_destroy(swe_ensemble *e) {
    if (!e) return SWE_OK;
    if (e->stream) cudaStreamSynchronize(e->stream);
    clear_graphs(e);
    for (swe_handle *h : e->members) swe_destroy(h);
    cudaFree(e->d_sync);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
    return SWE_OK;
}

extern "C" swe_status swe_ensemble_member(swe_ensemble *e, int k, swe_handle **member) {
    if (!e || !member || k < 0 || k >= (int)e->members.size()) return SWE_EINVAL;
    *member = e->members[k];
    return SWE_OK;
}

extern "C" swe_status swe_ensemble_run(swe_ensemble *e, int64_t nsteps) {
    const SweRange range_("swe_ensemble_run");
    if (!e || nsteps < 0) return SWE_EINVAL;
    if (nsteps == 0) return SWE_OK;
    swe_status s = upload(e);
    if (s != SWE_OK) return s;
    // one persistent launch per call (split only where steps x blocks of a
    // scenario would overflow its 32-bit work counter)
    const int64_t max_chunk = std::max<int64_t>(1, ((int64_t)1 << 31) / std::max(1, e->max_tiles));
    while (nsteps > 0) {
        const int chunk = (int)std::min<int64_t>(nsteps, max_chunk);
        cudaGraphExec_t g;
        if (e->graph_ok && graph_for(e, chunk, &g) == SWE_OK) {
            if (cudaGraphLaunch(g, e->stream) != cudaSuccess) return SWE_ECUDA;
        } else {
            if (launch_any(e, chunk) != cudaSuccess) return SWE_ECUDA;
        }
        nsteps -= chunk;
    }
    for (swe_handle *h : e->members)
        if (handle_regions_stale(h) != SWE_OK) return SWE_ECUDA;
    return check(e);
}

extern "C" swe_status swe_ensemble_set_timeout(swe_ensemble *e, double seconds, int extra_arrivals) {
    if (!e || !(seconds > 0) || extra_arrivals < 0) return SWE_EINVAL;
    e->timeout_ns = (unsigned long long)(seconds * 1e9);
    e->extra = extra_arrivals;
    clear_graphs(e);
    if (cudaMemsetAsync(e->d_sync, 0, ENS_WORDS(e->members.size()) * sizeof(unsigned), e->stream) != cudaSuccess)
        return SWE_ECUDA;
    return SWE_OK;
}

extern "C" swe_status swe_ensemble_autotune(swe_ensemble *e, int trial_steps, int *block_cols, int *tile_rows) {
    if (!e || trial_steps < 1) return SWE_EINVAL;
    const int n = (int)e->members.size();
    // save every member's state (device copies) and time
    std::vector<std::vector<float>> saved;
    std::vector<double> times(n);
    std::vector<void *> tmp(n, nullptr);
    for (int k = 0; k < n; ++k) {
        SweConst *c;
        bool set;
        handle_view(e->members[k], &c, nullptr, nullptr, nullptr, nullptr, &set);
        if (!set) return SWE_ESTATE;
        const size_t N = (size_t)c->nx * c->ny;
        if (cudaMalloc(&tmp[k], 4 * N * sizeof(float)) != cudaSuccess) {
            for (void *p : tmp) cudaFree(p);
            return SWE_ENOMEM;
        }
        float *f = (float *)tmp[k];
        swe_status s = swe_get_state_ex(e->members[k], f, f + N, f + 2 * N, f + 3 * N, SWE_FP32, SWE_DEVICE);
        if (s == SWE_OK) s = swe_get_time(e->members[k], &times[k]);
        if (s != SWE_OK) { for (void *p : tmp) cudaFree(p); return s; }
    }
    auto restore = [&]() -> swe_status {
        for (int k = 0; k < n; ++k) {
            SweConst *c;
            handle_view(e->members[k], &c, nullptr, nullptr, nullptr, nullptr, nullptr);
            const size_t N = (size_t)c->nx * c->ny;
            const float *f = (const float *)tmp[k];
            swe_status s = swe_set_state_ex(e->members[k], f, f + N, f + 2 * N, f + 3 * N, SWE_FP32, SWE_DEVICE);
            if (s == SWE_OK) s = swe_set_time(e->members[k], times[k]);
            if (s != SWE_OK) return s;
        }
        return SWE_OK;
    };
    const int cand_bw[2] = {128, 256};
    const int cand_th[7] = {16, 32, 64, 96, 128, 192, 256};
    float best = INFINITY;
    int best_bw = e->bw, best_th = e->th;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    swe_status s = SWE_OK;
    for (int bw : cand_bw)
        for (int th : cand_th) {
            e->bw = bw;
            e->th = th;
            for (swe_handle *h : e->members)
                if ((s = (swe_status)handle_retile(h, bw, th)) != SWE_OK) goto done;
            clear_graphs(e);
            if ((s = restore()) != SWE_OK) goto done;
            // one untimed run builds the graph and warms up; then the timed run
            if ((s = swe_ensemble_run(e, 1)) != SWE_OK) goto done;
            if ((s = restore()) != SWE_OK) goto done;
            if ((s = upload(e)) != SWE_OK) goto done;
            {
                cudaGraphExec_t g;
                const bool use_graph = e->graph_ok && graph_for(e, trial_steps, &g) == SWE_OK;
                cudaEventRecord(e0, e->stream);
                if (use_graph) cudaGraphLaunch(g, e->stream);
                else launch_any(e, trial_steps);
                cudaEventRecord(e1, e->stream);
                if ((s = check(e)) != SWE_OK) goto done;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; best_bw = bw; best_th = th; }
            }
        }
    e->bw = best_bw;
    e->th = best_th;
    for (swe_handle *h : e->members)
        if ((s = (swe_status)handle_retile(h, best_bw, best_th)) != SWE_OK) goto done;
    clear_graphs(e);
    s = restore();
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (void *p : tmp) cudaFree(p);
    if (block_cols) *block_cols = e->bw;
    if (tile_rows) *tile_rows = e->th;
    return s;
}
