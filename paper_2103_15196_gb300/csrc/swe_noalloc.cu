// swe_step_noalloc: one FP32 step on caller-owned device buffers, with all
// the working memory the step needs taken from a fixed array compiled into
// this library instead of from cudaMalloc.
//
// Who needs this: callers that must not allocate device memory once they are
// running.  Examples are real-time loops where cudaMalloc's implicit device
// synchronisation would stall the other streams of the application, and host
// applications whose own memory manager owns all device memory (a pool sized
// at start-up, with nothing left for a library to take).  Such a caller
// passes the input and output state; everything else lives in `g_scratch`
// below.
//
// Limits and sharing rules:
//   * The array holds SWE_NOALLOC_SCRATCH_BYTES (1 MiB), carved into the step
//     bookkeeping (~0.2 KB), two censuses (one int per HGS block each), the
//     skip flags (one byte per block), the block work list (one int per block
//     plus two), the per-row source table (one int per row plus one) and the
//     Manning constants, each region rounded up to 256 bytes.  With the
//     default blocks (248 x 32 cells below 2^22 cells, 248 x 64 below 2^26,
//     248 x 128 above) a 32768 x 32768 grid has 34,048 blocks and needs about
//     0.55 MiB; a grid fits while 13 bytes per block + 4 bytes per row stay
//     below ~1 MiB.  Larger grids are rejected with SWE_EINVAL.
//   * Every GPU that loads the library holds its own copy of the array until
//     the process exits.  All calls on one GPU share it and it keeps the last
//     call's contents; each call first resets the parts that must start from
//     a known value.  Two calls whose work overlaps on the same GPU (for
//     example on two streams) race on the array and give wrong results.
//   * The first call on a device looks the array's address up with
//     cudaGetSymbolAddress while that device is current; make that first
//     call before any stream capture begins.
//   * state_in is modified: the momentum of its dry cells is set to zero in
//     place, as swe_set_state does for the library's own buffers.
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>

#include "../../include/swe.h"
#include "swe_internal.h"
#include "swe_trace.h"

using namespace swe_impl;

#define SWE_NOALLOC_SCRATCH_BYTES (1u << 20)

static __device__ __align__(256) unsigned char g_scratch[SWE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;   // guards the lookups from several host threads

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

float float_floor(double e) {
    float f = (float)e;
    if ((double)f > e) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}

swe_status err(swe_status s, const char *) { return s; }

// Address of this device's copy of g_scratch (looked up once per device).
swe_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(SWE_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return err(SWE_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return err(SWE_ECUDA, "cudaGetSymbolAddress(g_scratch) failed");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SWE_OK;
}

}  // namespace

extern "C" swe_status swe_step_noalloc(const swe_params *pp, double manning_n, void *state_in,
                                       void *state_out, void *cuda_stream, double *dt_taken) {
    const SweRange range_("swe_step_noalloc");
    if (!pp || !state_in || !state_out || state_in == state_out) return err(SWE_EINVAL, "bad pointer argument");
    const swe_params &p = *pp;
    if ((reinterpret_cast<uintptr_t>(state_in) | reinterpret_cast<uintptr_t>(state_out)) & 15u)
        return err(SWE_EINVAL, "state buffers must be 16-byte aligned");
    if (p.precision != SWE_FP32) return err(SWE_EINVAL, "only the FP32 state layout is supported");
    if (p.nx < 1 || p.ny < 1 || (long long)p.nx * p.ny > (1ll << 31) - 1 || !(p.dx > 0) || !(p.g > 0) ||
        !(p.cfl_K > 0 && p.cfl_K < 1) || !(p.eps_wet > 0) || !(p.dt_max > 0) || !(p.psi >= 0 && p.psi < 1) ||
        !(p.A_J >= 0) || !(p.m_exp >= 0) || !(p.C_J >= 0) || !(p.d50 > 0) || !(p.s_rel > 1) ||
        !(p.C_Sh >= 0) || (p.aj_mode != 0 && p.aj_mode != 1) || p.tile_rows < 0 || (p.tile_rows % 8) != 0 ||
        (p.block_cols != 0 && p.block_cols != 128 && p.block_cols != 256) || !(manning_n >= 0) ||
        !std::isfinite(manning_n))
        return err(SWE_EINVAL, "invalid parameters");
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // block shape and constants, chosen as swe_create chooses them
    const long long ncell = (long long)p.nx * p.ny;
    const int bw = p.block_cols ? p.block_cols : (p.nx <= 120 ? 128 : 256);
    const int th = p.tile_rows ? p.tile_rows : (ncell >= (1ll << 26) ? 128 : (ncell >= (1ll << 22) ? 64 : 32));
    SweConst c{};
    c.nx = p.nx; c.ny = p.ny; c.tw = bw - 8; c.th = th;
    c.tiles_x = (p.nx + c.tw - 1) / c.tw;
    c.tiles_y = (p.ny + c.th - 1) / c.th;
    c.man_shift = 30; c.man_w = 1;
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
    c.psi = p.psi; c.K = p.cfl_K; c.dt_max = p.dt_max;
    c.neg_tol = p.neg_tol >= 0 ? p.neg_tol : 1e-4;
    c.eps_f = float_floor(p.eps_wet);
    swe_fill_f32(c);
    swe_set_regions(c);

    // carve the scratch: bookkeeping | census x2 | skip flags | work list | source rows |
    // region census | region flags x2 | Manning tables
    const size_t ntiles = (size_t)c.tiles_x * c.tiles_y;
    const size_t off_dev = 0;
    const size_t off_cen0 = align256(off_dev + sizeof(SweDev));
    const size_t off_cen1 = align256(off_cen0 + ntiles * sizeof(int));
    const size_t off_skip = align256(off_cen1 + ntiles * sizeof(int));
    const size_t off_work = align256(off_skip + ntiles);
    const size_t off_rows = align256(off_work + (ntiles + 2) * sizeof(int));
    const size_t nreg = (size_t)c.regions_x * c.regions_y;
    const size_t off_rc0 = align256(off_rows + ((size_t)p.ny + 1) * sizeof(int));
    const size_t off_rn0 = align256(off_rc0 + nreg * sizeof(int));
    const size_t off_rn1 = align256(off_rn0 + nreg);
    const size_t off_gn2 = align256(off_rn1 + nreg);
    const size_t off_ajn = off_gn2 + 128;
    const size_t total = off_ajn + 128;
    if (total > SWE_NOALLOC_SCRATCH_BYTES) return err(SWE_EINVAL, "grid too large for the fixed 1 MiB scratch");

    unsigned char *base = nullptr;
    swe_status s = scratch_address((void **)&base);
    if (s != SWE_OK) return s;

    SweBufs b{};
    b.buf[0] = state_in;
    b.buf[1] = state_out;
    b.census[0] = (int *)(base + off_cen0);
    b.census[1] = (int *)(base + off_cen1);
    b.skipped = base + off_skip;
    b.work = (int *)(base + off_work);
    b.src_rowptr = (const int *)(base + off_rows);
    b.rcen = (int *)(base + off_rc0);
    b.rneed[0] = base + off_rn0;
    b.rneed[1] = base + off_rn1;
    b.src_x = nullptr;
    b.hyd_t = nullptr; b.hyd_q = nullptr; b.qb = nullptr;
    b.gn2 = base + off_gn2;
    b.ajn = base + off_ajn;
    b.dev = (SweDev *)(base + off_dev);
    b.partials = nullptr;

    // reset what must start from known values: the bookkeeping (state^0 in
    // buf[0], t = 0, no clip), the empty source table and the Manning constants;
    // the census and skip flags are rewritten by the census kernel
    SweDev d0{};
    d0.t_end = INFINITY;
    const float gn2 = (float)((p.g * manning_n) * manning_n);
    const float ajn = (float)(0.05 * manning_n * manning_n * manning_n);
    cudaError_t e = cudaMemcpyAsync(b.dev, &d0, sizeof(SweDev), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + off_rows, 0, ((size_t)p.ny + 1) * sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + off_gn2, &gn2, sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + off_ajn, &ajn, sizeof(float), cudaMemcpyHostToDevice, stream);
    // census + Eq. 7 maxima of the input (dry cells' momentum in state_in is
    // set to zero, as swe_set_state does), dt, the step, and the commit
    if (e == cudaSuccess) e = launch_init<float>(c, b, stream);
    if (e == cudaSuccess) e = launch_between<float>(c, b, 2, stream);
    if (e == cudaSuccess) e = launch_step<float>(c, b, bw, stream);
    if (e == cudaSuccess) e = launch_between<float>(c, b, 1, stream);
    SweDev d1{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&d1, b.dev, sizeof(SweDev), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return err(SWE_ECUDA, cudaGetErrorString(e));
    if (d1.status) return err(SWE_ENUMERIC, "numerical failure (non-finite value or negative depth)");
    if (dt_taken) *dt_taken = d1.dt_last;
    return SWE_OK;
}
