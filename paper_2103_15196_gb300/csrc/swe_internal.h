// Internal declarations shared by the C-ABI host code and the kernel
// translation units (one per precision).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// Step bookkeeping that lives in device memory so a whole sequence of steps
// can be queued (or captured in a CUDA graph) without host round trips.
// Written by the one-thread `between` kernel, read by the step kernel.
struct SweDev {
    double t;             // time of the current state
    double dt;            // dt of the step scheduled next (0: none)
    double dt_unclipped;  // Eq. 7 value before the t_end clip
    double t_end;         // clip target of swe_advance (+inf when stepping freely)
    double dHs;           // depth added to each source cell by the scheduled step
    double inflow_total;  // FP64 total inflow volume since set_state
    double dt_last;       // dt of the last committed step
    double dtdx, hdt, c4, cb;  // dt/h, dt/2, dt/(4h), dt/(h(1-psi)) of the scheduled step
    long long n;          // index of the current state: state^n lives in buf[n & 1]
    int scheduled;        // a step with dt > 0 is prepared
    int done;             // t reached t_end
    int binding;          // Eq. 7 term behind dt
    int binding_last;
    unsigned status;      // 1: non-finite value, 2: depth below -neg_tol
    int active_tiles;     // blocks computed by the running step
    int active_last;      // blocks computed by the last committed step
    unsigned long long cells_computed;  // cells in blocks computed, summed over steps
    unsigned long long cells_copied;    // cells in blocks copied (skipped, buffers differed)
    unsigned long long acc[3];  // running maxima (bit patterns) of |v|, |v|+sqrt(gH), |J0|
    double vp, vs, jm;    // maxima of the current state, kept by `between`
    int rescan;           // 1: the region census is stale; the next compaction rebuilds it and scans every block
};

// Model constants (plain data, passed by value).
struct SweConst {
    int nx, ny;
    int tw, th;             // HGS block: tw columns x th rows
    int tiles_x, tiles_y;
    int regions_x, regions_y;  // HGS regions of SWE_REGION x SWE_REGION blocks
    int man_shift, man_w;   // Manning table: index (y >> shift) * man_w + (x >> shift)
    int sediment_on, aj_mode, m_is_2, hgs, literal_D, nk, has_qb;
    int nsrc;               // number of source cells
    int bc[4];              // W, E, S, N boundaries: 0 wall (mirror), 1 open (repeat the boundary cell)
    int has_rain;           // per-cell water source present
    int has_beta;           // per-cell infiltration rate present
    double g, dx, eps, coef, cjh, ksh, A_J, m_exp, sm1, d50, C_J, psi, K, dt_max, neg_tol;
    float eps_f;            // largest float <= eps: (float)H > eps_f <=> (double)H > eps
    // the same, rounded to FP32; inv_dx = 1/h, inv_4dx = 1/(4h), inv_dxp = 1/(h (1-psi)): the step
    // coefficients of the FP32 kernels are dt times these (ptxas can re-form them from dt)
    struct { float g, eps, coef, cjh, ksh, A_J, m_exp, sm1, d50, neg_tol, inv_dx, inv_4dx, inv_dxp; } f;
};

// Fills the FP32 copies of the model constants.
inline void swe_fill_f32(SweConst &c) {
    c.f.g = (float)c.g; c.f.eps = (float)c.eps; c.f.coef = (float)c.coef; c.f.cjh = (float)c.cjh;
    c.f.ksh = (float)c.ksh; c.f.A_J = (float)c.A_J; c.f.m_exp = (float)c.m_exp; c.f.sm1 = (float)c.sm1;
    c.f.d50 = (float)c.d50; c.f.neg_tol = (float)c.neg_tol;
    c.f.inv_dx = (float)(1.0 / c.dx); c.f.inv_4dx = (float)(1.0 / (4.0 * c.dx));
    c.f.inv_dxp = (float)(1.0 / (c.dx * (1.0 - c.psi)));
}

// HGS region: SWE_REGION x SWE_REGION blocks (Sec. 3's second level above the blocks).
#define SWE_REGION 8

inline void swe_set_regions(SweConst &c) {
    c.regions_x = (c.tiles_x + SWE_REGION - 1) / SWE_REGION;
    c.regions_y = (c.tiles_y + SWE_REGION - 1) / SWE_REGION;
}

// Device pointers of one solver instance.
struct SweBufs {
    void *buf[2];               // AoS state cells {H, Hu, Hv, b}, ping-pong
    int *census[2];             // Index_block of K1 for state^n (census[n & 1])
    unsigned char *skipped;     // per block: 1 = both buffers equal on the block
    int *work;                  // blocks to run this step: [0] count, [1] unused, [2..] block indices
    int *rcen;                  // HGS region census of the state being stepped: blocks with census > 0
    unsigned char *rneed[2];    // per region: it or an edge neighbour held water in state^n (rneed[n & 1])
    const void *gn2;            // g n^2 table (element type = state type)
    const void *ajn;            // 0.05 n^3 table (Eq. 4 numerator)
    const int *src_rowptr;      // ny + 1 offsets into src_x
    const int *src_x;           // source-cell columns, grouped by row
    const double *hyd_t, *hyd_q;
    const void *qb;             // optional bed source per cell (state type)
    const void *rain;           // optional water source per cell, m/s (state type)
    const void *beta;           // optional infiltration rate per cell, m/s (state type)
    SweDev *dev;
    double *partials;           // diagnostics scratch: 3 doubles per block
};

// Launchers implemented per precision (swe_f32.cu / swe_f64.cu).
namespace swe_impl {
template <typename T> size_t step_smem_bytes(int bw);
// grid: 0 launches one CUDA block per grid block; > 0 launches at most that
// many blocks, each walking the work list (for sparse steps).  list: form the
// work list first (false only right after launch_between_compact on the
// same stream, which formed it)
template <typename T>
cudaError_t launch_step(const SweConst &c, const SweBufs &b, int bw, cudaStream_t s, int grid = 0, bool list = true);
template <typename T> cudaError_t launch_init(const SweConst &c, const SweBufs &b, cudaStream_t s);
template <typename T> cudaError_t launch_between(const SweConst &c, const SweBufs &b, int commit, cudaStream_t s);
// launch_between(commit = 1) followed by the next step's work list, in one launch
template <typename T> cudaError_t launch_between_compact(const SweConst &c, const SweBufs &b, cudaStream_t s);
template <typename T> cudaError_t launch_diag(const SweConst &c, const SweBufs &b, int nblocks, cudaStream_t s);
template <typename T> cudaError_t launch_convert_in(const SweConst &c, void *dst, const void *H, const void *Hu,
                                                    const void *Hv, const void *bb, int src_is_f64, cudaStream_t s);
template <typename T> cudaError_t launch_convert_out(const SweConst &c, const void *src, void *H, void *Hu,
                                                     void *Hv, void *bb, int dst_is_f64, cudaStream_t s);
template <typename T> cudaError_t launch_bed_source(const SweConst &c, const SweBufs &b, cudaStream_t s);
}  // namespace swe_impl

// Internal hooks of the C-ABI handle used by the ensemble (swe_ensemble.cu).
struct swe_handle;
namespace swe_impl {
bool handle_view(swe_handle *h, SweConst **c, SweBufs **b, cudaStream_t *s, int *bw, int *precision, bool *state_set);
// Changes the HGS block shape (bw threads, th rows), recomputing the census
// of the current state; the state and time are untouched.
int handle_retile(swe_handle *h, int bw, int th);
// Re-prepares dt without an advance clip (after swe_advance) if needed.
int handle_free_stepping(swe_handle *h);
// Device pointer of the current state buffer (synchronises the stream).
void *handle_current_state(swe_handle *h);
// The current state was modified outside the step kernels: forget which
// dry blocks the ping-pong buffers agree on.
int handle_state_changed(swe_handle *h);
// The state was stepped by kernels that do not keep the HGS region census
// (the ensemble's): the next compaction rebuilds it.
int handle_regions_stale(swe_handle *h);
}  // namespace swe_impl

#define SWE_STATUS_TIMEOUT 4u   // device status bit: a bounded grid barrier gave up

