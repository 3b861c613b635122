/*
 * swe.h -- C ABI of the GB300 (sm_103a) CSPH-TVD + Exner solver.
 *
 * One time step advances the coupled Saint-Venant + Exner system written as
 * Eq. 6 of Khrapov & Khoperskov (2020): U = (H, Hu, Hv, b) with the Exner law
 * of Eq. 1 (porosity psi), the solid discharge of Eq. 2-3 (Grass law with
 * bed-slope term, A_J constant or from Eq. 4), the Shamov threshold of Eq. 5,
 * and the time step of the stability bound Eq. 7.  The step runs the paper's
 * kernels K1 (wet census of each block, the hierarchical grid system), K2-K6
 * (Lagrangian predictor/corrector) and K7-K8 (Eulerian fluxes and update) of
 * Sec. 3 as one fused CUDA kernel per step plus a one-thread kernel that forms
 * dt.  Everything runs on one GPU; state stays resident in device memory.
 *
 * Conventions, for every call:
 *   - Returns a swe_status; nothing is thrown across the ABI.  After a
 *     non-OK status, swe_last_error(handle) gives a one-line reason.
 *   - Arrays are row-major [ny][nx], x fastest.  Host arrays are read or
 *     written synchronously inside the call and stay owned by the caller.
 *   - The library owns all device memory it allocates (cudaMalloc) and frees
 *     it in swe_destroy.  Device pointers passed in (the *_device variants)
 *     stay owned by the caller and are only read/written on the handle's stream.
 *   - A handle is bound to the CUDA device current at swe_create and to the
 *     stream given there; calls on one handle must not overlap.
 *   - Call order: create -> set_manning (optional, default n = 0.03) ->
 *     set_sources (optional) -> set_state -> step/advance -> get_state.
 *     Stepping before set_state returns SWE_ESTATE.
 */
#ifndef SWE_H
#define SWE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swe_handle swe_handle;

typedef enum {
    SWE_OK = 0,
    SWE_EINVAL = 1,   /* invalid argument (sizes, parameters, null pointers) */
    SWE_ENOMEM = 2,   /* device or host allocation failed */
    SWE_ECUDA = 3,    /* a CUDA runtime call failed */
    SWE_ENUMERIC = 4, /* non-finite result, or a depth below -neg_tol */
    SWE_ETIMEOUT = 5, /* a bounded device wait gave up */
    SWE_ESTATE = 6    /* call out of order (e.g. step before set_state) */
} swe_status;

enum { SWE_FP64 = 0, SWE_FP32 = 1 };          /* state/flux precision */
enum { SWE_HOST = 0, SWE_DEVICE = 1 };        /* where a buffer lives */

/* Model parameters (plain data, copied at swe_create).  swe_params_default
 * fills the defaults named below. */
typedef struct {
    int nx, ny;          /* grid size in cells (>= 1 each) */
    double dx;           /* cell size h in metres (Eq. 7: h is the cell size) */
    double g;            /* gravity, 9.81 */
    double cfl_K;        /* Courant number K of Eq. 7, 0 < K < 1; default 0.4 */
    double eps_wet;      /* wet threshold Eps of kernel K1; default 1e-4 m */
    double dt_max;       /* cap on dt when no Eq. 7 term is finite; default 1 s */
    double psi;          /* porosity of Eq. 1, 0 <= psi < 1; default 0.4 */
    int sediment_on;     /* Exner coupling on (1) / off (0); default 1 */
    int aj_mode;         /* 0: constant A_J (Eq. 3); 1: A_J from Eq. 4; default 0 */
    double A_J;          /* Grass coefficient of Eq. 3; default 0.001 */
    double m_exp;        /* Grass exponent m of Eq. 3; default 2 */
    double C_J;          /* bed-slope coefficient of Eq. 2; default 2.0 */
    double d50;          /* median grain size, Eq. 4-5; default 5e-4 m */
    double s_rel;        /* relative density rho_s/rho, Eq. 4; default 2.65 */
    double C_Sh;         /* Shamov coefficient of Eq. 5; default 5.0 */
    int dt_literal_D;    /* 1: D of Eq. 7 as printed, 0: C_J-scaled D; default 0 */
    int precision;       /* SWE_FP64 or SWE_FP32; default SWE_FP32 */
    int hgs_skip;        /* skip dry blocks (K1 rule of Sec. 3); default 1 */
    int tile_rows;       /* rows per block strip, a multiple of 8; 0 = chosen by the library */
    int block_cols;      /* threads (columns) per block, 128 or 256; 0 = auto */
    double neg_tol;      /* H' < -neg_tol => SWE_ENUMERIC; default 1e-10 (FP64), 1e-4 (FP32) */
    int bc[4];           /* boundary of the W (x = 0), E, S (y = 0), N sides: SWE_BC_WALL (default,
                            reflective: the even extension, normal momentum negated) or SWE_BC_OPEN
                            (zero-gradient outflow: the boundary cell repeated; the paper names no
                            outflow condition, so this is a reading) */
} swe_params;

enum { SWE_BC_WALL = 0, SWE_BC_OPEN = 1 };

/* Diagnostics of the current state (swe_get_diag). Volumes are FP64 sums
 * times h^2 over all cells. */
typedef struct {
    double t;               /* simulated time of the current state */
    double dt_last;         /* dt of the last step taken */
    double dt_next;         /* dt the next step will take (Eq. 7, before any t_end clip) */
    int binding;            /* Eq. 7 term that set dt_last: 0 h/(2 vp), 1 h/vs, 2 h^2/(2D), 3 dt_max, 4 t_end */
    double water_volume;    /* sum H h^2 */
    double sediment_volume; /* sum b h^2 */
    double inflow_volume;   /* total volume added by sources since set_state */
    int64_t steps;          /* steps taken since set_state */
    int64_t wet_cells;      /* cells with H > eps_wet */
    int32_t active_tiles;   /* blocks computed in the last step (HGS) */
    int32_t total_tiles;    /* blocks per step */
    int32_t tile_x, tile_y; /* HGS block size in cells */
    uint32_t status;        /* device status bits: 1 non-finite, 2 negative depth,
                               8 an index outside its buffer (checked build only) */
    uint64_t cells_computed;/* cells of computed blocks, summed over steps since set_state */
    uint64_t cells_copied;  /* cells of skipped blocks that were copied, summed likewise */
} swe_diag;

/* Fills *p with the defaults above for an nx x ny grid of cell size dx. */
swe_status swe_params_default(swe_params *p, int nx, int ny, double dx);

/* Creates a solver for the grid and model of *p on the current CUDA device,
 * issuing all work on `cuda_stream` (a cudaStream_t; NULL = default stream).
 * Allocates two state buffers and small tables in device memory. */
swe_status swe_create(const swe_params *p, void *cuda_stream, swe_handle **out);

/* Frees all device and host memory of the handle (NULL is accepted). */
swe_status swe_destroy(swe_handle *h);

/* Manning coefficient n_M(x, y) (Sec. 3, an input field of the Main block),
 * used by bottom friction and by Eq. 4.  block = 0 or 1: n holds nx*ny
 * per-cell values; block = B (a power of two): n holds ceil(ny/B) x ceil(nx/B)
 * values, one per B x B block.  Values must be finite and >= 0. */
swe_status swe_set_manning(swe_handle *h, const double *n, int block);

/* Water sources sigma of Eq. 6 (row 1): the inflow Q(t) [m^3/s], piecewise
 * linear through (t[k], Q[k]), k < nk, constant beyond its ends, is spread
 * evenly over the cells flagged in mask (uint8, nx*ny, nonzero = source; these
 * are the Index_Q cells of kernel K1).  Water enters with zero momentum.
 * mask = NULL or nk = 0 removes all sources.  t must be increasing. */
swe_status swe_set_sources(swe_handle *h, const uint8_t *mask, const double *t,
                           const double *Q, int nk);

/* Bed source q_b^+ - q_b^- of Eq. 1 per cell (nx*ny values, m/s of bed
 * material per unit area); NULL removes it.  Default: none. */
swe_status swe_set_bed_source(swe_handle *h, const double *q);

/* Per-cell water source sigma of Eq. 6 row 1 in m/s (rain > 0, evaporation
 * < 0), host array [ny][nx] (copied); H' gains dt sigma each step.  NULL
 * removes it.  While set, dry blocks are not skipped (rain wets them). */
swe_status swe_set_rain(swe_handle *h, const double *sigma);

/* Per-cell infiltration (absorption) rate beta >= 0 of Sec. 3 in m/s, host
 * array [ny][nx] (copied); each step a cell loses min(dt beta, H') of depth
 * and the same fraction of its momentum (the paper names beta(x, y) but no
 * law; this is a reading).  NULL removes it.  SWE_EINVAL for a negative or
 * non-finite rate. */
swe_status swe_set_infiltration(swe_handle *h, const double *beta);

/* Sets the state (H, Hu, Hv, b) from host FP64 arrays of nx*ny values and
 * resets t to 0.  Dry cells (H <= eps_wet) are given zero momentum. */
swe_status swe_set_state(swe_handle *h, const double *H, const double *Hu,
                         const double *Hv, const double *b);

/* As swe_set_state, with the arrays' type (SWE_FP64 / SWE_FP32) and location
 * (SWE_HOST / SWE_DEVICE, device pointers on this handle's device) given. */
swe_status swe_set_state_ex(swe_handle *h, const void *H, const void *Hu, const void *Hv,
                            const void *b, int dtype, int where);

/* Copies the current state out to host FP64 arrays (any may be NULL). */
swe_status swe_get_state(swe_handle *h, double *H, double *Hu, double *Hv, double *b);

/* As swe_get_state with the output type and location given. */
swe_status swe_get_state_ex(swe_handle *h, void *H, void *Hu, void *Hv, void *b,
                            int dtype, int where);

/* One time step with dt from Eq. 7; *dt_taken (nullable) receives it.
 * Synchronises the stream and checks the device status word. */
swe_status swe_step(swe_handle *h, double *dt_taken);

/* Steps until t reaches t_end; the last dt is clipped so t lands exactly on
 * t_end.  Runs captured CUDA graphs of several steps and polls a device flag
 * once per graph replay.  *steps_taken (nullable) receives the step count. */
swe_status swe_advance(swe_handle *h, double t_end, int64_t *steps_taken);

/* Exactly nsteps steps (dt from Eq. 7, no t_end) queued on the stream without
 * host synchronisation; the status word is checked by swe_sync / swe_get_diag. */
swe_status swe_run_steps(swe_handle *h, int64_t nsteps);

/* Waits for the handle's stream and checks the device status word. */
swe_status swe_sync(swe_handle *h);

/* Current time, and setting it (the hydrograph is evaluated at absolute t). */
swe_status swe_get_time(swe_handle *h, double *t);
swe_status swe_set_time(swe_handle *h, double t);

/* Diagnostics of the current state (runs an FP64 reduction over the grid). */
swe_status swe_get_diag(swe_handle *h, swe_diag *out);

/* Index_block of kernel K1 for the current state: wet-or-source cell count of
 * each HGS block, row-major [tiles_y][tiles_x]; out may be NULL to query the
 * block grid size only. */
swe_status swe_get_census(swe_handle *h, int32_t *out, int *tiles_x, int *tiles_y);

/* Block shape tuning (Sec. 3 sizes blocks for the hardware; no law): times
 * trial_steps steps of the current state for each candidate shape (128 or
 * 256 columns x 16..256 rows, not beyond the grid), keeps the fastest and
 * restores the state and time exactly (results never depend on the shape;
 * the inflow total and step counter restart as after swe_set_state).
 * Outputs (nullable) the chosen shape.  Needs the state set (SWE_ESTATE);
 * SWE_ENOMEM if the state copy cannot be allocated. */
swe_status swe_autotune(swe_handle *h, int trial_steps, int *block_cols, int *tile_rows);

/* One FP32 step without any device allocation.  There is no counterpart of
 * this in the paper.  It is for callers that cannot allocate device memory
 * while they run: real-time loops that cannot afford cudaMalloc's implicit
 * device synchronisation, and applications whose own allocator owns all
 * device memory (a pool reserved at start-up leaves nothing for a library to
 * take).  The caller owns both state buffers: state_in and state_out are
 * distinct, 16-byte aligned device arrays of nx*ny cells, each cell four
 * floats {H, Hu, Hv, b} (row-major [ny][nx]).  state_in is read, and the
 * momentum of its dry cells is set to zero in place (as swe_set_state does);
 * state_out receives the state one Eq. 7 time step later (t = 0 for the
 * hydrograph; no sources; uniform Manning n = manning_n).  *dt_taken (host,
 * nullable) gets the step.  p->precision must be SWE_FP32.
 * Working memory (HGS census, skip flags, block list, step bookkeeping) comes
 * from a fixed 1 MiB array inside the library, one copy per GPU, kept until
 * the process exits.  A grid fits while 13 bytes per HGS block plus 4 bytes
 * per row stay below about 1 MiB (32768 x 32768 with the default blocks needs
 * 0.55 MiB); larger grids return SWE_EINVAL.  All calls on a GPU share that
 * array: calls whose work overlaps on one GPU (say, on two streams) race and
 * must be serialised by the caller.  The first call on a device looks the
 * array up (cudaGetSymbolAddress) with that device current; make it before
 * any stream capture.  Synchronises cuda_stream. */
swe_status swe_step_noalloc(const swe_params *p, double manning_n, void *state_in,
                            void *state_out, void *cuda_stream, double *dt_taken);

/* ---------------------------------------------------------------------
 * Batched ensembles: independent scenarios (grids of uneven sizes and
 * parameters, each with its own dt and time) advanced together by one
 * persistent launch per swe_ensemble_run call, captured in a CUDA graph.
 * Each step of each scenario is exactly the single-grid step above (same
 * kernels, bit-identical results).  Not in the paper: the paper runs one
 * scenario per GPU (Sec. 3); batching keeps a GB300 busy with many small
 * grids. */
typedef struct swe_ensemble swe_ensemble;

/* Most scenarios in one ensemble (the scenario table travels in the
 * persistent launch's parameters). */
#define SWE_ENSEMBLE_MAX 64

/* n scenarios (1 <= n <= SWE_ENSEMBLE_MAX, else SWE_EINVAL), params[k] for
 * scenario k (all SWE_FP32, same block_cols and tile_rows; 0 = library
 * defaults).  Each scenario is a solver handle created on the ensemble's
 * stream (NULL: a private stream). */
swe_status swe_ensemble_create(int n, const swe_params *params, void *cuda_stream, swe_ensemble **out);
swe_status swe_ensemble_destroy(swe_ensemble *e);

/* The handle of scenario k, for swe_set_state / swe_set_manning /
 * swe_set_sources / swe_get_state / swe_get_diag (owned by the ensemble). */
swe_status swe_ensemble_member(swe_ensemble *e, int k, swe_handle **member);

/* Advances every scenario by nsteps steps of its own Eq. 7 dt (no t_end clip)
 * in one persistent launch.  The launch's blocks form one group per scenario,
 * sized so that the scenarios' steps take about as long; a group runs its
 * scenario's (step, block) items by dataflow: the scenario's next step starts
 * as soon as its own previous step is complete, with no barrier across
 * scenarios.  A block whose scenario has no item it could start (its current
 * step all taken, or all its steps done) runs an open item of another
 * scenario meanwhile; which block runs an item does not change its result.
 * Every scenario's state must be set.  SWE_ETIMEOUT if a block's wait for a
 * scenario's step gave up (see set_timeout). */
swe_status swe_ensemble_run(swe_ensemble *e, int64_t nsteps);

/* Times each candidate block shape (128 or 256 columns x 16..256 rows) for
 * trial_steps steps on the current states, keeps the fastest, and restores
 * the states and times (step counters and inflow totals restart).  Outputs
 * (nullable) the chosen shape. */
swe_status swe_ensemble_autotune(swe_ensemble *e, int trial_steps, int *block_cols, int *tile_rows);

/* Time limit of each wait of the persistent launch for a scenario's step
 * (default 2 s), after which every block stops and swe_ensemble_run returns
 * SWE_ETIMEOUT with the context still usable.  extra_arrivals > 0 makes every
 * scenario step wait for that many work items that do not exist: a test hook
 * that exercises the time limit (the scenarios' states are then undefined).
 * Use 0 otherwise. */
swe_status swe_ensemble_set_timeout(swe_ensemble *e, double seconds, int extra_arrivals);

/* ---------------------------------------------------------------------
 * Tensor-core self-test (no counterpart in the paper): checks, on the
 * current device, the BF16 x BF16 -> FP32 tcgen05 MMA path that the bed
 * surrogate's convolution kernels use.  C[128][n] = A[128][k] * B[n][k]^T;
 * A and B are BF16 bit patterns (row-major host arrays), C is FP32 (host).
 * n = 16 or 32, k a multiple of 16 in 16..256.  SWE_ETIMEOUT if the MMA did
 * not complete within its bounded wait. */
swe_status swe_nn_tc_selftest(int n, int k, const uint16_t *A, const uint16_t *B, float *C);

/* Turns the Exner coupling (Eq. 1-5) on or off for the following steps and
 * re-forms dt (Eq. 7) for the current state. */
swe_status swe_set_sediment(swe_handle *h, int on);

/* ---------------------------------------------------------------------
 * Learned bed surrogate (a project addition, not in the paper): a 6-layer
 * 3x3 convolutional network, 32 channels, BF16 weights and activations with
 * FP32 accumulation on the tensor cores (tcgen05), that predicts the bed
 * change over a window of K coupled steps (Eq. 1-6) from the state two
 * coupled steps into the window.  Inputs are the solver state cut into T x T
 * tiles (batch index ty * ceil(nx/T) + tx) with 8 channels:
 *   0  (H - norm[0]) / norm[1]         1  (b - norm[2]) / norm[3]
 *   2  u / norm[4]                     3  v / norm[4]
 *   4  the Shamov ratio |v| / v_k of Eq. 5 (at most 4; 0 on dry cells)
 *   5  the second difference (b - b_mid) - (b_mid - b_saved) / (2 norm[7])
 *   6  p = (b - b_saved) / (2 norm[7]): the change over the two steps,
 *      scaled so that p is their linear extrapolation to the window in
 *      output units (norm[7] = norm[6] / K); p minus channel 5 is the first
 *      step's extrapolation alone
 *   7  m = 1 where a cell within 4 cells (Chebyshev distance) changed its
 *      bed since b_saved, else 0 (the activity mask)
 * b_saved is the bed at the last swe_surrogate_save_bed call (the window's
 * start), b_mid the bed at the last swe_surrogate_save_mid call (after the
 * window's first coupled step).  The network output is m (c + p), c the last
 * convolution: a learned correction of the linear extrapolation, zero where
 * nothing moved.  Output unit: norm[6] metres of bed change.  Device tensors:
 * X bf16 [B][T][T][8], targets/outputs float [B][T][T].  Training: MSE or L1
 * loss, Adam (lr given, betas 0.9/0.999). */
typedef struct swe_surrogate swe_surrogate;
typedef struct {
    int64_t windows, surrogate_windows, plain_windows, judged, takeover_window;
    double bed_time;          /* simulated seconds the bed advanced */
    double water_time;        /* simulated seconds the water advanced */
    double err_last, err_max, err_mean;  /* judged relative L1 error of the bed change */
    double err_zero_mean;     /* the same for predicting no change (1 by definition) */
    double err_persist_mean;  /* the same for repeating the last judged change */
    double err_linear_mean;   /* the same for the two-step linear extrapolation p alone */
    double elev_err_max;      /* judged relative L1 error of the bed elevation itself */
    int mode;                 /* 0: surrogate windows, 1: plain (after a takeover) */
} swe_surrogate_stats;

swe_status swe_surrogate_create(int tile, int max_batch, uint64_t seed, void *cuda_stream, swe_surrogate **out);
swe_status swe_surrogate_destroy(swe_surrogate *s);
/* The 8 normalisation constants above; norm[1], norm[3..7] must be > 0. */
swe_status swe_surrogate_set_norm(swe_surrogate *s, const float norm[8]);
/* Training loss of swe_surrogate_train_step: 0 mean squared error (the
 * default), 1 mean absolute error (the judged error is a relative L1). */
swe_status swe_surrogate_set_loss(swe_surrogate *s, int kind);
/* Forward pass of B tiles (X device bf16, out device float). */
swe_status swe_surrogate_forward(swe_surrogate *s, const void *X, float *out, int B);
/* One training step on B tiles (forward, loss, backward, Adam);
 * *loss_out (host) gets the mean loss before the update. */
swe_status swe_surrogate_train_step(swe_surrogate *s, const void *X, const float *target, int B, float lr,
                                    float *loss_out);
/* Layer (0..5) parameters, FP32 host array W[nout][9*cin] then bias[nout]
 * (cin 8 for layer 0, else 32; nout 1 for layer 5, else 32); dir 0 get, 1 set. */
swe_status swe_surrogate_params(swe_surrogate *s, int layer, float *host, int dir);
/* Gradients of the last training step, same layout as swe_surrogate_params. */
swe_status swe_surrogate_grads(swe_surrogate *s, int layer, float *host);
/* Device pointer of an internal buffer: 0..4 layer outputs (bf16, 32 channels,
 * row-planar [B][T][4][T][8]), 5 the network output. */
swe_status swe_surrogate_buffer(swe_surrogate *s, int index, void **ptr);
/* save_bed remembers the FP32 handle's current bed (the window's start),
 * save_mid the bed after the window's first coupled step; pack_state writes
 * the handle's current state (after the second) as input tiles (device X,
 * channels as above, relative to the saved beds); *batch gets the tile count;
 * pack_target writes the bed change since save_bed in output units (device
 * float). */
swe_status swe_surrogate_pack_state(swe_surrogate *s, swe_handle *h, void *X, int *batch);
swe_status swe_surrogate_save_bed(swe_surrogate *s, swe_handle *h);
swe_status swe_surrogate_save_mid(swe_surrogate *s, swe_handle *h);
swe_status swe_surrogate_pack_target(swe_surrogate *s, swe_handle *h, float *target);
/* Predicts the window's bed change from the handle's current state (two
 * coupled steps after save_bed, save_mid between them) and sets the bed to
 * the saved bed plus that change.  The network runs only on the
 * halo tiles (116 x 116 interior cells plus a 6-cell margin, as 128 x 128
 * images) that hold a cell of the activity mask; elsewhere the prediction is
 * exactly 0.  Device work of a few kernels and one host sync for the tile
 * count.  Errors: SWE_EINVAL (handle not FP32, state not set, or domain
 * larger than max_batch tiles), SWE_ENOMEM (first call's scratch), SWE_ECUDA,
 * SWE_ETIMEOUT (a convolution's bounded wait gave up). */
swe_status swe_surrogate_apply(swe_surrogate *s, swe_handle *h);
/* Runs nwindows windows, each worth K coupled steps of bed evolution (K/f
 * must be at least 2).  A surrogate window saves the bed, runs two coupled
 * steps (saving the bed between them), predicts the window's bed change (on
 * the active halo tiles, as swe_surrogate_apply does), advances the water
 * K/f - 2 further steps and sets the bed to the saved bed plus the prediction
 * (replacing what those steps did to it); its bed time is f times its water
 * time.  Every judge_every-th window instead runs K coupled
 * steps and judges the prediction against them; a judged bed-change error
 * above `bound` hands the rest to the plain solver.  *st accumulates (zero
 * it before the first call). */
swe_status swe_surrogate_run(swe_surrogate *s, swe_handle *h, int nwindows, int K, int f, int judge_every,
                             double bound, swe_surrogate_stats *st);

/* One-line description of the last error on the handle ("" if none). */
const char *swe_last_error(const swe_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* SWE_H */
