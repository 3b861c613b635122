/*
 * FP64 CPU oracle for one CSPH-TVD + Exner time step on a 2D grid.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never calls it and shares no code, header or table with it.
 *
 * Paper: Khrapov & Khoperskov, "Application of GPUs for self-consistent
 * modelling of shallow water dynamics and sediment transport" (2020).
 * The step follows the paper's kernel order K1..K8 (Sec. 3) applied to the
 * coupled Saint-Venant + Exner system of Eq. 6, with the Exner law of Eq. 1-5
 * and the stability bound of Eq. 7.  The paper does not print the discrete
 * CSPH-TVD scheme; every place where this code fixes a choice the paper leaves
 * open is marked READING and listed in the design notes.  Fidelity to the
 * authors' own discretisation is therefore parity unpinned; what pins this
 * reading are the tests' closed forms, invariants and analytic solutions
 * (lake at rest, conservation, Stoker/Ritter dam breaks, Manning decay, the
 * Exner diffusion mode, HLL identities, symmetry, Eq. 7 hand cases).
 *
 * Layout: all arrays are row-major [ny][nx], x fastest, FP64.
 * Every stage is a separate full pass over an extended rectangle that carries
 * R = 4 ghost/halo cells on each side, so a reader can check each formula in
 * isolation.  Ghost cells are the even (mirror) extension of the grid: H, b
 * and the tangential momentum are mirrored, the normal momentum changes sign
 * (reflective walls).  Every derived quantity is evaluated on that extension
 * with the same formulas as in the interior.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, so every
 * operation rounds exactly as written), optional -fopenmp for row loops.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_R 4 /* stencil radius of one fused step, in cells of the input state */

typedef struct {
    int nx, ny;          /* grid size in cells */
    double dx;           /* cell size h (Eq. 7: h is the cell size) */
    double g;            /* gravity */
    double cfl_K;        /* Courant number K, 0 < K < 1 (Eq. 7) */
    double eps_wet;      /* wet threshold Eps of kernel K1 */
    double dt_max;       /* cap on dt when every Eq. 7 term is unbounded (READING) */
    double psi;          /* porosity psi of Eq. 1, 0 <= psi < 1 */
    int sediment_on;     /* Exner coupling on/off */
    int aj_mode;         /* 0: constant A_J (Eq. 3), 1: A_J from Eq. 4 */
    double A_J;          /* Grass coefficient (Eq. 3) */
    double m_exp;        /* Grass exponent m (Eq. 3) */
    double C_J;          /* bed-slope coefficient C_J (Eq. 2) */
    double d50;          /* median grain size (Eq. 4, Eq. 5) */
    double s_rel;        /* relative density s = rho_s / rho (Eq. 4) */
    double C_Sh;         /* Shamov coefficient (Eq. 5) */
    int dt_literal_D;    /* 1: D of Eq. 7 exactly as printed; 0: C_J-scaled D (READING) */
    int hgs_skip;        /* hierarchical-grid dry-tile skip (kernel K1) */
    int tile_x, tile_y;  /* HGS block size L x K */
    int frozen_hydro;    /* test hook: hydro state frozen, only b evolves */
    double neg_tol;      /* H' < -neg_tol is reported as a numerical failure */
    int bc[4];           /* boundary of the W, E, S, N sides: 0 reflective wall, 1 open */
} orc_params;

typedef struct {
    double vp;    /* max |v| over wet cells          (Eq. 7, upsilon_p) */
    double vs;    /* max |v| + sqrt(g H) over wet    (Eq. 7, upsilon_s) */
    double J0max; /* max |J0_b| over wet cells       (Eq. 7, D numerator) */
} orc_dtterms;

typedef struct {
    double dt;          /* step taken */
    int binding;        /* 0: h/(2vp), 1: h/vs, 2: h^2/(2D), 3: dt_max, 4: t_end clip */
    double inflow_vol;  /* water volume added by sources during the step */
    double rain_vol;    /* water volume added by the per-cell source (rain) */
    double outflow_vol; /* water volume that left through open boundaries */
    double infil_vol;   /* water volume lost to infiltration */
    long n_negative;    /* cells with H' < 0 */
    long n_bad;         /* cells with H' < -neg_tol or a non-finite result */
    long active_tiles;  /* tiles computed (HGS) */
} orc_stepinfo;

/* ---------------------------------------------------------------- helpers */

/* Ghost index of i for the boundaries below 0 (lo_open) and at n (hi_open):
 * a reflective wall is the even (mirror) extension, the normal momentum
 * changing sign on every reflection; an open boundary repeats its boundary
 * cell, momentum unchanged (zero-gradient outflow, READING: the paper names
 * no outflow condition).  Walls on both sides give the 2n-periodic even
 * extension. */
static int ext_index(int i, int n, int lo_open, int hi_open, double *sign)
{
    double s = 1.0;
    for (;;) {
        if (i < 0) {
            if (lo_open) { i = 0; break; }
            i = -1 - i; s = -s;
        } else if (i >= n) {
            if (hi_open) { i = n - 1; break; }
            i = 2 * n - 1 - i; s = -s;
        } else {
            break;
        }
    }
    *sign = s;
    return i;
}

/* minmod TVD limiter (READING: the paper names "TVD-limiters" without the law). */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* The limiter, exported for its unit test. */
double orc_minmod(double a, double b) { return minmod(a, b); }

/* HLL flux of one conserved quantity U with physical flux F between left and
 * right states, for wave-speed bounds sL <= sR.  The caller passes the
 * shallow-water bounds sL = min(uL - cL, uR - cR), sR = max(uL + cL, uR + cR)
 * (celerity c = sqrt(g H*) on wet cells); the fluxes are the advective ones of
 * Eq. 6, the pressure and bed-slope terms living in the source Phi. */
double orc_hll(double UL, double UR, double FL, double FR, double sL, double sR)
{
    if (sL >= 0.0) return FL;
    if (sR <= 0.0) return FR;
    return ((sR * FL - sL * FR) + (sL * sR) * (UR - UL)) / (sR - sL);
}

/* Grass bed-load discharge J0 = A_J v |v|^m (Eq. 3), gated by the Shamov
 * critical velocity v_k = C_Sh d50^(1/3) H^(1/6) (Eq. 5): erosion only when
 * |v| > v_k, written exactly as |v|^6 > C_Sh^6 d50^2 H.  A_J is constant
 * (Eq. 3) or given by Eq. 4 with the cell depth.  Dry cells carry no load. */
static void grass_J0(const orc_params *p, int wet, double H, double n,
                     double vx, double vy, double *Jx, double *Jy, double *Jabs)
{
    *Jx = 0.0; *Jy = 0.0; *Jabs = 0.0;
    if (!p->sediment_on || !wet) return;
    double s2 = vx * vx + vy * vy;
    double ksh = pow(p->C_Sh, 6.0) * (p->d50 * p->d50);
    if (!(s2 * s2 * s2 > ksh * H)) return;
    double AJ;
    if (p->aj_mode == 1) {
        double num = 0.05 * n * n * n;
        AJ = num / (((p->s_rel - 1.0) * sqrt(p->g * H)) * p->d50);
    } else {
        AJ = p->A_J;
    }
    double vm = (p->m_exp == 2.0) ? s2 : pow(s2, 0.5 * p->m_exp); /* |v|^m */
    *Jx = (AJ * vx) * vm;
    *Jy = (AJ * vy) * vm;
    *Jabs = (AJ * vm) * sqrt(s2);
}

/* Manning friction coefficient c_f = g n^2 / max(H,Eps)^(4/3); the friction
 * rate of a particle moving at speed |v| is c_f |v| (READING: standard Manning
 * law for the paper's "bottom friction" and n_M field, applied point-implicitly). */
static double manning_cf(const orc_params *p, double H, double n)
{
    double Hm = H > p->eps_wet ? H : p->eps_wet;
    double H43 = Hm * cbrt(Hm);
    return ((p->g * n) * n) / H43;
}

/* --------------------------------------------------------- K3: Eq. 7 terms */

int orc_dt_terms(const orc_params *p, const double *H, const double *Hu,
                 const double *Hv, const double *nman, orc_dtterms *out)
{
    double vp = 0.0, vs = 0.0, jm = 0.0;
    long N = (long)p->nx * p->ny;
    for (long k = 0; k < N; ++k) {
        if (!(H[k] > p->eps_wet)) continue;
        double u = Hu[k] / H[k], v = Hv[k] / H[k];
        double va = sqrt(u * u + v * v);
        double c = va + sqrt(p->g * H[k]);
        if (va > vp) vp = va;
        if (c > vs) vs = c;
        double jx, jy, ja;
        grass_J0(p, 1, H[k], nman[k], u, v, &jx, &jy, &ja);
        if (ja > jm) jm = ja;
    }
    out->vp = vp; out->vs = vs; out->J0max = jm;
    return 0;
}

/* tau = K min(h/(2 vp), h/vs, h^2/(2D)), terms with a zero denominator are
 * ignored; D = C_J max|J0|/(1-psi) (READING: the diffusion coefficient that
 * Eq. 2 implies) or max|J0|/(1-psi) as printed when dt_literal_D is set. */
double orc_dt(const orc_params *p, const orc_dtterms *t, int *binding)
{
    double h = p->dx;
    double best = INFINITY;
    int which = 3;
    if (t->vp > 0.0) { double a = h / (2.0 * t->vp); if (a < best) { best = a; which = 0; } }
    if (t->vs > 0.0) { double a = h / t->vs; if (a < best) { best = a; which = 1; } }
    if (p->sediment_on && t->J0max > 0.0) {
        double D = (p->dt_literal_D ? t->J0max : p->C_J * t->J0max) / (1.0 - p->psi);
        double a = (h * h) / (2.0 * D);
        if (a < best) { best = a; which = 2; }
    }
    double dt = p->cfl_K * best;
    if (!(dt < p->dt_max)) { dt = p->dt_max; which = 3; }
    if (binding) *binding = which;
    return dt;
}

/* ------------------------------------------------------------ K1: census */

/* Index_block of kernel K1: per tile, the number of cells with H > Eps or a
 * source flag. */
void orc_census(const orc_params *p, const double *H, const uint8_t *src, int *counts)
{
    int ntx = (p->nx + p->tile_x - 1) / p->tile_x;
    int nty = (p->ny + p->tile_y - 1) / p->tile_y;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            int c = 0;
            for (int j = ty * p->tile_y; j < (ty + 1) * p->tile_y && j < p->ny; ++j)
                for (int i = tx * p->tile_x; i < (tx + 1) * p->tile_x && i < p->nx; ++i) {
                    long k = (long)j * p->nx + i;
                    if (H[k] > p->eps_wet || (src && src[k])) ++c;
                }
            counts[ty * ntx + tx] = c;
        }
}

/* ------------------------------------------------- K2..K8 on a rectangle */

typedef struct {
    int x0, y0, W, Hh; /* extended rectangle origin (x0 - R, y0 - R) and size */
    double *H, *b, *u, *v, *n;  /* t_n state on the extension (ghosts filled) */
    int *wet;
    double *ax, *ay;            /* K2: forces at t_n */
    double *vtx, *vty, *Hh_;    /* K4: v at t_{n+1/2} and particle depth H^{n+1/2} */
    double *bx, *by;            /* K5: forces at t_{n+1/2} */
    double *wx, *wy;            /* K6: Lagrangian end velocity at t_{n+1} */
    double *Jx, *Jy, *Ja;       /* Grass discharge from the transport velocity */
    double *cf;                 /* Manning coefficient from H^n */
} ext_t;

#define E(e, i, j) ((long)((j) - (e)->y0) * (e)->W + ((i) - (e)->x0))

/* Pressure + bed-slope force per unit mass (Eq. 6 Phi row 2, -g H grad(H+b);
 * READING on the sign: the printed +gH grad(H+b) sits on the right-hand side of
 * dU/dt + ... = Phi, physically the force is -g H grad(H+b)).
 * Central form (READING): a = -g/(2h) (eta_E' - eta_W') * Hs/H^n, where Hs is
 * the particle depth at the stage (H^n for K2, H^{n+1/2} = H^n/A for K5) and
 * H^n the particle mass per unit area: summed over cells, H^n a telescopes
 * into face differences of g Hs^2/2 on a flat bed (momentum-conservative,
 * dam-break shocks converge to the right states), the acceleration stays
 * bounded by g |d eta| / (2 h A), and a flat free surface feels no force.
 * Wet/dry rule (READING): a dry neighbour whose bed lies at or above the
 * cell's free surface acts as a wall (its level is taken equal to the cell's
 * own level).  Dry cells feel no force. */
static void forces(const orc_params *p, ext_t *e, const double *Hs, const double *eta,
                   int i0, int i1, int j0, int j1, double *fx, double *fy)
{
    double coef = p->g / (2.0 * p->dx);
    for (int j = j0; j < j1; ++j)
        for (int i = i0; i < i1; ++i) {
            long c = E(e, i, j);
            if (!e->wet[c]) { fx[c] = 0.0; fy[c] = 0.0; continue; }
            double ec = eta[c];
            long nb[4] = { E(e, i + 1, j), E(e, i - 1, j), E(e, i, j + 1), E(e, i, j - 1) };
            double en[4];
            for (int q = 0; q < 4; ++q) {
                long k = nb[q];
                en[q] = (!e->wet[k] && e->b[k] >= ec) ? ec : eta[k];
            }
            double r = Hs[c] / e->H[c];
            fx[c] = -(coef * (en[0] - en[1])) * r;
            fy[c] = -(coef * (en[2] - en[3])) * r;
        }
}

static double *xalloc(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

/* Computes state^{n+1} on [x0,x1) x [y0,y1) from state^n, for a given dt and a
 * given source depth increment dHs (added to source-flagged cells).  Writes
 * only the rectangle of the full-size output arrays.  qb (nullable) is the
 * per-cell bed source q_b^+ - q_b^- of Eq. 1; rain (nullable) a per-cell
 * water source sigma of Eq. 6 row 1 in m/s (rain > 0, evaporation < 0);
 * beta (nullable) the absorption (infiltration) rate of Sec. 3 in m/s >= 0,
 * a loss capped by the water present that takes its share of momentum
 * (READING: the paper names beta(x, y) but gives no law).
 * Returns the number of cells with H' < -neg_tol or a non-finite result;
 * *nneg counts H' < 0; *outflow (nullable) gets the volume of water that
 * left the grid through the rectangle's part of the domain boundary. */
long orc_step_rect(const orc_params *p, const double *H, const double *Hu,
                   const double *Hv, const double *b, const double *nman,
                   const uint8_t *src, const double *qb, const double *rain, const double *beta,
                   double dHs, double dt, int x0, int y0, int x1, int y1,
                   double *Ho, double *Huo, double *Hvo, double *bo, long *nneg, double *outflow,
                   double *infil)
{
    const int R = ORC_R;
    ext_t e;
    e.x0 = x0 - R; e.y0 = y0 - R;
    e.W = (x1 - x0) + 2 * R; e.Hh = (y1 - y0) + 2 * R;
    long NE = (long)e.W * e.Hh;
    e.H = xalloc(NE); e.b = xalloc(NE); e.u = xalloc(NE); e.v = xalloc(NE); e.n = xalloc(NE);
    e.wet = (int *)calloc((size_t)NE, sizeof(int));
    e.ax = xalloc(NE); e.ay = xalloc(NE); e.vtx = xalloc(NE); e.vty = xalloc(NE);
    e.Hh_ = xalloc(NE); e.bx = xalloc(NE); e.by = xalloc(NE); e.wx = xalloc(NE); e.wy = xalloc(NE);
    e.Jx = xalloc(NE); e.Jy = xalloc(NE); e.Ja = xalloc(NE); e.cf = xalloc(NE);
    double *eta = xalloc(NE), *etah = xalloc(NE);

    /* ghost fill (walls: even extension, normal momentum negated; open
     * sides: the boundary cell repeated) and cell
     * velocities v = (Hu, Hv)/H for wet cells, v = 0 for dry cells */
    for (int j = y0 - R; j < y1 + R; ++j)
        for (int i = x0 - R; i < x1 + R; ++i) {
            double sx, sy;
            int ii = ext_index(i, p->nx, p->bc[0], p->bc[1], &sx);
            int jj = ext_index(j, p->ny, p->bc[2], p->bc[3], &sy);
            long k = (long)jj * p->nx + ii, c = E(&e, i, j);
            double h = H[k];
            e.H[c] = h; e.b[c] = b[k]; e.n[c] = nman[k];
            e.wet[c] = h > p->eps_wet;
            e.u[c] = e.wet[c] ? (sx * Hu[k]) / h : 0.0;
            e.v[c] = e.wet[c] ? (sy * Hv[k]) / h : 0.0;
            eta[c] = h + b[k];
            e.cf[c] = manning_cf(p, h, nman[k]);
        }

    double hdt = 0.5 * dt;
    if (!p->frozen_hydro) {
        /* K2: forces at t_n (predictor), needed on R-2 */
        forces(p, &e, e.H, eta, x0 - 2, x1 + 2, y0 - 2, y1 + 2, e.ax, e.ay);
        /* K4: velocity at t_{n+1/2}, point-implicit Manning with |v^n|:
         *   vt = (v + dt/2 a) / (1 + dt/2 c_f |v|)                  on R-2
         * particle area ratio from the central divergence of v^n and the
         * particle depth H^{n+1/2} = H^n / A:
         *   A = 1 + dt/2 (D_x u + D_y v)                            on R-3 */
        for (int j = y0 - 2; j < y1 + 2; ++j)
            for (int i = x0 - 2; i < x1 + 2; ++i) {
                long c = E(&e, i, j);
                double va = sqrt(e.u[c] * e.u[c] + e.v[c] * e.v[c]);
                double den = 1.0 + hdt * (e.cf[c] * va);
                e.vtx[c] = (e.u[c] + hdt * e.ax[c]) / den;
                e.vty[c] = (e.v[c] + hdt * e.ay[c]) / den;
            }
        double c4 = dt / (4.0 * p->dx);
        for (int j = y0 - 3; j < y1 + 3; ++j)
            for (int i = x0 - 3; i < x1 + 3; ++i) {
                long c = E(&e, i, j);
                double A = 1.0 + c4 * ((e.u[E(&e, i + 1, j)] - e.u[E(&e, i - 1, j)])
                                     + (e.v[E(&e, i, j + 1)] - e.v[E(&e, i, j - 1)]));
                e.Hh_[c] = e.H[c] / A;
                etah[c] = e.Hh_[c] + e.b[c];
            }
        /* K5: forces at t_{n+1/2} from the particle free surface H^{n+1/2} + b
         * (bed frozen during the Lagrangian stage, READING), wet flags of t_n */
        forces(p, &e, e.Hh_, etah, x0 - 2, x1 + 2, y0 - 2, y1 + 2, e.bx, e.by);
        /* K6: Lagrangian end velocity, point-implicit Manning with |vt|:
         *   w = (v + dt a^{n+1/2}) / (1 + dt c_f |vt|)                on R-2 */
        for (int j = y0 - 2; j < y1 + 2; ++j)
            for (int i = x0 - 2; i < x1 + 2; ++i) {
                long c = E(&e, i, j);
                double va = sqrt(e.vtx[c] * e.vtx[c] + e.vty[c] * e.vty[c]);
                double den = 1.0 + dt * (e.cf[c] * va);
                e.wx[c] = (e.u[c] + dt * e.bx[c]) / den;
                e.wy[c] = (e.v[c] + dt * e.by[c]) / den;
            }
    } else {
        /* frozen hydro (test hook): transport and end velocity are v^n */
        for (long c = 0; c < NE; ++c) {
            e.vtx[c] = e.u[c]; e.vty[c] = e.v[c]; e.wx[c] = e.u[c]; e.wy[c] = e.v[c];
        }
    }
    /* Grass discharge at t_{n+1/2} from the transport velocity, on R-1 */
    for (int j = y0 - 1; j < y1 + 1; ++j)
        for (int i = x0 - 1; i < x1 + 1; ++i) {
            long c = E(&e, i, j);
            grass_J0(p, e.wet[c], e.H[c], e.n[c], e.vtx[c], e.vty[c], &e.Jx[c], &e.Jy[c], &e.Ja[c]);
        }

    /* K7: Eulerian face fluxes at t_{n+1/2}.  Piecewise-linear reconstruction
     * of H^n, the free surface eta^n = H^n + b, the normal transport velocity
     * and both end-velocity components
     * with the minmod limiter, then HLL for mass and both momenta (Eq. 6, F and
     * G rows 1-3) and the Exner face discharge (Eq. 2 + Eq. 3, row 4).
     * Face arrays: fx[k][j][i] is the x-face between (i,j) and (i+1,j) for
     * i = x0-1 .. x1-1; fy likewise for y-faces. */
    int FW = (x1 - x0) + 1, FH = (y1 - y0) + 1;
    int RW = x1 - x0, RH = y1 - y0;
    double *FX[4], *FY[4];
    for (int q = 0; q < 4; ++q) { FX[q] = xalloc((long)FW * RH); FY[q] = xalloc((long)RW * FH); }
    double cjh = (0.5 * p->C_J) / p->dx;
    for (int dir = 0; dir < 2; ++dir) {
        int ilo = dir == 0 ? x0 - 1 : x0, ihi = x1;
        int jlo = dir == 0 ? y0 : y0 - 1, jhi = y1;
        int di = dir == 0 ? 1 : 0, dj = dir == 0 ? 0 : 1;
        const double *un = dir == 0 ? e.vtx : e.vty;
        const double *Jn = dir == 0 ? e.Jx : e.Jy;
        for (int j = jlo; j < jhi; ++j)
            for (int i = ilo; i < ihi; ++i) {
                /* cells m1 = c-1, c, e = c+1, p2 = c+2 along the face normal */
                long cm = E(&e, i - di, j - dj), cc = E(&e, i, j);
                long ce = E(&e, i + di, j + dj), cp = E(&e, i + 2 * di, j + 2 * dj);
                const double *qs[5] = { e.H, eta, un, e.wx, e.wy };
                double qL[5], qR[5];
                for (int q = 0; q < 5; ++q) {
                    const double *f = qs[q];
                    double sc = minmod(f[cc] - f[cm], f[ce] - f[cc]);
                    double se = minmod(f[ce] - f[cc], f[cp] - f[ce]);
                    qL[q] = f[cc] + 0.5 * sc;
                    qR[q] = f[ce] - 0.5 * se;
                }
                /* hydrostatic face depths (READING, keeps a lake at rest exactly
                 * and depths non-negative over steep terrain): face bed from
                 * the reconstructed surface and depth, b_L = eta_L - H_L, the
                 * face sill b_f = max(b_L, b_R), H*_{L,R} = max(0, eta_{L,R} - b_f) */
                double bL = qL[1] - qL[0], bR = qR[1] - qR[0];
                double bf = bL > bR ? bL : bR;
                double HL = qL[1] - bf, HR = qR[1] - bf;
                if (!(HL > 0.0)) HL = 0.0;
                if (!(HR > 0.0)) HR = 0.0;
                double uL = qL[2], uR = qR[2];
                /* HLL wave-speed bounds of the shallow-water Riemann problem
                 * (READING: the paper solves "the Riemann problem ... using the
                 * HLL method"), celerity sqrt(g H*) on wet cells, 0 on dry ones */
                double cL = e.wet[cc] ? sqrt(p->g * HL) : 0.0;
                double cR = e.wet[ce] ? sqrt(p->g * HR) : 0.0;
                double aL = uL - cL, aR = uR - cR, bL2 = uL + cL, bR2 = uR + cR;
                double sL = aL < aR ? aL : aR, sR = bL2 > bR2 ? bL2 : bR2;
                double Fm = orc_hll(HL, HR, HL * uL, HR * uR, sL, sR);
                double UxL = HL * qL[3], UxR = HR * qR[3];
                double Fx = orc_hll(UxL, UxR, UxL * uL, UxR * uR, sL, sR);
                double UyL = HL * qL[4], UyR = HR * qR[4];
                double Fy = orc_hll(UyL, UyR, UyL * uL, UyR * uR, sL, sR);
                /* Exner face discharge (Eq. 2, READING): the advective Grass
                 * load from the upwind cell by the sign of the summed cell
                 * transport velocities, minus the bed-slope diffusion
                 * C_J |J0| grad b with the face mean of |J0| (the printed
                 * sign(J0)|J0| form read as the diffusion |J0| grad b that
                 * the text says Eq. 2 produces). */
                double Jf = 0.0;
                if (p->sediment_on) {
                    double su = un[cc] + un[ce];
                    double Jadv = su > 0.0 ? Jn[cc] : (su < 0.0 ? Jn[ce] : 0.0);
                    Jf = Jadv - (cjh * (e.Ja[cc] + e.Ja[ce])) * (e.b[ce] - e.b[cc]);
                }
                double vals[4] = { Fm, Fx, Fy, Jf };
                for (int q = 0; q < 4; ++q) {
                    if (dir == 0) FX[q][(long)(j - y0) * FW + (i - (x0 - 1))] = vals[q];
                    else          FY[q][(long)(j - (y0 - 1)) * RW + (i - x0)] = vals[q];
                }
            }
    }

    /* K8: Eulerian update at t_{n+1} (Eq. 6 rows 1-3, Eq. 1 for b):
     *   H'  = H^n - dt/h (dF + dG) + source
     *   Hw' = H^n w - dt/h (dF_w + dG_w)
     *   b'  = b^n - dt/(h (1-psi)) (dJx + dJy) + dt q/(1-psi)
     * Cells left with H' <= Eps carry no momentum. */
    double dtdx = dt / p->dx;
    double cb = dtdx / (1.0 - p->psi);
    double cq = dt / (1.0 - p->psi);
    long bad = 0, neg = 0;
    double lost = 0.0;
    for (int j = y0; j < y1; ++j)
        for (int i = x0; i < x1; ++i) {
            long c = E(&e, i, j), k = (long)j * p->nx + i;
            long fe = (long)(j - y0) * FW + (i - x0 + 1), fw = fe - 1;
            long fn = (long)(j - y0 + 1) * RW + (i - x0), fs = fn - RW;
            double hn, hun, hvn;
            if (!p->frozen_hydro) {
                hn = e.H[c] - dtdx * ((FX[0][fe] - FX[0][fw]) + (FY[0][fn] - FY[0][fs]));
                if (src && src[k]) hn = hn + dHs;
                if (rain) hn = hn + dt * rain[k];
                hun = e.H[c] * e.wx[c] - dtdx * ((FX[1][fe] - FX[1][fw]) + (FY[1][fn] - FY[1][fs]));
                hvn = e.H[c] * e.wy[c] - dtdx * ((FX[2][fe] - FX[2][fw]) + (FY[2][fn] - FY[2][fs]));
                if (beta) {
                    /* infiltration: at most the water present, with its share of momentum */
                    double loss = dt * beta[k];
                    if (loss > hn) loss = hn > 0.0 ? hn : 0.0;
                    if (loss > 0.0) {
                        double r = (hn - loss) / hn;
                        hn = hn - loss;
                        hun = hun * r;
                        hvn = hvn * r;
                        lost += loss;
                    }
                }
                if (!(hn > p->eps_wet)) { hun = 0.0; hvn = 0.0; }
            } else {
                hn = H[k]; hun = Hu[k]; hvn = Hv[k];
            }
            double bn = e.b[c] - cb * ((FX[3][fe] - FX[3][fw]) + (FY[3][fn] - FY[3][fs]));
            if (qb) bn = bn + cq * qb[k];
            Ho[k] = hn; Huo[k] = hun; Hvo[k] = hvn; bo[k] = bn;
            if (hn < 0.0) ++neg;
            if (!(hn >= -p->neg_tol) || !isfinite(hn) || !isfinite(bn) || !isfinite(hun) || !isfinite(hvn)) ++bad;
        }
    if (nneg) *nneg = neg;
    if (infil) *infil = lost * (p->dx * p->dx);
    if (outflow) {
        /* mass fluxes through the domain's boundary faces (zero at walls) */
        double out = 0.0, ah = dt * p->dx;
        for (int j = y0; j < y1; ++j) {
            long r = (long)(j - y0) * FW;
            if (x0 == 0) out -= ah * FX[0][r];
            if (x1 == p->nx) out += ah * FX[0][r + (x1 - x0)];
        }
        for (int i = x0; i < x1; ++i) {
            if (y0 == 0) out -= ah * FY[0][i - x0];
            if (y1 == p->ny) out += ah * FY[0][(long)(y1 - y0) * RW + (i - x0)];
        }
        *outflow = out;
    }

    for (int q = 0; q < 4; ++q) { free(FX[q]); free(FY[q]); }
    free(e.H); free(e.b); free(e.u); free(e.v); free(e.n); free(e.wet);
    free(e.ax); free(e.ay); free(e.vtx); free(e.vty); free(e.Hh_); free(e.bx); free(e.by);
    free(e.wx); free(e.wy); free(e.Jx); free(e.Jy); free(e.Ja); free(e.cf);
    free(eta); free(etah);
    return bad;
}

/* ------------------------------------------------------------- sources */

/* Integral of the piecewise-linear hydrograph Q(t) (constant beyond the end
 * points) over [ta, tb]; sigma of Eq. 6 row 1 on the flagged inflow cells. */
double orc_hydro_integral(int nk, const double *tk, const double *Qk, double ta, double tb)
{
    if (nk <= 0 || !(tb > ta)) return 0.0;
    double s = 0.0;
    /* left constant extension */
    if (ta < tk[0]) { double e = tb < tk[0] ? tb : tk[0]; s += Qk[0] * (e - ta); }
    for (int k = 0; k + 1 < nk; ++k) {
        double a = ta > tk[k] ? ta : tk[k];
        double c = tb < tk[k + 1] ? tb : tk[k + 1];
        if (!(c > a)) continue;
        double span = tk[k + 1] - tk[k];
        double qa = Qk[k] + (Qk[k + 1] - Qk[k]) * ((a - tk[k]) / span);
        double qc = Qk[k] + (Qk[k + 1] - Qk[k]) * ((c - tk[k]) / span);
        s += 0.5 * (qa + qc) * (c - a);
    }
    if (tb > tk[nk - 1]) { double a = ta > tk[nk - 1] ? ta : tk[nk - 1]; s += Qk[nk - 1] * (tb - a); }
    return s;
}

/* ---------------------------------------------------- one complete step */

/* K1 census -> K3 dt (clipped to t_end - t) -> sources -> K2..K8 on every
 * active tile (HGS: a tile is computed when it or one of its four edge
 * neighbours holds water or a source; otherwise its state is carried over).
 * Returns the count of bad cells (0 = success). */
long orc_step(const orc_params *p, const double *H, const double *Hu, const double *Hv,
              const double *b, const double *nman, const uint8_t *src, const double *qb,
              const double *rain, const double *beta, int nk, const double *tk, const double *Qk,
              double t, double t_end,
              double *Ho, double *Huo, double *Hvo, double *bo, orc_stepinfo *info)
{
    orc_dtterms terms;
    orc_dt_terms(p, H, Hu, Hv, nman, &terms);
    int binding;
    double dt = orc_dt(p, &terms, &binding);
    if (t_end > t && t_end - t < dt) { dt = t_end - t; binding = 4; }

    long N = (long)p->nx * p->ny, nsrc = 0;
    if (src) for (long k = 0; k < N; ++k) nsrc += src[k] ? 1 : 0;
    double vol = nsrc ? orc_hydro_integral(nk, tk, Qk, t, t + dt) : 0.0;
    double dHs = nsrc ? vol / ((double)nsrc * (p->dx * p->dx)) : 0.0;

    /* the rectangle step is independent of how the grid is cut, so tiles
     * also serve as the unit of (OpenMP) work when the skip is off */
    int tx = p->tile_x > 0 ? p->tile_x : 64, ty = p->tile_y > 0 ? p->tile_y : 64;
    int ntx = (p->nx + tx - 1) / tx, nty = (p->ny + ty - 1) / ty;
    int *cen = NULL;
    const int skip = p->hgs_skip && !rain;   /* rain wets dry tiles: no skipping */
    if (skip) {
        orc_params q = *p;
        q.tile_x = tx; q.tile_y = ty;
        cen = (int *)calloc((size_t)ntx * nty, sizeof(int));
        orc_census(&q, H, src, cen);
    }
    long bad = 0, neg = 0, active = 0;
    double outflow = 0.0, infil = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad, neg, active, outflow, infil) collapse(2)
#endif
    for (int by = 0; by < nty; ++by)
        for (int bx = 0; bx < ntx; ++bx) {
            int x0 = bx * tx, y0 = by * ty;
            int x1 = x0 + tx < p->nx ? x0 + tx : p->nx, y1 = y0 + ty < p->ny ? y0 + ty : p->ny;
            int act = 1;
            if (skip) {
                int l = bx > 0 ? bx - 1 : bx, r = bx < ntx - 1 ? bx + 1 : bx;
                int s = by > 0 ? by - 1 : by, nn = by < nty - 1 ? by + 1 : by;
                act = cen[by * ntx + bx] > 0 || cen[by * ntx + l] > 0 || cen[by * ntx + r] > 0
                   || cen[s * ntx + bx] > 0 || cen[nn * ntx + bx] > 0;
            }
            if (act) {
                long ng = 0;
                double of = 0.0, il = 0.0;
                bad += orc_step_rect(p, H, Hu, Hv, b, nman, src, qb, rain, beta, dHs, dt, x0, y0, x1, y1,
                                     Ho, Huo, Hvo, bo, &ng, &of, &il);
                neg += ng;
                outflow += of;
                infil += il;
                ++active;
            } else {
                for (int j = y0; j < y1; ++j)
                    for (int i = x0; i < x1; ++i) {
                        long k = (long)j * p->nx + i;
                        Ho[k] = H[k]; Huo[k] = Hu[k]; Hvo[k] = Hv[k]; bo[k] = b[k];
                    }
            }
        }
    free(cen);
    if (info) {
        double rv = 0.0;
        if (rain) for (long k = 0; k < N; ++k) rv += rain[k];
        info->dt = dt; info->binding = binding; info->inflow_vol = vol;
        info->rain_vol = rv * dt * (p->dx * p->dx);
        info->outflow_vol = outflow;
        info->infil_vol = infil;
        info->n_negative = neg; info->n_bad = bad; info->active_tiles = active;
    }
    return bad;
}

int orc_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
