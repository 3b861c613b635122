// CSPH-TVD + Exner step kernels for sm_103a, templated on the state type
// (float: production path with FP64 accumulators; double: parity build).
//
// Paper: Khrapov & Khoperskov (2020), Sec. 2 (Eq. 1-7) and Sec. 3 (kernels
// K1-K8, hierarchical grid system).  The paper runs K1..K8 as eight kernels;
// here K2-K8 are one streaming kernel per step so the state makes a single
// HBM round trip (16 B read + 16 B write per cell in FP32):
//
//   * A block owns BW consecutive columns (one thread per column) and a strip
//     of `th` rows; it writes the middle BW-8 columns (the stencil radius of
//     one step is 4 cells: K4/K6 need radius 2, K7's reconstruction 2 more).
//   * The block sweeps its strip row by row.  At sweep position s it loads
//     row s, forms the particle depth H^{n+1/2} (K4) of row s-1, the forces,
//     predictor and corrector velocities and Grass load (K2, K4-K6) of row s-2,
//     the x- and y-face fluxes (K7) of row s-4 and updates row s-4 (K8).
//     Intermediate rows live in small shared-memory rings, so nothing but the
//     state itself touches HBM.
//   * The epilogue forms, for the new state, the wet census of the block
//     (K1's Index_block), the maxima behind the Eq. 7 time step, and a status
//     word.  A one-thread `between` kernel turns the maxima into dt (FP64).
//   * HGS (Sec. 3): a block is computed when it or one of its four edge
//     neighbours holds water or a source; otherwise its state is carried over,
//     and not even copied when both ping-pong buffers already agree.
//
// Ghost cells: the state is extended evenly across each wall (H, b and the
// tangential momentum mirrored, the normal momentum negated), and every
// derived quantity is computed on that extension with the interior formulas.
//
// The double instantiation evaluates every formula in the same order as the
// FP64 CPU oracle (compiled without FMA contraction), so the two agree to a
// few ulps per step.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "swe_internal.h"

namespace swe_impl {

// ------------------------------------------------------------ checked build
//
// Built with -DSWE_CHECKED (the library's checked variant, for tests), every
// global access of the step kernel first tests its index against its buffer:
// an index outside sets SWE_STATUS_BOUNDS in the device status word and the
// access is skipped.  In the production build SWE_IN is the constant true.
#define SWE_STATUS_BOUNDS 8u
// source terms compiled into a step-kernel variant (template parameter SRC)
#define SWE_SRC_INFLOW 1
#define SWE_SRC_FIELDS 2
#ifdef SWE_CHECKED
__device__ inline bool swe_in(long long i, long long n, SweDev *dev) {
    if (i >= 0 && i < n) return true;
    atomicOr(&dev->status, SWE_STATUS_BOUNDS);
    return false;
}
#define SWE_IN(i, n) swe_in((long long)(i), (long long)(n), B.dev)
#else
#define SWE_IN(i, n) true
#endif
// cells of the grid, entries of the Manning tables
#define SWE_NCELL ((long long)c.nx * c.ny)
#define SWE_NMAN ((long long)((((c.ny - 1) >> c.man_shift) + 1) * c.man_w))

// ------------------------------------------------------------ state cells

template <typename T> struct CellIO;
template <> struct CellIO<float> {
    __device__ static inline void load(const void *base, long long k, float &H, float &Hu, float &Hv, float &b) {
        float4 c = __ldg(reinterpret_cast<const float4 *>(base) + k);
        H = c.x; Hu = c.y; Hv = c.z; b = c.w;
    }
    // L2-coherent load, for data other blocks of the same launch rewrite
    __device__ static inline void load_cg(const void *base, long long k, float &H, float &Hu, float &Hv, float &b) {
        float4 c = __ldcg(reinterpret_cast<const float4 *>(base) + k);
        H = c.x; Hu = c.y; Hv = c.z; b = c.w;
    }
    __device__ static inline void copy_cg(const void *src, void *dst, long long k) {
        reinterpret_cast<float4 *>(dst)[k] = __ldcg(reinterpret_cast<const float4 *>(src) + k);
    }
    __device__ static inline void store(void *base, long long k, float H, float Hu, float Hv, float b) {
        reinterpret_cast<float4 *>(base)[k] = make_float4(H, Hu, Hv, b);
    }
    __device__ static inline void copy(const void *src, void *dst, long long k) {
        reinterpret_cast<float4 *>(dst)[k] = __ldg(reinterpret_cast<const float4 *>(src) + k);
    }
};
template <> struct CellIO<double> {
    __device__ static inline void load(const void *base, long long k, double &H, double &Hu, double &Hv, double &b) {
        const double2 *p = reinterpret_cast<const double2 *>(base) + 2 * k;
        double2 a = __ldg(p), c = __ldg(p + 1);
        H = a.x; Hu = a.y; Hv = c.x; b = c.y;
    }
    __device__ static inline void load_cg(const void *base, long long k, double &H, double &Hu, double &Hv, double &b) {
        const double2 *p = reinterpret_cast<const double2 *>(base) + 2 * k;
        double2 a = __ldcg(p), c = __ldcg(p + 1);
        H = a.x; Hu = a.y; Hv = c.x; b = c.y;
    }
    __device__ static inline void copy_cg(const void *src, void *dst, long long k) {
        const double2 *s = reinterpret_cast<const double2 *>(src) + 2 * k;
        double2 *d = reinterpret_cast<double2 *>(dst) + 2 * k;
        d[0] = __ldcg(s);
        d[1] = __ldcg(s + 1);
    }
    __device__ static inline void store(void *base, long long k, double H, double Hu, double Hv, double b) {
        double2 *p = reinterpret_cast<double2 *>(base) + 2 * k;
        p[0] = make_double2(H, Hu);
        p[1] = make_double2(Hv, b);
    }
    __device__ static inline void copy(const void *src, void *dst, long long k) {
        const double2 *s = reinterpret_cast<const double2 *>(src) + 2 * k;
        double2 *d = reinterpret_cast<double2 *>(dst) + 2 * k;
        d[0] = __ldg(s);
        d[1] = __ldg(s + 1);
    }
};

// ------------------------------------------------------------ scalar math

__device__ inline float mm_sqrt(float x) { return sqrtf(x); }
__device__ inline double mm_sqrt(double x) { return sqrt(x); }
// x^(4/3) for x >= eps > 0 (Manning)
__device__ inline float pow43(float x) { return x * cbrtf(x); }
__device__ inline double pow43(double x) { return x * cbrt(x); }
__device__ inline float mm_pow(float x, float y) { return powf(x, y); }
__device__ inline double mm_pow(double x, double y) { return pow(x, y); }
__device__ inline bool mm_finite(float x) { return isfinite(x); }
__device__ inline bool mm_finite(double x) { return isfinite(x); }

// minmod limiter: 0 unless both slopes share a sign, else the smaller one.
template <typename T> __device__ inline T minmod(T a, T b) {
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

// HLL flux with wave-speed bounds sL <= sR.
template <typename T> __device__ inline T hll(T UL, T UR, T FL, T FR, T sL, T sR) {
    if (sL >= T(0)) return FL;
    if (sR <= T(0)) return FR;
    return ((sR * FL - sL * FR) + (sL * sR) * (UR - UL)) / (sR - sL);
}

// wet test with FP64 semantics: (double)H > eps
__device__ inline bool is_wet(float H, const SweConst &c) { return H > c.eps_f; }
__device__ inline bool is_wet(double H, const SweConst &c) { return H > c.eps; }

// Even extension of index i onto [0, n); sgn = -1 after an odd number of reflections.
// Ghost index of i for the boundaries below 0 (lo_open) and at n (hi_open):
// a wall mirrors (the normal momentum's sign flips on every reflection), an
// open side repeats its boundary cell.  Walls on both sides give the
// 2n-periodic even extension.  (The loop ends within a few turns for the
// stencil's reach; the bound only guards it.)
__device__ inline int ext_index(int i, int n, int lo_open, int hi_open, int &sgn) {
    int s = 1;
    for (int it = 0; it < 64; ++it) {
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
    if (i < 0 || i >= n) i = i < 0 ? 0 : n - 1;   // never outside the grid
    sgn = s;
    return i;
}

template <typename T> struct K {  // step constants in the state precision
    T g, eps, coef, cjh, ksh, A_J, m_exp, sm1, d50, neg_tol;
    T dt, dtdx, hdt, c4, cb, dHs;
    T hdtc, dtc;  // FP32: dt/2 g/(2h) and dt g/(2h), the force terms' factors (unused in FP64)
};

template <typename T> struct Ar;  // precision-specific arithmetic (below)

// Grass discharge (Eq. 3) gated by the Shamov velocity (Eq. 5, written as
// |v|^6 > C_Sh^6 d50^2 H); A_J constant or from Eq. 4.
template <typename T, bool GEN = true>
__device__ inline void grass(const SweConst &c, const K<T> &k, bool wet, T H, T ajn, T vx, T vy,
                             T &Jx, T &Jy, T &Ja) {
    Jx = T(0); Jy = T(0); Ja = T(0);
    if (!c.sediment_on || !wet) return;
    T s2 = vx * vx + vy * vy;
    if (!(s2 * s2 * s2 > k.ksh * H)) return;
    // GEN = false compiles only the default laws (constant A_J, m = 2)
    T AJ = (GEN && c.aj_mode == 1) ? ajn / ((k.sm1 * mm_sqrt(k.g * H)) * k.d50) : k.A_J;
    T vm = (!GEN || c.m_is_2) ? s2 : mm_pow(s2, T(0.5) * k.m_exp);
    Ar<T>::scale2(AJ, vx, vy, vm, Jx, Jy);
    Ja = (AJ * vm) * mm_sqrt(s2);
}

// Free-surface difference eta_p' - eta_m' across a cell on one axis, for the
// pressure + bed-slope force per unit mass -(g/2h) (eta_p' - eta_m') * ratio
// (K2 / K5; ratio = stage depth / H^n: 1 at t_n, H^{n+1/2}/H^n = 1/A at the
// half step), where a dry neighbour whose bed is at or above the cell's level
// ec counts as a wall (eta' = ec).
template <typename T>
__device__ inline T axis_diff(T ec, T eta_p, T b_p, bool wet_p, T eta_m, T b_m, bool wet_m) {
    T ep = (!wet_p && b_p >= ec) ? ec : eta_p;
    T em = (!wet_m && b_m >= ec) ? ec : eta_m;
    return ep - em;
}

template <typename T> __device__ inline unsigned long long max_bits(T x);
template <> __device__ inline unsigned long long max_bits<float>(float x) { return (unsigned long long)__float_as_uint(x); }
template <> __device__ inline unsigned long long max_bits<double>(double x) { return (unsigned long long)__double_as_longlong(x); }

template <typename T> __device__ inline T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { T w = __shfl_xor_sync(0xffffffffu, v, o); v = w > v ? w : v; }
    return v;
}
__device__ inline int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T> __device__ inline void atomic_max_acc(unsigned long long *a, T v);
template <> __device__ inline void atomic_max_acc<float>(unsigned long long *a, float v) {
    atomicMax(a, (unsigned long long)__float_as_uint(v));
}
template <> __device__ inline void atomic_max_acc<double>(unsigned long long *a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// --------------------------------------------------------- block epilogue

template <typename T, int BW>
__device__ inline void block_finish(int cnt, T m0, T m1, T m2, unsigned st, int tile,
                                    int *census_out, SweDev *dev, int count_active) {
    __shared__ int s_cnt[BW / 32];
    __shared__ T s_m[3][BW / 32];
    __shared__ unsigned s_st[BW / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    cnt = warp_sum(cnt);
    m0 = warp_max(m0); m1 = warp_max(m1); m2 = warp_max(m2);
    st = __reduce_or_sync(0xffffffffu, st);
    if (lane == 0) { s_cnt[wid] = cnt; s_m[0][wid] = m0; s_m[1][wid] = m1; s_m[2][wid] = m2; s_st[wid] = st; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tc = 0; T a = T(0), b = T(0), c = T(0); unsigned s = 0;
        for (int w = 0; w < BW / 32; ++w) {
            tc += s_cnt[w];
            a = s_m[0][w] > a ? s_m[0][w] : a;
            b = s_m[1][w] > b ? s_m[1][w] : b;
            c = s_m[2][w] > c ? s_m[2][w] : c;
            s |= s_st[w];
        }
        census_out[tile] = tc;
        if (a > T(0)) atomic_max_acc<T>(&dev->acc[0], a);
        if (b > T(0)) atomic_max_acc<T>(&dev->acc[1], b);
        if (c > T(0)) atomic_max_acc<T>(&dev->acc[2], c);
        if (s) atomicOr(&dev->status, s);
        if (count_active) atomicAdd(&dev->active_tiles, 1);
    }
}

// Per-cell terms of Eq. 7 and the census for a new state value.
template <typename T>
__device__ inline void cell_epilogue(const SweConst &c, const K<T> &k, T hn, T hun, T hvn, T bn, T ajn,
                                     bool src, int &cnt, T &m0, T &m1, T &m2, unsigned &st) {
    bool wet = is_wet(hn, c);
    cnt += (wet || src) ? 1 : 0;
    if (wet) {
        T u = hun / hn, v = hvn / hn;
        T va = mm_sqrt(u * u + v * v);
        T cs = va + mm_sqrt(k.g * hn);
        m0 = va > m0 ? va : m0;
        m1 = cs > m1 ? cs : m1;
        T jx, jy, ja;
        grass<T>(c, k, true, hn, ajn, u, v, jx, jy, ja);
        m2 = ja > m2 ? ja : m2;
    }
    if (!(hn >= -k.neg_tol)) st |= 2u;
    if (!mm_finite(hn) || !mm_finite(bn) || !mm_finite(hun) || !mm_finite(hvn)) st |= 1u;
}

// Per-step coefficients; coherent = read through L2 (volatile), for a
// persistent launch whose other blocks rewrote them.
struct StepCoef { double dt, dtdx, hdt, c4, cb, dHs; };
__device__ inline StepCoef step_coef(const SweDev *dev, bool coherent) {
    StepCoef r;
    if (coherent) {
        const volatile SweDev *v = dev;
        r.dt = v->dt; r.dtdx = v->dtdx; r.hdt = v->hdt; r.c4 = v->c4; r.cb = v->cb; r.dHs = v->dHs;
    } else {
        r.dt = dev->dt; r.dtdx = dev->dtdx; r.hdt = dev->hdt; r.c4 = dev->c4; r.cb = dev->cb; r.dHs = dev->dHs;
    }
    return r;
}

template <typename T> __device__ inline K<T> load_k(const SweConst &c, const SweDev *dev, bool coherent = false);
template <> __device__ inline K<double> load_k<double>(const SweConst &c, const SweDev *dev, bool coherent) {
    K<double> k;
    k.g = c.g; k.eps = c.eps; k.coef = c.coef; k.cjh = c.cjh; k.ksh = c.ksh;
    k.A_J = c.A_J; k.m_exp = c.m_exp; k.sm1 = c.sm1; k.d50 = c.d50; k.neg_tol = c.neg_tol;
    const StepCoef r = step_coef(dev, coherent);
    k.dt = r.dt; k.dtdx = r.dtdx; k.hdt = r.hdt; k.c4 = r.c4; k.cb = r.cb; k.dHs = r.dHs;
    k.hdtc = 0.0; k.dtc = 0.0;
    return k;
}
// FP32: the model constants come pre-rounded in the kernel parameters (so
// they can stay in the constant bank); the per-step ones from the bookkeeping.
template <> __device__ inline K<float> load_k<float>(const SweConst &c, const SweDev *dev, bool coherent) {
    K<float> k;
    k.g = c.f.g; k.eps = c.f.eps; k.coef = c.f.coef; k.cjh = c.f.cjh; k.ksh = c.f.ksh;
    k.A_J = c.f.A_J; k.m_exp = c.f.m_exp; k.sm1 = c.f.sm1; k.d50 = c.f.d50; k.neg_tol = c.f.neg_tol;
    const StepCoef r = step_coef(dev, coherent);
    k.dt = (float)r.dt;
    k.dtdx = k.dt * c.f.inv_dx; k.hdt = 0.5f * k.dt; k.c4 = k.dt * c.f.inv_4dx;
    k.cb = k.dt * c.f.inv_dxp; k.dHs = (float)r.dHs;
    k.hdtc = k.hdt * c.f.coef; k.dtc = k.dt * c.f.coef;
    return k;
}

// ---------------------------------------------------------- step kernel

// Fast even extension for row indices within one reflection of the grid;
// falls back to the general form for grids thinner than the stencil.
__device__ inline int reflect(int i, int n, int lo_open, int hi_open, int &sgn) {
    if (i >= 0 && i < n) { sgn = 1; return i; }
    return ext_index(i, n, lo_open, hi_open, sgn);
}

// Precision-specific arithmetic.  FP32 (production): hardware reciprocal,
// exp2/log2 power, a branch-free limiter and one reciprocal shared by the
// three HLL fluxes.  FP64 (parity): IEEE division, cbrt and the oracle's
// operation order.
// HLL fluxes of mass and both momenta sharing the bounds sL <= sR.
template <typename T>
__device__ inline void hll3(T HL, T HR, T uL, T uR, T wxL, T wxR, T wyL, T wyR, T sL, T sR,
                            T &Fm, T &Fx, T &Fy) {
    T UxL = HL * wxL, UxR = HR * wxR, UyL = HL * wyL, UyR = HR * wyR;
    Fm = hll(HL, HR, HL * uL, HR * uR, sL, sR);
    Fx = hll(UxL, UxR, UxL * uL, UxR * uR, sL, sR);
    Fy = hll(UyL, UyR, UyL * uL, UyR * uR, sL, sR);
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <typename T> struct Ar;
template <> struct Ar<double> {
    __device__ static inline void div2(double a, double b, double d, double &x, double &y) { x = a / d; y = b / d; }
    __device__ static inline double minmod(double a, double b) { return swe_impl::minmod(a, b); }
    // Manning coefficient g n^2 / H^(4/3)
    __device__ static inline double manning(double gn2, double H) { return gn2 / (H * cbrt(H)); }
    // K4 particle depth H / A; the K5 depth ratio H^{n+1/2} / H^n
    __device__ static inline double depth(double H, double A, double &iA) { iA = 0.0; return H / A; }
    __device__ static inline double ratio(double hc, double Hc, double) { return hc / Hc; }
    // K4 numerator v + dt/2 a^n and K6 numerator v + dt a^{n+1/2}, from the
    // free-surface difference d, in the oracle's order of operations
    __device__ static inline double k4_num(const K<double> &k, double u, double d) {
        return u + k.hdt * (-(k.coef * d) * 1.0);
    }
    __device__ static inline double k6_factor(const K<double> &, double ratio) { return ratio; }
    __device__ static inline double k6_num(const K<double> &k, double u, double d, double ratio) {
        return u + k.dt * (-(k.coef * d) * ratio);
    }
    // both axes at once (x, y): the K4 / K6 velocities, the Grass load
    // components
    __device__ static inline void k4_vel(const K<double> &k, double u, double v, double dx, double dy, double den,
                                         double &x, double &y) {
        div2(k4_num(k, u, dx), k4_num(k, v, dy), den, x, y);
    }
    __device__ static inline void k6_vel(const K<double> &k, double u, double v, double dx, double dy, double q,
                                         double den, double &x, double &y) {
        div2(k6_num(k, u, dx, q), k6_num(k, v, dy, q), den, x, y);
    }
    __device__ static inline void scale2(double a, double vx, double vy, double vm, double &x, double &y) {
        x = (a * vx) * vm;
        y = (a * vy) * vm;
    }

    // HLL fluxes of one face from the hydrostatic face depths, the normal
    // velocities and celerities, in the oracle's order of operations
    __device__ static inline void hll_face(double HL, double HR, double uL, double uR, double cL, double cR,
                                           double wxL, double wxR, double wyL, double wyR,
                                           double &Fm, double &Fx, double &Fy) {
        const double aL = uL - cL, aR = uR - cR, pL = uL + cL, pR = uR + cR;
        const double sL = aL < aR ? aL : aR, sR = pL > pR ? pL : pR;
        hll3<double>(HL, HR, uL, uR, wxL, wxR, wyL, wyR, sL, sR, Fm, Fx, Fy);
    }
};
template <> struct Ar<float> {
    // Pairs of the same operation on the x and y components run as one packed
    // FP32x2 instruction (each lane rounds as the scalar operation would): the
    // step is bound by instruction issue, and a packed instruction takes one
    // issue slot for two results.
    __device__ static inline void div2(float a, float b, float d, float &x, float &y) {
        const float r = 1.0f / d;
        const float2 q = __fmul2_rn(make_float2(a, b), make_float2(r, r));
        x = q.x; y = q.y;
    }
    // the median of (a, b, 0): 0 unless a and b share a sign, else the one
    // nearer zero (four min/max, no branch)
    __device__ static inline float minmod(float a, float b) {
        return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.f));
    }
    // g n^2 H^(-4/3) through exp2/log2 (no reciprocal)
    __device__ static inline float manning(float gn2, float H) { return gn2 * exp2f(-1.33333333f * log2f(H)); }
    // the reciprocal of A is kept: it is the K5 depth ratio of the same cell.
    // Written as an explicit rcp.approx and a rounded product, so that no
    // compiled copy of the sweep rewrites it (into a division, say) and the
    // value carried to the next position is the one every copy would form.
    __device__ static inline float depth(float H, float A, float &iA) {
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iA) : "f"(A));
        return __fmul_rn(H, iA);
    }
    __device__ static inline float ratio(float, float, float iA) { return iA; }
    // the same numerators with the constant factors folded: one FMA per axis
    __device__ static inline float k4_num(const K<float> &k, float u, float d) { return fmaf(-k.hdtc, d, u); }
    __device__ static inline float k6_factor(const K<float> &k, float ratio) { return k.dtc * ratio; }
    __device__ static inline float k6_num(const K<float> &, float u, float d, float q) { return fmaf(-q, d, u); }
    __device__ static inline void k4_vel(const K<float> &k, float u, float v, float dx, float dy, float den,
                                         float &x, float &y) {
        const float2 n = __ffma2_rn(make_float2(-k.hdtc, -k.hdtc), make_float2(dx, dy), make_float2(u, v));
        div2(n.x, n.y, den, x, y);
    }
    __device__ static inline void k6_vel(const K<float> &, float u, float v, float dx, float dy, float q,
                                         float den, float &x, float &y) {
        const float2 n = __ffma2_rn(make_float2(-q, -q), make_float2(dx, dy), make_float2(u, v));
        div2(n.x, n.y, den, x, y);
    }
    __device__ static inline void scale2(float a, float vx, float vy, float vm, float &x, float &y) {
        const float2 j = __fmul2_rn(__fmul2_rn(make_float2(a, a), make_float2(vx, vy)), make_float2(vm, vm));
        x = j.x; y = j.y;
    }
    // HLL with the bounds clamped to sL <= 0 <= sR: the same flux in all three
    // cases (sL >= 0 gives F_L, sR <= 0 gives F_R), so no branch.  With the
    // advective fluxes F = U u it is F = U_L alpha + U_R beta,
    // alpha = (sR uL - sL sR)/(sR - sL), beta = (sL sR - sL uR)/(sR - sL);
    // mirrored states (a wall) give beta = -alpha exactly: zero mass flux.
    // sL = sR = 0 only when both sides are at rest with no depth: zero flux.
    __device__ static inline void hll_face(float HL, float HR, float uL, float uR, float cL, float cR,
                                           float wxL, float wxR, float wyL, float wyR,
                                           float &Fm, float &Fx, float &Fy) {
        const float sL = min3f(uL - cL, uR - cR, 0.f);
        const float sR = max3f(uL + cL, uR + cR, 0.f);
        const float inv = 1.0f / fmaxf(sR - sL, 1e-30f);
        const float a = sR * inv, bm = sL * inv, cc = a * sL;
        const float al = fmaf(a, uL, -cc), be = fmaf(-bm, uR, cc);
        // rounded products and sum written out: no contraction choice is left
        // to the compiler, so every compiled copy of the sweep agrees bit for bit
        const float P = __fmul_rn(HL, al), Q = __fmul_rn(HR, be);
        Fm = __fadd_rn(P, Q);
        Fx = fmaf(P, wxL, __fmul_rn(Q, wxR));
        Fy = fmaf(P, wyL, __fmul_rn(Q, wyR));
    }
};

// Face states of one cell along one axis from its two neighbours: limited
// slope sigma = minmod(q - q_m, q_p - q); minus-side face value q - sigma/2,
// plus-side face value q + sigma/2.
template <typename T> __device__ inline void cell_faces(T qm, T q, T qp, T &lo, T &hi) {
    const T sg = Ar<T>::minmod(q - qm, qp - q);
    hi = q + T(0.5) * sg;
    lo = q - T(0.5) * sg;
}

// Fluxes through a face with at least one wet cell, from reconstructed states
// (L: H, eta, un, wx, wy of the minus cell's plus face; R: the plus cell's
// minus face), the wet flags, the cells' normal transport velocity, Grass
// load and bed.  (A face between two dry cells carries exactly zero flux.)
template <typename T>
__device__ inline void face_flux2(const SweConst &c, const K<T> &k, const T L[5], const T R[5],
                                  bool wet_c, bool wet_e, T un_c, T un_e, T Jn_c, T Jn_e, T Ja_c, T Ja_e,
                                  T b_c, T b_e, T &Fm, T &Fx, T &Fy, T &Fj) {
    const T bL = L[1] - L[0], bR = R[1] - R[0];
    const T bf = bL > bR ? bL : bR;
    T HL = L[1] - bf, HR = R[1] - bf;
    if (!(HL > T(0))) HL = T(0);
    if (!(HR > T(0))) HR = T(0);
    const T cL = wet_c ? mm_sqrt(k.g * HL) : T(0);
    const T cR = wet_e ? mm_sqrt(k.g * HR) : T(0);
    Ar<T>::hll_face(HL, HR, L[2], R[2], cL, cR, L[3], R[3], L[4], R[4], Fm, Fx, Fy);
    Fj = T(0);
    if (c.sediment_on) {
        const T su = un_c + un_e;
        const T Jadv = su > T(0) ? Jn_c : (su < T(0) ? Jn_e : T(0));
        Fj = Jadv - (k.cjh * (Ja_c + Ja_e)) * (b_e - b_c);
    }
}

// Per-cell terms of Eq. 7 and the census for a new state value.  cnt holds
// the census count in its low 24 bits and the status bits from bit 24 (one
// register for both).
template <typename T, bool GEN = true>
__device__ inline void cell_epilogue2(const SweConst &c, const K<T> &k, T hn, T hun, T hvn, T bn, T ajn,
                                      bool src, unsigned &cnt, T &m0, T &m1, T &m2, T epsw) {
    const bool wet = hn > epsw;
    cnt += (wet || src) ? 1u : 0u;
    if (wet) {
        T u, v;
        Ar<T>::div2(hun, hvn, hn, u, v);
        const T va = mm_sqrt(u * u + v * v);
        const T cs = va + mm_sqrt(k.g * hn);
        m0 = va > m0 ? va : m0;
        m1 = cs > m1 ? cs : m1;
        T jx, jy, ja;
        grass<T, GEN>(c, k, true, hn, ajn, u, v, jx, jy, ja);
        m2 = ja > m2 ? ja : m2;
    }
    if (!(hn >= -k.neg_tol)) cnt |= 2u << 24;
    if (!mm_finite(((hn + bn) + hun) + hvn)) cnt |= 1u << 24;
}

// Shared-memory rings; each row is padded by 2 entries on both sides so the
// edge threads' out-of-block neighbour reads stay in bounds (those threads'
// results are never used).  Quantities read together are stored together
// (V2: 8 B in FP32, V4: 16 B), so one shared-memory instruction moves them.
template <typename T> struct alignas(2 * sizeof(T)) V2 { T x, y; };
template <typename T> struct alignas(4 * sizeof(T) < 16 ? 4 * sizeof(T) : 16) V4 { T a, b, c, d; };

template <typename T, int BW> struct StepSmem {
    static constexpr int RW = BW + 4;
    V2<T> hb[8][RW];                    // state (H, b), rows s-7..s
    T u[4][RW];                         // cell velocity u^n, rows s-3..s (v^n: registers)
    V2<T> hj[4][RW];                    // (K4 particle depth H^{n+1/2}, Grass |J|)
    V2<T> U[4][RW], W[4][RW], J[4][RW]; // K4 transport velocity, K6 end velocity, Grass load (x, y)
    V4<T> qw[2][RW];                    // x-direction minus-face states (H, eta, ux, wx) ...
    T qy[2][RW];                        // ... and wy
    V4<T> xf[2][RW];                    // x-face fluxes (face t|t+1): mass, x-mom, y-mom, Exner
};

template <typename T> __device__ inline T tab(const void *p, int i) { return reinterpret_cast<const T *>(p)[i]; }

// The sweep of one block.  pos<P>(s) runs the pipeline at sweep position s;
// the sweep advances two positions per loop iteration, P = s mod 2 is known
// at compile time and every ring row is a per-iteration bank base plus a
// constant offset:
//   load row s | K4 depth, row s-1 | K2 K4 K5 K6 + Grass, row s-2 |
//   K8 update, row s-5 | x-faces, row s-4 | per-cell limited face states,
//   row s-3, and the y-face (s-4|s-3).
// Every read of a neighbour column refers to a row finished at an earlier
// position, so one __syncthreads per position suffices.
template <typename T, int BW, bool COHERENT, int SRC, bool GEN> struct Sweep {
    static constexpr int RW = StepSmem<T, BW>::RW;
    StepSmem<T, BW> &S;
    const SweConst &c;
    const SweBufs &B;
    const K<T> &k;
    const void *in;
    void *out;
    int y0, y1, x, xx, mcol, o;
    T sxT;
    bool out_lane;
    int gn2_row, aj_row;
    T gn2, ajo, aj_out;
    T qE[5], qN[5];
    T G1[4], dG[4];         // the last y-face fluxes, and their difference to the ones before (K8's y term)
    T vA[2], vB[2];         // own-column v^n of rows s-P, s-P+1 and of the two rows before
    T iA[2];                // own-column 1/A of K4 (FP32), by the parity of the position that formed it
    unsigned cnt;           // census count (low 24 bits) | status bits << 24
    T m0, m1, m2;
    T aH, aHu, aHv, ab, bH, bHu, bHv, bb0;
    int asy, bsy;
    V2<T> *hbk[4];          // 2-row banks of the 8-row (H, b) ring holding rows 2m-2j, 2m-2j+1
    int q4c, q4o;           // offsets of the current / previous 2-row bank of the 4-row rings
    T epsw;                 // the wet threshold (is_wet), held in a register in the persistent launch
    __device__ __forceinline__ bool wet_cell(T H) const { return H > epsw; }

    // Ring row r lives in slot r mod 8 (H, b) or r mod 4 (the 4-row rings).
    // For a sweep position s = 2m + P, row s-D = 2m + d with d = P - D, i.e.
    // in the bank of rows 2(m + fd), 2(m + fd) + 1, fd = floor(d / 2).
    template <int P, int D> struct FD {
        static constexpr int v = (P - D) >= 0 ? (P - D) / 2 : -((1 - (P - D)) / 2);
    };
    template <int P, int D> __device__ __forceinline__ V2<T> *HB() const {
        return hbk[-FD<P, D>::v] + ((P - D) & 1) * RW;
    }
    template <int P, int D, typename E> __device__ __forceinline__ E *q4(E (&a)[4][RW]) const {
        return &a[0][0] + ((FD<P, D>::v & 1) ? q4o : q4c) + ((P - D) & 1) * RW;
    }
    __device__ __forceinline__ void set_banks(int s) {
        const int m = s >> 1;
#pragma unroll
        for (int j = 0; j < 4; ++j) hbk[j] = &S.hb[2 * ((m - j) & 3)][0];
        q4c = 2 * RW * (m & 1);
        q4o = 2 * RW * ((m & 1) ^ 1);
        vB[0] = vA[0]; vB[1] = vA[1];
    }

    __device__ Sweep(StepSmem<T, BW> &S_, const SweConst &c_, const SweBufs &B_, const K<T> &k_)
        : S(S_), c(c_), B(B_), k(k_) {}

    __device__ __forceinline__ void load_cell(long long kk, T &H, T &Hu, T &Hv, T &b) const {
        if (COHERENT) CellIO<T>::load_cg(in, kk, H, Hu, Hv, b);
        else CellIO<T>::load(in, kk, H, Hu, Hv, b);
    }

    // FULL: every stage's row is inside the strip (s in [y0 + 5, y1 + 3]), so
    // the row-range tests are dropped (the same arithmetic, fewer branches).
    template <int P, bool FULL> __device__ __forceinline__ void pos(int s) {
        static_assert(P == 0 || P == 1, "two positions per bank");
        constexpr int PM3_2 = (P + 1) & 1, PM4_2 = P & 1, PM5_2 = (P + 1) & 1;
        T v_s = T(0);
        // ---------------- load row s (ghost rows by even extension)
        if (FULL || (s >= y0 - 4 && s <= y1 + 3)) {
            const T H = aH, Hu = aHu, Hv = aHv, bb = ab;
            const T syT = T(asy);
            aH = bH; aHu = bHu; aHv = bHv; ab = bb0; asy = bsy;
            if (s + 2 <= y1 + 3) {
                const int yy = reflect(s + 2, c.ny, c.bc[2], c.bc[3], bsy);
                if (SWE_IN((long long)yy * c.nx + xx, SWE_NCELL)) load_cell((long long)yy * c.nx + xx, bH, bHu, bHv, bb0);
            }
            const bool wet = wet_cell(H);
            HB<P, 0>()[o] = V2<T>{H, bb};
            T u = T(0);
            if (wet) Ar<T>::div2(sxT * Hu, syT * Hv, H, u, v_s);
            q4<P, 0>(S.u)[o] = u;
            vA[P] = v_s;
        }
        // ---------------- K4 (part): particle depth at t_{n+1/2}, row s-1
        if (FULL || (s - 1 >= y0 - 3 && s - 1 <= y1 + 2)) {
            const T A = T(1) + k.c4 * ((q4<P, 1>(S.u)[o + 1] - q4<P, 1>(S.u)[o - 1]) + (v_s - vB[P]));
            q4<P, 1>(S.hj)[o].x = Ar<T>::depth(HB<P, 1>()[o].x, A, iA[P]);
        }
        // ---------------- K2, K4, K5, K6 and Grass load, row s-2
        if (FULL || (s - 2 >= y0 - 2 && s - 2 <= y1 + 1)) {
            const int r = s - 2;
            const V2<T> C = HB<P, 2>()[o];
            const T Hc = C.x;
            const bool wet = wet_cell(Hc);
            T vtx = T(0), vty = T(0), wxv = T(0), wyv = T(0), jx = T(0), jy = T(0), ja = T(0);
            if (wet) {
                const T bc = C.y, u = q4<P, 2>(S.u)[o], v = vB[P];
                int sy;
                const int my = reflect(r, c.ny, c.bc[2], c.bc[3], sy) >> c.man_shift;
                if (my != gn2_row && SWE_IN(my * c.man_w + mcol, SWE_NMAN)) {
                    gn2_row = my;
                    gn2 = tab<T>(B.gn2, my * c.man_w + mcol);
                    if (GEN && c.aj_mode == 1) ajo = tab<T>(B.ajn, my * c.man_w + mcol);
                }
                const V2<T> E = HB<P, 2>()[o + 1], Wc = HB<P, 2>()[o - 1];
                const V2<T> N = HB<P, 1>()[o], Sc = HB<P, 3>()[o];
                const T HE = E.x, bE = E.y, HW = Wc.x, bW = Wc.y, HN = N.x, bN = N.y, HS = Sc.x, bS = Sc.y;
                const bool wE = wet_cell(HE), wW = wet_cell(HW), wN = wet_cell(HN), wS = wet_cell(HS);
                // K2: forces at t_n (free-surface differences per axis)
                const T ec = Hc + bc;
                const T dx2 = axis_diff<T>(ec, HE + bE, bE, wE, HW + bW, bW, wW);
                const T dy2 = axis_diff<T>(ec, HN + bN, bN, wN, HS + bS, bS, wS);
                // K4: predictor velocity, point-implicit Manning at |v^n|
                const T cf = Ar<T>::manning(gn2, Hc);
                const T va = mm_sqrt(u * u + v * v);
                const T den = T(1) + k.hdt * (cf * va);
                Ar<T>::k4_vel(k, u, v, dx2, dy2, den, vtx, vty);
                // K5: forces at t_{n+1/2} from H^{n+1/2} + b, wet flags of t_n
                const T hc = q4<P, 2>(S.hj)[o].x, ech = hc + bc;
                const T hE = q4<P, 2>(S.hj)[o + 1].x, hW = q4<P, 2>(S.hj)[o - 1].x;
                const T hN = q4<P, 1>(S.hj)[o].x, hS = q4<P, 3>(S.hj)[o].x;
                const T q = Ar<T>::k6_factor(k, Ar<T>::ratio(hc, Hc, iA[P ^ 1]));
                const T dx5 = axis_diff<T>(ech, hE + bE, bE, wE, hW + bW, bW, wW);
                const T dy5 = axis_diff<T>(ech, hN + bN, bN, wN, hS + bS, bS, wS);
                // K6: corrector (Lagrangian end) velocity, Manning at |vt|
                const T vat = mm_sqrt(vtx * vtx + vty * vty);
                const T den2 = T(1) + k.dt * (cf * vat);
                Ar<T>::k6_vel(k, u, v, dx5, dy5, q, den2, wxv, wyv);
                grass<T, GEN>(c, k, true, Hc, ajo, vtx, vty, jx, jy, ja);
            }
            q4<P, 2>(S.U)[o] = V2<T>{vtx, vty};
            q4<P, 2>(S.W)[o] = V2<T>{wxv, wyv};
            q4<P, 2>(S.J)[o] = V2<T>{jx, jy};
            q4<P, 2>(S.hj)[o].y = ja;
        }
        // ---------------- K8: update row s-5
        if ((FULL || (s - 5 >= y0 && s - 5 <= y1 - 1)) && out_lane) {
            const int r = s - 5;
            const V2<T> C = HB<P, 5>()[o];
            const T Hc = C.x, bc = C.y;
            bool src = false;
            if ((SRC & SWE_SRC_INFLOW) && c.nsrc > 0 && SWE_IN(r + 1, c.ny + 1))
                for (int q = B.src_rowptr[r]; q < B.src_rowptr[r + 1]; ++q)
                    if (SWE_IN(q, c.nsrc)) src |= (B.src_x[q] == x);
            const V4<T> f = S.xf[PM5_2][o], fw = S.xf[PM5_2][o - 1];
            const V2<T> w = q4<P, 5>(S.W)[o];
            T hn = Hc - k.dtdx * ((f.a - fw.a) + dG[0]);
            // the source increment is read only for the few source cells (not
            // held in a register through the sweep)
            if (src) hn = hn + T(COHERENT ? ((const volatile SweDev *)B.dev)->dHs : B.dev->dHs);
            if ((SRC & SWE_SRC_FIELDS) && c.has_rain && SWE_IN((long long)r * c.nx + x, SWE_NCELL))
                hn = hn + k.dt * tab<T>(B.rain, (long long)r * c.nx + x);
            T hun = Hc * w.x - k.dtdx * ((f.b - fw.b) + dG[1]);
            T hvn = Hc * w.y - k.dtdx * ((f.c - fw.c) + dG[2]);
            if ((SRC & SWE_SRC_FIELDS) && c.has_beta && SWE_IN((long long)r * c.nx + x, SWE_NCELL)) {
                // infiltration: at most the water present, with its share of momentum
                T loss = k.dt * tab<T>(B.beta, (long long)r * c.nx + x);
                if (loss > hn) loss = hn > T(0) ? hn : T(0);
                if (loss > T(0)) {
                    const T ratio = (hn - loss) / hn;
                    hn = hn - loss;
                    hun = hun * ratio;
                    hvn = hvn * ratio;
                }
            }
            if (!wet_cell(hn)) { hun = T(0); hvn = T(0); }
            const T bn = bc - k.cb * ((f.d - fw.d) + dG[3]);
            if (SWE_IN((long long)r * c.nx + x, SWE_NCELL)) CellIO<T>::store(out, (long long)r * c.nx + x, hn, hun, hvn, bn);
            if (GEN && c.aj_mode == 1 && (r >> c.man_shift) != aj_row && SWE_IN((r >> c.man_shift) * c.man_w + mcol, SWE_NMAN)) {
                aj_row = r >> c.man_shift;
                aj_out = tab<T>(B.ajn, aj_row * c.man_w + mcol);
            }
            cell_epilogue2<T, GEN>(c, k, hn, hun, hvn, bn, aj_out, src, cnt, m0, m1, m2, epsw);
        }
        // ---------------- x-faces of row s-4 (face t|t+1): own plus-face state
        // (from the previous position) and the minus-face state of t+1
        if (FULL || (s - 4 >= y0 && s - 4 <= y1 - 1)) {
            const V2<T> C = HB<P, 4>()[o], E = HB<P, 4>()[o + 1];
            const bool wc = wet_cell(C.x), we = wet_cell(E.x);
            T f0 = T(0), f1 = T(0), f2 = T(0), f3 = T(0);
            if (wc || we) {
                const V4<T> q = S.qw[PM4_2][o + 1];
                const T R[5] = {q.a, q.b, q.c, q.d, S.qy[PM4_2][o + 1]};
                const V2<T> Uc = q4<P, 4>(S.U)[o], Ue = q4<P, 4>(S.U)[o + 1];
                const V2<T> Jc = q4<P, 4>(S.J)[o], Je = q4<P, 4>(S.J)[o + 1];
                face_flux2<T>(c, k, qE, R, wc, we, Uc.x, Ue.x, Jc.x, Je.x, q4<P, 4>(S.hj)[o].y,
                              q4<P, 4>(S.hj)[o + 1].y, C.y, E.y, f0, f1, f2, f3);
            }
            S.xf[PM4_2][o] = V4<T>{f0, f1, f2, f3};
        }
        // ---------------- per-cell limited face states (K7 reconstruction), row s-3,
        // and the y-face (s-4 | s-3)
        if (FULL || (s - 3 >= y0 - 1 && s - 3 <= y1)) {
            const V2<T> C = HB<P, 3>()[o], Wc = HB<P, 3>()[o - 1], E = HB<P, 3>()[o + 1];
            const V2<T> Sc = HB<P, 4>()[o], N = HB<P, 2>()[o];
            const T H0 = C.x, b0 = C.y, Hm = Wc.x, Hp = E.x, Hs = Sc.x, Hn = N.x;
            const bool w0 = wet_cell(H0), ws = wet_cell(Hs);
            const bool need = w0 || ws || wet_cell(Hm) || wet_cell(Hp) || wet_cell(Hn);
            T G[4] = {T(0), T(0), T(0), T(0)};
            if (need) {
                const T e0 = H0 + b0;
                T lo, hi, lo2;
                // x direction: (H, eta, ux, wx, wy) at t-1, t, t+1
                const V2<T> U3m = q4<P, 3>(S.U)[o - 1], U3 = q4<P, 3>(S.U)[o], U3p = q4<P, 3>(S.U)[o + 1];
                const V2<T> W3m = q4<P, 3>(S.W)[o - 1], W3 = q4<P, 3>(S.W)[o], W3p = q4<P, 3>(S.W)[o + 1];
                cell_faces<T>(Hm, H0, Hp, lo, hi); qE[0] = hi;
                cell_faces<T>(Hm + Wc.y, e0, Hp + E.y, lo2, hi); qE[1] = hi;
                T lo3, lo4;
                cell_faces<T>(U3m.x, U3.x, U3p.x, lo3, hi); qE[2] = hi;
                cell_faces<T>(W3m.x, W3.x, W3p.x, lo4, hi); qE[3] = hi;
                S.qw[PM3_2][o] = V4<T>{lo, lo2, lo3, lo4};
                cell_faces<T>(W3m.y, W3.y, W3p.y, lo, hi); S.qy[PM3_2][o] = lo; qE[4] = hi;
                // y direction: (H, eta, uy, wx, wy) at rows r-1, r, r+1 (own column)
                const V2<T> U4 = q4<P, 4>(S.U)[o], U2 = q4<P, 2>(S.U)[o];
                const V2<T> W4 = q4<P, 4>(S.W)[o], W2 = q4<P, 2>(S.W)[o];
                T qS[5], hn5[5];
                cell_faces<T>(Hs, H0, Hn, qS[0], hn5[0]);
                cell_faces<T>(Hs + Sc.y, e0, Hn + N.y, qS[1], hn5[1]);
                cell_faces<T>(U4.y, U3.y, U2.y, qS[2], hn5[2]);
                cell_faces<T>(W4.x, W3.x, W2.x, qS[3], hn5[3]);
                cell_faces<T>(W4.y, W3.y, W2.y, qS[4], hn5[4]);
                if ((FULL || s - 3 >= y0) && (ws || w0))
                    face_flux2<T>(c, k, qN, qS, ws, w0, U4.y, U3.y, q4<P, 4>(S.J)[o].y, q4<P, 3>(S.J)[o].y,
                                  q4<P, 4>(S.hj)[o].y, q4<P, 3>(S.hj)[o].y, Sc.y, b0, G[0], G[1], G[2], G[3]);
#pragma unroll
                for (int q = 0; q < 5; ++q) qN[q] = hn5[q];
            }
            if (FULL || s - 3 >= y0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) { dG[q] = G[q] - G1[q]; G1[q] = G[q]; }
            }
        }
        __syncthreads();
    }
};

// One step of one block (column band bx, row strip by).  COHERENT selects
// L2-coherent reads of the state, census and bookkeeping, needed when other
// blocks of the same (persistent) launch rewrote them since its start.
// SRC compiles in the source terms of the update (SWE_SRC_INFLOW: the inflow
// hydrograph; SWE_SRC_FIELDS: the rain and infiltration fields), GEN
// the general transport laws (A_J from Eq. 4, m != 2); without them (not in
// use) the kernel is markedly smaller, which its instruction fetch rewards.
template <typename T, int BW, bool COHERENT, int SRC, bool GEN>
__device__ __forceinline__ void step_tile(const SweConst &c, const SweBufs &B, int bx, int by, StepSmem<T, BW> &S) {
    SweDev *dev = B.dev;
    const volatile SweDev *vdev = dev;
    if (!(COHERENT ? vdev->scheduled : dev->scheduled)) return;
    const int t = threadIdx.x;
    const int tile = by * c.tiles_x + bx;
    const long long n = COHERENT ? vdev->n : dev->n;
    const int par = (int)(n & 1);
    const void *in = par ? B.buf[1] : B.buf[0];
    void *out = par ? B.buf[0] : B.buf[1];
    const int *cen_in = par ? B.census[1] : B.census[0];
    int *cen_out = par ? B.census[0] : B.census[1];
    const int tx0 = bx * c.tw;                       // first output column
    const int y0 = by * c.th, y1 = min(y0 + c.th, c.ny);

    // ---- K1 / HGS: skip dry blocks (Sec. 3, kernel_ES rule: the block or one
    // of its four edge neighbours must hold water)
    if (c.hgs) {
        int l = bx > 0 ? bx - 1 : bx, r = bx < c.tiles_x - 1 ? bx + 1 : bx;
        int d = by > 0 ? by - 1 : by, u = by < c.tiles_y - 1 ? by + 1 : by;
        auto cen = [&](int i) {
            return SWE_IN(i, c.tiles_x * c.tiles_y) ? (COHERENT ? __ldcg(cen_in + i) : cen_in[i]) : 0;
        };
        // every count and the skip flag loaded first (one wait for memory, not
        // one per term of a short-circuit test); the skip flag was written by
        // whichever block ran this tile last
        const int k0 = cen(tile), k1 = cen(by * c.tiles_x + l), k2 = cen(by * c.tiles_x + r);
        const int k3 = cen(d * c.tiles_x + bx), k4 = cen(u * c.tiles_x + bx);
        const bool was_skipped = COHERENT ? __ldcg(B.skipped + tile) != 0 : B.skipped[tile] != 0;
        const bool active = (k0 > 0) | (k1 > 0) | (k2 > 0) | (k3 > 0) | (k4 > 0);
        if (!active) {
            if (!was_skipped) {
                int x1 = min(tx0 + c.tw, c.nx);
                for (int y = y0; y < y1; ++y)
                    for (int x = tx0 + t; x < x1; x += BW) {
                        if (!SWE_IN((long long)y * c.nx + x, SWE_NCELL)) continue;
                        if (COHERENT) CellIO<T>::copy_cg(in, out, (long long)y * c.nx + x);
                        else CellIO<T>::copy(in, out, (long long)y * c.nx + x);
                    }
            }
            if (t == 0) {
                if (!was_skipped)
                    atomicAdd(&dev->cells_copied, (unsigned long long)(min(tx0 + c.tw, c.nx) - tx0) * (y1 - y0));
                cen_out[tile] = 0;
                B.skipped[tile] = 1;
            }
            return;
        }
        if (t == 0) B.skipped[tile] = 0;
    }
    if (t == 0) atomicAdd(&dev->cells_computed, (unsigned long long)(min(tx0 + c.tw, c.nx) - tx0) * (y1 - y0));

    const K<T> k = load_k<T>(c, COHERENT ? const_cast<const SweDev *>(dev) : dev, COHERENT);
    Sweep<T, BW, COHERENT, SRC, GEN> w(S, c, B, k);
    w.in = in; w.out = out; w.y0 = y0; w.y1 = y1;
    w.x = tx0 - 4 + t;                               // this thread's column
    int sx;
    // columns more than 4 past the grid feed no output cell; clamped, their
    // ghost index stays a few reflections away even on a 1-column grid
    w.xx = reflect(min(w.x, c.nx + 3), c.nx, c.bc[0], c.bc[1], sx);
    w.sxT = T(sx);
    w.mcol = w.xx >> c.man_shift;
    w.out_lane = (t >= 4) && (t < BW - 4) && (w.x < c.nx);
    if constexpr (sizeof(T) == 4) {
        // a persistent launch reads the scenario's threshold at a block-uniform
        // parameter offset; the move keeps one register copy for the sweep
        if (COHERENT) asm volatile("mov.b32 %0, %1;" : "=f"(w.epsw) : "f"(c.eps_f));
        else w.epsw = c.eps_f;
    } else {
        w.epsw = T(c.eps);
    }
    w.o = t + 2;                                     // padded smem index
    w.gn2_row = -1; w.aj_row = -1;
    w.gn2 = T(0); w.ajo = T(0); w.aj_out = T(0);
#pragma unroll
    for (int q = 0; q < 5; ++q) { w.qE[q] = T(0); w.qN[q] = T(0); }
#pragma unroll
    for (int q = 0; q < 4; ++q) { w.G1[q] = T(0); w.dG[q] = T(0); }
    w.vA[0] = w.vA[1] = T(0);
    w.iA[0] = w.iA[1] = T(0);
    w.cnt = 0u; w.m0 = T(0); w.m1 = T(0); w.m2 = T(0);
    // A warp whose columns all lie more than 4 past the grid (in the last
    // column band) feeds no output cell: the one step of an output cell
    // reaches 4 columns, and the 4th of them only through its loaded state.
    // In the persistent ensemble launch (COHERENT), where the grids are small
    // and last bands common, such a warp takes part in the barriers and
    // nothing else; the live column next to it reads its never-written ring
    // slots only for values that feed no output (as at the block's own
    // edge).  The single-grid kernel computes them (at 16384^2 they are 1.3 %
    // of the work, and the branch around the sweep made that kernel slower).
    const bool live = COHERENT ? (tx0 - 4 + (t & ~31) < c.nx + 4) : true;
    if (!live) {
        for (int s = y0 - 8; s <= y1 + 4; s += 2) { __syncthreads(); __syncthreads(); }
    } else {
        int yy = reflect(y0 - 4, c.ny, c.bc[2], c.bc[3], w.asy);
        if (SWE_IN((long long)yy * c.nx + w.xx, SWE_NCELL)) w.load_cell((long long)yy * c.nx + w.xx, w.aH, w.aHu, w.aHv, w.ab);
        yy = reflect(y0 - 3, c.ny, c.bc[2], c.bc[3], w.bsy);
        if (SWE_IN((long long)yy * c.nx + w.xx, SWE_NCELL)) w.load_cell((long long)yy * c.nx + w.xx, w.bH, w.bHu, w.bHv, w.bb0);
        // sweep positions y0-8 .. y1+4 in pairs (y0 is a multiple of 8)
        for (int s = y0 - 8; s <= y1 + 4; s += 2) {
            w.set_banks(s);
            if (s >= y0 + 5 && s + 1 <= y1 + 3) {
                w.template pos<0, true>(s);
                w.template pos<1, true>(s + 1);
            } else {
                w.template pos<0, false>(s);
                w.template pos<1, false>(s + 1);
            }
        }
    }
    block_finish<T, BW>((int)(w.cnt & 0xffffffu), w.m0, w.m1, w.m2, w.cnt >> 24, tile, cen_out, dev, 1);
}

// The 32 per-warp counts in v[] replaced by their exclusive prefix sums and
// the total written to *total, by one warp (lane = its lane index).
__device__ __forceinline__ void warp_exclusive_scan32(int *v, int lane, int *total) {
    const int own = v[lane];
    int x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    v[lane] = x - own;
    if (lane == 31) *total = x;
}

// The blocks the next step must run (HGS, Sec. 3: regions of SWE_REGION x
// SWE_REGION blocks above the blocks, compacted): those active by the K1 rule
// (the block or one of its four edge neighbours holds water or a source) and
// dry ones whose two state buffers still differ (one copy carries them over).
// Only the blocks of regions that hold water, or border one that does, in
// the current state or the previous one are examined: a block elsewhere is
// dry with dry neighbours, was carried over already, and has census 0 in the
// buffer the next census goes to.  The region census of the state (blocks
// with census > 0) is counted over the previous step's list, the only blocks
// whose census can be > 0; when that list is stale (after a state is set or
// changed outside the step) it is counted over every block and every block is
// examined.  The list goes to work[2..] with the count
// in work[0]; the census of the next state is written as 0 for every examined
// block left out.  Without the dry-block skip every block is listed.  One
// block of 1024 threads (T: the state type, for one instance per precision's
// translation unit).  The step index and the rescan flag are read through a
// volatile pointer: in between_compact_kernel thread 0 has just rewritten them.
template <typename T>
__device__ __forceinline__ void compact_body(const SweConst &c, const SweBufs &B) {
    __shared__ int wsum[32];
    __shared__ int base, chunk, nscan;
    __shared__ int rlist[1024];
    const volatile SweDev *vd = B.dev;
    const long long n = vd->n;
    const int par = (int)(n & 1);
    const int *cen = par ? B.census[1] : B.census[0];
    int *cen_next = par ? B.census[0] : B.census[1];
    const int nt = c.tiles_x * c.tiles_y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    if (!c.hgs) {   // every block, in order; the region census is not kept meanwhile
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += 1024) B.work[2 + t] = t;
        if (threadIdx.x == 0) {
            B.work[0] = nt;
            B.dev->rescan = 1;
        }
        return;
    }
    const int nreg = c.regions_x * c.regions_y;
    int *rc = B.rcen;
    unsigned char *rn = par ? B.rneed[1] : B.rneed[0];
    const unsigned char *rn_prev = par ? B.rneed[0] : B.rneed[1];
    const bool rescan = vd->rescan != 0;
    // the region census of this state: blocks with census > 0
    for (int r = threadIdx.x; r < nreg; r += 1024) rc[r] = 0;
    __syncthreads();
    const int nlast = rescan ? nt : B.work[0];
    for (int i = threadIdx.x; i < nlast; i += 1024) {
        const int t = rescan ? i : B.work[2 + i];
        if (cen[t] > 0) atomicAdd(rc + (t / c.tiles_x / SWE_REGION) * c.regions_x + (t % c.tiles_x) / SWE_REGION, 1);
    }
    __syncthreads();
    // regions examined, in chunks of 1024: their blocks, in chunks of 1024.
    // A region's flag for this state (it or an edge neighbour holds water) is
    // formed by the thread that examines it, from loads issued together
    // (clamped neighbour indices, no short-circuit test).
    for (int r0 = 0; r0 < nreg; r0 += 1024) {
        const int r = r0 + (int)threadIdx.x;
        bool scan = false;
        if (r < nreg) {
            const int rx = r % c.regions_x, ry = r / c.regions_x;
            const int q0 = rc[r], q1 = rc[rx > 0 ? r - 1 : r], q2 = rc[rx < c.regions_x - 1 ? r + 1 : r];
            const int q3 = rc[ry > 0 ? r - c.regions_x : r], q4 = rc[ry < c.regions_y - 1 ? r + c.regions_x : r];
            const bool prev = rn_prev[r] != 0;
            const bool wet = (q0 > 0) | (q1 > 0) | (q2 > 0) | (q3 > 0) | (q4 > 0);
            rn[r] = wet ? 1 : 0;
            scan = rescan || wet || prev;
        }
        unsigned m = __ballot_sync(0xffffffffu, scan);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        if (w == 0) warp_exclusive_scan32(wsum, lane, &nscan);
        __syncthreads();
        if (scan) rlist[wsum[w] + __popc(m & ((1u << lane) - 1u))] = r;
        __syncthreads();
        const int ns = nscan;
        for (int j0 = 0; j0 < ns * SWE_REGION * SWE_REGION; j0 += 1024) {
            const int j = j0 + (int)threadIdx.x;
            bool need = false;
            int tile = 0;
            if (j < ns * SWE_REGION * SWE_REGION) {
                const int reg = rlist[j / (SWE_REGION * SWE_REGION)], q = j % (SWE_REGION * SWE_REGION);
                const int bx = (reg % c.regions_x) * SWE_REGION + q % SWE_REGION;
                const int by = (reg / c.regions_x) * SWE_REGION + q / SWE_REGION;
                if (bx < c.tiles_x && by < c.tiles_y) {
                    tile = by * c.tiles_x + bx;
                    const int l = bx > 0 ? bx - 1 : bx, rr = bx < c.tiles_x - 1 ? bx + 1 : bx;
                    const int d = by > 0 ? by - 1 : by, u = by < c.tiles_y - 1 ? by + 1 : by;
                    const int k0 = cen[tile], k1 = cen[by * c.tiles_x + l], k2 = cen[by * c.tiles_x + rr];
                    const int k3 = cen[d * c.tiles_x + bx], k4 = cen[u * c.tiles_x + bx];
                    const bool skipped = B.skipped[tile] != 0;
                    const bool active = (k0 > 0) | (k1 > 0) | (k2 > 0) | (k3 > 0) | (k4 > 0);
                    need = active || !skipped;
                    if (!need) cen_next[tile] = 0;
                }
            }
            m = __ballot_sync(0xffffffffu, need);
            __syncthreads();   // rlist of this chunk stays read-only; wsum is reused below
            if (lane == 0) wsum[w] = __popc(m);
            __syncthreads();
            if (w == 0) warp_exclusive_scan32(wsum, lane, &chunk);
            __syncthreads();
            if (need) B.work[2 + base + wsum[w] + __popc(m & ((1u << lane) - 1u))] = tile;
            __syncthreads();
            if (threadIdx.x == 0) base += chunk;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        B.work[0] = base;
        if (rescan) B.dev->rescan = 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) compact_kernel(SweConst c, SweBufs B) { compact_body<T>(c, B); }

// One step: CUDA block i runs entries i, i + gridDim.x, ... of the work list
// (a column band x row strip each).  Launched with one CUDA block per grid
// block (dense steps) each runs at most one entry and the blocks past the
// list's end return at once; a smaller grid (sparse steps) walks the list.
// FP32: 24 warps per SM at 80 registers for every dense variant: three
// 256-column blocks (73 KB of shared memory each) or six 128-column blocks
// (37 KB each), whose barriers wait for 4 warps instead of 8 (on grids of
// 2^25 cells and more 1.6-2.3 % faster than the 256-column blocks despite
// twice the halo columns; on smaller grids, with fewer blocks than resident
// slots, slower).  The variants with source terms or the general laws spill
// 20-60 bytes at 80 registers and are still 10-25 % faster than at 16 warps
// per SM.  The list-walking variant runs a wave of two blocks per SM over few
// blocks, where the sweep's latency counts: it gets the registers of two
// blocks per SM.
template <typename T, int BW, int SRC, bool GEN, bool WALK>
__global__ void __launch_bounds__(BW, sizeof(T) == 4 ? (WALK ? 2 : (BW == 128 ? 6 : 3)) : 1)
step_kernel(SweConst c, SweBufs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<T, BW> &S = *reinterpret_cast<StepSmem<T, BW> *>(smem_raw);
    const int count = B.work[0];
    if constexpr (!WALK) {   // dense: at most one entry per CUDA block
        const int i = blockIdx.x;
        if (i >= count) return;
        const int tile = B.work[2 + i];
        if (!SWE_IN(tile, c.tiles_x * c.tiles_y)) return;
        step_tile<T, BW, false, SRC, GEN>(c, B, tile % c.tiles_x, tile / c.tiles_x, S);
    } else {
        for (int i = blockIdx.x; i < count; i += gridDim.x) {
            const int tile = B.work[2 + i];
            if (!SWE_IN(tile, c.tiles_x * c.tiles_y)) return;
            step_tile<T, BW, false, SRC, GEN>(c, B, tile % c.tiles_x, tile / c.tiles_x, S);
        }
    }
}

// ----------------------------------------------- census + Eq. 7 terms of a state

// Canonicalises a freshly set state (dry cells carry no momentum) and forms
// the census and the Eq. 7 maxima for it.  One block per HGS tile.
template <typename T, int BW>
__global__ void __launch_bounds__(BW) init_kernel(SweConst c, SweBufs B) {
    SweDev *dev = B.dev;
    const long long n = dev->n;
    void *buf = (n & 1) ? B.buf[1] : B.buf[0];
    const int bx = blockIdx.x, by = blockIdx.y, tile = by * c.tiles_x + bx;
    const int x0 = bx * c.tw, y0 = by * c.th;
    const int x1 = min(x0 + c.tw, c.nx), y1 = min(y0 + c.th, c.ny);
    K<T> k;
    k.g = T(c.g); k.eps = T(c.eps); k.ksh = T(c.ksh); k.A_J = T(c.A_J); k.m_exp = T(c.m_exp);
    k.sm1 = T(c.sm1); k.d50 = T(c.d50); k.neg_tol = T(c.neg_tol);
    int cnt = 0;
    T m0 = T(0), m1 = T(0), m2 = T(0);
    unsigned st = 0;
    for (int y = y0; y < y1; ++y)
        for (int x = x0 + (int)threadIdx.x; x < x1; x += BW) {
            long long kk = (long long)y * c.nx + x;
            T H, Hu, Hv, bb;
            CellIO<T>::load(buf, kk, H, Hu, Hv, bb);
            if (!is_wet(H, c)) { Hu = T(0); Hv = T(0); CellIO<T>::store(buf, kk, H, Hu, Hv, bb); }
            bool src = false;
            for (int q = B.src_rowptr[y]; q < B.src_rowptr[y + 1]; ++q) src |= (B.src_x[q] == x);
            int mi = (y >> c.man_shift) * c.man_w + (x >> c.man_shift);
            cell_epilogue<T>(c, k, H, Hu, Hv, bb, tab<T>(B.ajn, mi), src, cnt, m0, m1, m2, st);
        }
    block_finish<T, BW>(cnt, m0, m1, m2, st, tile, (n & 1) ? B.census[1] : B.census[0], dev, 0);
    if (threadIdx.x == 0) {
        B.skipped[tile] = 0;
        if (tile == 0) dev->rescan = 1;   // the first compaction rebuilds the region census
    }
}

// ------------------------------------------------------ dt (K3) and bookkeeping

// Piecewise-linear hydrograph integral over [ta, tb] (constant beyond the
// ends), summed piece by piece in knot order.  Hydrographs of up to 4 knots
// are read into registers first, in one batch of loads (the loop then unrolls
// on constant indices); longer ones are read knot by knot.
__device__ inline double hydro_integral(int nk, const double *tk, const double *Qk, double ta, double tb) {
    if (nk <= 0 || !(tb > ta)) return 0.0;
    if (nk <= 4) {
        double t[4], q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            t[j] = j < nk ? tk[j] : 0.0;
            q[j] = j < nk ? Qk[j] : 0.0;
        }
        double s = 0.0;
        if (ta < t[0]) { double e = tb < t[0] ? tb : t[0]; s += q[0] * (e - ta); }
        double tl = t[0], ql = q[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j + 1 < nk) {
                tl = t[j + 1]; ql = q[j + 1];
                double a = ta > t[j] ? ta : t[j];
                double b = tb < t[j + 1] ? tb : t[j + 1];
                if (b > a) {
                    double span = t[j + 1] - t[j];
                    double qa = q[j] + (q[j + 1] - q[j]) * ((a - t[j]) / span);
                    double qb = q[j] + (q[j + 1] - q[j]) * ((b - t[j]) / span);
                    s += 0.5 * (qa + qb) * (b - a);
                }
            }
        }
        if (tb > tl) { double a = ta > tl ? ta : tl; s += ql * (tb - a); }
        return s;
    }
    double s = 0.0;
    if (ta < tk[0]) { double e = tb < tk[0] ? tb : tk[0]; s += Qk[0] * (e - ta); }
    for (int j = 0; j + 1 < nk; ++j) {
        double a = ta > tk[j] ? ta : tk[j];
        double b = tb < tk[j + 1] ? tb : tk[j + 1];
        if (!(b > a)) continue;
        double span = tk[j + 1] - tk[j];
        double qa = Qk[j] + (Qk[j + 1] - Qk[j]) * ((a - tk[j]) / span);
        double qb = Qk[j] + (Qk[j + 1] - Qk[j]) * ((b - tk[j]) / span);
        s += 0.5 * (qa + qb) * (b - a);
    }
    if (tb > tk[nk - 1]) { double a = ta > tk[nk - 1] ? ta : tk[nk - 1]; s += Qk[nk - 1] * (tb - a); }
    return s;
}

template <typename T> __device__ inline double acc_value(unsigned long long bits);
template <> __device__ inline double acc_value<float>(unsigned long long bits) { return (double)__uint_as_float((unsigned)bits); }
template <> __device__ inline double acc_value<double>(unsigned long long bits) { return __longlong_as_double((long long)bits); }


// One thread.  mode 1 (commit) first commits the step that just ran, if one
// was scheduled (n += 1, t += dt, the maxima gathered by its epilogue become
// the current ones); mode 2 (init) takes the maxima the census kernel
// gathered for a freshly set state; mode 0 only re-prepares.  It then forms
// dt of the next step from Eq. 7 (FP64), clipped to t_end - t, the source
// increment and the step coefficients.  The bookkeeping is read first, in one
// batch of L2-coherent loads (so the body also runs inside a persistent
// launch, after other blocks wrote it, and waits for memory once, not once per
// field), and written back with plain stores.
template <typename T>
__device__ void between_body(const SweConst &c, const SweBufs &B, int mode) {
    SweDev *d = B.dev;
    const int nsrc = c.nsrc;
    const int sched = __ldcg(&d->scheduled), binding = __ldcg(&d->binding), active = __ldcg(&d->active_tiles);
    const long long n = __ldcg(&d->n);
    const double t0 = __ldcg(&d->t), t_end = __ldcg(&d->t_end), dt0 = __ldcg(&d->dt);
    const double dHs0 = __ldcg(&d->dHs), inflow0 = __ldcg(&d->inflow_total);
    const unsigned long long a0 = __ldcg(&d->acc[0]), a1 = __ldcg(&d->acc[1]), a2 = __ldcg(&d->acc[2]);
    double vp = __ldcg(&d->vp), vs = __ldcg(&d->vs), jm = __ldcg(&d->jm);
    double t = t0;
    bool take = mode == 2;
    if (mode == 1 && sched) {
        t = binding == 4 ? t_end : t0 + dt0;  // a clipped step lands on t_end
        d->n = n + 1;
        d->t = t;
        d->dt_last = dt0;
        d->binding_last = binding;
        d->inflow_total = inflow0 + dHs0 * ((double)nsrc * (c.dx * c.dx));
        d->active_last = active;
        take = true;
    }
    if (take) {
        vp = acc_value<T>(a0);
        vs = acc_value<T>(a1);
        jm = acc_value<T>(a2);
        d->vp = vp; d->vs = vs; d->jm = jm;
        d->acc[0] = 0ull; d->acc[1] = 0ull; d->acc[2] = 0ull;
    }
    const double h = c.dx;
    double best = INFINITY;
    int which = 3;
    if (vp > 0.0) { double a = h / (2.0 * vp); if (a < best) { best = a; which = 0; } }
    if (vs > 0.0) { double a = h / vs; if (a < best) { best = a; which = 1; } }
    if (c.sediment_on && jm > 0.0) {
        double D = (c.literal_D ? jm : c.C_J * jm) / (1.0 - c.psi);
        double a = (h * h) / (2.0 * D);
        if (a < best) { best = a; which = 2; }
    }
    double dt = c.K * best;
    if (!(dt < c.dt_max)) { dt = c.dt_max; which = 3; }
    d->dt_unclipped = dt;
    if (t_end < INFINITY) {
        double rem = t_end - t;
        if (!(rem > 0.0)) { dt = 0.0; d->done = 1; }
        else if (rem < dt) { dt = rem; which = 4; }
    }
    d->dt = dt;
    d->binding = which;
    d->scheduled = dt > 0.0 ? 1 : 0;
    double vol = (nsrc > 0 && dt > 0.0) ? hydro_integral(c.nk, B.hyd_t, B.hyd_q, t, t + dt) : 0.0;
    d->dHs = nsrc > 0 ? vol / ((double)nsrc * (c.dx * c.dx)) : 0.0;
    const double dtdx = dt / c.dx;
    d->dtdx = dtdx;
    d->hdt = 0.5 * dt;
    d->c4 = dt / (4.0 * c.dx);
    d->cb = dtdx / (1.0 - c.psi);
    d->active_tiles = 0;
}

template <typename T>
__global__ void between_kernel(SweConst c, SweBufs B, int mode) { between_body<T>(c, B, mode); }

// The end of a step and the start of the next in one launch: thread 0 commits
// the step and forms the next dt (between_body, mode 1), then the block lists
// the blocks of the next step (compact_body) from the census just committed.
// (Listing twice for one state gives the same list, so a step may still be
// preceded by its own compaction.)
template <typename T>
__global__ void __launch_bounds__(1024) between_compact_kernel(SweConst c, SweBufs B) {
    if (threadIdx.x == 0) between_body<T>(c, B, 1);
    __syncthreads();
    compact_body<T>(c, B);
}

// b += dt q / (1 - psi) on the freshly written buffer (Eq. 1 bed source).
template <typename T>
__global__ void bed_source_kernel(SweConst c, SweBufs B) {
    SweDev *d = B.dev;
    if (!d->scheduled) return;
    void *out = ((d->n + 1) & 1) ? B.buf[1] : B.buf[0];
    const T cq = T(d->dt / (1.0 - c.psi));
    const long long N = (long long)c.nx * c.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < N; kk += (long long)gridDim.x * blockDim.x) {
        T H, Hu, Hv, bb;
        CellIO<T>::load(out, kk, H, Hu, Hv, bb);
        bb = bb + cq * tab<T>(B.qb, (int)kk);
        CellIO<T>::store(out, kk, H, Hu, Hv, bb);
    }
}

// ------------------------------------------------------------ diagnostics

// FP64 sums of H and b and the wet count, in a fixed order: per-block
// partials here, then a one-block pass.
template <typename T, int BW>
__global__ void __launch_bounds__(BW) diag_partial_kernel(SweConst c, SweBufs B) {
    const void *buf = (B.dev->n & 1) ? B.buf[1] : B.buf[0];
    const long long N = (long long)c.nx * c.ny;
    double sh = 0.0, sb = 0.0, sw = 0.0;
    for (long long kk = blockIdx.x * (long long)BW + threadIdx.x; kk < N; kk += (long long)gridDim.x * BW) {
        T H, Hu, Hv, bb;
        CellIO<T>::load(buf, kk, H, Hu, Hv, bb);
        sh += (double)H; sb += (double)bb; sw += is_wet(H, c) ? 1.0 : 0.0;
    }
    __shared__ double r[3][BW];
    r[0][threadIdx.x] = sh; r[1][threadIdx.x] = sb; r[2][threadIdx.x] = sw;
    __syncthreads();
    for (int w = BW / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 3; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) B.partials[3 * blockIdx.x + q] = r[q][0];
}

__global__ void diag_final_kernel(SweBufs B, int nblocks, double *out3);

// ------------------------------------------------------------ conversion

template <typename T>
__global__ void convert_in_kernel(SweConst c, void *dst, const void *H, const void *Hu, const void *Hv,
                                  const void *bb, int f64) {
    const long long N = (long long)c.nx * c.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < N; kk += (long long)gridDim.x * blockDim.x) {
        T a, b2, c2, d2;
        if (f64) {
            a = T(((const double *)H)[kk]); b2 = T(((const double *)Hu)[kk]);
            c2 = T(((const double *)Hv)[kk]); d2 = T(((const double *)bb)[kk]);
        } else {
            a = T(((const float *)H)[kk]); b2 = T(((const float *)Hu)[kk]);
            c2 = T(((const float *)Hv)[kk]); d2 = T(((const float *)bb)[kk]);
        }
        CellIO<T>::store(dst, kk, a, b2, c2, d2);
    }
}

template <typename T>
__global__ void convert_out_kernel(SweConst c, const void *src, void *H, void *Hu, void *Hv, void *bb, int f64) {
    const long long N = (long long)c.nx * c.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < N; kk += (long long)gridDim.x * blockDim.x) {
        T a, b2, c2, d2;
        CellIO<T>::load(src, kk, a, b2, c2, d2);
        if (f64) {
            if (H) ((double *)H)[kk] = (double)a;
            if (Hu) ((double *)Hu)[kk] = (double)b2;
            if (Hv) ((double *)Hv)[kk] = (double)c2;
            if (bb) ((double *)bb)[kk] = (double)d2;
        } else {
            if (H) ((float *)H)[kk] = (float)a;
            if (Hu) ((float *)Hu)[kk] = (float)b2;
            if (Hv) ((float *)Hv)[kk] = (float)c2;
            if (bb) ((float *)bb)[kk] = (float)d2;
        }
    }
}

}  // namespace swe_impl
