// Generic launchers; each precision's translation unit includes this file and
// instantiates the templates for its own state type.
#pragma once
#include <atomic>

#include "swe_kernels.cuh"

namespace swe_impl {

template <typename T> size_t step_smem_bytes(int bw) {
    return bw == 128 ? sizeof(StepSmem<T, 128>) : sizeof(StepSmem<T, 256>);
}

// One step: the work list of the blocks to run (compact_kernel, left out
// when the launch before it on the stream, between_compact_kernel, formed
// it), then one CUDA block per grid block, the unlisted ones returning at
// once.  The kernel variant compiles only the terms in use: the inflow, and
// the rain and infiltration fields (SRC bits), the general transport laws
// (GEN); every dense FP32 variant runs 24 warps per SM (three 256-column or
// six 128-column blocks).
template <typename T, int BW, int SRC, bool GEN>
static cudaError_t launch_step_v(const SweConst &c, const SweBufs &b, cudaStream_t s, int grid, bool list) {
    // the shared-memory opt-in is a per-device function attribute: one bit
    // per device (devices beyond 64 set it on every launch)
    static std::atomic<unsigned long long> configured{0};
    const size_t smem = sizeof(StepSmem<T, BW>);
    const int nt = c.tiles_x * c.tiles_y;
    const bool walk = grid > 0 && grid < nt;
    auto kern = walk ? step_kernel<T, BW, SRC, GEN, true> : step_kernel<T, BW, SRC, GEN, false>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (!bit || !(configured.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(step_kernel<T, BW, SRC, GEN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel<T, BW, SRC, GEN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit, std::memory_order_release);
    }
    if (list) compact_kernel<T><<<1, 1024, 0, s>>>(c, b);
    kern<<<walk ? grid : nt, BW, smem, s>>>(c, b);
    return cudaGetLastError();
}

inline int source_terms(const SweConst &c) {
    return (c.nsrc > 0 ? SWE_SRC_INFLOW : 0) | ((c.has_rain || c.has_beta) ? SWE_SRC_FIELDS : 0);
}
inline bool uses_general_laws(const SweConst &c) { return c.aj_mode == 1 || !c.m_is_2; }

template <typename T, int BW, int SRC>
static cudaError_t launch_step_s(const SweConst &c, const SweBufs &b, cudaStream_t s, int grid, bool list) {
    return uses_general_laws(c) ? launch_step_v<T, BW, SRC, true>(c, b, s, grid, list)
                                : launch_step_v<T, BW, SRC, false>(c, b, s, grid, list);
}

template <typename T, int BW>
static cudaError_t launch_step_bw(const SweConst &c, const SweBufs &b, cudaStream_t s, int grid, bool list) {
    if constexpr (sizeof(T) == 8) {
        // the FP64 build (parity): the general variant
        return launch_step_v<T, BW, SWE_SRC_INFLOW | SWE_SRC_FIELDS, true>(c, b, s, grid, list);
    } else {
        switch (source_terms(c)) {
        case 0: return launch_step_s<T, BW, 0>(c, b, s, grid, list);
        case SWE_SRC_INFLOW: return launch_step_s<T, BW, SWE_SRC_INFLOW>(c, b, s, grid, list);
        case SWE_SRC_FIELDS: return launch_step_s<T, BW, SWE_SRC_FIELDS>(c, b, s, grid, list);
        default: return launch_step_s<T, BW, SWE_SRC_INFLOW | SWE_SRC_FIELDS>(c, b, s, grid, list);
        }
    }
}

template <typename T>
cudaError_t launch_step(const SweConst &c, const SweBufs &b, int bw, cudaStream_t s, int grid, bool list) {
    if (bw == 128) return launch_step_bw<T, 128>(c, b, s, grid, list);
    return launch_step_bw<T, 256>(c, b, s, grid, list);
}

template <typename T> cudaError_t launch_init(const SweConst &c, const SweBufs &b, cudaStream_t s) {
    dim3 grid(c.tiles_x, c.tiles_y);
    init_kernel<T, 256><<<grid, 256, 0, s>>>(c, b);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_between(const SweConst &c, const SweBufs &b, int commit, cudaStream_t s) {
    between_kernel<T><<<1, 1, 0, s>>>(c, b, commit);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_between_compact(const SweConst &c, const SweBufs &b, cudaStream_t s) {
    between_compact_kernel<T><<<1, 1024, 0, s>>>(c, b);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_diag(const SweConst &c, const SweBufs &b, int nblocks, cudaStream_t s) {
    diag_partial_kernel<T, 256><<<nblocks, 256, 0, s>>>(c, b);
    return cudaGetLastError();
}

static inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

template <typename T> cudaError_t launch_convert_in(const SweConst &c, void *dst, const void *H, const void *Hu,
                                                    const void *Hv, const void *bb, int f64, cudaStream_t s) {
    convert_in_kernel<T><<<grid_for((long long)c.nx * c.ny), 256, 0, s>>>(c, dst, H, Hu, Hv, bb, f64);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_convert_out(const SweConst &c, const void *src, void *H, void *Hu,
                                                     void *Hv, void *bb, int f64, cudaStream_t s) {
    convert_out_kernel<T><<<grid_for((long long)c.nx * c.ny), 256, 0, s>>>(c, src, H, Hu, Hv, bb, f64);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_bed_source(const SweConst &c, const SweBufs &b, cudaStream_t s) {
    bed_source_kernel<T><<<grid_for((long long)c.nx * c.ny), 256, 0, s>>>(c, b);
    return cudaGetLastError();
}

#define SWE_INSTANTIATE(T)                                                                                        \
    template size_t step_smem_bytes<T>(int);                                                                      \
    template cudaError_t launch_step<T>(const SweConst &, const SweBufs &, int, cudaStream_t, int, bool);        \
    template cudaError_t launch_init<T>(const SweConst &, const SweBufs &, cudaStream_t);                        \
    template cudaError_t launch_between<T>(const SweConst &, const SweBufs &, int, cudaStream_t);                \
    template cudaError_t launch_between_compact<T>(const SweConst &, const SweBufs &, cudaStream_t);             \
    template cudaError_t launch_diag<T>(const SweConst &, const SweBufs &, int, cudaStream_t);                   \
    template cudaError_t launch_convert_in<T>(const SweConst &, void *, const void *, const void *, const void *, \
                                              const void *, int, cudaStream_t);                                   \
    template cudaError_t launch_convert_out<T>(const SweConst &, const void *, void *, void *, void *, void *,   \
                                               int, cudaStream_t);                                                \
    template cudaError_t launch_bed_source<T>(const SweConst &, const SweBufs &, cudaStream_t);

}  // namespace swe_impl
