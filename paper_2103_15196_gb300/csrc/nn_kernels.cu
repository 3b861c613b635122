// Tensor-core kernels of the learned bed surrogate (BF16 operands, FP32
// accumulation in tensor memory), plus a self-test GEMM of the same MMA path.
#include <cuda_bf16.h>
#include <algorithm>
#include <stdint.h>

#include "../../include/swe.h"
#include "nn_tc.cuh"

using namespace swe_nn;

namespace {

constexpr int kPolls = 1 << 22;   // bounded mbarrier wait (~0.3 s)

// C[128][n] = A[128][k] * B[n][k]^T: one CTA of 128 threads; operand tiles
// in two 64 KB shared buffers (zero-filled), K-major no-swizzle layout.
template <int N>
__global__ void __launch_bounds__(128) tc_selftest_kernel(const __nv_bfloat16 *__restrict__ A,
                                                          const __nv_bfloat16 *__restrict__ B, float *__restrict__ C,
                                                          int K, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sa = sm;
    unsigned char *sb = sm + 65536;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 131072);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 131072 + 16);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int i = t; i < 131072 / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int kb = K / 8;
    for (int i = t; i < 128 * kb; i += 128) {
        const int r = i / kb, c = i % kb;
        *reinterpret_cast<uint4 *>(sa + kmajor_off(r, c * 8, 128)) =
            *reinterpret_cast<const uint4 *>(A + (size_t)r * K + c * 8);
    }
    for (int i = t; i < N * kb; i += 128) {
        const int r = i / kb, c = i % kb;
        *reinterpret_cast<uint4 *>(sb + kmajor_off(r, c * 8, N)) =
            *reinterpret_cast<const uint4 *>(B + (size_t)r * K + c * 8);
    }
    fence_async_smem();
    if (warp == 0) tmem_alloc(tslot, 32);
    if (t == 0) mbar_init(mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (t == 0) {
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ad = smem_desc(smem_u32(sa) + kk * 128 * 32, 128 * 16, 128);
            const uint64_t bd = smem_desc(smem_u32(sb) + kk * N * 32, N * 16, 128);
            mma_bf16(tmem, ad, bd, idesc_bf16_f32(N), kk > 0 ? 1u : 0u);
        }
        mma_commit(mbar);
    }
    bool ok = __syncthreads_and(mbar_wait(mbar, 0, kPolls));
    if (!ok) {
        if (t == 0) atomicOr(err, 1);
        ok = __syncthreads_and(mbar_wait(mbar, 0, kPolls));   // let MMAs in flight finish before freeing TMEM
    }
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        const int row = warp * 32 + lane;
#pragma unroll
        for (int j = 0; j < N; ++j) C[row * N + j] = v[j];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace

extern "C" swe_status swe_nn_tc_selftest(int n, int k, const uint16_t *A, const uint16_t *B, float *C) {
    if ((n != 16 && n != 32) || k < 16 || k > 256 || (k % 16) || !A || !B || !C) return SWE_EINVAL;
    void *dA = nullptr, *dB = nullptr, *dC = nullptr;
    int *derr = nullptr;
    swe_status st = SWE_OK;
    const size_t smem = 131072 + 64;
    if (cudaMalloc(&dA, 128 * k * 2) != cudaSuccess || cudaMalloc(&dB, n * k * 2) != cudaSuccess ||
        cudaMalloc(&dC, 128 * n * 4) != cudaSuccess || cudaMalloc(&derr, 4) != cudaSuccess) {
        st = SWE_ENOMEM;
    } else {
        cudaMemcpy(dA, A, 128 * k * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, n * k * 2, cudaMemcpyHostToDevice);
        cudaMemset(derr, 0, 4);
        cudaError_t e;
        if (n == 16) {
            cudaFuncSetAttribute(tc_selftest_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_selftest_kernel<16><<<1, 128, smem>>>((const __nv_bfloat16 *)dA, (const __nv_bfloat16 *)dB,
                                                     (float *)dC, k, derr);
        } else {
            cudaFuncSetAttribute(tc_selftest_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_selftest_kernel<32><<<1, 128, smem>>>((const __nv_bfloat16 *)dA, (const __nv_bfloat16 *)dB,
                                                     (float *)dC, k, derr);
        }
        e = cudaDeviceSynchronize();
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(C, dC, 128 * n * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = SWE_ECUDA;
        else if (herr) st = SWE_ETIMEOUT;
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(derr);
    return st;
}

// ======================================================================
// 3x3 convolutions (stride 1, zero padding 1) of the bed surrogate as
// implicit GEMMs on the tensor cores.  Activations are NHWC BF16 with 8
// (input) or 32 channels; weights are K-major BF16 [nout][k], k = tap * cin +
// c, tap = (dy + 1) * 3 + (dx + 1).  One CTA of 128 threads computes 128
// consecutive pixels of one image row x nout channels; the FP32 accumulator
// lives in tensor memory (128 lanes x nout columns).
// ======================================================================

namespace swe_nn {

enum { EPI_RELU = 0, EPI_OUT = 1, EPI_MASK = 2 };

template <int CIN> struct ConvK {
    static constexpr int K = 9 * CIN;
    static constexpr int KP = (K + 15) / 16 * 16;   // padded to whole MMAs
};

// Forward (EPI_RELU: bias + ReLU -> NHWC32; EPI_OUT: channel 0 + bias -> float
// per pixel) or input gradient (EPI_MASK: times (mask > 0) -> NHWC32).
template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(128)
conv3x3_tc(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt, const float *__restrict__ bias,
           const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ Y, float *__restrict__ Yf, int H,
           int W, int *err) {
    constexpr int KP = ConvK<CIN>::KP;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sa = sm;                              // 128 x KP
    unsigned char *sb = sm + 128 * KP * 2;               // NOUT x KP
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + NOUT * KP * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * 128, y = blockIdx.y, img = blockIdx.z;
    const size_t plane = (size_t)H * W;
    const __nv_bfloat16 *Xi = X + (size_t)img * plane * CIN;

    // A: im2col of the 128-pixel segment (zero outside the image)
    if (CIN == 32) {
        const int cg = t & 3, pb = t >> 2;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = y + tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int p = pb + 32 * pp, xx = x0 + p + dx;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v = *reinterpret_cast<const uint4 *>(Xi + ((size_t)yy * W + xx) * CIN + cg * 8);
                *reinterpret_cast<uint4 *>(sa + kmajor_off(p, tap * CIN + cg * 8, 128)) = v;
            }
        }
    } else {
        const int p = t;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = y + tap / 3 - 1, xx = x0 + p + tap % 3 - 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = *reinterpret_cast<const uint4 *>(Xi + ((size_t)yy * W + xx) * CIN);
            *reinterpret_cast<uint4 *>(sa + kmajor_off(p, tap * CIN, 128)) = v;
        }
        for (int k = 9 * CIN; k < KP; k += 8)
            *reinterpret_cast<uint4 *>(sa + kmajor_off(p, k, 128)) = make_uint4(0, 0, 0, 0);
    }
    // B: the weights
    for (int i = t; i < NOUT * (KP / 8); i += 128) {
        const int r = i / (KP / 8), c = i % (KP / 8);
        *reinterpret_cast<uint4 *>(sb + kmajor_off(r, c * 8, NOUT)) =
            *reinterpret_cast<const uint4 *>(Wt + (size_t)r * KP + c * 8);
    }
    fence_async_smem();
    if (warp == 0) tmem_alloc(tslot, 32);
    if (t == 0) mbar_init(mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (t == 0) {
#pragma unroll 1
        for (int kk = 0; kk < KP / 16; ++kk) {
            const uint64_t ad = smem_desc(smem_u32(sa) + kk * 128 * 32, 128 * 16, 128);
            const uint64_t bd = smem_desc(smem_u32(sb) + kk * NOUT * 32, NOUT * 16, 128);
            mma_bf16(tmem, ad, bd, idesc_bf16_f32(NOUT), kk > 0 ? 1u : 0u);
        }
        mma_commit(mbar);
    }
    bool ok = __syncthreads_and(mbar_wait(mbar, 0, kPolls));
    if (!ok) {
        if (t == 0) atomicOr(err, 1);
        ok = __syncthreads_and(mbar_wait(mbar, 0, kPolls));
    }
    tc_fence_after();
    if (ok) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        const int p = warp * 32 + lane, xx = x0 + p;
        if (xx < W) {
            const size_t pix = (size_t)img * plane + (size_t)y * W + xx;
            if (EPI == EPI_OUT) {
                Yf[pix] = v[0] + bias[0];
            } else {
                __align__(16) __nv_bfloat16 o[32];
                if (EPI == EPI_RELU) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) o[j] = __float2bfloat16(fmaxf(v[j] + bias[j], 0.f));
                } else {
                    __align__(16) __nv_bfloat16 m[32];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        reinterpret_cast<uint4 *>(m)[q] = reinterpret_cast<const uint4 *>(mask + pix * 32)[q];
#pragma unroll
                    for (int j = 0; j < 32; ++j) o[j] = __float2bfloat16(__bfloat162float(m[j]) > 0.f ? v[j] : 0.f);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(Y + pix * 32)[q] = reinterpret_cast<uint4 *>(o)[q];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// cp.async of 16 bytes into shared memory; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Persistent form of conv3x3_tc: one CTA per SM keeps the weights in shared
// memory and walks 128-pixel tiles (round-robin over the grid).  Two A
// buffers and two TMEM accumulator halves pipeline the work: while the MMAs
// of tile i run, the CTA stores the result of tile i-1 and streams the im2col
// of tile i+1 in with cp.async.
template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(128, 1)
conv3x3_tcp(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt, const float *__restrict__ bias,
            const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ Y, float *__restrict__ Yf, int H,
            int W, int nimg, int *err) {
    constexpr int KP = ConvK<CIN>::KP;
    constexpr int ABYTES = 128 * KP * 2;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sa0 = sm;
    unsigned char *sa1 = sm + ABYTES;
    unsigned char *sb = sm + 2 * ABYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + NOUT * KP * 2);   // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int segs = (W + 127) / 128;
    const long long ntile = (long long)nimg * H * segs;
    const size_t plane = (size_t)H * W;

    // weights, and the zero K-padding columns of both A buffers
    for (int i = t; i < NOUT * (KP / 8); i += 128) {
        const int r = i / (KP / 8), c = i % (KP / 8);
        *reinterpret_cast<uint4 *>(sb + kmajor_off(r, c * 8, NOUT)) =
            *reinterpret_cast<const uint4 *>(Wt + (size_t)r * KP + c * 8);
    }
    for (int k = 9 * CIN; k < KP; k += 8) {
        *reinterpret_cast<uint4 *>(sa0 + kmajor_off(t, k, 128)) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(sa1 + kmajor_off(t, k, 128)) = make_uint4(0, 0, 0, 0);
    }

    auto load_tile = [&](long long tile, unsigned char *sa) {
        const int img = (int)(tile / ((long long)H * segs));
        const int rem = (int)(tile % ((long long)H * segs));
        const int y = rem / segs, x0 = (rem % segs) * 128;
        const __nv_bfloat16 *Xi = X + (size_t)img * plane * CIN;
        if (CIN == 32) {
            const int cg = t & 3, pb = t >> 2;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int yy = y + tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int p = pb + 32 * pp, xx = x0 + p + dx;
                    const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
                    const __nv_bfloat16 *src = in ? Xi + ((size_t)yy * W + xx) * CIN + cg * 8 : X;
                    cp_async16(sa + kmajor_off(p, tap * CIN + cg * 8, 128), src, in ? 16 : 0);
                }
            }
        } else {
            const int p = t;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int yy = y + tap / 3 - 1, xx = x0 + p + tap % 3 - 1;
                const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
                const __nv_bfloat16 *src = in ? Xi + ((size_t)yy * W + xx) * CIN : X;
                cp_async16(sa + kmajor_off(p, tap * CIN, 128), src, in ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    auto epilogue = [&](long long tile, uint32_t taddr) {
        const int img = (int)(tile / ((long long)H * segs));
        const int rem = (int)(tile % ((long long)H * segs));
        const int y = rem / segs, x0 = (rem % segs) * 128;
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), v);
        const int p = warp * 32 + lane, xx = x0 + p;
        if (xx >= W) return;
        const size_t pix = (size_t)img * plane + (size_t)y * W + xx;
        if (EPI == EPI_OUT) {
            Yf[pix] = v[0] + bias[0];
        } else {
            __align__(16) __nv_bfloat16 o[32];
            if (EPI == EPI_RELU) {
#pragma unroll
                for (int j = 0; j < 32; ++j) o[j] = __float2bfloat16(fmaxf(v[j] + bias[j], 0.f));
            } else {
                __align__(16) __nv_bfloat16 m[32];
#pragma unroll
                for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(m)[q] = reinterpret_cast<const uint4 *>(mask + pix * 32)[q];
#pragma unroll
                for (int j = 0; j < 32; ++j) o[j] = __float2bfloat16(__bfloat162float(m[j]) > 0.f ? v[j] : 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(Y + pix * 32)[q] = reinterpret_cast<uint4 *>(o)[q];
        }
    };

    if (warp == 0) tmem_alloc(tslot, 64);
    if (t == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); }
    long long tile = blockIdx.x;
    if (tile < ntile) load_tile(tile, sa0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t ph[2] = {0, 0};
    bool ok = true;
    long long prev = -1;
    int it = 0;
    for (; tile < ntile && ok; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        unsigned char *sa = buf ? sa1 : sa0;
        cp_async_wait_all();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
#pragma unroll 1
            for (int kk = 0; kk < KP / 16; ++kk) {
                const uint64_t ad = smem_desc(smem_u32(sa) + kk * 128 * 32, 128 * 16, 128);
                const uint64_t bd = smem_desc(smem_u32(sb) + kk * NOUT * 32, NOUT * 16, 128);
                mma_bf16(tmem + buf * 32, ad, bd, idesc_bf16_f32(NOUT), kk > 0 ? 1u : 0u);
            }
            mma_commit(&mbar[buf]);
        }
        if (prev >= 0) {
            const int pb = buf ^ 1;
            ok = __syncthreads_and(mbar_wait(&mbar[pb], ph[pb], kPolls));
            ph[pb] ^= 1;
            tc_fence_after();
            if (ok) epilogue(prev, tmem + pb * 32);
        }
        const long long next = tile + gridDim.x;
        if (ok && next < ntile) load_tile(next, buf ? sa0 : sa1);
        prev = tile;
    }
    if (ok && prev >= 0) {
        const int pb = (it - 1) & 1;
        ok = __syncthreads_and(mbar_wait(&mbar[pb], ph[pb], kPolls));
        ph[pb] ^= 1;
        tc_fence_after();
        if (ok) epilogue(prev, tmem + pb * 32);
    }
    if (!ok) {
        if (t == 0) atomicOr(err, 1);
        __syncthreads_and(mbar_wait(&mbar[0], ph[0], kPolls));
        __syncthreads_and(mbar_wait(&mbar[1], ph[1], kPolls));
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// Row-streaming form of the convolution (used by the surrogate): no im2col.
// A CTA owns one 128-pixel column band of an image and a run of output rows.
// Each input row it needs is loaded once, into a shared-memory slot of 136
// pixels (x0-1 .. x0+134) in the K-major layout, the 136 rows of each 8-channel
// column block contiguous (16 bytes per pixel, blocks CBS bytes apart).  The
// A operand of tap (dy, dx) is then that slot read from pixel dx+1 on: the
// same layout with the descriptor's start moved by 16 (dx+1) bytes.  With 32
// channels a tap is two MMAs (K = 16 channels each, LBO = CBS); with 8
// channels one MMA covers the taps (dy, dx) and (dy, dx+1), LBO = 16 bytes
// (one pixel), and the weights carry a zero block for the unused pair
// partner.  Five row slots and two TMEM accumulator halves pipeline the rows:
// while the MMAs of row y run, the CTA stores row y-1, and rows y+2 and y+3
// stream in with cp.async.
template <int CIN> struct RowConv {
    static constexpr int KR = CIN == 8 ? 96 : 9 * CIN;   // K of the MMA sequence
    static constexpr int RP = 136;                        // pixels per row slot
    static constexpr int CBS = RP * 16 + 16;              // column-block stride (padded against bank conflicts)
    static constexpr int SLOT = (CIN / 8) * CBS;
    static constexpr int NS = 5;                          // row slots
    template <int NOUT> static constexpr size_t smem() { return (size_t)NOUT * KR * 2 + (size_t)NS * SLOT + 64; }
};

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(128)
conv3x3_row(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt, const float *__restrict__ bias,
            const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ Y, float *__restrict__ Yf, int H,
            int W, int rows, int *err) {
    using RC = RowConv<CIN>;
    constexpr int KPS = ConvK<CIN>::KP;
    constexpr int KR = RC::KR, NMMA = KR / 16, CB = CIN / 8, CBS = RC::CBS, SLOT = RC::SLOT, NS = RC::NS;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sb = sm;                       // NOUT x KR
    unsigned char *slots = sm + NOUT * KR * 2;    // NS x SLOT
    uint64_t *mbar = reinterpret_cast<uint64_t *>(slots + NS * SLOT);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * 128, ya = blockIdx.y * rows, img = blockIdx.z;
    const int yb = min(ya + rows, H);
    const size_t plane = (size_t)H * W;
    const __nv_bfloat16 *Xi = X + (size_t)img * plane * CIN;

    // weights, in the order of the MMA sequence
    for (int i = t; i < NOUT * (KR / 8); i += 128) {
        const int r = i / (KR / 8), kb = i % (KR / 8);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (CIN == 8) {
            const int dyi = kb / 4, dxs = kb % 4;
            if (dxs < 3) v = *reinterpret_cast<const uint4 *>(Wt + (size_t)r * KPS + (dyi * 3 + dxs) * 8);
        } else {
            v = *reinterpret_cast<const uint4 *>(Wt + (size_t)r * KPS + kb * 8);
        }
        *reinterpret_cast<uint4 *>(sb + kmajor_off(r, kb * 8, NOUT)) = v;
    }

    // slot of input row yy (yy >= -1)
    auto slot_of = [&](int yy) { return slots + ((yy + NS) % NS) * SLOT; };
    // one cp.async group per call (empty when the row is not needed)
    auto load_row = [&](int yy, bool need) {
        if (need) {
            unsigned char *slot = slot_of(yy);
            const bool rin = yy >= 0 && yy < H;
            for (int i = t; i < RC::RP * CB; i += 128) {
                const int j = i / CB, cb = i % CB;
                const int xx = x0 - 1 + j;
                const bool in = rin && xx >= 0 && xx < W;
                const __nv_bfloat16 *src = in ? Xi + ((size_t)yy * W + xx) * CIN + cb * 8 : X;
                cp_async16(slot + cb * CBS + j * 16, src, in ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    auto epilogue = [&](int y, uint32_t taddr) {
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), v);
        const int p = warp * 32 + lane, xx = x0 + p;
        if (xx >= W) return;
        const size_t pix = (size_t)img * plane + (size_t)y * W + xx;
        if (EPI == EPI_OUT) {
            Yf[pix] = v[0] + bias[0];
        } else {
            __align__(16) __nv_bfloat16 o[32];
            if (EPI == EPI_RELU) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) o[jj] = __float2bfloat16(fmaxf(v[jj] + bias[jj], 0.f));
            } else {
                __align__(16) __nv_bfloat16 m[32];
#pragma unroll
                for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(m)[q] = reinterpret_cast<const uint4 *>(mask + pix * 32)[q];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) o[jj] = __float2bfloat16(__bfloat162float(m[jj]) > 0.f ? v[jj] : 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(Y + pix * 32)[q] = reinterpret_cast<uint4 *>(o)[q];
        }
    };

    if (warp == 0) tmem_alloc(tslot, 64);
    if (t == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); }
    load_row(ya - 1, true);
    load_row(ya, true);
    load_row(ya + 1, true);
    load_row(ya + 2, ya + 2 <= yb);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phases = 0;   // bit h: parity of the next phase of mbar[h]
    bool ok = true;
    int it = 0;
    for (int y = ya; y < yb && ok; ++y, ++it) {
        const int half = it & 1;
        // rows y-1 .. y+1 have landed (only the group of row y+2 may be pending)
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
#pragma unroll 1
            for (int m = 0; m < NMMA; ++m) {
                uint32_t astart, lbo;
                if (CIN == 8) {
                    const int dyi = m / 2, pair = m % 2;
                    astart = smem_u32(slot_of(y + dyi - 1)) + pair * 2 * 16;
                    lbo = 16;
                } else {
                    const int tap = m / 2, hc = m % 2, dyi = tap / 3, dxi = tap % 3;
                    astart = smem_u32(slot_of(y + dyi - 1)) + hc * 2 * CBS + dxi * 16;
                    lbo = CBS;
                }
                const uint64_t ad = smem_desc(astart, lbo, 128);
                const uint64_t bd = smem_desc(smem_u32(sb) + m * NOUT * 32, NOUT * 16, 128);
                mma_bf16(tmem + half * 32, ad, bd, idesc_bf16_f32(NOUT), m > 0 ? 1u : 0u);
            }
            mma_commit(&mbar[half]);
        }
        if (it > 0) {
            const int pb = half ^ 1;
            ok = __syncthreads_and(mbar_wait(&mbar[pb], (phases >> pb) & 1u, kPolls));
            phases ^= 1u << pb;
            tc_fence_after();
            if (ok) epilogue(y - 1, tmem + pb * 32);
        }
        // the slot of row y+3 held row y-2, last read by the MMAs of row y-1
        if (ok) load_row(y + 3, y + 3 <= yb);
    }
    if (ok && it > 0) {
        const int pb = (it - 1) & 1;
        ok = __syncthreads_and(mbar_wait(&mbar[pb], (phases >> pb) & 1u, kPolls));
        phases ^= 1u << pb;
        tc_fence_after();
        if (ok) epilogue(yb - 1, tmem + pb * 32);
    }
    if (!ok) {
        // let MMAs in flight finish before the tensor memory is freed
        if (t == 0) atomicOr(err, 1);
        __syncthreads_and(mbar_wait(&mbar[0], phases & 1u, kPolls));
        __syncthreads_and(mbar_wait(&mbar[1], (phases >> 1) & 1u, kPolls));
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// Weight gradient: dW[k][n] = sum_p Xpatch[p][k] dY[p][n] (k = tap*CIN + c;
// row 9*CIN is a row of ones, giving the bias gradient sum_p dY[p][n]).
// GEMM D[k][n] = A[k][p] B[n][p]^T over 128-pixel chunks, A and B K-major
// over pixels, built by transposing the NHWC loads in shared memory.  Each
// CTA sums `rows` image rows; partial[cta][MT*128][NOUT] is reduced later.
// DYC: channels stored per pixel in dY (32, or 8 for the output layer).
template <int CIN, int NOUT, int DYC>
__global__ void __launch_bounds__(128)
wgrad_tc(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ dY, float *__restrict__ partial,
         int H, int W, int rows, int *err) {
    constexpr int MT = (9 * CIN + 1 + 127) / 128;       // M tiles of 128 k-rows
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sa = sm;                             // MT x (128 x 128)
    unsigned char *sb = sm + MT * 128 * 128 * 2;        // NOUT x 128
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + NOUT * 128 * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int img = blockIdx.y, y0 = blockIdx.x * rows;
    const size_t plane = (size_t)H * W;
    const __nv_bfloat16 *Xi = X + (size_t)img * plane * CIN;
    const __nv_bfloat16 *Di = dY + (size_t)img * plane * DYC;
    const __nv_bfloat16 one = __float2bfloat16(1.f), zero = __float2bfloat16(0.f);

    // zero the tiles once (padding rows stay zero); the ones row is rewritten below
    for (int i = t; i < (MT * 128 * 128 * 2 + NOUT * 128 * 2) / 16; i += 128)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    {
        const int kr = 9 * CIN;   // ones row
        __nv_bfloat16 *base = reinterpret_cast<__nv_bfloat16 *>(sa + (kr / 128) * 128 * 128 * 2);
        for (int p = t; p < 128; p += 128)
            *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(base) + kmajor_off(kr % 128, p, 128)) = one;
    }
    if (warp == 0) tmem_alloc(tslot, 128);
    if (t == 0) mbar_init(mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool ok = true, first = true;
    const int nseg = (W + 127) / 128;
#pragma unroll 1
    for (int yy = y0; yy < min(y0 + rows, H) && ok; ++yy) {
#pragma unroll 1
        for (int sgi = 0; sgi < nseg && ok; ++sgi) {
            const int x0 = sgi * 128;
            // A: the 9 shifted copies of X, transposed to rows (tap, c) x pixels
            const int p = t;
            const int xp = x0 + p;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int sy = yy + tap / 3 - 1, sx = xp + tap % 3 - 1;
                const bool in = xp < W && sy >= 0 && sy < H && sx >= 0 && sx < W;
#pragma unroll
                for (int cg = 0; cg < CIN / 8; ++cg) {
                    __align__(16) __nv_bfloat16 v[8];
                    if (in) reinterpret_cast<uint4 *>(v)[0] =
                        *reinterpret_cast<const uint4 *>(Xi + ((size_t)sy * W + sx) * CIN + cg * 8);
                    else reinterpret_cast<uint4 *>(v)[0] = make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int kr = tap * CIN + cg * 8 + j;
                        *reinterpret_cast<__nv_bfloat16 *>(sa + (kr / 128) * 128 * 128 * 2 + kmajor_off(kr % 128, p, 128)) = v[j];
                    }
                }
            }
            {   // ones row: 1 for pixels inside the image
                const int kr = 9 * CIN;
                *reinterpret_cast<__nv_bfloat16 *>(sa + (kr / 128) * 128 * 128 * 2 + kmajor_off(kr % 128, p, 128)) =
                    xp < W ? one : zero;
            }
            // B: dY transposed to rows n x pixels
            {
                __align__(16) __nv_bfloat16 v[DYC];
                if (xp < W) {
#pragma unroll
                    for (int q = 0; q < DYC / 8; ++q)
                        reinterpret_cast<uint4 *>(v)[q] = reinterpret_cast<const uint4 *>(Di + ((size_t)yy * W + xp) * DYC)[q];
                } else {
#pragma unroll
                    for (int q = 0; q < DYC / 8; ++q) reinterpret_cast<uint4 *>(v)[q] = make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int n = 0; n < (DYC < NOUT ? DYC : NOUT); ++n)
                    *reinterpret_cast<__nv_bfloat16 *>(sb + kmajor_off(n, p, NOUT)) = v[n];
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (t == 0) {
#pragma unroll 1
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll 1
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint64_t ad = smem_desc(smem_u32(sa + mt * 128 * 128 * 2) + kk * 128 * 32, 128 * 16, 128);
                        const uint64_t bd = smem_desc(smem_u32(sb) + kk * NOUT * 32, NOUT * 16, 128);
                        mma_bf16(tmem + mt * NOUT, ad, bd, idesc_bf16_f32(NOUT), (first && kk == 0) ? 0u : 1u);
                    }
                mma_commit(mbar);
            }
            first = false;
            ok = __syncthreads_and(mbar_wait(mbar, phase, kPolls));
            phase ^= 1;
            tc_fence_after();
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(err, 1);
        __syncthreads_and(mbar_wait(mbar, phase ^ 1, kPolls));
    }
    if (ok && !first) {
        float *out = partial + ((size_t)img * gridDim.x + blockIdx.x) * (MT * 128) * NOUT;
        for (int mt = 0; mt < MT; ++mt) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + mt * NOUT, v);
            const int row = mt * 128 + warp * 32 + lane;
#pragma unroll
            for (int n = 0; n < NOUT; ++n) out[(size_t)row * NOUT + n] = v[n];
        }
    } else if (ok) {
        float *out = partial + ((size_t)img * gridDim.x + blockIdx.x) * (MT * 128) * NOUT;
        for (int i = t; i < MT * 128 * NOUT; i += 128) out[i] = 0.f;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace swe_nn

// ======================================================================
// Elementwise kernels of the surrogate: weight layouts, Adam, the loss,
// input packing from solver states and the bed update.
// ======================================================================

namespace swe_nn {

// Reduce wgrad partials over CTAs/images: g[row][n] = sum_i partial[i][row][n].
__global__ void reduce_partials(const float *__restrict__ partial, int count, int rows, int nout, float *__restrict__ g) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * nout) return;
    float s = 0.f;
    for (int i = 0; i < count; ++i) s += partial[(size_t)i * rows * nout + idx];
    g[idx] = s;
}

// Master weights W[nout][9*cin] (FP32) -> forward BF16 [NOUTP][KP] and the
// flipped/transposed input-gradient BF16 [cin][KPD] with
// Wd[c][tap' * cind + n] = W[n][(8 - tap') * cin + c] (cind: padded nout).
__global__ void prep_weights(const float *__restrict__ Wm, int nout, int cin, int noutp, int kp,
                             __nv_bfloat16 *__restrict__ Wf, int cind, int kpd, __nv_bfloat16 *__restrict__ Wd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < noutp * kp) {
        const int n = idx / kp, k = idx % kp;
        const float v = (n < nout && k < 9 * cin) ? Wm[(size_t)n * 9 * cin + k] : 0.f;
        Wf[idx] = __float2bfloat16(v);
    }
    if (Wd && idx < cin * kpd) {
        const int c = idx / kpd, k = idx % kpd;
        float v = 0.f;
        if (k < 9 * cind) {
            const int tp = k / cind, n = k % cind;
            if (n < nout) v = Wm[(size_t)n * 9 * cin + (8 - tp) * cin + c];
        }
        Wd[idx] = __float2bfloat16(v);
    }
}

// Adam on FP32 parameters with gradient g[k][n] read from the transposed
// wgrad layout: param index (n, k) <- g[k * nout_g + n]; bias from row bias_row.
__global__ void adam_update(float *__restrict__ Wm, float *__restrict__ m, float *__restrict__ v, int nout, int kin,
                            const float *__restrict__ g, int nout_g, float *__restrict__ bias, float *__restrict__ mb,
                            float *__restrict__ vb, int bias_row, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = nout * kin;
    if (idx < nw) {
        const int n = idx / kin, k = idx % kin;
        const float gr = g[(size_t)k * nout_g + n];
        const float mm = b1 * m[idx] + (1.f - b1) * gr, vv = b2 * v[idx] + (1.f - b2) * gr * gr;
        m[idx] = mm; v[idx] = vv;
        Wm[idx] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    } else if (idx < nw + nout) {
        const int n = idx - nw;
        const float gr = g[(size_t)bias_row * nout_g + n];
        const float mm = b1 * mb[n] + (1.f - b1) * gr, vv = b2 * vb[n] + (1.f - b2) * gr * gr;
        mb[n] = mm; vb[n] = vv;
        bias[n] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    }
}

// dOut = 2 (out - target) / count as channel 0 of an NHWC8 BF16 tensor;
// the squared error is summed (per block) for the loss.
__global__ void loss_grad(const float *__restrict__ out, const float *__restrict__ target, size_t count,
                          __nv_bfloat16 *__restrict__ dOut, float *__restrict__ loss_sum) {
    __shared__ float red[256];
    float s = 0.f;
    const float scale = 2.f / (float)count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        s += d * d;
        __align__(16) __nv_bfloat16 o[8];
        o[0] = __float2bfloat16(scale * d);
#pragma unroll
        for (int j = 1; j < 8; ++j) o[j] = __float2bfloat16(0.f);
        reinterpret_cast<uint4 *>(dOut)[i] = reinterpret_cast<uint4 *>(o)[0];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss_sum, red[0]);
}

// Solver state (AoS float4 {H, Hu, Hv, b}, nx x ny) -> NHWC8 BF16 tiles of
// T x T (tile (tx, ty) of the domain -> batch index ty * ntx + tx), zeros
// beyond the domain.  Channels: (H, Hu, Hv, b) normalised as
// (x - norm[j]) / norm[4 + j]; the cell velocity (u, v) / norm[10]; and the
// Grass load direction of Eq. 3 with m = 2, v |v|^2, where the Shamov gate of
// Eq. 5 is open (|v|^6 > ksh H), over norm[11].  Dry cells: zero velocity.
__global__ void pack_state(const float4 *__restrict__ state, int nx, int ny, int T, int ntx, const float *__restrict__ norm,
                           float eps, float ksh, __nv_bfloat16 *__restrict__ X, size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane);
        const int r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        __align__(16) __nv_bfloat16 o[8];
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool in = x < nx && y < ny;
        if (in) c = state[(size_t)y * nx + x];
        const float f[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = __float2bfloat16(in ? (f[j] - norm[j]) / norm[4 + j] : 0.f);
        float u = 0.f, v = 0.f, jx = 0.f, jy = 0.f;
        if (in && c.x > eps) {
            u = c.y / c.x;
            v = c.z / c.x;
            const float s2 = u * u + v * v;
            if (s2 * s2 * s2 > ksh * c.x) { jx = u * s2; jy = v * s2; }
        }
        o[4] = __float2bfloat16(u / norm[10]);
        o[5] = __float2bfloat16(v / norm[10]);
        o[6] = __float2bfloat16(jx / norm[11]);
        o[7] = __float2bfloat16(jy / norm[11]);
        reinterpret_cast<uint4 *>(X)[i] = reinterpret_cast<uint4 *>(o)[0];
    }
}

// b += pred * out_std + out_mean on the solver state, for the cells of the tiles.
__global__ void apply_bed(float4 *__restrict__ state, int nx, int ny, int T, int ntx, const float *__restrict__ pred,
                          const float *__restrict__ norm, size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane);
        const int r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        if (x < nx && y < ny) state[(size_t)y * nx + x].w += pred[i] * norm[9] + norm[8];
    }
}

}  // namespace swe_nn

// ======================================================================
// The surrogate object (host side): layer buffers and launches.
// Network: 6 conv3x3 layers, 4(+4 zero) -> 32 -> 32 -> 32 -> 32 -> 32 -> 1,
// ReLU on the hidden layers, linear output; BF16 weights/activations, FP32
// accumulation, FP32 master weights with Adam.
// ======================================================================

#include <cmath>
#include <cstdlib>
#include <random>
#include <vector>

#include "swe_internal.h"

namespace {

struct NnLayer {
    int cin, nout, noutp, kp, cind, kpd, mt;
    float *Wm = nullptr, *m = nullptr, *v = nullptr, *bias = nullptr, *mb = nullptr, *vb = nullptr;
    __nv_bfloat16 *Wf = nullptr, *Wd = nullptr;
    float *grad = nullptr;   // [mt*128][noutp]
};

template <int CIN, int NOUT, int EPI> size_t conv_smem() { return (size_t)(128 + NOUT) * ConvK<CIN>::KP * 2 + 64; }
template <int CIN, int NOUT, int DYC> size_t wgrad_smem() {
    constexpr int MT = (9 * CIN + 1 + 127) / 128;
    return (size_t)MT * 128 * 128 * 2 + (size_t)NOUT * 128 * 2 + 64;
}

}  // namespace

struct swe_surrogate {
    int T = 1024, maxB = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    NnLayer L[6];
    __nv_bfloat16 *X0 = nullptr, *A[5] = {}, *dA[5] = {}, *dOut = nullptr;
    float *out = nullptr, *partial = nullptr, *loss = nullptr, *norm = nullptr, *tgt = nullptr, *bsave = nullptr;
    int *err = nullptr;
    size_t partial_floats = 0;
    long adam_t = 0;
    std::vector<void *> allocs;
    float h_norm[12] = {0, 0, 0, 0, 1, 1, 1, 1, 0, 1, 1, 1};
};

namespace {

cudaError_t salloc(swe_surrogate *s, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) { s->allocs.push_back(*p); cudaMemsetAsync(*p, 0, bytes, s->stream); }
    return e;
}

int grid_n(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 32); }

int g_persist = -1;   // 1: persistent pipelined convolutions (default), 0: one CTA per tile

template <int CIN, int NOUT, int EPI>
cudaError_t conv(swe_surrogate *s, const __nv_bfloat16 *X, const NnLayer &l, const __nv_bfloat16 *Wt, const float *bias,
                 const __nv_bfloat16 *mask, __nv_bfloat16 *Y, float *Yf, int B) {
    if (g_persist < 0) {
        // SWE_NN_CONV: 1 row-streaming (default), 2 persistent im2col, 0 one CTA per tile
        const char *e = getenv("SWE_NN_CONV");
        g_persist = (e && (e[0] == '0' || e[0] == '2')) ? e[0] - '0' : 1;
    }
    if (g_persist == 1) {
        // row-streaming kernel
        // at least 30 KB: at most 7 CTAs (448 TMEM columns) per SM
        const size_t smem = std::max<size_t>(RowConv<CIN>::template smem<NOUT>(), 30 * 1024);
        cudaFuncSetAttribute(conv3x3_row<CIN, NOUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int rows = 16;
        dim3 grid((s->T + 127) / 128, (s->T + rows - 1) / rows, B);
        conv3x3_row<CIN, NOUT, EPI><<<grid, 128, smem, s->stream>>>(X, Wt, bias, mask, Y, Yf, s->T, s->T, rows, s->err);
        return cudaGetLastError();
    }
    if (g_persist == 2) {
        const size_t smem = (size_t)(2 * 128 + NOUT) * ConvK<CIN>::KP * 2 + 64;
        cudaFuncSetAttribute(conv3x3_tcp<CIN, NOUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long ntile = (long long)B * s->T * ((s->T + 127) / 128);
        const int grid = (int)std::min<long long>(ntile, sms);
        conv3x3_tcp<CIN, NOUT, EPI><<<grid, 128, smem, s->stream>>>(X, Wt, bias, mask, Y, Yf, s->T, s->T, B, s->err);
        return cudaGetLastError();
    }
    const size_t smem = conv_smem<CIN, NOUT, EPI>();
    cudaFuncSetAttribute(conv3x3_tc<CIN, NOUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((s->T + 127) / 128, s->T, B);
    conv3x3_tc<CIN, NOUT, EPI><<<grid, 128, smem, s->stream>>>(X, Wt, bias, mask, Y, Yf, s->T, s->T, s->err);
    return cudaGetLastError();
}

constexpr int kWgradRows = 16;

template <int CIN, int NOUT, int DYC>
cudaError_t wgrad(swe_surrogate *s, const __nv_bfloat16 *X, const __nv_bfloat16 *dY, NnLayer &l, int B) {
    const size_t smem = wgrad_smem<CIN, NOUT, DYC>();
    cudaFuncSetAttribute(wgrad_tc<CIN, NOUT, DYC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((s->T + kWgradRows - 1) / kWgradRows, B);
    wgrad_tc<CIN, NOUT, DYC><<<grid, 128, smem, s->stream>>>(X, dY, s->partial, s->T, s->T, kWgradRows, s->err);
    const int rows = l.mt * 128;
    reduce_partials<<<(rows * NOUT + 255) / 256, 256, 0, s->stream>>>(s->partial, (int)(grid.x * grid.y), rows, NOUT,
                                                                      l.grad);
    return cudaGetLastError();
}

cudaError_t prep(swe_surrogate *s, NnLayer &l) {
    const int n = std::max(l.noutp * l.kp, l.Wd ? l.cin * l.kpd : 0);
    prep_weights<<<(n + 255) / 256, 256, 0, s->stream>>>(l.Wm, l.nout, l.cin, l.noutp, l.kp, l.Wf, l.cind, l.kpd, l.Wd);
    return cudaGetLastError();
}

cudaError_t forward_all(swe_surrogate *s, const __nv_bfloat16 *X, float *out, int B) {
    cudaError_t e = conv<8, 32, EPI_RELU>(s, X, s->L[0], s->L[0].Wf, s->L[0].bias, nullptr, s->A[0], nullptr, B);
    for (int i = 1; i < 5 && e == cudaSuccess; ++i)
        e = conv<32, 32, EPI_RELU>(s, s->A[i - 1], s->L[i], s->L[i].Wf, s->L[i].bias, nullptr, s->A[i], nullptr, B);
    if (e == cudaSuccess) e = conv<32, 16, EPI_OUT>(s, s->A[4], s->L[5], s->L[5].Wf, s->L[5].bias, nullptr, nullptr, out, B);
    return e;
}

swe_status check_err(swe_surrogate *s) {
    int h = 0;
    if (cudaMemcpyAsync(&h, s->err, 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return SWE_ECUDA;
    if (h) { cudaMemsetAsync(s->err, 0, 4, s->stream); return SWE_ETIMEOUT; }
    return SWE_OK;
}

}  // namespace

extern "C" swe_status swe_surrogate_destroy(swe_surrogate *s) {
    if (!s) return SWE_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return SWE_OK;
}

extern "C" swe_status swe_surrogate_create(int tile, int max_batch, uint64_t seed, void *cuda_stream, swe_surrogate **out) {
    if (!out || tile < 128 || (tile % 128) || max_batch < 1) return SWE_EINVAL;
    *out = nullptr;
    swe_surrogate *s = new swe_surrogate();
    s->T = tile;
    s->maxB = max_batch;
    if (cuda_stream) s->stream = (cudaStream_t)cuda_stream;
    else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess) s->own_stream = true;
    else { delete s; return SWE_ECUDA; }
    const int cins[6] = {8, 32, 32, 32, 32, 32}, nouts[6] = {32, 32, 32, 32, 32, 1};
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    const size_t pix = (size_t)max_batch * tile * tile;
    cudaError_t e = cudaSuccess;
    size_t maxpart = 0;
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
        NnLayer &l = s->L[i];
        l.cin = cins[i]; l.nout = nouts[i];
        l.noutp = l.nout == 1 ? 16 : 32;
        l.kp = (9 * l.cin + 15) / 16 * 16;
        l.cind = l.nout == 1 ? 8 : 32;
        l.kpd = (9 * l.cind + 15) / 16 * 16;
        l.mt = (9 * l.cin + 1 + 127) / 128;
        const int nw = l.nout * 9 * l.cin;
        e = salloc(s, (void **)&l.Wm, nw * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.m, nw * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.v, nw * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.bias, 32 * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.mb, 32 * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.vb, 32 * 4);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.Wf, (size_t)l.noutp * l.kp * 2);
        if (e == cudaSuccess && i > 0) e = salloc(s, (void **)&l.Wd, (size_t)l.cin * l.kpd * 2);
        if (e == cudaSuccess) e = salloc(s, (void **)&l.grad, (size_t)l.mt * 128 * l.noutp * 4);
        // He initialisation for the hidden layers, a small output layer
        std::vector<float> w(nw);
        const int fan_in = 9 * l.cin;
        const float sd = i == 5 ? 0.01f : std::sqrt(2.f / fan_in);
        for (int n = 0; n < l.nout; ++n)
            for (int k = 0; k < 9 * l.cin; ++k) {
                const int c = k % l.cin;
                (void)c;
                w[(size_t)n * 9 * l.cin + k] = sd * nd(rng);
            }
        if (e == cudaSuccess) e = cudaMemcpyAsync(l.Wm, w.data(), nw * 4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = prep(s, l);
        maxpart = std::max(maxpart, (size_t)l.mt * 128 * l.noutp);
    }
    if (e == cudaSuccess) e = salloc(s, (void **)&s->X0, pix * 8 * 2);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
        e = salloc(s, (void **)&s->A[i], pix * 32 * 2);
        if (e == cudaSuccess) e = salloc(s, (void **)&s->dA[i], pix * 32 * 2);
    }
    if (e == cudaSuccess) e = salloc(s, (void **)&s->dOut, pix * 8 * 2);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->out, pix * 4);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->tgt, pix * 4);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->bsave, pix * 4);
    s->partial_floats = maxpart * (size_t)max_batch * ((tile + kWgradRows - 1) / kWgradRows);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->partial, s->partial_floats * 4);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->loss, 16);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->norm, 64);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->err, 16);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->norm, s->h_norm, 48, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        swe_surrogate_destroy(s);
        return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
    }
    *out = s;
    return SWE_OK;
}

extern "C" swe_status swe_surrogate_set_norm(swe_surrogate *s, const float norm[12]) {
    if (!s || !norm) return SWE_EINVAL;
    for (int j : {4, 5, 6, 7, 9, 10, 11})
        if (!(norm[j] > 0)) return SWE_EINVAL;
    std::copy(norm, norm + 12, s->h_norm);
    if (cudaMemcpyAsync(s->norm, s->h_norm, 48, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) return SWE_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_forward(swe_surrogate *s, const void *X, float *out, int B) {
    if (!s || !X || !out || B < 1 || B > s->maxB) return SWE_EINVAL;
    if (forward_all(s, (const __nv_bfloat16 *)X, out, B) != cudaSuccess) return SWE_ECUDA;
    return check_err(s);
}

extern "C" swe_status swe_surrogate_train_step(swe_surrogate *s, const void *Xv, const float *target, int B, float lr,
                                              float *loss_out) {
    if (!s || !Xv || !target || B < 1 || B > s->maxB || !(lr > 0)) return SWE_EINVAL;
    const __nv_bfloat16 *X = (const __nv_bfloat16 *)Xv;
    const size_t pix = (size_t)B * s->T * s->T;
    cudaError_t e = forward_all(s, X, s->out, B);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, 4, s->stream);
    if (e == cudaSuccess) {
        loss_grad<<<grid_n(pix), 256, 0, s->stream>>>(s->out, target, pix, s->dOut, s->loss);
        e = cudaGetLastError();
    }
    // backward: gradient w.r.t. the pre-activations of layers 5..1, then weights
    if (e == cudaSuccess) e = conv<8, 32, EPI_MASK>(s, s->dOut, s->L[5], s->L[5].Wd, nullptr, s->A[4], s->dA[4], nullptr, B);
    for (int i = 4; i >= 1 && e == cudaSuccess; --i)
        e = conv<32, 32, EPI_MASK>(s, s->dA[i], s->L[i], s->L[i].Wd, nullptr, s->A[i - 1], s->dA[i - 1], nullptr, B);
    if (e == cudaSuccess) e = wgrad<32, 16, 8>(s, s->A[4], s->dOut, s->L[5], B);
    for (int i = 4; i >= 1 && e == cudaSuccess; --i) e = wgrad<32, 32, 32>(s, s->A[i - 1], s->dA[i], s->L[i], B);
    if (e == cudaSuccess) e = wgrad<8, 32, 32>(s, X, s->dA[0], s->L[0], B);
    // Adam
    ++s->adam_t;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)s->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)s->adam_t));
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
        NnLayer &l = s->L[i];
        const int kin = 9 * l.cin, n = l.nout * kin + l.nout;
        adam_update<<<(n + 255) / 256, 256, 0, s->stream>>>(l.Wm, l.m, l.v, l.nout, kin, l.grad, l.noutp, l.bias, l.mb,
                                                            l.vb, kin, lr, b1, b2, eps, c1, c2);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = prep(s, l);
    }
    float h = 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, s->loss, 4, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return SWE_ECUDA;
    swe_status st = check_err(s);
    if (loss_out) *loss_out = h / (float)pix;
    return st;
}

// Weights and biases of layer `layer` as FP32: W[nout][9*cin] (k = tap*cin + c)
// then bias[nout].  get (dir 0) or set (dir 1); host arrays.
extern "C" swe_status swe_surrogate_params(swe_surrogate *s, int layer, float *host, int dir) {
    if (!s || !host || layer < 0 || layer > 5) return SWE_EINVAL;
    NnLayer &l = s->L[layer];
    const size_t nw = (size_t)l.nout * 9 * l.cin;
    cudaError_t e;
    if (dir == 0) {
        e = cudaMemcpyAsync(host, l.Wm, nw * 4, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host + nw, l.bias, l.nout * 4, cudaMemcpyDeviceToHost, s->stream);
    } else {
        e = cudaMemcpyAsync(l.Wm, host, nw * 4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(l.bias, host + nw, l.nout * 4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = prep(s, l);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

// Gradients of the last train_step for layer `layer`: dW[nout][9*cin] then
// dbias[nout] (FP32 host array), for checks against a CPU reference.
extern "C" swe_status swe_surrogate_grads(swe_surrogate *s, int layer, float *host) {
    if (!s || !host || layer < 0 || layer > 5) return SWE_EINVAL;
    NnLayer &l = s->L[layer];
    const int kin = 9 * l.cin;
    std::vector<float> g((size_t)l.mt * 128 * l.noutp);
    if (cudaMemcpyAsync(g.data(), l.grad, g.size() * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return SWE_ECUDA;
    for (int n = 0; n < l.nout; ++n) {
        for (int k = 0; k < kin; ++k) host[(size_t)n * kin + k] = g[(size_t)k * l.noutp + n];
        host[(size_t)l.nout * kin + n] = g[(size_t)kin * l.noutp + n];
    }
    return SWE_OK;
}

// Internal activation buffers (device pointers) for tests: index 0..4 = the
// outputs of layers 1..5 (NHWC32 BF16), 5 = the output (FP32 per pixel).
extern "C" swe_status swe_surrogate_buffer(swe_surrogate *s, int index, void **ptr) {
    if (!s || !ptr || index < 0 || index > 5) return SWE_EINVAL;
    *ptr = index < 5 ? (void *)s->A[index] : (void *)s->out;
    return SWE_OK;
}

// ---------------------------------------------------------------- solver coupling

static bool handle_state(swe_handle *h, SweConst **c, void **cur, cudaStream_t *st) {
    SweBufs *b;
    int prec;
    bool set;
    if (!swe_impl::handle_view(h, c, &b, st, nullptr, &prec, &set) || !set || prec != SWE_FP32) return false;
    *cur = swe_impl::handle_current_state(h);
    return *cur != nullptr;
}

extern "C" swe_status swe_surrogate_pack_state(swe_surrogate *s, swe_handle *h, void *X, int *batch) {
    SweConst *c;
    void *cur;
    cudaStream_t hs;
    if (!s || !h || !X || !handle_state(h, &c, &cur, &hs)) return SWE_EINVAL;
    const int ntx = (c->nx + s->T - 1) / s->T, nty = (c->ny + s->T - 1) / s->T;
    if (ntx * nty > s->maxB) return SWE_EINVAL;
    const size_t total = (size_t)ntx * nty * s->T * s->T;
    pack_state<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->norm,
                                                     c->eps_f, c->f.ksh, (__nv_bfloat16 *)X, total);
    if (batch) *batch = ntx * nty;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

namespace {
__global__ void bed_tiles(const float4 *__restrict__ state, int nx, int ny, int T, int ntx, float *__restrict__ b,
                          size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane), r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        b[i] = (x < nx && y < ny) ? state[(size_t)y * nx + x].w : 0.f;
    }
}
__global__ void make_target(const float *__restrict__ b0, const float *__restrict__ b1, const float *__restrict__ norm,
                            float *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = ((b1[i] - b0[i]) - norm[8]) / norm[9];
}
}  // namespace

// Target of a sample: the handle's bed now minus the bed saved by the last
// swe_surrogate_save_bed call, normalised, in the tile layout (device out).
extern "C" swe_status swe_surrogate_save_bed(swe_surrogate *s, swe_handle *h) {
    SweConst *c;
    void *cur;
    cudaStream_t hs;
    if (!s || !h || !handle_state(h, &c, &cur, &hs)) return SWE_EINVAL;
    const int ntx = (c->nx + s->T - 1) / s->T, nty = (c->ny + s->T - 1) / s->T;
    if (ntx * nty > s->maxB) return SWE_EINVAL;
    const size_t total = (size_t)ntx * nty * s->T * s->T;
    bed_tiles<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->bsave, total);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_pack_target(swe_surrogate *s, swe_handle *h, float *target) {
    SweConst *c;
    void *cur;
    cudaStream_t hs;
    if (!s || !h || !target || !handle_state(h, &c, &cur, &hs)) return SWE_EINVAL;
    const int ntx = (c->nx + s->T - 1) / s->T, nty = (c->ny + s->T - 1) / s->T;
    const size_t total = (size_t)ntx * nty * s->T * s->T;
    bed_tiles<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->tgt, total);
    make_target<<<grid_n(total), 256, 0, s->stream>>>(s->bsave, s->tgt, s->norm, target, total);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

// Predicts the bed change of one window from the handle's current state and
// adds it to the bed (b += pred * std + mean) in place.
extern "C" swe_status swe_surrogate_apply(swe_surrogate *s, swe_handle *h) {
    SweConst *c;
    void *cur;
    cudaStream_t hs;
    if (!s || !h || !handle_state(h, &c, &cur, &hs)) return SWE_EINVAL;
    const int ntx = (c->nx + s->T - 1) / s->T, nty = (c->ny + s->T - 1) / s->T;
    if (ntx * nty > s->maxB) return SWE_EINVAL;
    const int B = ntx * nty;
    const size_t total = (size_t)B * s->T * s->T;
    pack_state<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->norm, c->eps_f,
                                                     c->f.ksh, s->X0, total);
    if (forward_all(s, s->X0, s->out, B) != cudaSuccess) return SWE_ECUDA;
    apply_bed<<<grid_n(total), 256, 0, s->stream>>>((float4 *)cur, c->nx, c->ny, s->T, ntx, s->out, s->norm, total);
    if (cudaGetLastError() != cudaSuccess) return SWE_ECUDA;
    swe_status st = check_err(s);
    if (st == SWE_OK) st = (swe_status)swe_impl::handle_state_changed(h);
    return st;
}

namespace {
// Judged-window error sums (FP64): |b0 + pred - b1|, |b1 - b0|, |b1|,
// |last - (b1 - b0)| over the cells of the domain.
__global__ void judge_sums(const float *__restrict__ b0, const float *__restrict__ b1, const float *__restrict__ pred,
                           const float *__restrict__ last, const float *__restrict__ norm, int nx, int ny, int T, int ntx,
                           size_t total, double *__restrict__ out) {
    __shared__ double red[4][256];
    double a = 0, b = 0, c = 0, d = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane), r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        if (x >= nx || y >= ny) continue;
        const double ch = (double)b1[i] - (double)b0[i];
        const double pr = (double)pred[i] * norm[9] + norm[8];
        a += fabs(pr - ch);
        b += fabs(ch);
        c += fabs((double)b1[i]);
        d += fabs((double)last[i] - ch);
    }
    red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c; red[3][threadIdx.x] = d;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) atomicAdd(&out[q], red[q][0]);
}
__global__ void diff_into(const float *__restrict__ b0, const float *__restrict__ b1, float *__restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d[i] = b1[i] - b0[i];
}
}  // namespace

// Surrogate-accelerated run (morphological acceleration, a project addition):
// each window stands for K coupled steps of the bed.  In a surrogate window
// the network predicts the window's bed change from the window's start state,
// the water alone is advanced K/f steps (Exner coupling off), and the
// prediction is added to the bed: the bed's simulated time advances f times
// faster than the water's.  Every judge_every-th window is judged instead:
// the plain coupled solver runs the K steps from the same start state, the
// relative L1 error of the predicted bed change against it is recorded (and,
// for reference, that of a zero change and of repeating the last judged
// change), and the run continues from the plain result.  A judged error above
// `bound` hands every remaining window to the plain solver.
extern "C" swe_status swe_surrogate_run(swe_surrogate *s, swe_handle *h, int nwindows, int K, int f, int judge_every,
                                       double bound, swe_surrogate_stats *st) {
    SweConst *c;
    void *cur;
    cudaStream_t hs;
    if (!s || !h || !st || nwindows < 0 || K < 1 || f < 1 || (K % f) || judge_every < 1 || !(bound > 0) ||
        !handle_state(h, &c, &cur, &hs))
        return SWE_EINVAL;
    const int ntx = (c->nx + s->T - 1) / s->T, nty = (c->ny + s->T - 1) / s->T;
    const int B = ntx * nty;
    if (B > s->maxB) return SWE_EINVAL;
    const size_t total = (size_t)B * s->T * s->T;
    double *dsum = nullptr;
    float *last = nullptr;
    if (cudaMalloc(&dsum, 4 * sizeof(double)) != cudaSuccess) return SWE_ENOMEM;
    if (cudaMalloc(&last, total * 4) != cudaSuccess) { cudaFree(dsum); return SWE_ENOMEM; }
    cudaMemsetAsync(last, 0, total * 4, s->stream);
    double err_sum = 0, zero_sum = 0, pers_sum = 0;
    swe_status rc = SWE_OK;
    for (int w = 0; w < nwindows && rc == SWE_OK; ++w) {
        double t0 = 0, t1 = 0;
        if ((rc = swe_get_time(h, &t0)) != SWE_OK) break;
        if (st->mode == 1) {                                     // plain coupled window
            if ((rc = swe_run_steps(h, K)) != SWE_OK || (rc = swe_get_time(h, &t1)) != SWE_OK) break;
            st->bed_time += t1 - t0;
            st->water_time += t1 - t0;
            ++st->plain_windows;
        } else if (w % judge_every == 0) {                       // judged window
            handle_state(h, &c, &cur, &hs);
            pack_state<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->norm, c->eps_f,
                                                     c->f.ksh, s->X0, total);
            bed_tiles<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->bsave, total);
            if (forward_all(s, s->X0, s->out, B) != cudaSuccess) { rc = SWE_ECUDA; break; }
            if ((rc = check_err(s)) != SWE_OK) break;
            if ((rc = swe_run_steps(h, K)) != SWE_OK || (rc = swe_get_time(h, &t1)) != SWE_OK) break;
            handle_state(h, &c, &cur, &hs);
            bed_tiles<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->tgt, total);
            cudaMemsetAsync(dsum, 0, 4 * sizeof(double), s->stream);
            judge_sums<<<grid_n(total), 256, 0, s->stream>>>(s->bsave, s->tgt, s->out, last, s->norm, c->nx, c->ny,
                                                            s->T, ntx, total, dsum);
            diff_into<<<grid_n(total), 256, 0, s->stream>>>(s->bsave, s->tgt, last, total);
            double hsum[4];
            if (cudaMemcpyAsync(hsum, dsum, sizeof hsum, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
                cudaStreamSynchronize(s->stream) != cudaSuccess) { rc = SWE_ECUDA; break; }
            const double ref = hsum[1] > 0 ? hsum[1] : 1e-300;
            const double err = hsum[0] / ref;
            st->err_last = err;
            st->err_max = std::max(st->err_max, err);
            st->elev_err_max = std::max(st->elev_err_max, hsum[0] / (hsum[2] > 0 ? hsum[2] : 1e-300));
            err_sum += err;
            zero_sum += 1.0;
            pers_sum += hsum[3] / ref;
            ++st->judged;
            st->err_mean = err_sum / st->judged;
            st->err_zero_mean = zero_sum / st->judged;
            st->err_persist_mean = pers_sum / st->judged;
            st->bed_time += t1 - t0;
            st->water_time += t1 - t0;
            if (err > bound) { st->mode = 1; st->takeover_window = w; }
        } else {                                                 // surrogate window
            handle_state(h, &c, &cur, &hs);
            pack_state<<<grid_n(total), 256, 0, s->stream>>>((const float4 *)cur, c->nx, c->ny, s->T, ntx, s->norm, c->eps_f,
                                                     c->f.ksh, s->X0, total);
            if (forward_all(s, s->X0, s->out, B) != cudaSuccess) { rc = SWE_ECUDA; break; }
            if ((rc = check_err(s)) != SWE_OK) break;
            if ((rc = swe_set_sediment(h, 0)) != SWE_OK) break;
            rc = swe_run_steps(h, K / f);
            swe_status r2 = swe_set_sediment(h, 1);
            if (rc == SWE_OK) rc = r2;
            if (rc != SWE_OK || (rc = swe_get_time(h, &t1)) != SWE_OK) break;
            handle_state(h, &c, &cur, &hs);
            apply_bed<<<grid_n(total), 256, 0, s->stream>>>((float4 *)cur, c->nx, c->ny, s->T, ntx, s->out, s->norm, total);
            if (cudaStreamSynchronize(s->stream) != cudaSuccess) { rc = SWE_ECUDA; break; }
            rc = (swe_status)swe_impl::handle_state_changed(h);
            st->bed_time += (t1 - t0) * f;
            st->water_time += t1 - t0;
            ++st->surrogate_windows;
        }
        ++st->windows;
    }
    cudaFree(dsum);
    cudaFree(last);
    return rc;
}
