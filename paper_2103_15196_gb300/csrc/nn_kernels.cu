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
// implicit GEMMs on the tensor cores.  Activations are BF16 with 8 (input)
// or 32 channels in the row-planar layout below; weights are K-major BF16
// [nout][k], k = tap * cin + c, tap = (dy + 1) * 3 + (dx + 1).  FP32
// accumulators live in tensor memory (128 pixel lanes x nout columns).
// ======================================================================

namespace swe_nn {

enum { EPI_RELU = 0, EPI_OUT = 1, EPI_MASK = 2 };

// Activations are stored row-planar: [image][y][channel block][x][8]
// (BF16), so that one row of one 8-channel block is contiguous.  With 8
// channels this is plain NHWC.  Element offset of channel block cb of pixel
// (x, y) of image img, for C channels:
__device__ __forceinline__ size_t act_off(int img, int y, int x, int cb, int C, int H, int W) {
    return ((((size_t)img * H + y) * (C / 8) + cb) * W + x) * 8;
}

template <int CIN> struct ConvK {
    static constexpr int K = 9 * CIN;
    static constexpr int KP = (K + 15) / 16 * 16;   // padded to whole MMAs
};

// 3x3 convolution with zero padding on the tensor cores (tcgen05, BF16 x
// BF16 -> FP32 in tensor memory), no im2col.  Epilogues: EPI_RELU (forward,
// hidden layer): bias + ReLU -> BF16; EPI_OUT (the output layer): m (channel
// 0 + bias + p) -> FP32 per pixel, where p and m are channels 6 (the linear
// extrapolation of the bed change) and 7 (the activity mask) of the network
// input, passed as `mask`; EPI_MASK (input gradient): times (mask > 0) ->
// BF16.
//
// A CTA owns one 128-pixel column band of an image and a run of output rows,
// computed four at a time.  Each input row is loaded once, by bulk copies of
// its contiguous row segments (one per 8-channel block, pixels x0-1 ..
// x0+134 clipped to the image), into a slot laid out K-major: the 136 pixels
// of a channel block 16 bytes apart, blocks CBS bytes apart.  The A operand
// of column tap dx is that slot read from pixel dx+1 on (the descriptor's
// start moved by 16 (dx+1) bytes); with 8 input channels one MMA covers two
// neighbouring column taps (LBO = 16 bytes).
//
// An input row feeds at most three of the four output rows, through the
// weights of row taps dy = +1, 0, -1 (in that order of output row).  The
// weights of each K-slice (column tap and channel half) are stored as a
// 3-block array [W(dy=+1); W(0); W(-1)] of NOUT rows each, so that one MMA per
// input row and K-slice covers all the output rows it feeds: N = NOUT x
// (rows fed), B = the matching sub-range of the array, D = the accumulator
// columns of those rows (row r at column r NOUT).  A batch of four output
// rows takes 6 x 6 + 1 MMAs (32 channels; 6 x 2 + 1 with 8) instead of 4 x 18:
// the MMA cost is per instruction (about 151 cycles for any N <= 256), so
// wider MMAs are faster.  The extra MMA zeroes the accumulator (zero A and B).
// Pixels outside the image stay at the zeros written when the CTA starts;
// rows outside it are not loaded and their MMAs are not issued.
//
// Warp roles, with no block-wide barrier in the row loop:
//   warp 4, lane 0  - producer: bulk copies of input rows into a ring of NS
//                     slots (mbarrier `full` per slot), each slot refilled
//                     once `freed`;
//   warp 5, lane 0  - MMA issuer: a batch of four output rows into one of two
//                     TMEM stages; tcgen05.commit to `accf` (stage ready) and
//                     `freed` (input rows no later batch needs);
//   warps 0-3       - epilogue: wait `accf`, read the stage from TMEM row by
//                     row, release it (`acce`), convert and store.
// Output row j (y = ya + j) reads input rows q = j, j+1, j+2 (y-1, y, y+1).
// All waits are bounded; a timeout raises a shared abort flag that ends every
// role's waits, the producer and the MMA issuer then let their copies and MMAs
// in flight finish, and *err is set.
template <int CIN, int NOUT> struct WsConv {
    static constexpr int CB = CIN / 8;
    static constexpr int CBS = 136 * 16;                  // 2176 B: a 128-byte multiple (bulk-copy destination)
    static constexpr int SLOT = CB * CBS;
    static constexpr int NSLICE = CIN == 8 ? 2 : 6;       // K-slices per input row
    static constexpr int WSL = 3 * NOUT * 16 * 2;         // bytes of one K-slice's 3-block weight array
    static constexpr int ZERO = 128 * 16 * 2;             // a zero 128 x 16 tile
    static constexpr int NS = 10;                         // input row slots: a batch's 6 + the next 4
    static constexpr int SC = 4 * NOUT;                   // TMEM columns of a stage (four rows)
    static constexpr int TCOLS = SC * 2 <= 32 ? 32 : (SC * 2 <= 64 ? 64 : (SC * 2 <= 128 ? 128 : 256));
    static constexpr size_t smem() {
        return (size_t)NSLICE * WSL + ZERO + (size_t)NS * SLOT + (2 * NS + 4) * 8 + 16;
    }
};

// Bounded wait on an mbarrier phase: try_wait (which suspends briefly in
// hardware) without sleeping for the first polls, then with a short back-off.
__device__ __forceinline__ bool ws_wait(uint64_t *mbar, uint32_t parity, volatile int *abort, bool honour_abort) {
    for (int i = 0; i < kPolls; ++i) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (honour_abort && *abort) return false;
        if (i > 256) __nanosleep(64);
    }
    *abort = 1;
    return false;
}

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(192)
conv3x3_ws(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt,
           const float *__restrict__ bias, const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ Y,
           float *__restrict__ Yf, int H, int W, int rows, int *err) {
    using WC = WsConv<CIN, NOUT>;
    constexpr int KPS = ConvK<CIN>::KP;
    constexpr int CB = WC::CB, CBS = WC::CBS, SLOT = WC::SLOT, NSLICE = WC::NSLICE, WSL = WC::WSL;
    constexpr int NS = WC::NS, SC = WC::SC;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sw = sm;                                   // NSLICE x WSL weight arrays
    unsigned char *zero = sw + NSLICE * WSL;                  // zero tile
    unsigned char *slots = zero + WC::ZERO;                   // NS x SLOT
    uint64_t *full = reinterpret_cast<uint64_t *>(slots + NS * SLOT);
    uint64_t *freed = full + NS;
    uint64_t *accf = freed + NS;
    uint64_t *acce = accf + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * 128, ya = blockIdx.y * rows, img = blockIdx.z;
    const int nrows = min(ya + rows, H) - ya;                 // >= 1
    const int nin = nrows + 2;
    const size_t plane = (size_t)H * W;

    // weights: slice s, block blk (row tap dyi = 2 - blk), output channel co,
    // 16-channel K chunk kc of 8
    for (int i = t; i < NSLICE * 3 * NOUT * 2; i += blockDim.x) {
        const int kc = i & 1, n = (i >> 1) % (3 * NOUT), sl = (i >> 1) / (3 * NOUT);
        const int blk = n / NOUT, co = n % NOUT, dyi = 2 - blk;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (CIN == 8) {
            const int dx = 2 * sl + kc;
            if (dx < 3) v = *reinterpret_cast<const uint4 *>(Wt + (size_t)co * KPS + (dyi * 3 + dx) * 8);
        } else {
            const int dx = sl >> 1, h = sl & 1;
            v = *reinterpret_cast<const uint4 *>(Wt + (size_t)co * KPS + (dyi * 3 + dx) * CIN + h * 16 + kc * 8);
        }
        *reinterpret_cast<uint4 *>(sw + sl * WSL + kmajor_off(n, kc * 8, 3 * NOUT)) = v;
    }
    // zero tile and slots: pixels outside the image are never written again
    for (int i = t; i < (WC::ZERO + NS * SLOT) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(zero)[i] = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    if (warp == 0) tmem_alloc(tslot, WC::TCOLS);
    if (t == 0) {
        for (int q = 0; q < NS; ++q) { mbar_init(&full[q], 1); mbar_init(&freed[q], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 4); }
        *abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nbatch = (nrows + 3) / 4;

    if (warp == 4) {
        if (lane == 0) {
            const int xs = max(x0 - 1, 0), xe = min(x0 + 135, W);   // pixels [xs, xe) of the row segment
            const uint32_t seg = (uint32_t)(xe - xs) * 16;
            int q = 0;
            bool ok = true;
            for (; q < nin; ++q) {
                const int sl = q % NS, yy = ya - 1 + q;
                if (q >= NS && !(ok = ws_wait(&freed[sl], (uint32_t)((q / NS) - 1) & 1u, abort, true))) break;
                if (yy < 0 || yy >= H) {      // not loaded: its MMAs are not issued
                    mbar_arrive(&full[sl]);
                    continue;
                }
                mbar_arrive_expect_tx(&full[sl], CB * seg);
#pragma unroll
                for (int cb = 0; cb < CB; ++cb)
                    bulk_load(slots + sl * SLOT + cb * CBS + (xs - (x0 - 1)) * 16, X + act_off(img, yy, xs, cb, CIN, H, W),
                              seg, &full[sl]);
            }
            if (!ok) atomicOr(err, 1);
            // the copies of the last rows issued must land before the CTA ends
            for (int p = max(0, q - NS); p < q; ++p) ws_wait(&full[p % NS], (uint32_t)(p / NS) & 1u, abort, false);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            int landed = 0, freed_rows = 0;
            bool ok = true, any = false;
            const uint64_t zd = smem_desc(smem_u32(zero), 128 * 16, 128);
            for (int b = 0; b < nbatch && ok; ++b) {
                const int j0 = 4 * b, nb = min(4, nrows - j0), st = b & 1;
                while (ok && landed < j0 + nb + 2) {
                    ok = ws_wait(&full[landed % NS], (uint32_t)(landed / NS) & 1u, abort, true);
                    if (ok) ++landed;
                }
                if (ok && b >= 2) ok = ws_wait(&acce[st], (uint32_t)((b / 2) - 1) & 1u, abort, true);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dst = tmem + st * SC;
                mma_bf16(dst, zd, zd, idesc_bf16_f32(SC), 0u);
#pragma unroll 1
                for (int yi = 0; yi < nb + 2; ++yi) {
                    const int q = j0 + yi, yy = ya - 1 + q;
                    if (yy < 0 || yy >= H) continue;
                    const int r_lo = max(0, yi - 2), r_hi = min(nb - 1, yi);
                    if (r_lo > r_hi) continue;
                    const int cnt = r_hi - r_lo + 1, off = 2 - (yi - r_lo);   // first block: row tap yi - r_lo
                    const uint32_t slot = smem_u32(slots + (q % NS) * SLOT);
#pragma unroll
                    for (int sl = 0; sl < NSLICE; ++sl) {
                        uint32_t aoff, lbo;
                        if (CIN == 8) { aoff = sl * 2 * 16; lbo = 16; }
                        else { aoff = (sl & 1) * 2 * CBS + (sl >> 1) * 16; lbo = CBS; }
                        const uint64_t ad = smem_desc(slot + aoff, lbo, 128);
                        const uint64_t bd = smem_desc(smem_u32(sw + sl * WSL) + off * NOUT * 16, 3 * NOUT * 16, 128);
                        mma_bf16(dst + r_lo * NOUT, ad, bd, idesc_bf16_f32(cnt * NOUT), 1u);
                    }
                }
                mma_commit(&accf[st]);
                // input rows no later batch reads: q < j0 + nb (the next batch starts at row j0 + 4)
                for (; freed_rows < j0 + nb; ++freed_rows) mma_commit(&freed[freed_rows % NS]);
                any = true;
            }
            if (!ok) atomicOr(err, 1);
            // MMAs in flight must finish before the tensor memory is freed
            if (any) {
                const int jl = freed_rows - 1;
                ws_wait(&freed[jl % NS], (uint32_t)(jl / NS) & 1u, abort, false);
            }
        }
    } else {
        for (int b = 0; b < nbatch; ++b) {
            const int j0 = 4 * b, nb = min(4, nrows - j0), st = b & 1;
            if (!ws_wait(&accf[st], (uint32_t)(b / 2) & 1u, abort, true)) {
                if (lane == 0) atomicOr(err, 1);
                break;
            }
            tc_fence_after();
            const int p = warp * 32 + lane, xx = x0 + p;
            for (int r = 0; r < nb; ++r) {
                const uint32_t ta = tmem + st * SC + r * NOUT + ((uint32_t)(warp * 32) << 16);
                const int y = ya + j0 + r;
                if (NOUT == 16) {
                    float v[16];
                    tmem_ld16(ta, v);
                    if (r == nb - 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acce[st]);
                    }
                    if (xx < W && EPI == EPI_OUT) {
                        const size_t pix = (size_t)img * plane + (size_t)y * W + xx;
                        const __nv_bfloat162 pm = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * 8 + 6);
                        Yf[pix] = __high2float(pm) * (v[0] + bias[0] + __low2float(pm));
                    }
                } else {
                    float v[32];
                    tmem_ld32(ta, v);
                    if (r == nb - 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acce[st]);
                    }
                    if (xx >= W) continue;
                    __align__(16) __nv_bfloat16 o[32];
                    if (EPI == EPI_RELU) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) o[jj] = __float2bfloat16(fmaxf(v[jj] + bias[jj], 0.f));
                    } else {
                        __align__(16) __nv_bfloat16 mk[32];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            reinterpret_cast<uint4 *>(mk)[q] =
                                *reinterpret_cast<const uint4 *>(mask + act_off(img, y, xx, q, 32, H, W));
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            o[jj] = __float2bfloat16(__bfloat162float(mk[jj]) > 0.f ? v[jj] : 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4 *>(Y + act_off(img, y, xx, q, 32, H, W)) = reinterpret_cast<uint4 *>(o)[q];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, WC::TCOLS);
}

// Weight gradient: dW[k][n] = sum_p Xpatch[p][k] dY[p][n] (k = tap*CIN + c;
// row 9*CIN is a row of ones, giving the bias gradient sum_p dY[p][n]).
// GEMM D[k][n] = A[k][p] B[n][p]^T over 128-pixel chunks, A and B K-major
// over pixels, built by transposing the activation loads in shared memory.  Each
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
                        *reinterpret_cast<const uint4 *>(X + act_off(img, sy, sx, cg, CIN, H, W));
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
                        reinterpret_cast<uint4 *>(v)[q] = *reinterpret_cast<const uint4 *>(dY + act_off(img, yy, xp, q, DYC, H, W));
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

// Loss gradient as channel 0 of an NHWC8 BF16 tensor, m the activity mask
// (channel 7 of the input X; out = m (...)), d = out - target:
//   l1 = 0: mean squared error, dOut = 2 m d / count;
//   l1 = 1: mean absolute error, dOut = m sign(d) / count (0 at d = 0).
// The per-pixel loss is summed (per block).
__global__ void loss_grad(const float *__restrict__ out, const float *__restrict__ target,
                          const __nv_bfloat16 *__restrict__ X, size_t count, int l1, __nv_bfloat16 *__restrict__ dOut,
                          float *__restrict__ loss_sum) {
    __shared__ float red[256];
    float s = 0.f;
    const float scale = (l1 ? 1.f : 2.f) / (float)count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        const float gd = l1 ? (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) : d;
        s += l1 ? fabsf(d) : d * d;
        __align__(16) __nv_bfloat16 o[8];
        o[0] = __float2bfloat16(__bfloat162float(X[i * 8 + 7]) * scale * gd);
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
// beyond the domain.  The channels (see cell_features): (H, b) normalised as
// (x - norm[j]) / norm[j + 1], the cell velocity (u, v) / norm[4], the
// Shamov ratio |v| / v_k of Eq. 5, the second difference of the bed over the
// window's two coupled steps, their linear extrapolation p, and the activity
// mask.  Dry cells: zero velocity and ratio.
#ifndef SWE_ACT_R
#define SWE_ACT_R 4
#endif
constexpr int kActR = SWE_ACT_R;   // Chebyshev radius of the activity mask

__device__ __forceinline__ size_t tile_index(int x, int y, int T, int ntx) {
    return ((size_t)(y / T) * ntx + x / T) * T * T + (size_t)(y % T) * T + x % T;
}

// Channels 0-6 of the network input for one cell with state c, the bed b0 at
// the window's start and b1 after its first coupled step (c.w is the bed
// after the second): 0, 1 (H, b) normalised; 2, 3 the velocity (u, v) /
// norm[4]; 4 the Shamov ratio |v| / v_k = (|v|^6 / (C_Sh^6 d50^2 H))^(1/6)
// (Eq. 5), at most 4; 5 the second difference (b2 - b1) - (b1 - b0) and 6 the
// two-step change b2 - b0, both over 2 norm[7]: in output units, channel 6
// is the linear extrapolation of the two steps to the window, and channel
// 6 - channel 5 that of the first step alone.
__device__ __forceinline__ void cell_features(const float4 c, float b0, float b1, const float *__restrict__ norm,
                                              float eps, float ksh, float f[8]) {
    f[0] = (c.x - norm[0]) / norm[1];
    f[1] = (c.w - norm[2]) / norm[3];
    if (c.x > eps) {
        const float u = c.y / c.x, v = c.z / c.x, s2 = u * u + v * v;
        f[2] = u / norm[4];
        f[3] = v / norm[4];
        const float r6 = (s2 * s2 * s2) / (ksh * c.x);
        f[4] = fminf(exp2f(log2f(r6) * (1.0f / 6.0f)), 4.f);
    }
    const float h7 = 2.f * norm[7];
    f[5] = ((c.w - b1) - (b1 - b0)) / h7;
    f[6] = (c.w - b0) / h7;
}

// Row pass of the activity mask: act[y][x] = 1 if a cell of row y within
// kActR columns of x changed its bed since the saved bed (tile layout).
__global__ void activity_rows(const float4 *__restrict__ state, int nx, int ny, int T, int ntx,
                              const float *__restrict__ bsave, uint8_t *__restrict__ act) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        uint8_t a = 0;
        for (int xx = max(0, x - kActR); xx <= min(nx - 1, x + kActR); ++xx)
            a |= state[(size_t)y * nx + xx].w != bsave[tile_index(xx, y, T, ntx)];
        act[i] = a;
    }
}

// Network input tiles (channels: see the surrogate's header comment); the
// column pass of the activity mask is done here.
__global__ void pack_state(const float4 *__restrict__ state, int nx, int ny, int T, int ntx, const float *__restrict__ norm,
                           float eps, float ksh, const float *__restrict__ bsave, const float *__restrict__ bsave1,
                           const uint8_t *__restrict__ act, __nv_bfloat16 *__restrict__ X, size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane);
        const int r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        __align__(16) __nv_bfloat16 o[8];
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (x < nx && y < ny) {
            cell_features(state[(size_t)y * nx + x], bsave[i], bsave1[i], norm, eps, ksh, f);
            uint8_t a = 0;
            for (int yy = max(0, y - kActR); yy <= min(ny - 1, y + kActR); ++yy) a |= act[(size_t)yy * nx + x];
            f[7] = a ? 1.f : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16(f[j]);
        reinterpret_cast<uint4 *>(X)[i] = reinterpret_cast<uint4 *>(o)[0];
    }
}

// b = b_saved + pred * norm[6] on the solver state, for the cells of the tiles.
__global__ void apply_bed(float4 *__restrict__ state, int nx, int ny, int T, int ntx, const float *__restrict__ pred,
                          const float *__restrict__ bsave, const float *__restrict__ norm, size_t total) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane);
        const int r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        if (x < nx && y < ny) state[(size_t)y * nx + x].w = bsave[i] + pred[i] * norm[6];
    }
}

// ---- prediction on active halo tiles (the surrogate windows)
//
// The network is fully convolutional with a receptive field of kHalo cells
// (six 3x3 layers), so a cell's prediction needs only the kHalo-cell
// neighbourhood.  The domain is cut into interior tiles of kTC x kTC cells;
// the network runs only on the tiles whose activity mask holds a 1 (where it
// is all zero the output m (z + bias + p) is exactly 0), each as a kTI x kTI
// image of the interior and a kHalo-cell margin from its neighbours.  An
// image never reaches beyond the domain: at the domain's edges it is shifted
// inwards, so its own edge (where every layer pads with zeros) is the
// domain's, as in a whole-domain image (domains of at least kTI x kTI).
constexpr int kTI = 128;
constexpr int kHalo = 6;
constexpr int kTC = kTI - 2 * kHalo;

// first row / column of the image of interior tile t along an axis of n cells
__device__ __forceinline__ int halo_origin(int t, int n) { return min(max(t * kTC - kHalo, 0), n - kTI); }

// chg: 1 where the bed differs from the saved bed (row-major); pcell: the
// linear extrapolation (b - b_saved) / (2 norm[7]) of the two coupled steps,
// rounded to BF16 as the network reads it (tile layout of the saved bed).
__global__ void bed_change(const float4 *__restrict__ state, int nx, int ny, int T, int ntx,
                           const float *__restrict__ bsave, const float *__restrict__ norm, uint8_t *__restrict__ chg,
                           float *__restrict__ pcell) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        const size_t j = tile_index(x, y, T, ntx);
        const float b = state[i].w, b0 = bsave[j];
        chg[i] = b != b0;
        pcell[j] = __bfloat162float(__float2bfloat16((b - b0) / (2.f * norm[7])));
    }
}

// Row pass of the activity mask, row-major: actr[y][x] = 1 if a cell of row y
// within kActR columns of x changed its bed.
__global__ void act_rows_rm(const uint8_t *__restrict__ chg, int nx, int ny, uint8_t *__restrict__ actr) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        uint8_t a = 0;
        for (int xx = max(0, x - kActR); xx <= min(nx - 1, x + kActR); ++xx) a |= chg[(size_t)y * nx + xx];
        actr[i] = a;
    }
}

// flag[tile] = 1 for the interior tiles with a 1 in their activity mask: a
// row-dilated 1 in one of their columns within kActR rows of their rows.
__global__ void tile_flags(const uint8_t *__restrict__ actr, int nx, int ny, int ntcx, int ntcy, int *__restrict__ flag) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (!actr[i]) continue;
        const int y = (int)(i / nx), x = (int)(i % nx), tx = x / kTC;
        for (int ty = max(0, (y - kActR) / kTC); ty <= min(ntcy - 1, (y + kActR) / kTC); ++ty)
            if (y >= ty * kTC - kActR && y < ty * kTC + kTC + kActR) flag[ty * ntcx + tx] = 1;
    }
}

// The active tiles in order (list[0..count)) and each tile's place in that
// list (slot, -1 for an inactive tile); clears the flags.  One block of 1024.
__global__ void __launch_bounds__(1024) compact_tiles(int *__restrict__ flag, int nt, int *__restrict__ list,
                                                      int *__restrict__ slot, int *__restrict__ count) {
    __shared__ int wsum[32];
    __shared__ int base, chunk;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int t0 = 0; t0 < nt; t0 += 1024) {
        const int t = t0 + (int)threadIdx.x;
        const bool on = t < nt && flag[t] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int i = 0; i < 32; ++i) { const int v = wsum[i]; wsum[i] = acc; acc += v; }
            chunk = acc;
        }
        __syncthreads();
        if (t < nt) {
            const int k = on ? base + wsum[w] + __popc(m & ((1u << lane) - 1u)) : -1;
            slot[t] = k;
            if (on) list[k] = t;
            flag[t] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) base += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// Network input (NHWC8 BF16, the channels of pack_state) of the active tiles
// list[first .. first + nimg): kTI x kTI pixels each.
__global__ void gather_tiles(const float4 *__restrict__ state, int nx, int ny, int T, int ntx, const float *__restrict__ norm,
                             float eps, float ksh, const float *__restrict__ bsave, const float *__restrict__ bsave1,
                             const uint8_t *__restrict__ actr, const int *__restrict__ list, int first, int nimg,
                             int ntcx, __nv_bfloat16 *__restrict__ X) {
    const size_t total = (size_t)nimg * kTI * kTI;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / (kTI * kTI)), r = (int)(i % (kTI * kTI));
        const int tile = list[first + b];
        const int y = halo_origin(tile / ntcx, ny) + r / kTI, x = halo_origin(tile % ntcx, nx) + r % kTI;
        __align__(16) __nv_bfloat16 o[8];
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        {
            const size_t j = tile_index(x, y, T, ntx);
            cell_features(state[(size_t)y * nx + x], bsave[j], bsave1[j], norm, eps, ksh, f);
            uint8_t a = 0;
            for (int yy = max(0, y - kActR); yy <= min(ny - 1, y + kActR); ++yy) a |= actr[(size_t)yy * nx + x];
            f[7] = a ? 1.f : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16(f[j]);
        reinterpret_cast<uint4 *>(X)[i] = reinterpret_cast<uint4 *>(o)[0];
    }
}

// The prediction of every cell (tile layout of the saved bed): the interior
// pixels of the images of list[first .. first + nimg) (out: nimg x kTI x kTI),
// 0 for the cells of inactive tiles (written with the first chunk).
__global__ void scatter_pred(int nx, int ny, int T, int ntx, const float *__restrict__ out, const int *__restrict__ slot,
                             int ntcx, int first, int nimg, float *__restrict__ predc) {
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        const int ty = y / kTC, tx = x / kTC;
        const int sl = slot[ty * ntcx + tx];
        float v;
        if (sl < 0) {
            if (first != 0) continue;
            v = 0.f;
        } else {
            if (sl < first || sl >= first + nimg) continue;
            v = out[((size_t)(sl - first) * kTI + (y - halo_origin(ty, ny))) * kTI + (x - halo_origin(tx, nx))];
        }
        predc[tile_index(x, y, T, ntx)] = v;
    }
}

}  // namespace swe_nn

// ======================================================================
// The surrogate object (host side): layer buffers and launches.
// Network: 6 conv3x3 layers, 4(+4 zero) -> 32 -> 32 -> 32 -> 32 -> 32 -> 1,
// ReLU on the hidden layers, linear output; BF16 weights/activations, FP32
// accumulation, FP32 master weights with Adam.
// ======================================================================

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <random>
#include <vector>

#include "swe_internal.h"
#include "swe_trace.h"

namespace {

struct NnLayer {
    int cin, nout, noutp, kp, cind, kpd, mt;
    float *Wm = nullptr, *m = nullptr, *v = nullptr, *bias = nullptr, *mb = nullptr, *vb = nullptr;
    __nv_bfloat16 *Wf = nullptr, *Wd = nullptr;
    float *grad = nullptr;   // [mt*128][noutp]
};

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
    float *bsave1 = nullptr;   // the bed after the window's first coupled step
    int *err = nullptr;
    size_t partial_floats = 0;
    long adam_t = 0;
    std::vector<void *> allocs;
    uint8_t *act = nullptr;
    // prediction on active halo tiles: changed cells, per-cell linear
    // extrapolation and prediction (tile layout), tile flags / list / slots
    uint8_t *chg = nullptr;
    float *pcell = nullptr, *predc = nullptr;
    int *tflag = nullptr, *tlist = nullptr, *tslot = nullptr, *tcount = nullptr;
    int tcap = 0;
    int l1 = 0;   // training loss: 0 mean squared error, 1 mean absolute error
    float h_norm[8] = {0, 1, 0, 1, 1, 1, 1, 1};
};

namespace {

cudaError_t salloc(swe_surrogate *s, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) { s->allocs.push_back(*p); cudaMemsetAsync(*p, 0, bytes, s->stream); }
    return e;
}

int grid_n(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 32); }

// T: the images' side (the training tiles, or the halo tiles of prediction)
template <int CIN, int NOUT, int EPI>
cudaError_t conv(swe_surrogate *s, const __nv_bfloat16 *X, const NnLayer &l, const __nv_bfloat16 *Wt, const float *bias,
                 const __nv_bfloat16 *mask, __nv_bfloat16 *Y, float *Yf, int B, int T) {
    (void)l;
    using WC = WsConv<CIN, NOUT>;
    auto kern = conv3x3_ws<CIN, NOUT, EPI>;
    // enough shared memory that the CTAs of one SM fit its 512 TMEM columns
    static const size_t smem = std::max<size_t>(WC::smem(), (size_t)(227 * 1024) / (512 / WC::TCOLS) - 1024);
    // the function attributes and the resident CTA count, per device (the
    // attributes are per-device settings; devices beyond 64 redo them)
    static std::atomic<int> resident_of[64];
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    int resident = (dev >= 0 && dev < 64) ? resident_of[dev].load(std::memory_order_acquire) : 0;
    if (resident == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        int sms = 0, smem_sm = 0, reserved = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess) return e;
        // CTAs per SM: shared memory, tensor memory (512 columns), threads
        const int per_sm = std::min({smem_sm / (int)(smem + reserved), 512 / WC::TCOLS, 2048 / 192});
        resident = std::max(1, per_sm) * sms;
        if (dev >= 0 && dev < 64) resident_of[dev].store(resident, std::memory_order_release);
    }
    // one wave: the column bands x images share the resident CTAs, each CTA
    // streams a run of rows (a multiple of 4, at least 8, to amortise its set-up)
    const int bands = (T + 127) / 128;
    const int groups = std::max(1, resident / (bands * B));
    const int rows = std::max(8, ((T + groups - 1) / groups + 3) / 4 * 4);
    dim3 grid(bands, (T + rows - 1) / rows, B);
    kern<<<grid, 192, smem, s->stream>>>(X, Wt, bias, mask, Y, Yf, T, T, rows, s->err);
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

cudaError_t forward_all(swe_surrogate *s, const __nv_bfloat16 *X, float *out, int B, int T) {
    cudaError_t e = conv<8, 32, EPI_RELU>(s, X, s->L[0], s->L[0].Wf, s->L[0].bias, nullptr, s->A[0], nullptr, B, T);
    for (int i = 1; i < 5 && e == cudaSuccess; ++i)
        e = conv<32, 32, EPI_RELU>(s, s->A[i - 1], s->L[i], s->L[i].Wf, s->L[i].bias, nullptr, s->A[i], nullptr, B, T);
    if (e == cudaSuccess) e = conv<32, 16, EPI_OUT>(s, s->A[4], s->L[5], s->L[5].Wf, s->L[5].bias, X, nullptr, out, B, T);
    return e;
}
cudaError_t forward_all(swe_surrogate *s, const __nv_bfloat16 *X, float *out, int B) { return forward_all(s, X, out, B, s->T); }

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
        // He initialisation for the hidden layers
        std::vector<float> w(nw);
        const int fan_in = 9 * l.cin;
        // zero output layer: the untrained network is the linear extrapolation itself
        const float sd = i == 5 ? 0.f : std::sqrt(2.f / fan_in);
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
    if (e == cudaSuccess) e = salloc(s, (void **)&s->bsave1, pix * 4);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->act, pix);
    s->partial_floats = maxpart * (size_t)max_batch * ((tile + kWgradRows - 1) / kWgradRows);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->partial, s->partial_floats * 4);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->loss, 16);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->norm, 64);
    if (e == cudaSuccess) e = salloc(s, (void **)&s->err, 16);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->norm, s->h_norm, sizeof s->h_norm, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        swe_surrogate_destroy(s);
        return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
    }
    *out = s;
    return SWE_OK;
}

extern "C" swe_status swe_surrogate_set_norm(swe_surrogate *s, const float norm[8]) {
    if (!s || !norm) return SWE_EINVAL;
    for (int j : {1, 3, 4, 5, 6, 7})
        if (!(norm[j] > 0)) return SWE_EINVAL;
    std::copy(norm, norm + 8, s->h_norm);
    if (cudaMemcpyAsync(s->norm, s->h_norm, sizeof s->h_norm, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return SWE_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_set_loss(swe_surrogate *s, int kind) {
    if (!s || (kind != 0 && kind != 1)) return SWE_EINVAL;
    s->l1 = kind;
    return SWE_OK;
}

extern "C" swe_status swe_surrogate_forward(swe_surrogate *s, const void *X, float *out, int B) {
    const SweRange range_("swe_surrogate_forward");
    if (!s || !X || !out || B < 1 || B > s->maxB) return SWE_EINVAL;
    if (forward_all(s, (const __nv_bfloat16 *)X, out, B) != cudaSuccess) return SWE_ECUDA;
    return check_err(s);
}

extern "C" swe_status swe_surrogate_train_step(swe_surrogate *s, const void *Xv, const float *target, int B, float lr,
                                              float *loss_out) {
    const SweRange range_("swe_surrogate_train_step");
    if (!s || !Xv || !target || B < 1 || B > s->maxB || !(lr > 0)) return SWE_EINVAL;
    const __nv_bfloat16 *X = (const __nv_bfloat16 *)Xv;
    const size_t pix = (size_t)B * s->T * s->T;
    cudaError_t e = forward_all(s, X, s->out, B);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, 4, s->stream);
    if (e == cudaSuccess) {
        loss_grad<<<grid_n(pix), 256, 0, s->stream>>>(s->out, target, X, pix, s->l1, s->dOut, s->loss);
        e = cudaGetLastError();
    }
    // backward: gradient w.r.t. the pre-activations of layers 5..1, then weights
    if (e == cudaSuccess) e = conv<8, 32, EPI_MASK>(s, s->dOut, s->L[5], s->L[5].Wd, nullptr, s->A[4], s->dA[4], nullptr, B, s->T);
    for (int i = 4; i >= 1 && e == cudaSuccess; --i)
        e = conv<32, 32, EPI_MASK>(s, s->dA[i], s->L[i], s->L[i].Wd, nullptr, s->A[i - 1], s->dA[i - 1], nullptr, B, s->T);
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
// outputs of layers 1..5 (32-channel BF16, row-planar), 5 = the output (FP32 per pixel).
extern "C" swe_status swe_surrogate_buffer(swe_surrogate *s, int index, void **ptr) {
    if (!s || !ptr || index < 0 || index > 5) return SWE_EINVAL;
    *ptr = index < 5 ? (void *)s->A[index] : (void *)s->out;
    return SWE_OK;
}

// ---------------------------------------------------------------- solver coupling

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
        out[i] = (b1[i] - b0[i]) / norm[6];
}

// Judged-window error sums (FP64) over the cells of the domain, ch = b1 - b0
// the plain solver's bed change:  |pred - ch|, |ch|, |b1|, |last - ch|,
// |p - ch| (p: the linear extrapolation as the network reads it).
__global__ void judge_sums(const float *__restrict__ b0, const float *__restrict__ b1, const float *__restrict__ pred,
                           const float *__restrict__ last, const float *__restrict__ pcell,
                           const float *__restrict__ norm, int nx, int ny, int T, int ntx, size_t total,
                           double *__restrict__ out) {
    __shared__ double red[5][256];
    double q[5] = {0, 0, 0, 0, 0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = (size_t)T * T;
        const int bt = (int)(i / plane), r = (int)(i % plane);
        const int y = (bt / ntx) * T + r / T, x = (bt % ntx) * T + r % T;
        if (x >= nx || y >= ny) continue;
        const double ch = (double)b1[i] - (double)b0[i];
        q[0] += fabs((double)pred[i] * norm[6] - ch);
        q[1] += fabs(ch);
        q[2] += fabs((double)b1[i]);
        q[3] += fabs((double)last[i] - ch);
        q[4] += fabs((double)pcell[i] * norm[6] - ch);
    }
    for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) atomicAdd(&out[k], red[k][0]);
}
__global__ void diff_into(const float *__restrict__ b0, const float *__restrict__ b1, float *__restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d[i] = b1[i] - b0[i];
}

// The handle as the surrogate sees it: its FP32 state, tile grid and stream.
struct Coupling {
    SweConst *c = nullptr;
    void *cur = nullptr;
    cudaStream_t hs = nullptr;
    int ntx = 0, nty = 0;
    size_t total = 0;
};

bool couple(swe_surrogate *s, swe_handle *h, Coupling &k) {
    SweBufs *b;
    int prec;
    bool set;
    if (!s || !h || !swe_impl::handle_view(h, &k.c, &b, &k.hs, nullptr, &prec, &set) || !set || prec != SWE_FP32)
        return false;
    k.cur = swe_impl::handle_current_state(h);
    k.ntx = (k.c->nx + s->T - 1) / s->T;
    k.nty = (k.c->ny + s->T - 1) / s->T;
    k.total = (size_t)k.ntx * k.nty * s->T * s->T;
    return k.cur != nullptr && k.ntx * k.nty <= s->maxB;
}

// Orders the surrogate's stream after the solver's work so far.
swe_status after_solver(swe_surrogate *s, const Coupling &k) {
    if (k.hs == s->stream) return SWE_OK;
    return cudaStreamSynchronize(k.hs) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

// Orders the solver's next work after the surrogate's work so far.
swe_status before_solver(swe_surrogate *s, const Coupling &k) {
    if (k.hs == s->stream) return cudaGetLastError() == cudaSuccess ? SWE_OK : SWE_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

void launch_save(swe_surrogate *s, const Coupling &k, float *dst) {
    bed_tiles<<<grid_n(k.total), 256, 0, s->stream>>>((const float4 *)k.cur, k.c->nx, k.c->ny, s->T, k.ntx, dst, k.total);
}

void launch_pack(swe_surrogate *s, const Coupling &k, __nv_bfloat16 *X) {
    const size_t n = (size_t)k.c->nx * k.c->ny;
    activity_rows<<<grid_n(n), 256, 0, s->stream>>>((const float4 *)k.cur, k.c->nx, k.c->ny, s->T, k.ntx, s->bsave, s->act);
    pack_state<<<grid_n(k.total), 256, 0, s->stream>>>((const float4 *)k.cur, k.c->nx, k.c->ny, s->T, k.ntx, s->norm,
                                                       k.c->eps_f, k.c->f.ksh, s->bsave, s->bsave1, s->act, X, k.total);
}

// The network's prediction for every cell of the coupled domain into
// s->predc (tile layout), from the bed saved by launch_save and the current
// state: the activity mask, the list of active halo tiles, and the network
// on those tiles only, in batches that fit the activation buffers.
swe_status predict_tiles(swe_surrogate *s, const Coupling &k) {
    using namespace swe_nn;
    const int nx = k.c->nx, ny = k.c->ny;
    const size_t n = (size_t)nx * ny;
    const int ntcx = (nx + kTC - 1) / kTC, ntcy = (ny + kTC - 1) / kTC, nt = ntcx * ntcy;
    if (!s->chg) {
        const size_t pix = (size_t)s->maxB * s->T * s->T;
        if (salloc(s, (void **)&s->chg, pix) != cudaSuccess || salloc(s, (void **)&s->pcell, pix * 4) != cudaSuccess ||
            salloc(s, (void **)&s->predc, pix * 4) != cudaSuccess || salloc(s, (void **)&s->tcount, 16) != cudaSuccess)
            return SWE_ENOMEM;
    }
    if (nt > s->tcap) {
        const int cap = std::max(nt, 64);
        if (salloc(s, (void **)&s->tflag, (size_t)cap * 4) != cudaSuccess ||
            salloc(s, (void **)&s->tlist, (size_t)cap * 4) != cudaSuccess ||
            salloc(s, (void **)&s->tslot, (size_t)cap * 4) != cudaSuccess)
            return SWE_ENOMEM;
        s->tcap = cap;
    }
    const float4 *st = (const float4 *)k.cur;
    bed_change<<<grid_n(n), 256, 0, s->stream>>>(st, nx, ny, s->T, k.ntx, s->bsave, s->norm, s->chg, s->pcell);
    if (nx < kTI || ny < kTI) {   // smaller than one halo image: the network on the whole-domain tiles
        launch_pack(s, k, s->X0);
        if (forward_all(s, s->X0, s->out, k.ntx * k.nty) != cudaSuccess) return SWE_ECUDA;
        return cudaMemcpyAsync(s->predc, s->out, k.total * 4, cudaMemcpyDeviceToDevice, s->stream) == cudaSuccess
                   ? SWE_OK : SWE_ECUDA;
    }
    act_rows_rm<<<grid_n(n), 256, 0, s->stream>>>(s->chg, nx, ny, s->act);
    tile_flags<<<grid_n(n), 256, 0, s->stream>>>(s->act, nx, ny, ntcx, ntcy, s->tflag);
    compact_tiles<<<1, 1024, 0, s->stream>>>(s->tflag, nt, s->tlist, s->tslot, s->tcount);
    int count = 0;
    if (cudaMemcpyAsync(&count, s->tcount, 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return SWE_ECUDA;
    const int cap = (int)(((size_t)s->maxB * s->T * s->T) / ((size_t)kTI * kTI));
    for (int first = 0; first == 0 || first < count; first += cap) {
        const int nimg = std::min(cap, count - first);
        if (nimg > 0) {
            gather_tiles<<<grid_n((size_t)nimg * kTI * kTI), 256, 0, s->stream>>>(
                st, nx, ny, s->T, k.ntx, s->norm, k.c->eps_f, k.c->f.ksh, s->bsave, s->bsave1, s->act, s->tlist, first,
                nimg, ntcx, s->X0);
            if (forward_all(s, s->X0, s->out, nimg, kTI) != cudaSuccess) return SWE_ECUDA;
        }
        scatter_pred<<<grid_n(n), 256, 0, s->stream>>>(nx, ny, s->T, k.ntx, s->out, s->tslot, ntcx, first, nimg, s->predc);
    }
    return cudaGetLastError() == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

// Sets the bed to saved + prediction (s->predc) and lets the handle re-form
// its census and dt for the new bed.
swe_status launch_apply(swe_surrogate *s, swe_handle *h, const Coupling &k) {
    apply_bed<<<grid_n(k.total), 256, 0, s->stream>>>((float4 *)k.cur, k.c->nx, k.c->ny, s->T, k.ntx, s->predc, s->bsave,
                                                      s->norm, k.total);
    const swe_status r = before_solver(s, k);
    if (r != SWE_OK) return r;
    return (swe_status)swe_impl::handle_state_changed(h);
}
}  // namespace

extern "C" swe_status swe_surrogate_pack_state(swe_surrogate *s, swe_handle *h, void *X, int *batch) {
    Coupling k;
    if (!X || !couple(s, h, k)) return SWE_EINVAL;
    swe_status st = after_solver(s, k);
    if (st != SWE_OK) return st;
    launch_pack(s, k, (__nv_bfloat16 *)X);
    if (batch) *batch = k.ntx * k.nty;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_save_bed(swe_surrogate *s, swe_handle *h) {
    Coupling k;
    if (!couple(s, h, k)) return SWE_EINVAL;
    swe_status st = after_solver(s, k);
    if (st != SWE_OK) return st;
    launch_save(s, k, s->bsave);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_save_mid(swe_surrogate *s, swe_handle *h) {
    Coupling k;
    if (!couple(s, h, k)) return SWE_EINVAL;
    swe_status st = after_solver(s, k);
    if (st != SWE_OK) return st;
    launch_save(s, k, s->bsave1);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_pack_target(swe_surrogate *s, swe_handle *h, float *target) {
    Coupling k;
    if (!target || !couple(s, h, k)) return SWE_EINVAL;
    swe_status st = after_solver(s, k);
    if (st != SWE_OK) return st;
    launch_save(s, k, s->tgt);
    make_target<<<grid_n(k.total), 256, 0, s->stream>>>(s->bsave, s->tgt, s->norm, target, k.total);
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? SWE_OK : SWE_ECUDA;
}

extern "C" swe_status swe_surrogate_apply(swe_surrogate *s, swe_handle *h) {
    const SweRange range_("swe_surrogate_apply");
    Coupling k;
    if (!couple(s, h, k)) return SWE_EINVAL;
    swe_status st = after_solver(s, k);
    if (st != SWE_OK) return st;
    if ((st = predict_tiles(s, k)) != SWE_OK || (st = check_err(s)) != SWE_OK) return st;
    return launch_apply(s, h, k);
}

extern "C" swe_status swe_surrogate_run(swe_surrogate *s, swe_handle *h, int nwindows, int K, int f, int judge_every,
                                       double bound, swe_surrogate_stats *st) {
    const SweRange range_("swe_surrogate_run");
    Coupling k;
    if (!st || nwindows < 0 || K < 2 || f < 1 || (K % f) || K / f < 2 || judge_every < 1 || !(bound > 0) ||
        !couple(s, h, k))
        return SWE_EINVAL;
    double *dsum = nullptr;
    float *last = nullptr;
    if (cudaMalloc(&dsum, 5 * sizeof(double)) != cudaSuccess) return SWE_ENOMEM;
    if (cudaMalloc(&last, k.total * 4) != cudaSuccess) { cudaFree(dsum); return SWE_ENOMEM; }
    cudaMemsetAsync(last, 0, k.total * 4, s->stream);
    double err_sum = 0, zero_sum = 0, pers_sum = 0, lin_sum = 0;
    swe_status rc = SWE_OK;
    // the network's prediction from the state two coupled steps into the
    // window (the beds at its start and after its first step saved)
    auto first_steps_and_predict = [&]() -> swe_status {
        swe_status r;
        if (!couple(s, h, k) || (r = after_solver(s, k)) != SWE_OK) return r == SWE_OK ? SWE_EINVAL : r;
        launch_save(s, k, s->bsave);
        if ((r = before_solver(s, k)) != SWE_OK || (r = swe_run_steps(h, 1)) != SWE_OK) return r;
        if (!couple(s, h, k) || (r = after_solver(s, k)) != SWE_OK) return r == SWE_OK ? SWE_EINVAL : r;
        launch_save(s, k, s->bsave1);
        if ((r = before_solver(s, k)) != SWE_OK || (r = swe_run_steps(h, 1)) != SWE_OK) return r;
        if (!couple(s, h, k) || (r = after_solver(s, k)) != SWE_OK) return r == SWE_OK ? SWE_EINVAL : r;
        if ((r = predict_tiles(s, k)) != SWE_OK) return r;
        return before_solver(s, k);   // the forward's error flag is read once per window
    };
    double t_next = 0;   // the time at the start of the next window (read once; each window ends by reading it)
    if (nwindows > 0) rc = swe_get_time(h, &t_next);
    for (int w = 0; w < nwindows && rc == SWE_OK; ++w) {
        const SweRange window_(st->mode == 1 ? "plain window" : (w % judge_every == 0 ? "judged window" : "surrogate window"));
        const double t0 = t_next;
        double t1 = 0;
        if (st->mode == 1) {                                     // plain coupled window
            if ((rc = swe_run_steps(h, K)) != SWE_OK || (rc = swe_get_time(h, &t1)) != SWE_OK) break;
            st->bed_time += t1 - t0;
            st->water_time += t1 - t0;
            ++st->plain_windows;
        } else if (w % judge_every == 0) {                       // judged window: K coupled steps
            if ((rc = first_steps_and_predict()) != SWE_OK) break;
            if ((rc = swe_run_steps(h, K - 2)) != SWE_OK || (rc = swe_get_time(h, &t1)) != SWE_OK) break;
            if (!couple(s, h, k) || (rc = after_solver(s, k)) != SWE_OK) { rc = rc == SWE_OK ? SWE_EINVAL : rc; break; }
            if ((rc = check_err(s)) != SWE_OK) break;
            launch_save(s, k, s->tgt);
            cudaMemsetAsync(dsum, 0, 5 * sizeof(double), s->stream);
            judge_sums<<<grid_n(k.total), 256, 0, s->stream>>>(s->bsave, s->tgt, s->predc, last, s->pcell, s->norm,
                                                              k.c->nx, k.c->ny, s->T, k.ntx, k.total, dsum);
            diff_into<<<grid_n(k.total), 256, 0, s->stream>>>(s->bsave, s->tgt, last, k.total);
            double q[5];
            if (cudaMemcpyAsync(q, dsum, sizeof q, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
                cudaStreamSynchronize(s->stream) != cudaSuccess) { rc = SWE_ECUDA; break; }
            const double ref = q[1] > 0 ? q[1] : 1e-300;
            const double err = q[0] / ref;
            st->err_last = err;
            st->err_max = std::max(st->err_max, err);
            st->elev_err_max = std::max(st->elev_err_max, q[0] / (q[2] > 0 ? q[2] : 1e-300));
            err_sum += err;
            zero_sum += 1.0;
            pers_sum += q[3] / ref;
            lin_sum += q[4] / ref;
            ++st->judged;
            st->err_mean = err_sum / st->judged;
            st->err_zero_mean = zero_sum / st->judged;
            st->err_persist_mean = pers_sum / st->judged;
            st->err_linear_mean = lin_sum / st->judged;
            st->bed_time += t1 - t0;
            st->water_time += t1 - t0;
            if (err > bound) { st->mode = 1; st->takeover_window = w; }
        } else {                                                 // surrogate window
            if ((rc = first_steps_and_predict()) != SWE_OK) break;
            // the remaining water steps run the coupled step as it is: the bed
            // they move is replaced by the prediction at the window's end
            if (K / f > 2 && (rc = swe_run_steps(h, K / f - 2)) != SWE_OK) break;
            if ((rc = swe_get_time(h, &t1)) != SWE_OK) break;
            if (!couple(s, h, k) || (rc = after_solver(s, k)) != SWE_OK) { rc = rc == SWE_OK ? SWE_EINVAL : rc; break; }
            if ((rc = check_err(s)) != SWE_OK || (rc = launch_apply(s, h, k)) != SWE_OK) break;
            st->bed_time += (t1 - t0) * f;
            st->water_time += t1 - t0;
            ++st->surrogate_windows;
        }
        ++st->windows;
        t_next = t1;
    }
    cudaStreamSynchronize(s->stream);
    cudaFree(dsum);
    cudaFree(last);
    return rc;
}
