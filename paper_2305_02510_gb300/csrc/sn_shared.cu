// One shared dense integer network driven by B independent input trains,
// propagated on the 5th-generation tensor cores (tcgen05).
//
// Per timestep t the synaptic input of all trains is one GEMM
//   Acc[B][n] = S(t-1)[B][n] . W[n][n]
// with S the 0/1 spikes of the previous step (Section 2.1: "the vector of
// spikes from the previous time step is multiplied by the weight matrix").
// Spikes and integer weights in [-8, 8] are exact in FP8 E4M3, and every sum
// (at most n * 8 in magnitude, n <= 2^21) is an integer below 2^24, exact in
// the FP32 accumulator: the GEMM runs as tcgen05.mma kind::f8f6f4 and is
// bit-exact integer arithmetic.  (kind::i8 does not exist on sm_103a.)
//
// Tile = 128 trains x 128 post-neurons, accumulated in TMEM over the K = n
// pre-neurons in 128-byte stages loaded by TMA (128B swizzle, 6 stages).
// Warp 0 lane 0 issues TMA, warp 1 lane 0 issues the MMAs; meanwhile warps
// 2..15 draw the tile's Poisson input of step t (one bit per train and neuron)
// and stage the tile's neuron parameters in shared memory.  Afterwards the
// sixteen warps read the accumulator rows (tcgen05.ld: warps w, w+4, w+8 and
// w+12 share TMEM lane quarter w, each taking 32 columns) and apply the integer LIF
// rule (Section 2.1 order).  When every block holds one tile for the whole
// launch (tiles <= blocks), the tile's V and r stay in TMEM next to the
// accumulator (columns 128.. and 256..), read from global memory at the
// launch's start and written back at its end; otherwise they make the round
// trip every step.  The global state is neuron-major ([n][B]: lane = train,
// so every load and store of V and r is one 128-byte line per warp); the
// spike bytes that are the next step's A operand go through a shared-memory
// transpose and leave as whole 128-byte rows.  A persistent cooperative
// launch runs all steps; a grid barrier separates them.  Every wait is
// bounded: on expiry the kernel latches SN_ETIMEOUT, drains its own copies
// and MMAs, frees its TMEM and returns.

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_device.cuh"
#include "sn_internal.h"
#include "sn_tc.cuh"

namespace sn {

constexpr int kTM = 128;                       // trains per tile (MMA M)
constexpr int kTN = 128;                       // post-neurons per tile (MMA N)
constexpr int kTK = 128;                       // bytes of K per stage (one 128B swizzle row)
constexpr int kStages = 6;
constexpr int kStageA = kTM * kTK;             // 16 KiB
constexpr int kStageBytes = (kTM + kTN) * kTK; // 32 KiB
constexpr int kShThreads = 512;
constexpr int kEpiParts = kShThreads / 128;        // warps per TMEM lane quarter
constexpr int kEpiCols = kTN / kEpiParts;          // accumulator columns per epilogue warp
static_assert(kEpiCols % 32 == 0, "an epilogue warp takes whole 32-column TMEM loads");
constexpr int kSub = 4;                      // state columns loaded together
// epilogue staging after the pipeline stages: spike bytes [128][kSaPitch],
// raster words and Poisson bits [128][4], parameters [5][128]
constexpr int kSaPitch = 144;                  // 128 B + 16: conflict-free 16-byte stores
constexpr int kEpiBytes = kTM * kSaPitch + 2 * kTM * 4 * 4 + 5 * kTN * 4;
constexpr unsigned kTmemCols = 128;
// When every block holds one tile for the whole launch, the tile's state
// stays in TMEM between steps: V at columns kVCol + c, r at kRCol + c of the
// train's lane (512 columns allocated: the accumulator's 128 and 256 of state).
constexpr unsigned kTmemColsRes = 512;
constexpr uint32_t kVCol = 128, kRCol = 256;

struct SharedArgs {
    int n, B, t0, steps, cap, words;
    int tiles_m, tiles;
    unsigned char *A0, *A1;        // spike operands [B][n] bytes, A_(t & 1) holds step t
    int *V, *r;                    // [n][B] (neuron-major)
    const int *th, *lk, *rs, *R;   // [n]
    const unsigned *prate;         // [n]
    const int *pamp;               // [n]
    const unsigned long long *pkey;// [B]
    unsigned *raster;              // [cap][B][words]
    Control *ctl;
};

template <bool kRes>
__global__ void __launch_bounds__(kShThreads, 1)
shared_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmW, SharedArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_addr(smem);
    unsigned char *sA = smem + kStages * kStageBytes;                 // [128][kSaPitch]
    unsigned *sR = (unsigned *)(sA + kTM * kSaPitch);                 // [128][4] raster words
    unsigned *sP = sR + kTM * 4;                                      // [128][4] Poisson bits
    int *sTh = (int *)(sP + kTM * 4), *sLk = sTh + kTN, *sRs = sLk + kTN, *sRf = sRs + kTN,
        *sAmp = sRf + kTN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&accbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        s_abort = 0;
    }
    constexpr unsigned kCols = kRes ? kTmemColsRes : kTmemCols;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_addr(&s_tmem)), "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int quarter = warp & 3, part = warp >> 2;
    const int bl = quarter * 32 + lane;                // tile row = TMEM lane
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);   // this warp's lane quarter
    if (kRes && blockIdx.x < a.tiles) {
        // the block's one tile: its state into TMEM for the whole launch
        const int m0 = (blockIdx.x % a.tiles_m) * kTM, n0 = (blockIdx.x / a.tiles_m) * kTN;
        for (int h = 0; h < kEpiCols / 16; ++h) {
            const int c0 = part * kEpiCols + h * 16;
            const int *Vp = a.V + (size_t)(n0 + c0) * a.B + m0 + bl;
            const int *rp = a.r + (size_t)(n0 + c0) * a.B + m0 + bl;
            uint32_t vv[16], rr[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                vv[q] = (uint32_t)__ldcg(Vp + (size_t)q * a.B);
                rr[q] = (uint32_t)__ldcg(rp + (size_t)q * a.B);
            }
            tmem_st16x2(trow + kVCol + c0, trow + kRCol + c0, vv, rr);
        }
    }
    const int kblocks = a.n / kTK;
    constexpr uint32_t idesc = idesc_e4m3_f32(kTM, kTN);
    unsigned g_prod = 0, g_mma = 0, tiles_done = 0;
    unsigned long long my_spikes = 0;
    bool overflow = false;

    for (int s = 0; s < a.steps && !s_abort; ++s) {
        const int t = a.t0 + s;
        const CUtensorMap *tmA = ((t + 1) & 1) ? &tmA1 : &tmA0;   // holds step t-1
        unsigned char *Aout = (t & 1) ? a.A1 : a.A0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
            const int m0 = (tile % a.tiles_m) * kTM, n0 = (tile / a.tiles_m) * kTN;
            if (warp == 0 && lane == 0) {
                // TMA producer
                for (int kb = 0; kb < kblocks; ++kb, ++g_prod) {
                    const int st = g_prod % kStages;
                    const unsigned round = g_prod / kStages;
                    if (round > 0 && !mbar_wait(smem_addr(&empty[st]), (round - 1) & 1u, a.ctl)) {
                        s_abort = 1;
                        break;
                    }
                    const uint32_t fb = smem_addr(&full[st]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                                 :: "r"(fb), "r"(kStageBytes) : "memory");
                    const uint32_t dA = sbase + st * kStageBytes;
                    tma_load_2d(dA, tmA, kb * kTK, m0, fb);
                    tma_load_2d(dA + kStageA, &tmW, kb * kTK, n0, fb);
                }
            } else if (warp == 1 && lane == 0) {
                // MMA issuer
                for (int kb = 0; kb < kblocks; ++kb, ++g_mma) {
                    const int st = g_mma % kStages;
                    const unsigned round = g_mma / kStages;
                    if (!mbar_wait(smem_addr(&full[st]), round & 1u, a.ctl)) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t dA = sbase + st * kStageBytes;
#pragma unroll
                    for (int kk = 0; kk < kTK / 32; ++kk)
                        mma_f8(tmem, umma_desc_sw128(dA + kk * 32), umma_desc_sw128(dA + kStageA + kk * 32), idesc,
                               (kb | kk) != 0);
                    mma_commit(smem_addr(&empty[st]));
                }
                mma_commit(smem_addr(&accbar));
            } else if (warp >= 2) {
                // the tile's external input of step t and its parameters,
                // while the tensor cores run
                const int tid = threadIdx.x - 64;
                for (int c = tid; c < kTN; c += kShThreads - 64) {
                    const int j = n0 + c;
                    sTh[c] = __ldg(a.th + j); sLk[c] = __ldg(a.lk + j); sRs[c] = __ldg(a.rs + j);
                    sRf[c] = __ldg(a.R + j); sAmp[c] = __ldg(a.pamp + j);
                }
                for (int i = tid; i < kTM * 4; i += kShThreads - 64) {
                    const int bl = i >> 2, w = i & 3;
                    const unsigned long long key = __ldg(a.pkey + m0 + bl);
                    unsigned bits = 0;
                    for (int q = 0; q < 32; ++q) {
                        const int j = n0 + w * 32 + q;
                        const unsigned thr = __ldg(a.prate + j);
                        if (thr && poisson_fires(key, (unsigned)t, (unsigned)j, thr)) bits |= 1u << q;
                    }
                    sP[i] = bits;
                }
            }
            __syncwarp();
            // epilogue: warps w, w+4, ... own TMEM lanes (tile rows) 32(w%4) ..,
            // each taking kEpiCols of the 128 columns
            const bool ok = mbar_wait(smem_addr(&accbar), tiles_done & 1u, a.ctl);
            ++tiles_done;
            if (!ok) s_abort = 1;
            __syncthreads();                   // Poisson bits and parameters staged
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int b = m0 + bl;
            for (int cc = 0; cc < kEpiCols / 32; ++cc) {
                const int c0 = part * kEpiCols + cc * 32;  // tile column of register 0
                const unsigned pb = sP[bl * 4 + (c0 >> 5)];
                unsigned bits = 0;
                uint32_t outw[8];
                if constexpr (kRes) {
                    // accumulator and state from TMEM, state back, 16
                    // columns at a time (the stores run even after a failed
                    // wait: tcgen05.st is warp-collective)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t col = (uint32_t)(c0 + 16 * h);
                        uint32_t v[16], vv[16], rr[16];
                        tmem_ld16x3(trow + col, trow + kVCol + col, trow + kRCol + col, v, vv, rr);
                        if (ok) {
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                uint32_t bytes = 0;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const int qq = q4 * 4 + e, q = h * 16 + qq, c = c0 + q;
                                    const int acc = __float2int_rn(__uint_as_float(v[qq]));
                                    const int ext = ((pb >> q) & 1u) ? sAmp[c] : 0;
                                    int vq = (int)vv[qq], rq = (int)rr[qq];
                                    const bool fire = lif_update_i32(vq, rq, acc, ext, sTh[c], sLk[c], sRs[c],
                                                                     sRf[c], overflow);
                                    vv[qq] = (uint32_t)vq;
                                    rr[qq] = (uint32_t)rq;
                                    bits |= (unsigned)fire << q;
                                    bytes |= (fire ? 0x38u : 0u) << (8 * e);      // E4M3 1.0
                                }
                                outw[h * 4 + q4] = bytes;
                            }
                        }
                        tmem_st16x2(trow + kVCol + col, trow + kRCol + col, vv, rr);
                    }
                    if (!ok) continue;
                } else {
                    uint32_t v[32];
                    tmem_ld32(trow + (uint32_t)c0, v);
                    if (!ok) continue;
                    const int j0 = n0 + c0;
                    // column q of this train at V[(j0 + q) * B + b], in groups of kSub
                    // columns whose loads are issued together
                    int *Vp = a.V + (size_t)j0 * a.B + b;
                    int *rp = a.r + (size_t)j0 * a.B + b;
#pragma unroll
                    for (int h = 0; h < 32 / kSub; ++h) {
                        int vin[kSub], rin[kSub];
#pragma unroll
                        for (int q = 0; q < kSub; ++q) {
                            vin[q] = __ldcg(Vp + (unsigned)((h * kSub + q) * a.B));
                            rin[q] = __ldcg(rp + (unsigned)((h * kSub + q) * a.B));
                        }
#pragma unroll
                        for (int q4 = 0; q4 < kSub / 4; ++q4) {
                            uint32_t bytes = 0;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int qq = q4 * 4 + e, q = h * kSub + qq, c = c0 + q;
                                const int acc = __float2int_rn(__uint_as_float(v[q]));
                                const int ext = ((pb >> q) & 1u) ? sAmp[c] : 0;
                                const bool fire = lif_update_i32(vin[qq], rin[qq], acc, ext, sTh[c], sLk[c], sRs[c],
                                                                 sRf[c], overflow);
                                bits |= (unsigned)fire << q;
                                bytes |= (fire ? 0x38u : 0u) << (8 * e);      // E4M3 1.0
                            }
                            outw[h * (kSub / 4) + q4] = bytes;
                        }
#pragma unroll
                        for (int q = 0; q < kSub; ++q) {
                            __stcg(Vp + (unsigned)((h * kSub + q) * a.B), vin[q]);
                            __stcg(rp + (unsigned)((h * kSub + q) * a.B), rin[q]);
                        }
                    }
                }
                uint4 *dst = (uint4 *)(sA + bl * kSaPitch + c0);
                dst[0] = make_uint4(outw[0], outw[1], outw[2], outw[3]);
                dst[1] = make_uint4(outw[4], outw[5], outw[6], outw[7]);
                sR[bl * 4 + (c0 >> 5)] = bits;
                my_spikes += (unsigned long long)__popc(bits);
            }
            __syncthreads();
            if (ok) {
                // spike bytes: 128-byte rows of A (the next step's operand);
                // raster: the tile's four words of each train
                for (int row = warp; row < kTM; row += kShThreads / 32)
                    *(uint32_t *)(Aout + (size_t)(m0 + row) * a.n + n0 + lane * 4) =
                        *(const uint32_t *)(sA + row * kSaPitch + lane * 4);
                if (threadIdx.x < kTM) {
                    const int row = threadIdx.x;
                    *(uint4 *)(a.raster + ((size_t)(t % a.cap) * a.B + m0 + row) * a.words + (n0 >> 5)) =
                        *(const uint4 *)(sR + row * 4);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            if (s_abort) break;
        }
        // the spike bytes written this step are read by TMA (async proxy) next step
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        __syncthreads();
        if (s_abort) break;
        if (!grid_barrier(a.ctl)) { s_abort = 1; break; }
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
    }

    // drain: TMA loads issued and MMAs committed by this block complete before
    // its shared memory and TMEM go away (bounded waits; no-ops when all
    // phases have already completed)
    if (warp == 0 && lane == 0) {
        for (unsigned i = g_prod > kStages ? g_prod - kStages : 0; i < g_prod; ++i)
            mbar_wait(smem_addr(&full[i % kStages]), (i / kStages) & 1u, a.ctl);
    }
    if (warp == 1 && lane == 0) {
        for (unsigned i = g_mma > kStages ? g_mma - kStages : 0; i < g_mma; ++i)
            mbar_wait(smem_addr(&empty[i % kStages]), (i / kStages) & 1u, a.ctl);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (kRes && blockIdx.x < a.tiles) {
        // the tile's state back to its neuron-major arrays
        const int m0 = (blockIdx.x % a.tiles_m) * kTM, n0 = (blockIdx.x / a.tiles_m) * kTN;
        for (int h = 0; h < kEpiCols / 16; ++h) {
            const int c0 = part * kEpiCols + h * 16;
            int *Vp = a.V + (size_t)(n0 + c0) * a.B + m0 + bl;
            int *rp = a.r + (size_t)(n0 + c0) * a.B + m0 + bl;
            uint32_t vv[16], rr[16];
            tmem_ld16x2(trow + kVCol + c0, trow + kRCol + c0, vv, rr);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                __stcg(Vp + (size_t)q * a.B, (int)vv[q]);
                __stcg(rp + (size_t)q * a.B, (int)rr[q]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(kCols));
    if (overflow) atomicCAS(&a.ctl->status, 0, (int)SN_EOVERFLOW);
    if (my_spikes) {
        atomicAdd(&a.ctl->spikes, my_spikes);
        atomicAdd(&a.ctl->events, my_spikes * (unsigned long long)a.n);
    }
}

size_t shared_smem_bytes() { return (size_t)kStages * kStageBytes + kEpiBytes + 1024; }

// [n][B] state -> [B][n] (the ABI's train-major order), 32 x 32 tiles
__global__ void shared_transpose_kernel(const int *src, int *dst, int n, int B) {
    __shared__ int tile[32][33];
    const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) tile[y][threadIdx.x] = src[(size_t)(j0 + y) * B + b0 + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) dst[(size_t)(b0 + y) * n + j0 + threadIdx.x] = tile[threadIdx.x][y];
}

cudaError_t launch_shared_transpose(const int *src, int *dst, int n, int B, cudaStream_t s) {
    shared_transpose_kernel<<<dim3(n / 32, B / 32), dim3(32, 8), 0, s>>>(src, dst, n, B);
    return cudaGetLastError();
}

cudaError_t max_grid_shared(int *grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (const void *f : {(const void *)shared_kernel<false>, (const void *)shared_kernel<true>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_smem_bytes());
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)shared_kernel<false>, kShThreads,
                                                      shared_smem_bytes());
    if (e != cudaSuccess) return e;
    // one block per SM: TMEM columns and the 128 KiB pipeline are per block
    *grid = (per > 0 ? 1 : 0) * sms;
    return cudaSuccess;
}

cudaError_t launch_shared(const void *tmaps, const SharedHostArgs &h, int grid, cudaStream_t s) {
    SharedArgs a;
    a.n = h.n; a.B = h.B; a.t0 = h.t0; a.steps = h.steps; a.cap = h.cap; a.words = h.n / 32;
    a.tiles_m = h.B / kTM;
    a.tiles = a.tiles_m * (h.n / kTN);
    a.A0 = h.A0; a.A1 = h.A1; a.V = h.V; a.r = h.r;
    a.th = h.th; a.lk = h.lk; a.rs = h.rs; a.R = h.R;
    a.prate = h.prate; a.pamp = h.pamp; a.pkey = h.pkey; a.raster = h.raster; a.ctl = h.ctl;
    const CUtensorMap *tm = (const CUtensorMap *)tmaps;
    const int g = grid < a.tiles ? grid : a.tiles;
    void *args[] = {(void *)&tm[0], (void *)&tm[1], (void *)&tm[2], (void *)&a};
    // the grid barrier's arrival count starts every launch at zero
    cudaError_t e = cudaMemsetAsync(&h.ctl->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    // one tile per block for the whole launch: the state stays in TMEM
    const void *f = g == a.tiles ? (const void *)shared_kernel<true> : (const void *)shared_kernel<false>;
    return cudaLaunchCooperativeKernel(f, dim3(g), dim3(kShThreads), args, shared_smem_bytes(), s);
}

}  // namespace sn
