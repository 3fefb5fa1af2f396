// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) contractions
// of the feedforward network: the forward synaptic input (ff_tc_fwd_kernel)
// and the backward's spike and weight gradients (ff_tc_kernel).  sn_ff.cu has
// the recurrences and the SIMT forms of these contractions.
//
// A delay-shifted contraction is a sum of plain GEMMs, one per delay d, with
// the weights restricted to the synapses of delay d (W_d = W masked by
// [D == d]) and the gradient or spike rows shifted by d steps (d * B rows):
//   gS[r][i] = sum_d sum_j gI[r + dB][j] W_d[i][j]
//   dW[i][j] = sum_d [D[i][j] = d] sum_r S[r - dB][i] gI[r][j]
// with r = t * B + b, rows outside [0, T * B) contributing zero (TMA fills
// coordinates outside a tensor with zeros).  FP32 weights and gradients enter
// as two-term BF16 splits x = hi + mid (about 16 significant bits), spikes as
// exact 0/1, and the cross products hi*hi + hi*mid + mid*hi are accumulated in
// FP32 (relative error near 2^-16 per product).
//
// The forward synaptic input I[r][j] = sum_d sum_i S[r - dB][i] W_d[i][j] runs
// as 4 passes (one per delay), each multiplying a 0/1 spike tile by the three
// BF16 parts hi + mid + lo of every weight (an exact split), so every product
// is exact.  The forward kernel accumulates one 64-input block of all passes
// at a time in TMEM (double-buffered) and adds each block's partial sums in
// FP32 (round to nearest) in registers of dedicated drain warps: a sequential
// sum over input blocks, so only 48 MMA steps ever accumulate in TMEM.
//
// One kernel runs a list of passes, each a K loop of 64-element (128-byte)
// blocks of an A and one or two B tensor maps at given coordinate offsets
// (both B tiles multiply the same A tile, which is loaded once), into one of
// up to four TMEM accumulators of a 128 x 128 output tile.  The structure is
// that of sn_shared.cu: warp 0 lane 0 issues TMA into a 4-stage ring, warp 1
// lane 0 issues the MMAs, then all eight warps drain the accumulators through
// shared memory into coalesced FP32 rows.  Work items are (tile, K split)
// pairs taken by a persistent grid; every wait is bounded.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_internal.h"
#include "sn_tc.cuh"

namespace sn {

namespace {

constexpr int kT = 128;                         // tile rows (M) and columns (N)
constexpr int kKB = 64;                         // BF16 elements of K per stage (128 bytes)
constexpr int kSt = 4;
constexpr int kStageA = kT * 128;               // 16 KiB
constexpr int kStageBytes = 3 * kStageA;        // A and up to two B tiles: 48 KiB
constexpr int kThreads = 256;
constexpr int kCPitch = kT + 4;                 // floats per staged output row

__global__ void __launch_bounds__(kThreads, 1) ff_tc_kernel(const __grid_constant__ FfTcMaps maps, FfTcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kSt], empty[kSt], accbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_started;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_addr(smem);
    const unsigned ncols = a.nacc <= 1 ? 128u : a.nacc == 2 ? 256u : 512u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSt; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&accbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_addr(&s_tmem)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = idesc_bf16_f32(kT, kT);
    unsigned g_prod = 0, g_mma = 0, items_done = 0;
    const int items = a.tiles_m * a.tiles_n * a.ksplit;

    for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x) {
        const int ks = item % a.ksplit, tile = item / a.ksplit;
        const int tm = tile % a.tiles_m, tn = tile / a.tiles_m;
        if (warp == 0 && lane == 0) {
            // TMA producer over every pass's K blocks of this split
            for (int p = 0; p < a.npass && !s_abort; ++p) {
                const FfTcPass &ps = a.pass[p];
                const int kb0 = (int)((long long)ps.kblocks * ks / a.ksplit);
                const int kb1 = (int)((long long)ps.kblocks * (ks + 1) / a.ksplit);
                for (int kb = kb0; kb < kb1; ++kb, ++g_prod) {
                    const int st = g_prod % kSt;
                    const unsigned round = g_prod / kSt;
                    if (round > 0 && !mbar_wait(smem_addr(&empty[st]), (round - 1) & 1u, a.ctl)) {
                        s_abort = 1;
                        break;
                    }
                    const uint32_t fb = smem_addr(&full[st]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                                 :: "r"(fb), "r"((1 + ps.nb) * kStageA) : "memory");
                    const uint32_t dA = sbase + st * kStageBytes;
                    tma_load_2d(dA, &maps.m[ps.amap], ps.a_x + kb * kKB, ps.a_y + tm * kT, fb);
                    tma_load_2d(dA + kStageA, &maps.m[ps.bmap], ps.b_x + kb * kKB, ps.b_y + tn * kT, fb);
                    if (ps.nb > 1)
                        tma_load_2d(dA + 2 * kStageA, &maps.m[ps.bmap2], ps.b_x + kb * kKB, ps.b_y2 + tn * kT, fb);
                }
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer; an accumulator's first MMA of this item overwrites it
            int started = 0;
            for (int p = 0; p < a.npass && !s_abort; ++p) {
                const FfTcPass &ps = a.pass[p];
                const int kb0 = (int)((long long)ps.kblocks * ks / a.ksplit);
                const int kb1 = (int)((long long)ps.kblocks * (ks + 1) / a.ksplit);
                const uint32_t tacc = tmem + (uint32_t)(ps.acc * kT);
                for (int kb = kb0; kb < kb1; ++kb, ++g_mma) {
                    const int st = g_mma % kSt;
                    const unsigned round = g_mma / kSt;
                    if (!mbar_wait(smem_addr(&full[st]), round & 1u, a.ctl)) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t dA = sbase + st * kStageBytes;
                    for (int q = 0; q < ps.nb; ++q) {
#pragma unroll
                        for (int kk = 0; kk < 128 / 32; ++kk) {
                            const int on = ((started >> ps.acc) & 1) | (q > 0) | (kk > 0);
                            mma_bf16(tacc, umma_desc_sw128(dA + kk * 32),
                                     umma_desc_sw128(dA + (1 + q) * kStageA + kk * 32), idesc, on);
                        }
                    }
                    started |= 1 << ps.acc;
                    mma_commit(smem_addr(&empty[st]));
                }
            }
            s_started = started;
            mma_commit(smem_addr(&accbar));
        }
        __syncwarp();
        const bool ok = mbar_wait(smem_addr(&accbar), items_done & 1u, a.ctl);
        ++items_done;
        if (!ok) s_abort = 1;
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // epilogue: warps w and w+4 read TMEM lane quarter w (tile rows), each
        // half of the columns; values go to a staged tile in the (now idle)
        // pipeline buffers, then leave as coalesced rows
        float *Cs = (float *)smem;                  // [128][kCPitch]
        const int quarter = warp & 3, half = warp >> 2;
        const int ml = quarter * 32 + lane, m = tm * kT + ml;
        const int started = s_started;
        for (int cc = 0; cc < 2; ++cc) {
            const int c0 = half * 64 + cc * 32;
            const int n0 = tn * kT + c0;
            float out[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) out[q] = 0.0f;
            const int nacc = a.mode == 1 ? a.nacc : 1;
            for (int d = 0; d < nacc; ++d) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(d * kT + c0), v);
                if (!ok || !((started >> d) & 1)) continue;
                if (a.mode == 0) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) out[q] = __uint_as_float(v[q]);
                } else if (m < a.M) {
                    // the weight gradient of (m, n) is that of its own delay
                    const uint8_t *Dr = a.D + (size_t)m * a.N;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (n0 + q < a.N && Dr[n0 + q] == d + 1) out[q] = __uint_as_float(v[q]);
                }
            }
            float4 *dst = (float4 *)(Cs + ml * kCPitch + c0);
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4)
                dst[q4] = make_float4(out[4 * q4], out[4 * q4 + 1], out[4 * q4 + 2], out[4 * q4 + 3]);
        }
        __syncthreads();
        if (ok) {
            float *C = a.C + (size_t)ks * a.cstride;
            const int ncol = min(kT, a.N - tn * kT);
            for (int row = warp; row < kT; row += kThreads / 32) {
                const int mm = tm * kT + row;
                if (mm >= a.M) break;
                float *crow = C + (size_t)mm * a.ldc + tn * kT;
                const float *srow = Cs + row * kCPitch;
                for (int c = lane; c < ncol; c += 32) crow[c] = srow[c];
            }
        }
        // the staged tile was written and read through the generic proxy; the
        // next item's TMA (async proxy) reuses those bytes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
    }

    // drain: copies issued and MMAs committed complete before shared memory and
    // TMEM go away (bounded waits; no-ops when the phases have completed)
    if (warp == 0 && lane == 0) {
        for (unsigned i = g_prod > kSt ? g_prod - kSt : 0; i < g_prod; ++i)
            mbar_wait(smem_addr(&full[i % kSt]), (i / kSt) & 1u, a.ctl);
    }
    if (warp == 1 && lane == 0) {
        for (unsigned i = g_mma > kSt ? g_mma - kSt : 0; i < g_mma; ++i)
            mbar_wait(smem_addr(&empty[i % kSt]), (i / kSt) & 1u, a.ctl);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(ncols));
}

// Forward synaptic input with block-wise accumulation.  384 threads: warp 0
// lane 0 issues TMA (K block outer, pass inner), warp 1 lane 0 issues the
// MMAs of one K block of every pass into TMEM buffer (block & 1) and commits
// it to accf[buf]; warps 4..11 (warp w: TMEM lane quarter w % 4, columns
// 64 * ((w - 4) / 4) ..+63) add each block's partial into FP32 registers and
// release the buffer through acce[buf] (8 arrivals).  Every pass has the
// same number of K blocks; a.C[m][n] = the sum (mode 0 layout).  A pass
// multiplies its A tile by kFwdParts B tiles (rows b_y + s * a.part_stride,
// s = 0 .. kFwdParts-1: the parts of one weight split), so a stage holds one
// A tile and kFwdParts B tiles and A is read once for all parts.
constexpr int kFwdTcThreads = 384;
constexpr int kFwdParts = 3;
constexpr int kFwdStageBytes = (1 + kFwdParts) * kStageA;   // 64 KiB
constexpr int kFwdSt = 3;

__global__ void __launch_bounds__(kFwdTcThreads, 1) ff_tc_fwd_kernel(const __grid_constant__ FfTcMaps maps,
                                                                     FfTcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kFwdSt], empty[kFwdSt], accf[2], acce[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_addr(smem);
    constexpr unsigned ncols = 256;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFwdSt; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&empty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_addr(&accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" :: "r"(smem_addr(&acce[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_addr(&s_tmem)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = idesc_bf16_f32(kT, kT);
    const int items = a.tiles_m * a.tiles_n;
    const int KB = a.pass[0].kblocks;
    unsigned g_prod = 0, g_mma = 0;

    if (warp == 0 && lane == 0) {
        for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x) {
            const int tm = item % a.tiles_m, tn = item / a.tiles_m;
            for (int kb = 0; kb < KB && !s_abort; ++kb)
                for (int p = 0; p < a.npass; ++p, ++g_prod) {
                    const FfTcPass &ps = a.pass[p];
                    const int st = g_prod % kFwdSt;
                    const unsigned round = g_prod / kFwdSt;
                    if (round > 0 && !mbar_wait(smem_addr(&empty[st]), (round - 1) & 1u, a.ctl)) {
                        s_abort = 1;
                        break;
                    }
                    const uint32_t fb = smem_addr(&full[st]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                                 :: "r"(fb), "r"(kFwdStageBytes) : "memory");
                    const uint32_t dA = sbase + st * kFwdStageBytes;
                    tma_load_2d(dA, &maps.m[ps.amap], ps.a_x + kb * kKB, ps.a_y + tm * kT, fb);
#pragma unroll
                    for (int q = 0; q < kFwdParts; ++q)
                        tma_load_2d(dA + (1 + q) * kStageA, &maps.m[ps.bmap], ps.b_x + kb * kKB,
                                    ps.b_y + q * a.part_stride + tn * kT, fb);
                }
        }
    } else if (warp == 1 && lane == 0) {
        unsigned g_chunk = 0;
        for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x)
            for (int kb = 0; kb < KB && !s_abort; ++kb, ++g_chunk) {
                const unsigned buf = g_chunk & 1u, use = g_chunk >> 1;
                if (use > 0 && !mbar_wait(smem_addr(&acce[buf]), (use - 1) & 1u, a.ctl)) { s_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t tacc = tmem + buf * kT;
                for (int p = 0; p < a.npass; ++p, ++g_mma) {
                    const int st = g_mma % kFwdSt;
                    const unsigned round = g_mma / kFwdSt;
                    if (!mbar_wait(smem_addr(&full[st]), round & 1u, a.ctl)) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t dA = sbase + st * kFwdStageBytes;
#pragma unroll
                    for (int q = 0; q < kFwdParts; ++q)
#pragma unroll
                        for (int kk = 0; kk < 128 / 32; ++kk)
                            mma_bf16(tacc, umma_desc_sw128(dA + kk * 32),
                                     umma_desc_sw128(dA + (1 + q) * kStageA + kk * 32), idesc,
                                     (p > 0) | (q > 0) | (kk > 0));
                    mma_commit(smem_addr(&empty[st]));
                }
                mma_commit(smem_addr(&accf[buf]));
            }
    } else if (warp >= 4) {
        const int quarter = warp & 3, half = (warp - 4) >> 2;
        unsigned g_chunk = 0;
        for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x) {
            const int tm = item % a.tiles_m, tn = item / a.tiles_m;
            float acc[64];
#pragma unroll
            for (int q = 0; q < 64; ++q) acc[q] = 0.0f;
            bool ok = true;
            for (int kb = 0; kb < KB; ++kb, ++g_chunk) {
                const unsigned buf = g_chunk & 1u, use = g_chunk >> 1;
                ok = ok && mbar_wait(smem_addr(&accf[buf]), use & 1u, a.ctl);
                __syncwarp();
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + buf * kT + (uint32_t)(half * 64 + h * 32), v);
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc[h * 32 + q] = __fadd_rn(acc[h * 32 + q], __uint_as_float(v[q]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(smem_addr(&acce[buf])) : "memory");
                if (!ok) break;
            }
            if (!ok) { s_abort = 1; break; }
            const int m = tm * kT + quarter * 32 + lane;
            const int n0 = tn * kT + half * 64;
            if (m < a.M) {
                float *crow = a.C + (size_t)m * a.ldc;
                if (n0 + 64 <= a.N && (a.ldc & 3) == 0) {
#pragma unroll
                    for (int q4 = 0; q4 < 16; ++q4)
                        *(float4 *)(crow + n0 + 4 * q4) =
                            make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 64; ++q)
                        if (n0 + q < a.N) crow[n0 + q] = acc[q];
                }
            }
        }
    }
    __syncwarp();

    // drain: copies issued and MMAs committed complete before shared memory and
    // TMEM go away (bounded waits; no-ops when the phases have completed)
    if (warp == 0 && lane == 0) {
        for (unsigned i = g_prod > kFwdSt ? g_prod - kFwdSt : 0; i < g_prod; ++i)
            mbar_wait(smem_addr(&full[i % kFwdSt]), (i / kFwdSt) & 1u, a.ctl);
    }
    if (warp == 1 && lane == 0) {
        for (unsigned i = g_mma > kFwdSt ? g_mma - kFwdSt : 0; i < g_mma; ++i)
            mbar_wait(smem_addr(&empty[i % kFwdSt]), (i / kFwdSt) & 1u, a.ctl);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(ncols));
}

// Weight parts: Wb[(d-1)*2 + s] = part s (hi, mid) of W_d ([rows_in][nout_p],
// rows_in = n_in rounded up to 128) for the backward; if Wf is given,
// Wf[(d-1)*3 + s] = part s (hi, mid, lo: hi + mid + lo = w exactly) of W_d
// transposed ([rows_out][nin_p]) for the forward.  Only each weight's own
// delay slot is written: the buffers are zeroed once when the context is
// set up and the delays never change, so every other slot stays zero.
// 32 x 32 tiles through shared memory (a grid-stride loop over tiles), so
// that both outputs leave as 64-byte row pieces.
__global__ void __launch_bounds__(256) ff_tc_weights_kernel(const float *__restrict__ W,
                                                            const uint8_t *__restrict__ D, int n_in, int n_out,
                                                            int nout_p, int rows_in, int nin_p, int rows_out,
                                                            __nv_bfloat16 *Wb, __nv_bfloat16 *Wf) {
    __shared__ __nv_bfloat16 sp[3][32][34];
    __shared__ uint8_t sd[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    const size_t bsz = (size_t)rows_in * nout_p, fsz = (size_t)rows_out * nin_p;
    const int ti = (n_in + 31) / 32, tj = (n_out + 31) / 32;
    const long long ntiles = (long long)ti * tj;
    for (long long tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int i0 = (int)(tl / tj) * 32, j0 = (int)(tl % tj) * 32;
        for (int y = ty; y < 32; y += 8) {
            const int i = i0 + y, j = j0 + tx;
            if (i >= n_in || j >= n_out) continue;
            const size_t q = (size_t)i * n_out + j;
            const int d = D[q];
            const float w = W[q];
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const float r1 = __fsub_rn(w, __bfloat162float(hi));
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            if (Wb) {
                const size_t b = (size_t)i * nout_p + j;
                Wb[(size_t)((d - 1) * 2 + 0) * bsz + b] = hi;
                Wb[(size_t)((d - 1) * 2 + 1) * bsz + b] = mid;
            }
            sp[0][y][tx] = hi;
            sp[1][y][tx] = mid;
            sp[2][y][tx] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid)));
            sd[y][tx] = (uint8_t)d;
        }
        if (!Wf) continue;
        __syncthreads();
        for (int y = ty; y < 32; y += 8) {
            const int j = j0 + y, i = i0 + tx;
            if (i >= n_in || j >= n_out) continue;
            const int d = sd[tx][y];
            const size_t f = (size_t)j * nin_p + i;
#pragma unroll
            for (int part = 0; part < 3; ++part) Wf[(size_t)((d - 1) * 3 + part) * fsz + f] = sp[part][tx][y];
        }
        __syncthreads();
    }
}

// Spike bits [rows][words] -> 0/1 BF16: rows S [rows][nin_p] and/or the
// transpose ST [n_in][rows_p], whichever is given (padding stays zero).  A
// block converts a 32 x 32 tile (rows r0.., inputs i0..) through shared
// memory, so both outputs leave as 64-byte row pieces.
__global__ void __launch_bounds__(256) ff_tc_spikes_kernel(const unsigned *__restrict__ bits, int rows, int n_in,
                                                           int words, int nin_p, int rows_p, __nv_bfloat16 *S,
                                                           __nv_bfloat16 *ST) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.x * 32, i0 = blockIdx.y * 32;   // rows on x: no 65535 limit
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    for (int y = ty; y < 32; y += 8) {
        const int r = r0 + y, i = i0 + tx;
        bool sp = false;
        if (r < rows && i < n_in) sp = (__ldg(bits + (size_t)r * words + (i >> 5)) >> (i & 31)) & 1u;
        tile[y][tx] = sp ? one : zero;
        if (S && r < rows && i < n_in) S[(size_t)r * nin_p + i] = sp ? one : zero;
    }
    if (!ST) return;
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int i = i0 + y, r = r0 + tx;
        if (i < n_in && r < rows) ST[(size_t)i * rows_p + r] = tile[tx][y];
    }
}

// Gradient gI [rows][n_out] -> two-term BF16 split G[s] ([rows][nout_p]) and,
// if GT is given, its transpose GT[s] ([n_out][rows_p]); 32 x 32 tiles
// through shared memory.
__global__ void __launch_bounds__(256) ff_tc_gsplit_kernel(const float *__restrict__ g, int rows, int n_out,
                                                           int nout_p, int rows_p, __nv_bfloat16 *G,
                                                           __nv_bfloat16 *GT) {
    __shared__ __nv_bfloat16 th[32][34], tm[32][34];
    const int r0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const size_t gsz = (size_t)rows * nout_p, tsz = (size_t)n_out * rows_p;
    for (int y = ty; y < 32; y += 8) {
        const int r = r0 + y, j = j0 + tx;
        float x = 0.0f;
        if (r < rows && j < n_out) x = __ldg(g + (size_t)r * n_out + j);
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 mid = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(hi)));
        th[y][tx] = hi;
        tm[y][tx] = mid;
        if (G && r < rows && j < n_out) {
            G[(size_t)r * nout_p + j] = hi;
            G[gsz + (size_t)r * nout_p + j] = mid;
        }
    }
    if (!GT) return;
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int j = j0 + y, r = r0 + tx;
        if (j < n_out && r < rows) {
            GT[(size_t)j * rows_p + r] = th[tx][y];
            GT[tsz + (size_t)j * rows_p + r] = tm[tx][y];
        }
    }
}

// Blocks for a grid-stride loop over 32 x 32 tiles: at most 1216 (eight per
// SM of a 152-SM part).
static int tile_grid(long long tiles) {
    const long long b = tiles < 1216 ? tiles : 1216;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t ff_tc_smem_bytes() { return (size_t)kSt * kStageBytes + 1024; }

cudaError_t ff_tc_gemm(const FfTcMaps &maps, const FfTcArgs &args, cudaStream_t s) {
    static_assert(kT * kCPitch * 4 <= kSt * kStageBytes, "staged output tile fits the stage buffers");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int p = 0; p < args.npass; ++p)
        if (args.pass[p].nb < 1 || args.pass[p].nb > 2) return cudaErrorInvalidValue;
    const size_t smem = ff_tc_smem_bytes();
    if ((e = cudaFuncSetAttribute((const void *)ff_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const int items = args.tiles_m * args.tiles_n * args.ksplit;
    const int grid = items < sms ? items : sms;
    ff_tc_kernel<<<grid, kThreads, smem, s>>>(maps, args);
    return cudaGetLastError();
}

cudaError_t ff_tc_forward(const FfTcMaps &maps, const FfTcArgs &args, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int p = 1; p < args.npass; ++p)
        if (args.pass[p].kblocks != args.pass[0].kblocks) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kFwdSt * kFwdStageBytes + 1024;
    if ((e = cudaFuncSetAttribute((const void *)ff_tc_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const int items = args.tiles_m * args.tiles_n;
    const int grid = items < sms ? items : sms;
    ff_tc_fwd_kernel<<<grid, kFwdTcThreads, smem, s>>>(maps, args);
    return cudaGetLastError();
}

cudaError_t ff_tc_weights(const float *W, const uint8_t *D, int n_in, int n_out, int nout_p, int rows_in,
                          void *Wb, int nin_p, int rows_out, void *Wf, cudaStream_t s) {
    ff_tc_weights_kernel<<<tile_grid((long long)((n_in + 31) / 32) * ((n_out + 31) / 32)), 256, 0, s>>>(
        W, D, n_in, n_out, nout_p, rows_in, nin_p, rows_out, (__nv_bfloat16 *)Wb, (__nv_bfloat16 *)Wf);
    return cudaGetLastError();
}

cudaError_t ff_tc_spikes(const unsigned *bits, int rows, int n_in, int words, int nin_p, int rows_p, void *S,
                         void *ST, cudaStream_t s) {
    // one block per tile: a grid-stride loop over tiles measured slower
    const dim3 grid((rows + 31) / 32, (n_in + 31) / 32);
    ff_tc_spikes_kernel<<<grid, 256, 0, s>>>(bits, rows, n_in, words, nin_p, rows_p, (__nv_bfloat16 *)S,
                                            (__nv_bfloat16 *)ST);
    return cudaGetLastError();
}

cudaError_t ff_tc_gsplit(const float *g, int rows, int n_out, int nout_p, int rows_p, void *G, void *GT,
                         cudaStream_t s) {
    const dim3 grid((rows + 31) / 32, (n_out + 31) / 32);
    ff_tc_gsplit_kernel<<<grid, 256, 0, s>>>(g, rows, n_out, nout_p, rows_p, (__nv_bfloat16 *)G,
                                            (__nv_bfloat16 *)GT);
    return cudaGetLastError();
}

}  // namespace sn
