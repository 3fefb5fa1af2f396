// Feedforward spiking network with per-synapse delays: exact forward
// simulation and the surrogate-gradient adjoint (backpropagation through
// time) with membrane checkpoints and recomputation.
//
// Layer l (1..L) maps n_in = n_{l-1} inputs to n_out = n_l LIF neurons with
// weights W[i][j] (row-major, i = pre) and delays D[i][j] in 1..4.  Because
// every delay is at least one step, the synaptic input of layer l at step t
// depends only on layer l-1 at steps <= t-1, so each layer is computed for
// all timesteps at once:
//   I[t][b][j] = sum_i W[i][j] * s_{l-1}[t - D[i][j]][b][i]      (delay GEMM)
// followed by the LIF recurrence of every (b, j) over t (Section 2.1 order:
// leak toward reset, add input, strict threshold, refractory mask, reset).
//
// Adjoint (per (b, j), backwards in t; reset detached, refractory mask
// constant, clamped-leak derivative [|V - reset| > leak]):
//   gu(t)  = gV(t) (1 - s(t)) + gs(t) m(t) / (1 + slope |u(t) - theta|)^2
//   gI(t)  = gu(t);   gV(t-1) = gu(t) L'(V(t-1))
//   gs_{l-1}[t][b][i] = sum_j W[i][j] gI[t + D[i][j]][b][j]
//   dW[i][j]          = sum_{t,b} gI[t][b][j] s_{l-1}[t - D[i][j]][b][i]
// u(t) is recomputed from membrane checkpoints stored every k steps.
//
// This file holds the recurrences and the CUDA-core (SIMT) forms of the three
// contractions; sn_ff_tc.cu holds their tensor-core forms, which the host
// code uses by default (sn_ff_set_engine).

#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_internal.h"

namespace sn {

constexpr int kFFDelays = 4;
constexpr unsigned short kBf16One = 0x3f80;          // 1.0 in BF16

// ---------------------------------------------------------------------------
// input spikes (bytes) -> bit rows [T*B][words], and, if sbf is given, BF16
// rows [T*B][ldbf] (1 or 0; the tensor cores' spike operand)
__global__ void ff_pack_kernel(const uint8_t *in, int rows, int n, int words, unsigned *out,
                               unsigned short *sbf, int ldbf) {
    const int lane = threadIdx.x & 31;
    constexpr int kU = 4;                      // words per warp and iteration (loads in flight)
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = (long long)rows * words;
    for (long long w0 = gw * kU; w0 < total; w0 += nw * kU) {
        bool bit[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const long long w = w0 + u;
            const long long r = w / words;
            const int i = (int)(w - r * words) * 32 + lane;
            bit[u] = w < total && i < n && in[r * n + i] != 0;
            if (sbf && w < total && i < n) sbf[r * ldbf + i] = bit[u] ? kBf16One : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const unsigned word = __ballot_sync(0xffffffffu, bit[u]);
            if (lane == 0 && w0 + u < total) out[w0 + u] = word;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward delay GEMM.  Block = 8 warps; a warp owns 32 output columns (one per
// lane) and kRowsPerWarp rows; the block shares the columns, so the weight
// chunk [32 inputs][32 columns] is staged once in shared memory.  dm holds,
// per 32-input chunk c and column j, one bit mask per delay d:
// bit (i - 32c) of dm[(c * n_out + j) * 4 + d - 1] is set iff D[i][j] == d.
constexpr int kFwdWarps = 8;
constexpr int kRowsPerWarp = 8;
constexpr int kFwdRows = kFwdWarps * kRowsPerWarp;

__global__ void __launch_bounds__(kFwdWarps * 32)
ff_delay_fwd_kernel(const unsigned *__restrict__ sprev, int words_in, const float *__restrict__ W,
                    const uint4 *__restrict__ dm, int n_in, int n_out, int B, int row0, int rows,
                    float *__restrict__ I) {
    __shared__ float ws[32][33];
    __shared__ unsigned sw[kFwdRows][kFFDelays];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int rbase = row0 + blockIdx.y * kFwdRows;
    float acc[kRowsPerWarp];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) acc[q] = 0.0f;
    const int chunks = (n_in + 31) / 32;
    for (int c = 0; c < chunks; ++c) {
        __syncthreads();
        // weights of the chunk: ws[ii][lane] = W[32c + ii][col]
        for (int ii = warp; ii < 32; ii += kFwdWarps) {
            const int i = c * 32 + ii;
            ws[ii][lane] = (i < n_in && col < n_out) ? W[(size_t)i * n_out + col] : 0.0f;
        }
        // delayed spike words of the block's rows
        for (int e = threadIdx.x; e < kFwdRows * kFFDelays; e += blockDim.x) {
            const int rr = e / kFFDelays, d = e % kFFDelays + 1;
            const int row = rbase + rr;
            unsigned v = 0;
            if (row < row0 + rows) {
                const int t = row / B, b = row - (row / B) * B;
                if (t - d >= 0) v = sprev[((size_t)(t - d) * B + b) * words_in + c];
            }
            sw[rr][d - 1] = v;
        }
        __syncthreads();
        uint4 m = make_uint4(0, 0, 0, 0);
        if (col < n_out) m = dm[(size_t)c * n_out + col];
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q) {
            const int rr = warp * kRowsPerWarp + q;
            const unsigned s1 = sw[rr][0], s2 = sw[rr][1], s3 = sw[rr][2], s4 = sw[rr][3];
            const unsigned mine = (s1 & m.x) | (s2 & m.y) | (s3 & m.z) | (s4 & m.w);
            unsigned any = s1 | s2 | s3 | s4;            // same for every lane
            float a = acc[q];
            while (any) {
                const int ii = __ffs(any) - 1;
                any &= any - 1u;
                if ((mine >> ii) & 1u) a = __fadd_rn(a, ws[ii][lane]);
            }
            acc[q] = a;
        }
    }
    if (col < n_out) {
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q) {
            const int row = rbase + warp * kRowsPerWarp + q;
            if (row < row0 + rows) I[(size_t)row * n_out + col] = acc[q];
        }
    }
}

// ---------------------------------------------------------------------------
// LIF recurrence of one layer over all steps.  Thread = (b, j); a warp covers
// 32 consecutive j of one sample, so its ballot is a spike word.
struct FFNeuron {
    float theta, leak, reset, slope;
    int refractory;
};

__device__ __forceinline__ float ff_leak(float v, float lk, float rs) {
    if (v > rs) { const float u = __fsub_rn(v, lk); return u > rs ? u : rs; }
    if (v < rs) { const float u = __fadd_rn(v, lk); return u < rs ? u : rs; }
    return rs;
}

// The inputs of a thread's next kScanChunk steps are copied into its own
// column of a shared-memory buffer by asynchronous 4-byte copies, one chunk
// ahead of their use (they do not depend on the recurrence): up to
// 2 * kScanChunk loads of a thread in flight without holding registers.
constexpr int kScanChunk = 16;
constexpr int kScanBlock = 256;

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__global__ void __launch_bounds__(kScanBlock) ff_scan_fwd_kernel(const float *__restrict__ I, int n, int words,
                                   int B, int T, int k, FFNeuron p, unsigned *__restrict__ S,
                                   float *__restrict__ vck, int *__restrict__ rck, float *__restrict__ counts,
                                   unsigned short *__restrict__ sbf, int ldbf) {
    __shared__ float sI[2][kScanChunk][kScanBlock];
    const int lane = threadIdx.x & 31;
    const int per_b = words * 32;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)B * per_b) return;          // whole warps exit together
    const int b = (int)(tid / per_b);
    const int j = (int)(tid - (long long)b * per_b);
    const bool live = j < n;
    float v = p.reset;
    int r = 0;
    float cnt = 0.0f;
    const size_t stride = (size_t)B * n;
    const float *Ip = I + (size_t)b * n + j;
    // chunk c of steps [c * kScanChunk, ...) into buffer c & 1; an empty
    // group past the last step keeps the wait count uniform
    auto issue = [&](int c) {
        const int t0 = c * kScanChunk;
        if (live)
            for (int q = 0; q < kScanChunk && t0 + q < T; ++q)
                cp_async4(&sI[c & 1][q][threadIdx.x], Ip + (size_t)(t0 + q) * stride);
        cp_async_commit();
    };
    issue(0);
    // output pointers advance by one step's row (the per-step index
    // arithmetic was most of the loop's instructions)
    unsigned *Sp = S + (size_t)b * words + (j >> 5);
    const size_t s_step = (size_t)B * words;
    unsigned short *bp = sbf ? sbf + (size_t)b * ldbf + j : nullptr;
    const size_t b_step = (size_t)B * ldbf;
    float *vp = vck + (size_t)b * n + j;
    int *rp = rck + (size_t)b * n + j;
    int until_ck = k;                                  // steps to the next checkpoint
    for (int c = 0; c * kScanChunk < T; ++c) {
        issue(c + 1);
        cp_async_wait_prev();                          // chunk c has landed (each thread reads its own copies)
        const int qn = min(kScanChunk, T - c * kScanChunk);
        for (int q = 0; q < qn; ++q) {
            bool s = false;
            if (live) {
                const float in = sI[c & 1][q][threadIdx.x];
                const float u = __fadd_rn(ff_leak(v, p.leak, p.reset), in);
                s = (u > p.theta) && (r == 0);
                if (s) { v = p.reset; r = p.refractory; }
                else { v = u; if (r > 0) r -= 1; }
                if (s) cnt += 1.0f;
            }
            const unsigned word = __ballot_sync(0xffffffffu, s);
            if (lane == 0) *Sp = word;
            Sp += s_step;
            if (bp) {
                if (live) *bp = s ? kBf16One : 0;
                bp += b_step;
            }
            if (--until_ck == 0) {
                until_ck = k;
                if (live) { *vp = v; *rp = r; }
                vp += stride;
                rp += stride;
            }
        }
    }
    if (live && counts) counts[(size_t)b * n + j] = cnt;
}

// Adjoint of the recurrence for one layer: segments of k steps from the last
// to the first; each is recomputed from its checkpoint (u kept in registers),
// then walked backwards.  gs = gradient w.r.t. the layer's spikes: per step
// ([T][B][n]) or, for the output layer, the count gradient gc [B][n] that
// every step shares.  A segment's inputs and spike gradients do not depend on
// the adjoint: those of segment sg - 1 are copied into the thread's own
// column of a shared-memory buffer (asynchronous 4-byte copies) while segment
// sg is computed, and its checkpoint is loaded into registers.
constexpr int kBwdBlock = 128;

template <int K>
__global__ void __launch_bounds__(kBwdBlock) ff_scan_bwd_kernel(const float *__restrict__ I, int n, int B, int T,
                                   FFNeuron p, const float *__restrict__ vck, const int *__restrict__ rck,
                                   const float *__restrict__ gs, const float *__restrict__ gc,
                                   float *__restrict__ gI) {
    __shared__ float sI[2][K][kBwdBlock], sG[2][K][kBwdBlock];
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)B * n) return;
    const int b = (int)(tid / n), j = (int)(tid - (long long)(tid / n) * n);
    const int segs = (T + K - 1) / K;
    const float gcount = gc ? gc[(size_t)b * n + j] : 0.0f;
    const size_t stride = (size_t)B * n;
    const float *Ib = I + (size_t)b * n + j;
    const float *Gb = gs ? gs + (size_t)b * n + j : nullptr;
    float *gIb = gI + (size_t)b * n + j;
    // segment sg's inputs (and spike gradients) into buffer sg & 1; an empty
    // group before the first segment keeps the wait count uniform
    auto issue = [&](int sg) {
        if (sg >= 0) {
            const int t0 = sg * K;
            for (int q = 0; q < K && t0 + q < T; ++q) {
                cp_async4(&sI[sg & 1][q][threadIdx.x], Ib + (size_t)(t0 + q) * stride);
                if (Gb) cp_async4(&sG[sg & 1][q][threadIdx.x], Gb + (size_t)(t0 + q) * stride);
            }
        }
        cp_async_commit();
    };
    // checkpoint of segment sg: the state after step sg * K - 1
    auto ckpt = [&](int sg, float &v0, int &r0) {
        v0 = p.reset;
        r0 = 0;
        if (sg > 0) {
            const size_t q = ((size_t)(sg - 1) * B + b) * n + j;
            v0 = __ldg(vck + q);
            r0 = __ldg(rck + q);
        }
    };
    float gv = 0.0f, vc;
    int rc;
    issue(segs - 1);
    ckpt(segs - 1, vc, rc);
    for (int sg = segs - 1; sg >= 0; --sg) {
        const int t0 = sg * K;
        issue(sg - 1);
        float vn = p.reset;
        int rn = 0;
        if (sg > 0) ckpt(sg - 1, vn, rn);
        cp_async_wait_prev();                          // segment sg has landed (own copies)
        const int buf = sg & 1;
        float v = vc;
        int r = rc;
        float u[K], vprev[K];
        bool sp[K], mk[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int t = t0 + q;
            vprev[q] = v;
            if (t < T) {
                u[q] = __fadd_rn(ff_leak(v, p.leak, p.reset), sI[buf][q][threadIdx.x]);
                mk[q] = (r == 0);
                sp[q] = (u[q] > p.theta) && mk[q];
                if (sp[q]) { v = p.reset; r = p.refractory; }
                else { v = u[q]; if (r > 0) r -= 1; }
            } else {
                u[q] = 0.0f; mk[q] = false; sp[q] = false;
            }
        }
#pragma unroll
        for (int q = K - 1; q >= 0; --q) {
            const int t = t0 + q;
            if (t >= T) continue;
            const float x = fabsf(u[q] - p.theta);
            const float den = 1.0f + p.slope * x;
            // 1 / den^2, correctly rounded (the same value as the division)
            const float sur = mk[q] ? __frcp_rn(__fmul_rn(den, den)) : 0.0f;
            const float g = Gb ? sG[buf][q][threadIdx.x] : gcount;
            const float gu = (sp[q] ? 0.0f : gv) + g * sur;
            gIb[(size_t)t * stride] = gu;
            const float dv = vprev[q] - p.reset;
            gv = (fabsf(dv) > p.leak) ? gu : 0.0f;
        }
        vc = vn;
        rc = rn;
    }
}

// ---------------------------------------------------------------------------
// Gradient w.r.t. the previous layer's spikes:
//   gsp[t][b][i] = sum_j W[i][j] * gI[t + D[i][j]][b][j]   (0 beyond T-1)
// Block = 8 warps over 32 inputs (one per lane) x 64 rows (8 per warp); the
// reduction over j runs in chunks of 32 staged in shared memory.
constexpr int kBdRows = 64;

__global__ void __launch_bounds__(256)
ff_bwd_data_kernel(const float *__restrict__ gI, const float *__restrict__ W, const uint8_t *__restrict__ D,
                   int n_in, int n_out, int B, int T, float *__restrict__ gsp) {
    __shared__ float wt[32][33];            // wt[jj][ii] = W[i][j]
    __shared__ uint8_t dt[32][33];          // dt[jj][ii] = D[i][j] - 1
    __shared__ float gs[kBdRows][kFFDelays][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int rbase = blockIdx.y * kBdRows;
    const int rows = T * B;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    for (int j0 = 0; j0 < n_out; j0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int ii = e / 32, jj = e % 32;        // coalesced over j
            const int ig = blockIdx.x * 32 + ii, jg = j0 + jj;
            const bool ok = ig < n_in && jg < n_out;
            wt[jj][ii] = ok ? W[(size_t)ig * n_out + jg] : 0.0f;
            dt[jj][ii] = ok ? (uint8_t)(D[(size_t)ig * n_out + jg] - 1) : (uint8_t)0;
        }
        for (int e = threadIdx.x; e < kBdRows * kFFDelays * 32; e += blockDim.x) {
            const int jj = e % 32, d = (e / 32) % kFFDelays + 1, rr = e / (32 * kFFDelays);
            const int row = rbase + rr;
            float g = 0.0f;
            if (row < rows && j0 + jj < n_out) {
                const int t = row / B, b = row - (row / B) * B;
                if (t + d < T) g = gI[((size_t)(t + d) * B + b) * n_out + j0 + jj];
            }
            gs[rr][d - 1][jj] = g;
        }
        __syncthreads();
        const int jn = min(32, n_out - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const float w = wt[jj][lane];
            const int d = dt[jj][lane];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = fmaf(w, gs[warp * 8 + q][d][jj], acc[q]);
        }
    }
    if (i < n_in) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int row = rbase + warp * 8 + q;
            if (row < rows) gsp[(size_t)row * n_in + i] = acc[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient, split over the rows (t, b) for parallelism:
//   part[sp][i][j] = sum_{rows of split sp} gI[row][j] * s_{l-1}[t - D[i][j]][b][i]
// Block = 8 warps: the block owns 32 inputs (i) x 256 outputs (j, one per
// thread); each thread keeps 32 accumulators, one per input.
__global__ void __launch_bounds__(256)
ff_dw_kernel(const float *__restrict__ gI, const unsigned *__restrict__ sprev, int words_in,
             const uint8_t *__restrict__ D, int n_in, int n_out, int B, int T, int splits,
             float *__restrict__ part) {
    const int j = blockIdx.x * 256 + threadIdx.x;
    const int c = blockIdx.y;                       // 32-input chunk
    const int sp = blockIdx.z;
    const int rows = T * B;
    const int r0 = (int)((long long)sp * rows / splits), r1 = (int)((long long)(sp + 1) * rows / splits);
    __shared__ unsigned sw[64][kFFDelays];
    int dsh[32];                                    // per input: delay - 1 (or -1 if absent)
#pragma unroll
    for (int ii = 0; ii < 32; ++ii) {
        const int i = c * 32 + ii;
        dsh[ii] = (i < n_in && j < n_out) ? (int)D[(size_t)i * n_out + j] - 1 : -1;
    }
    float acc[32];
#pragma unroll
    for (int ii = 0; ii < 32; ++ii) acc[ii] = 0.0f;
    for (int rb = r0; rb < r1; rb += 64) {
        __syncthreads();
        {
            const int e = threadIdx.x;              // 64 rows x 4 delays = 256 entries
            const int rr = e / kFFDelays, d = e % kFFDelays + 1;
            const int row = rb + rr;
            unsigned v = 0;
            if (row < r1) {
                const int t = row / B, b = row - (row / B) * B;
                if (t - d >= 0) v = sprev[((size_t)(t - d) * B + b) * words_in + c];
            }
            sw[rr][d - 1] = v;
        }
        __syncthreads();
        const int rn = min(64, r1 - rb);
        for (int rr = 0; rr < rn; ++rr) {
            const unsigned s1 = sw[rr][0], s2 = sw[rr][1], s3 = sw[rr][2], s4 = sw[rr][3];
            if ((s1 | s2 | s3 | s4) == 0u) continue;        // uniform over the block
            const float g = j < n_out ? gI[(size_t)(rb + rr) * n_out + j] : 0.0f;
#pragma unroll
            for (int ii = 0; ii < 32; ++ii) {
                const int d = dsh[ii];
                const unsigned w = d == 0 ? s1 : d == 1 ? s2 : d == 2 ? s3 : s4;
                if (d >= 0 && ((w >> ii) & 1u)) acc[ii] = __fadd_rn(acc[ii], g);
            }
        }
    }
    if (j < n_out) {
#pragma unroll
        for (int ii = 0; ii < 32; ++ii) {
            const int i = c * 32 + ii;
            if (i < n_in) part[((size_t)sp * n_in + i) * n_out + j] = acc[ii];
        }
    }
}

// Weight gradient from the spike lists (sparse form): input i's spikes are
// few, so
//   dW[i][j] = sum over spikes (t', b) of input i of gI[t' + D[i][j]][b][j]
// with t' + D < T.  One block per input (and per 2048-column slice): it
// compacts the rows (t', b) where the input spiked, in ascending order, into
// shared memory, then each thread accumulates its columns over that list.
constexpr int kDwJ = 8;                          // columns per thread
constexpr int kDwCols = 256 * kDwJ;              // columns per block

__global__ void __launch_bounds__(256)
ff_dw_sparse_kernel(const float *__restrict__ gI, const unsigned *__restrict__ sprev, int words_in,
                    const uint8_t *__restrict__ D, int n_in, int n_out, int B, int T, float *__restrict__ dW) {
    extern __shared__ int s_rows[];             // [T * B] spike rows of input i
    __shared__ int s_warp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x;
    const int jb = blockIdx.y * kDwCols;
    const int rows = T * B;
    const int c = i >> 5;
    const unsigned bit = 1u << (i & 31);
    int count = 0;
    for (int r0 = 0; r0 < rows; r0 += 256) {
        const int r = r0 + threadIdx.x;
        const bool sp = r < rows && (sprev[(size_t)r * words_in + c] & bit);
        const unsigned ball = __ballot_sync(0xffffffffu, sp);
        if (lane == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int v = s_warp[w];
            before += w < warp ? v : 0;
            total += v;
        }
        if (sp) s_rows[count + before + __popc(ball & ((1u << lane) - 1u))] = r;
        count += total;
        __syncthreads();
    }
    int dj[kDwJ];
    float acc[kDwJ];
#pragma unroll
    for (int q = 0; q < kDwJ; ++q) {
        const int j = jb + threadIdx.x + 256 * q;
        dj[q] = j < n_out ? (int)D[(size_t)i * n_out + j] : 0;
        acc[q] = 0.0f;
    }
    for (int k = 0; k < count; ++k) {
        const int r = s_rows[k];
        const int t = r / B, b = r - (r / B) * B;
#pragma unroll
        for (int q = 0; q < kDwJ; ++q) {
            const int tt = t + dj[q];
            if (dj[q] > 0 && tt < T)
                acc[q] = __fadd_rn(acc[q], __ldg(gI + ((size_t)tt * B + b) * n_out + jb + threadIdx.x + 256 * q));
        }
    }
#pragma unroll
    for (int q = 0; q < kDwJ; ++q) {
        const int j = jb + threadIdx.x + 256 * q;
        if (j < n_out) dW[(size_t)i * n_out + j] = acc[q];
    }
}

constexpr int kDwSparseMaxRows = 49152;          // spike-list capacity (192 KiB of shared memory)

__global__ void ff_dw_reduce_kernel(const float *__restrict__ part, int splits, long long count,
                                    float *__restrict__ dW) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int sp = 0; sp < splits; ++sp) s = __fadd_rn(s, part[(size_t)sp * count + q]);
        dW[q] = s;
    }
}

// ---------------------------------------------------------------------------
// launchers

static int blocks_for(long long work, int per) {
    long long b = (work + per - 1) / per;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t ff_pack(const uint8_t *in, int rows, int n, int words, unsigned *out, void *sbf, int ldbf,
                    cudaStream_t s) {
    const long long warps = (long long)rows * words;
    // a grid-stride loop over at most 2048 blocks (block launches, not
    // bandwidth, bound one word per warp)
    int nb = blocks_for(warps * 32 / 4, 256);
    nb = nb < 2048 ? nb : 2048;
    ff_pack_kernel<<<nb, 256, 0, s>>>(in, rows, n, words, out, (unsigned short *)sbf, ldbf);
    return cudaGetLastError();
}

cudaError_t ff_delay_fwd(const unsigned *sprev, int words_in, const float *W, const void *dm, int n_in,
                         int n_out, int B, int row0, int rows, float *I, cudaStream_t s) {
    dim3 grid((n_out + 31) / 32, (rows + kFwdRows - 1) / kFwdRows);
    ff_delay_fwd_kernel<<<grid, kFwdWarps * 32, 0, s>>>(sprev, words_in, W, (const uint4 *)dm, n_in, n_out, B,
                                                       row0, rows, I);
    return cudaGetLastError();
}

cudaError_t ff_scan_fwd(const float *I, int n, int B, int T, int k, float theta, float leak, float reset,
                        int refractory, unsigned *S, float *vck, int *rck, float *counts, void *sbf, int ldbf,
                        cudaStream_t s) {
    FFNeuron p{theta, leak, reset, 0.0f, refractory};
    const int words = (n + 31) / 32;
    const long long threads = (long long)B * words * 32;
    ff_scan_fwd_kernel<<<blocks_for(threads, kScanBlock), kScanBlock, 0, s>>>(I, n, words, B, T, k, p, S, vck, rck, counts,
                                                                (unsigned short *)sbf, ldbf);
    return cudaGetLastError();
}

cudaError_t ff_scan_bwd(const float *I, int n, int B, int T, int k, float theta, float leak, float reset,
                        int refractory, float slope, const float *vck, const int *rck, const float *gs,
                        const float *gc, float *gI, cudaStream_t s) {
    FFNeuron p{theta, leak, reset, slope, refractory};
    const long long threads = (long long)B * n;
    const int nb = blocks_for(threads, kBwdBlock);
    switch (k) {
        case 1: ff_scan_bwd_kernel<1><<<nb, kBwdBlock, 0, s>>>(I, n, B, T, p, vck, rck, gs, gc, gI); break;
        case 2: ff_scan_bwd_kernel<2><<<nb, kBwdBlock, 0, s>>>(I, n, B, T, p, vck, rck, gs, gc, gI); break;
        case 5: ff_scan_bwd_kernel<5><<<nb, kBwdBlock, 0, s>>>(I, n, B, T, p, vck, rck, gs, gc, gI); break;
        case 10: ff_scan_bwd_kernel<10><<<nb, kBwdBlock, 0, s>>>(I, n, B, T, p, vck, rck, gs, gc, gI); break;
        case 20: ff_scan_bwd_kernel<20><<<nb, kBwdBlock, 0, s>>>(I, n, B, T, p, vck, rck, gs, gc, gI); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t ff_bwd_data(const float *gI, const float *W, const uint8_t *D, int n_in, int n_out, int B, int T,
                        float *gsp, cudaStream_t s) {
    dim3 grid((n_in + 31) / 32, (T * B + kBdRows - 1) / kBdRows);
    ff_bwd_data_kernel<<<grid, 256, 0, s>>>(gI, W, D, n_in, n_out, B, T, gsp);
    return cudaGetLastError();
}

cudaError_t ff_dw(const float *gI, const unsigned *sprev, int words_in, const uint8_t *D, int n_in, int n_out,
                  int B, int T, int splits, float *part, float *dW, cudaStream_t s) {
    if (T * B <= kDwSparseMaxRows) {
        const size_t smem = (size_t)T * B * sizeof(int);
        cudaError_t e = cudaFuncSetAttribute((const void *)ff_dw_sparse_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 g(n_in, (n_out + kDwCols - 1) / kDwCols);
        ff_dw_sparse_kernel<<<g, 256, smem, s>>>(gI, sprev, words_in, D, n_in, n_out, B, T, dW);
        return cudaGetLastError();
    }
    dim3 grid((n_out + 255) / 256, (n_in + 31) / 32, splits);
    ff_dw_kernel<<<grid, 256, 0, s>>>(gI, sprev, words_in, D, n_in, n_out, B, T, splits, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long count = (long long)n_in * n_out;
    ff_dw_reduce_kernel<<<blocks_for(count, 256), 256, 0, s>>>(part, splits, count, dW);
    return cudaGetLastError();
}

cudaError_t ff_dw_reduce(const float *part, int splits, long long count, float *dW, cudaStream_t s) {
    ff_dw_reduce_kernel<<<blocks_for(count, 256), 256, 0, s>>>(part, splits, count, dW);
    return cudaGetLastError();
}

}  // namespace sn
