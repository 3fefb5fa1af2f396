// Single-network simulation kernels for sm_103a.
//
// Both kernels are persistent: one cooperative launch runs every requested
// timestep.  Each block owns a contiguous, 32-aligned range of neurons, so a
// warp's ballot over 32 neurons is exactly one raster word.
//
// One timestep (SuperNeuro Section 2.1 order; Section 2.2 strict threshold):
//   U: drain the ring slot of step t (pending synaptic input), apply the
//      clamped constant leak, add synaptic and external input, threshold,
//      refractory mask, reset; ballot -> raster word; warp-aggregated
//      compaction of the block's spikers into shared memory.
//   P: propagate (sparse: push each spiker's CSR row into ring slots t+d;
//      dense: gather the rows of all spikers into per-chunk partial sums).
//   STDP (optional): pair-based trace rule fused into the propagation phase;
//      only rows of spiking pre-neurons and columns of spiking post-neurons
//      are touched.
// Blocks meet at a grid barrier whose wait is bounded by a wall-clock limit;
// on expiry the kernel latches SN_ETIMEOUT and every block returns.

#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_device.cuh"
#include "sn_internal.h"

namespace sn {

// Phase U for the block's neurons [j0, j1).  `take_acc(j)` returns the pending
// synaptic input of j for this step.  Spikers go to s_list (block order is
// not deterministic; nothing downstream depends on it).
template <int MODE, bool STDP, typename TakeAcc>
__device__ __forceinline__ void phase_update(const NetArgs &a, int t, int j0, int j1, int *s_list,
                                             int *s_cnt, TakeAcc take_acc) {
    using V = typename Tr<MODE>::V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned *rrow = a.raster + (size_t)(t % a.cap) * a.words;
    V *Vp = (V *)a.V;
    const V *th = (const V *)a.th, *lk = (const V *)a.lk, *rs = (const V *)a.rs;
    bool overflow = false;
    for (int jb = j0; jb < j1; jb += blockDim.x) {
        const int j = jb + threadIdx.x;
        bool fire = false;
        if (j < j1) {
            V acc = take_acc(j);
            V ext = external_input<MODE>(a, t, j);
            V v = Vp[j];
            int rr = a.r[j];
            if constexpr (MODE == SN_F32)
                fire = lif_update_f32(v, rr, acc, ext, th[j], lk[j], rs[j], a.R[j]);
            else
                fire = lif_update_i32(v, rr, acc, ext, th[j], lk[j], rs[j], a.R[j], overflow);
            Vp[j] = v;
            a.r[j] = rr;
            if constexpr (STDP) {
                const float *xo = a.trace + (size_t)((t & 1) ^ 1) * a.n;
                float *xn = a.trace + (size_t)(t & 1) * a.n;
                xn[j] = __fadd_rn(__fmul_rn(a.decay, xo[j]), fire ? 1.0f : 0.0f);
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, fire);
        const int wbase = jb + warp * 32;
        if (lane == 0 && wbase < j1) rrow[wbase >> 5] = ball;
        if (ball) {
            int base = 0;
            if (lane == 0) base = atomicAdd(s_cnt, __popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (fire) s_list[base + __popc(ball & ((1u << lane) - 1u))] = j;
        }
    }
    if (MODE == SN_I32 && overflow) atomicCAS(&a.ctl->status, 0, (int)SN_EOVERFLOW);
}

// ---------------------------------------------------------------------------
// Sparse network: CSR push into a ring of D+1 slots.  Slot (t+d) mod (D+1)
// never equals slot t mod (D+1) for 1 <= d <= D, so a block may push right
// after its own update while other blocks are still draining slot t: one grid
// barrier per step suffices (two with STDP, which needs every spike of t).

constexpr int kBlock = 256;

template <int MODE, bool STDP>
__global__ void __launch_bounds__(kBlock) sparse_kernel(NetArgs a) {
    using A = typename Tr<MODE>::A;
    using V = typename Tr<MODE>::V;
    extern __shared__ int s_list[];            // chunk entries
    __shared__ int s_cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int j0 = blockIdx.x * a.chunk;
    const int j1 = min(a.n, j0 + a.chunk);
    A *ring = (A *)a.ring;
    unsigned long long my_spikes = 0, my_events = 0;

    __shared__ int s_stop;
    for (int s = 0; s < a.steps; ++s) {
        // thread 0 reads the status for the whole block (a uniform exit)
        if (threadIdx.x == 0) { s_cnt = 0; s_stop = ld_status(a.ctl); }
        __syncthreads();
        if (s_stop) break;
        const int t = a.t0 + s;
        const int cur = t % a.D1;
        A *slot = ring + (size_t)cur * a.n;
        phase_update<MODE, STDP>(a, t, j0, j1, s_list, &s_cnt, [&](int j) -> V {
            A v = slot[j];
            slot[j] = 0;
            return Tr<MODE>::from_acc(v);
        });
        __syncthreads();
        const int k = s_cnt;
        if (threadIdx.x == 0) my_spikes += (unsigned long long)k;

        if constexpr (STDP) {
            if (!grid_barrier(a.ctl)) break;
            const unsigned *rrow = a.raster + (size_t)(t % a.cap) * a.words;
            const float *xo = a.trace + (size_t)((t & 1) ^ 1) * a.n;
            // rows of spiking pre-neurons: LTD for every target, LTP where the
            // target spiked too; the updated weight is the one delivered.
            for (int q = warp; q < k; q += nwarp) {
                const int i = s_list[q];
                const float xi = xo[i];
                const long long beg = a.rowptr[i], end = a.rowptr[i + 1];
                for (long long p = beg + lane; p < end; p += 32) {
                    uint2 e = a.syn[p];
                    const int post = (int)(e.x & kPostMask);
                    const int d = (int)(e.x >> kPostBits) + 1;
                    float dw = 0.0f;
                    if (spiked(rrow, post)) dw = __fmul_rn(a.a_plus, xi);
                    dw = __fsub_rn(dw, __fmul_rn(a.a_minus, xo[post]));
                    float w = clampf(__fadd_rn(__uint_as_float(e.y), dw), a.wmin, a.wmax);
                    e.y = __float_as_uint(w);
                    a.syn[p].y = e.y;
                    int sl = cur + d;
                    if (sl >= a.D1) sl -= a.D1;
                    atomicAdd(ring + (size_t)sl * a.n + post, Tr<MODE>::to_acc(e.y));
                }
                if (lane == 0) my_events += (unsigned long long)(end - beg);
            }
            // columns of spiking post-neurons whose pre-neuron did not spike: LTP
            for (int q = warp; q < k; q += nwarp) {
                const int j = s_list[q];
                const long long beg = a.colptr[j], end = a.colptr[j + 1];
                for (long long p = beg + lane; p < end; p += 32) {
                    const uint2 c = a.csc[p];
                    const int pre = (int)c.x;
                    if (spiked(rrow, pre)) continue;
                    const float dw = __fmul_rn(a.a_plus, xo[pre]);
                    const float w = ld_scattered((const float *)&a.syn[c.y] + 1);
                    const float nw = clampf(__fadd_rn(w, dw), a.wmin, a.wmax);
                    // an update that rounds back to the same bits leaves the sector clean
                    if (__float_as_uint(nw) != __float_as_uint(w)) a.syn[c.y].y = __float_as_uint(nw);
                }
            }
        } else {
            // push: each warp takes spikers; lanes stride the row, four
            // synapses per lane in flight before their atomics.
            for (int q = warp; q < k; q += nwarp) {
                const int i = s_list[q];
                const long long beg = a.rowptr[i], end = a.rowptr[i + 1];
                for (long long p0 = beg; p0 < end; p0 += 128) {
                    uint2 e[4];
                    bool ok[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long p = p0 + lane + 32 * u;
                        ok[u] = p < end;
                        if (ok[u]) e[u] = __ldg(a.syn + p);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (!ok[u]) continue;
                        const int post = (int)(e[u].x & kPostMask);
                        int sl = cur + (int)(e[u].x >> kPostBits) + 1;
                        if (sl >= a.D1) sl -= a.D1;
                        atomicAdd(ring + (size_t)sl * a.n + post, Tr<MODE>::to_acc(e[u].y));
                    }
                }
                if (lane == 0) my_events += (unsigned long long)(end - beg);
            }
        }
        if (!grid_barrier(a.ctl)) break;
    }
    // run counters: one atomic per thread that counted anything
    if (my_spikes) atomicAdd(&a.ctl->spikes, my_spikes);
    if (my_events) atomicAdd(&a.ctl->events, my_events);
}

// ---------------------------------------------------------------------------
// Sparse push, register-resident variant (no STDP).  Block = 512 threads and
// every thread owns at most one neuron, so the neuron's state, parameters,
// Poisson source and CSR row bounds live in registers for the whole launch
// (V and r are written back at the end).  The spikers of a step are compacted
// with their row bounds; an exclusive scan of the row lengths flattens the
// block's synapse work, and every thread keeps eight independent synapse
// loads in flight before issuing their fixed-point atomics.

constexpr int kRegBlock = 512;
constexpr int kRegUnroll = 8;

template <int MODE>
__global__ void __launch_bounds__(kRegBlock) sparse_reg_kernel(NetArgs a) {
    using A = typename Tr<MODE>::A;
    using V = typename Tr<MODE>::V;
    __shared__ int s_j[kRegBlock];
    __shared__ long long s_beg[kRegBlock];
    __shared__ int s_off[kRegBlock + 1];
    __shared__ int s_wsum[kRegBlock / 32];
    __shared__ int s_cnt, s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * a.chunk;
    const int j1 = min(a.n, j0 + a.chunk);
    const int j = j0 + threadIdx.x;
    const bool mine = j < j1;
    V v = 0, th = 0, lk = 0, rs = 0, amp = 0;
    int rr = 0, R = 0, len = 0;
    unsigned thr = 0;
    long long beg = 0;
    if (mine) {
        v = ((const V *)a.V)[j];
        rr = a.r[j];
        th = ((const V *)a.th)[j];
        lk = ((const V *)a.lk)[j];
        rs = ((const V *)a.rs)[j];
        R = a.R[j];
        thr = a.prate[j];
        amp = ((const V *)a.pamp)[j];
        beg = a.rowptr[j];
        len = (int)(a.rowptr[j + 1] - beg);
    }
    A *ring = (A *)a.ring;
    unsigned long long my_spikes = 0, my_events = 0;
    bool overflow = false;
    for (int s = 0; s < a.steps; ++s) {
        if (threadIdx.x == 0) { s_cnt = 0; s_stop = ld_status(a.ctl); }
        __syncthreads();
        if (s_stop) break;
        const int t = a.t0 + s;
        const int cur = t % a.D1;
        bool fire = false;
        if (mine) {
            A *slot = ring + (size_t)cur * a.n;
            const V acc = Tr<MODE>::from_acc(slot[j]);
            slot[j] = 0;
            V ext = 0;
            if (t < a.ev_nsteps) {
                int lo = a.ev_off[t], hi = a.ev_off[t + 1];
                const int end = hi;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (a.ev_neuron[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo < end && a.ev_neuron[lo] == j) ext = ((const V *)a.ev_val)[lo];
            }
            if (thr && poisson_fires(a.pkey, (unsigned)t, (unsigned)j, thr)) {
                if (MODE == SN_F32) ext = __fadd_rn(ext, amp); else ext = ext + amp;
            }
            if constexpr (MODE == SN_F32) fire = lif_update_f32(v, rr, acc, ext, th, lk, rs, R);
            else fire = lif_update_i32(v, rr, acc, ext, th, lk, rs, R, overflow);
        }
        const unsigned ball = __ballot_sync(0xffffffffu, fire);
        const int wbase = j0 + warp * 32;
        if (lane == 0 && wbase < j1) a.raster[(size_t)(t % a.cap) * a.words + (wbase >> 5)] = ball;
        if (ball) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&s_cnt, __popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (fire) {
                const int q = base + __popc(ball & ((1u << lane) - 1u));
                s_j[q] = j;
                s_beg[q] = beg;
                s_off[q] = len;
            }
        }
        __syncthreads();
        const int k = s_cnt;
        // exclusive scan of the spikers' row lengths
        const int x = threadIdx.x < k ? s_off[threadIdx.x] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < kRegBlock / 32 ? s_wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < kRegBlock / 32) s_wsum[lane] = w;
        }
        __syncthreads();
        const int total = s_wsum[kRegBlock / 32 - 1];
        if (threadIdx.x < k) s_off[threadIdx.x] = (warp ? s_wsum[warp - 1] : 0) + incl - x;
        if (threadIdx.x == 0) s_off[k] = total;
        __syncthreads();
        if (threadIdx.x == 0) { my_spikes += (unsigned long long)k; my_events += (unsigned long long)total; }
        // flattened push: item e = synapse (e - s_off[q]) of spiker q
        int q = 0;
        for (int e0 = 0; e0 < total; e0 += kRegBlock * kRegUnroll) {
            uint2 sy[kRegUnroll];
            bool ok[kRegUnroll];
#pragma unroll
            for (int u = 0; u < kRegUnroll; ++u) {
                const int e = e0 + u * kRegBlock + threadIdx.x;
                ok[u] = e < total;
                if (ok[u]) {
                    while (s_off[q + 1] <= e) ++q;
                    sy[u] = __ldg(a.syn + s_beg[q] + (e - s_off[q]));
                }
            }
#pragma unroll
            for (int u = 0; u < kRegUnroll; ++u) {
                if (!ok[u]) continue;
                const int post = (int)(sy[u].x & kPostMask);
                int sl = cur + (int)(sy[u].x >> kPostBits) + 1;
                if (sl >= a.D1) sl -= a.D1;
                atomicAdd(ring + (size_t)sl * a.n + post, Tr<MODE>::to_acc(sy[u].y));
            }
        }
        if (!grid_barrier(a.ctl)) break;
    }
    if (mine) {
        ((V *)a.V)[j] = v;
        a.r[j] = rr;
    }
    if (MODE == SN_I32 && overflow) atomicCAS(&a.ctl->status, 0, (int)SN_EOVERFLOW);
    if (my_spikes) atomicAdd(&a.ctl->spikes, my_spikes);
    if (my_events) atomicAdd(&a.ctl->events, my_events);
}

static const void *sparse_reg_fn(int dtype) {
    return dtype == SN_F32 ? (const void *)sparse_reg_kernel<SN_F32> : (const void *)sparse_reg_kernel<SN_I32>;
}

cudaError_t max_grid_sparse_reg(int *grid) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int per = 1 << 30;
    for (int dt : {(int)SN_F32, (int)SN_I32}) {
        int p = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, sparse_reg_fn(dt), kRegBlock, 0);
        if (e != cudaSuccess) return e;
        per = p < per ? p : per;
    }
    *grid = per * sms;
    return cudaSuccess;
}

// The grid barrier's arrival count starts every launch at zero.
static cudaError_t reset_barrier(Control *ctl, cudaStream_t s) {
    return cudaMemsetAsync(&ctl->bar, 0, sizeof(GridBarrier), s);
}

cudaError_t launch_sparse_reg(const NetArgs &a, int dtype, int grid, cudaStream_t s) {
    void *args[] = {(void *)&a};
    cudaError_t e = reset_barrier(a.ctl, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(sparse_reg_fn(dtype), dim3(grid), dim3(kRegBlock), args, 0, s);
}

cudaError_t launch_sparse(const NetArgs &a, int dtype, int grid, int block, cudaStream_t s) {
    void *args[] = {(void *)&a};
    if (cudaError_t e = reset_barrier(a.ctl, s)) return e;
    const size_t smem = (size_t)a.chunk * sizeof(int);
    const void *fn;
    if (dtype == SN_F32)
        fn = a.stdp ? (const void *)sparse_kernel<SN_F32, true> : (const void *)sparse_kernel<SN_F32, false>;
    else
        fn = (const void *)sparse_kernel<SN_I32, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t max_grid_sparse(int dtype, int stdp, int block, int *grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    (void)dtype;
    (void)stdp;
    // the smallest residency of all variants, shared memory for a chunk of up
    // to 1024 neurons, so that any variant's cooperative launch fits
    per = 1 << 30;
    for (const void *fn : {(const void *)sparse_kernel<SN_F32, true>, (const void *)sparse_kernel<SN_F32, false>,
                           (const void *)sparse_kernel<SN_I32, false>}) {
        int p = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, block, 1024 * sizeof(int));
        if (e != cudaSuccess) return e;
        per = p < per ? p : per;
    }
    *grid = per * sms;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Dense network: W[n][n] row-major (row = pre), one grid barrier per step.
// Block c owns the column slab [c * cw, c * cw + cw), cw = 32 * CPL, and the
// neurons with the same indices.  Step t:
//   update(t):  own neurons (state in registers, parameters in shared
//               memory), input from the block's own ring slot t; spikes ->
//               spike bits of t (double buffer), raster;
//   grid barrier;
//   gather(t):  every block walks the spikers of step t in ascending order,
//               each warp taking every eighth row, and sums W[i][own columns]
//               (vector form: gather_vec, four rows per float4 instruction);
//               the warp partials are folded in a fixed order and stored as
//               the input arriving at t + delay.  With STDP the block also
//               updates its columns of the spiking rows (LTD, and LTP where the
//               column spiked) before using them, and its spiking columns in
//               the other rows (LTP), from the traces of step t-1.
// Every write to W[:, slab] and to the slab's ring comes from the owning
// block, so no other synchronisation is needed; the result does not depend on
// thread timing.

constexpr int kDListMax = 4096;                    // spikers held in shared memory

// Spike ranks of a spike-bit row: each thread copies the contiguous words
// [w0, w0 + per) from global memory into the shared copy `bits` and counts
// their spikes; an exclusive block scan gives the rank (position in ascending
// neuron order) of the thread's first spike.  Returns the row's spike count;
// two block barriers, after which the whole shared copy is visible.
struct RankSpan {
    int w0, w1, base;
};
__device__ int block_spike_ranks(const unsigned *g_bits, unsigned *bits, int words, int *s_scan, RankSpan &sp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (words + blockDim.x - 1) / blockDim.x;
    sp.w0 = min(words, (int)threadIdx.x * per);
    sp.w1 = min(words, sp.w0 + per);
    int c = 0;
    for (int w = sp.w0; w < sp.w1; ++w) {
        const unsigned b = g_bits[w];
        bits[w] = b;
        c += __popc(b);
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < nw ? s_scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) s_scan[lane] = v;
    }
    __syncthreads();
    sp.base = (warp ? s_scan[warp - 1] : 0) + incl - c;
    return s_scan[nw - 1];
}

// The spikers of this thread's words with rank in [lo, hi) into list[rank - lo].
__device__ __forceinline__ void emit_ranks(const unsigned *bits, const RankSpan &sp, int lo, int hi, int *list) {
    int rank = sp.base;
    for (int w = sp.w0; w < sp.w1 && rank < hi; ++w) {
        unsigned b = bits[w];
        while (b) {
            const int bpos = __ffs(b) - 1;
            b &= b - 1u;
            if (rank >= lo && rank < hi) list[rank - lo] = w * 32 + bpos;
            ++rank;
        }
    }
}

// Vector gather of one list chunk (no STDP; n % 4 == 0 and W 16-byte aligned).
// The slab's 32 * CPL columns are G = 8 * CPL float4 groups.  A warp loads
// RPI = 32 / min(G, 32) rows per instruction (lane l: sub-row l / LPR, group
// l % LPR, plus group + 32 when G = 64), so one instruction moves 512 bytes.
// The warp's rows are list[warp + nwarp * i], i = 0, 1, ...; sub-row q takes
// i = q, q + RPI, ... in ascending order.  U instructions stay in flight: the
// load for row i + RPI * U is issued as row i is added (register rotation).
template <int CPL>
struct VecGeom {
    static constexpr int G = 8 * CPL;                  // float4 groups of the slab
    static constexpr int LPR = G < 32 ? G : 32;        // lanes per row
    static constexpr int RPI = 32 / LPR;               // rows per instruction
    static constexpr int F = G > 32 ? G / 32 : 1;      // float4 per lane per row
    static constexpr int U = F > 1 ? 3 : (CPL == 4 ? 7 : 8);   // instructions in flight
};

template <int CPL>
__device__ __forceinline__ void gather_vec(const float *__restrict__ W, int n, int c0, const int *list,
                                           int cnt, int warp, int lane, float4 (&acc)[VecGeom<CPL>::F]) {
    using Gm = VecGeom<CPL>;
    constexpr int nwarp = kBlock / 32, RPI = Gm::RPI, F = Gm::F, U = Gm::U;
    const int q = lane / Gm::LPR, g = lane % Gm::LPR;
    // this lane's rows: list[warp + nwarp * (q + RPI * k)], k = 0 .. nk-1
    const int rows = cnt > warp ? (cnt - warp + nwarp - 1) / nwarp : 0;
    const int nk = rows > q ? (rows - q + RPI - 1) / RPI : 0;
    const int *lp = list + warp + nwarp * q;
    constexpr int lstep = nwarp * RPI;
    const float4 *wv = (const float4 *)(W + c0) + g;     // this lane's first group, row 0
    const size_t rs4 = (size_t)(n >> 2);                 // float4 per row
    const bool cv0 = c0 + 4 * g < n, cv1 = F > 1 && c0 + 4 * (g + 32) < n;
    float4 buf[U][F];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const bool ok = u < nk;
        const float4 *p = wv + (ok ? (size_t)lp[lstep * u] * rs4 : 0);
        buf[u][0] = (ok && cv0) ? __ldg(p) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (F > 1) buf[u][F - 1] = (ok && cv1) ? __ldg(p + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int k0 = 0; k0 < nk; k0 += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u;
            float4 x[F];
#pragma unroll
            for (int f = 0; f < F; ++f) x[f] = buf[u][f];
            const int kn = k + U;
            const bool ok = kn < nk;
            const float4 *p = wv + (ok ? (size_t)lp[lstep * kn] * rs4 : 0);
            buf[u][0] = (ok && cv0) ? __ldg(p) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (F > 1) buf[u][F - 1] = (ok && cv1) ? __ldg(p + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < nk) {
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    acc[f].x = __fadd_rn(acc[f].x, x[f].x);
                    acc[f].y = __fadd_rn(acc[f].y, x[f].y);
                    acc[f].z = __fadd_rn(acc[f].z, x[f].z);
                    acc[f].w = __fadd_rn(acc[f].w, x[f].w);
                }
            }
        }
    }
}

template <int CPL, bool STDP, bool VEC>
__global__ void __launch_bounds__(kBlock, CPL <= 2 ? 4 : 3) dense_kernel(NetArgs a) {
    extern __shared__ int smem[];
    constexpr int cw = 32 * CPL;
    constexpr int nwarp = kBlock / 32;
    using Gm = VecGeom<CPL>;
    int *list = smem;                                  // [kDListMax]
    // the spike-bit row of the step, read once from global memory
    unsigned *s_bits = (unsigned *)(smem + kDListMax);  // [words]
    // [nwarp][cw], vector path [nwarp][RPI][cw]; 16-byte aligned
    float *wpart = (float *)(smem + ((a.words + kDListMax + 3) & ~3));
    __shared__ int s_scan[kBlock / 32];
    __shared__ int s_stop;
    __shared__ float s_x[STDP ? kBlock : 1];           // pre-step traces of the slab's neurons
    __shared__ float s_carry[kBlock];                  // delay 1: the fold of the last step
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n;
    const int c0 = blockIdx.x * cw;
    const int j = c0 + threadIdx.x;
    const bool mine = threadIdx.x < cw && j < n;
    float *ring = (float *)a.ring;
    // the slab's neuron parameters stay in shared memory for the launch (the
    // registers go to the gather's loads in flight); state in registers
    __shared__ float s_th[kBlock], s_lk[kBlock], s_rs[kBlock], s_amp[kBlock];
    __shared__ int s_R[kBlock];
    __shared__ unsigned s_thr[kBlock];
    float v = 0;
    int rr = 0;
    if (mine) {
        v = ((const float *)a.V)[j];
        rr = a.r[j];
        s_th[threadIdx.x] = ((const float *)a.th)[j];
        s_lk[threadIdx.x] = ((const float *)a.lk)[j];
        s_rs[threadIdx.x] = ((const float *)a.rs)[j];
        s_R[threadIdx.x] = a.R[j];
        s_thr[threadIdx.x] = a.prate[j];
        s_amp[threadIdx.x] = ((const float *)a.pamp)[j];
    }
    unsigned long long my_spikes = 0;
    // with delay 1 the input of step t + 1 is this thread's own fold of step
    // t (kept in shared memory), and the pre-step trace its own update's (in
    // a register); both are also stored for the next launch
    float x_own = 0.0f;
    // a status latched by another block is read once per step without
    // waiting for it, and acted on at the end of the step
    int st = 0;
    if (threadIdx.x == 0) s_stop = ld_status(a.ctl);
    __syncthreads();
    if (s_stop) return;

    for (int s = 0; s < a.steps; ++s) {
        if (threadIdx.x == 0) st = ld_status(a.ctl);
        const int t = a.t0 + s;
        const int cur = t % a.D1;
        // ---- update(t)
        bool fire = false;
        if (mine) {
            const float acc = (s > 0 && a.dense_delay == 1) ? s_carry[threadIdx.x] : ring[(size_t)cur * n + j];
            float ext = 0.0f;
            if (t < a.ev_nsteps) {
                int lo = a.ev_off[t], hi = a.ev_off[t + 1];
                const int end = hi;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (a.ev_neuron[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo < end && a.ev_neuron[lo] == j) ext = ((const float *)a.ev_val)[lo];
            }
            const unsigned thr = s_thr[threadIdx.x];
            if (thr && poisson_fires(a.pkey, (unsigned)t, (unsigned)j, thr)) ext = __fadd_rn(ext, s_amp[threadIdx.x]);
            fire = lif_update_f32(v, rr, acc, ext, s_th[threadIdx.x], s_lk[threadIdx.x], s_rs[threadIdx.x],
                                  s_R[threadIdx.x]);
            if constexpr (STDP) {
                const float xo = s > 0 ? x_own : a.trace[(size_t)((t + 2) % 3) * n + j];
                s_x[threadIdx.x] = xo;
                x_own = __fadd_rn(__fmul_rn(a.decay, xo), fire ? 1.0f : 0.0f);
                a.trace[(size_t)(t % 3) * n + j] = x_own;
            }
        }
        if (threadIdx.x < cw) {
            const unsigned ball = __ballot_sync(0xffffffffu, fire);
            if (lane == 0 && c0 + warp * 32 < n) {
                const int word = (c0 >> 5) + warp;
                a.spk[(size_t)(t & 1) * a.words + word] = ball;
                a.raster[(size_t)(t % a.cap) * a.words + word] = ball;
                my_spikes += (unsigned long long)__popc(ball);
            }
        }
        if (!grid_barrier(a.ctl)) break;

        // ---- gather(t): input of t + delay (and STDP of step t)
        const unsigned *row_bits = s_bits;
        RankSpan span;
        const int k = block_spike_ranks(a.spk + (size_t)(t & 1) * a.words, s_bits, a.words, s_scan, span);
        const float *xo = STDP ? a.trace + (size_t)((t + 2) % 3) * n : nullptr;   // x(t-1)
        float acc[CPL];
        bool sc[CPL];
        float xc[CPL];
        float4 vacc[Gm::F];
#pragma unroll
        for (int f = 0; f < Gm::F; ++f) vacc[f] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            acc[q] = 0.0f;
            const int col = c0 + lane + 32 * q;
            sc[q] = false;
            xc[q] = 0.0f;
            if (STDP && col < n) { sc[q] = spiked(row_bits, col); xc[q] = s_x[lane + 32 * q]; }
        }
        for (int base = 0; base < k; base += kDListMax) {
            const int cnt = min(kDListMax, k - base);
            __syncthreads();
            emit_ranks(row_bits, span, base, base + cnt, list);
            __syncthreads();
            int r = warp;
            if constexpr (VEC) {
                gather_vec<CPL>(a.W, n, c0, list, cnt, warp, lane, vacc);
                continue;
            }
            if constexpr (!STDP) {
                // RF rows per warp in flight (16 columns-per-lane loads)
                constexpr int RF = CPL >= 8 ? 2 : 16 / CPL;
                for (; r + (RF - 1) * nwarp < cnt; r += RF * nwarp) {
                    float w16[RF][CPL];
#pragma unroll
                    for (int u = 0; u < RF; ++u) {
                        const float *row = a.W + (size_t)list[r + u * nwarp] * n;
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            const int col = c0 + lane + 32 * q;
                            w16[u][q] = col < n ? __ldg(row + col) : 0.0f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RF; ++u)
#pragma unroll
                        for (int q = 0; q < CPL; ++q) acc[q] = __fadd_rn(acc[q], w16[u][q]);
                }
            }
            if constexpr (STDP) {
                // up to RS spiking rows per warp in flight: their slab weights
                // and pre traces are loaded together, then each row in turn is
                // updated, written back and added (the order of the sum); the
                // loop takes every row, so the one-row loop below has none left
                constexpr int RS = CPL >= 4 ? 2 : 8 / CPL;
                for (; r < cnt; r += RS * nwarp) {
                    float wv[RS][CPL], xr[RS];
                    int ir[RS];
#pragma unroll
                    for (int u = 0; u < RS; ++u) {
                        const bool ok = r + u * nwarp < cnt;
                        ir[u] = ok ? list[r + u * nwarp] : -1;
                        xr[u] = ok ? xo[ir[u]] : 0.0f;
                        const float *row = a.W + (size_t)(ok ? ir[u] : 0) * n;
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            const int col = c0 + lane + 32 * q;
                            wv[u][q] = (ok && col < n) ? row[col] : 0.0f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RS; ++u) {
                        if (ir[u] < 0) break;
                        float *row = a.W + (size_t)ir[u] * n;
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            const int col = c0 + lane + 32 * q;
                            if (col >= n) continue;
                            float w = wv[u][q];
                            if (col != ir[u]) {
                                float dw = sc[q] ? __fmul_rn(a.a_plus, xr[u]) : 0.0f;
                                dw = __fsub_rn(dw, __fmul_rn(a.a_minus, xc[q]));
                                w = clampf(__fadd_rn(w, dw), a.wmin, a.wmax);
                                row[col] = w;
                            }
                            acc[q] = __fadd_rn(acc[q], w);
                        }
                    }
                }
            }
            for (; r < cnt; r += nwarp) {
                const int i = list[r];
                float *row = a.W + (size_t)i * n;
                const float xi = STDP ? xo[i] : 0.0f;
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const int col = c0 + lane + 32 * q;
                    if (col >= n) continue;
                    float w = row[col];
                    if (STDP && col != i) {
                        float dw = sc[q] ? __fmul_rn(a.a_plus, xi) : 0.0f;
                        dw = __fsub_rn(dw, __fmul_rn(a.a_minus, xc[q]));
                        w = clampf(__fadd_rn(w, dw), a.wmin, a.wmax);
                        row[col] = w;
                    }
                    acc[q] = __fadd_rn(acc[q], w);
                }
            }
            if constexpr (STDP) {
                // LTP in the spiking columns of this list chunk, rows that did not
                // spike; the rows are shared out over every warp of the grid (no
                // block writes a row the gather touches: those rows spiked)
                // Each element is one read-modify-write of its own weight, so the
                // reads of kLtpRows rows are issued together before any write.
                constexpr int kLtpRows = 4;
                const int gwarps = gridDim.x * nwarp;
                for (int i0 = blockIdx.x * nwarp + warp; i0 < n; i0 += kLtpRows * gwarps) {
                    for (int q0 = 0; q0 < cnt; q0 += 64) {
                        float val[kLtpRows][2], dw[kLtpRows];
                        bool act[kLtpRows];
#pragma unroll
                        for (int u = 0; u < kLtpRows; ++u) {
                            const int i = i0 + u * gwarps;
                            act[u] = i < n && !spiked(row_bits, i);
                            dw[u] = act[u] ? __fmul_rn(a.a_plus, xo[i]) : 0.0f;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int q = q0 + lane + 32 * h;
                                val[u][h] = (act[u] && q < cnt) ? ld_scattered(a.W + (size_t)i * n + list[q]) : 0.0f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kLtpRows; ++u) {
                            const int i = i0 + u * gwarps;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int q = q0 + lane + 32 * h;
                                if (act[u] && q < cnt) {
                                    // a weight whose update rounds back to itself (an old
                                    // pre-neuron's trace has decayed below its half ulp) is
                                    // not written: same bits, no dirty sector
                                    const float nv = clampf(__fadd_rn(val[u][h], dw[u]), a.wmin, a.wmax);
                                    if (__float_as_uint(nv) != __float_as_uint(val[u][h]))
                                        a.W[(size_t)i * n + list[q]] = nv;
                                }
                            }
                        }
                    }
                }
            }
        }
        // fold the warp partials in warp order (vector path: warp, then
        // sub-row); the input of t + delay
        if constexpr (VEC) {
            const int q = lane / Gm::LPR, g = lane % Gm::LPR;
#pragma unroll
            for (int f = 0; f < Gm::F; ++f)
                *(float4 *)&wpart[(warp * Gm::RPI + q) * cw + 4 * (g + 32 * f)] = vacc[f];
        } else {
#pragma unroll
            for (int q = 0; q < CPL; ++q) wpart[warp * cw + lane + 32 * q] = acc[q];
        }
        __syncthreads();
        if (mine) {
            float sum = 0.0f;
            constexpr int parts = VEC ? nwarp * Gm::RPI : nwarp;
#pragma unroll
            for (int w = 0; w < parts; ++w) sum = __fadd_rn(sum, wpart[w * cw + threadIdx.x]);
            ring[(size_t)((t + a.dense_delay) % a.D1) * n + j] = sum;
            s_carry[threadIdx.x] = sum;
        }
        if (threadIdx.x == 0) s_stop = st;
        __syncthreads();
        if (s_stop) break;
    }
    if (mine) {
        ((float *)a.V)[j] = v;
        a.r[j] = rr;
    }
    if (my_spikes) {
        atomicAdd(&a.ctl->spikes, my_spikes);
        atomicAdd(&a.ctl->events, my_spikes * (unsigned long long)n);
    }
}

// Failure-detection self-test: block 0 never arrives at the barrier, so the
// count stays one short of its target and every other block's wait runs out
// after kBarrierTimeoutNs, latching SN_ETIMEOUT (no fault, no trap).
__global__ void barrier_selftest_kernel(Control *ctl) {
    if (blockIdx.x == 0) return;
    grid_barrier(ctl);
}

cudaError_t launch_barrier_selftest(Control *ctl, int blocks, cudaStream_t s) {
    barrier_selftest_kernel<<<blocks, 32, 0, s>>>(ctl);
    return cudaGetLastError();
}

// Shared memory of a dense block: list chunk, the step's spike-bit row, warp
// partials (the vector path keeps RPI partials per warp: at most 4 * 32 * 4 B
// per warp for any CPL, as much as CPL = 4's scalar partials).
static size_t dense_smem(int words, int cpl) {
    const size_t part = (size_t)(kBlock / 32) * 32 * (cpl > 4 ? cpl : 4) * sizeof(float);
    return (size_t)((words + kDListMax + 3) & ~3) * sizeof(int) + part;
}

// vec: the vector gather (no STDP, n % 4 == 0, W 16-byte aligned)
static const void *dense_fn(int cpl, bool stdp, bool vec) {
    if (vec && !stdp) {
        switch (cpl) {
            case 1: return (const void *)dense_kernel<1, false, true>;
            case 2: return (const void *)dense_kernel<2, false, true>;
            case 4: return (const void *)dense_kernel<4, false, true>;
            default: return (const void *)dense_kernel<8, false, true>;
        }
    }
    switch (cpl) {
        case 1: return stdp ? (const void *)dense_kernel<1, true, false> : (const void *)dense_kernel<1, false, false>;
        case 2: return stdp ? (const void *)dense_kernel<2, true, false> : (const void *)dense_kernel<2, false, false>;
        case 4: return stdp ? (const void *)dense_kernel<4, true, false> : (const void *)dense_kernel<4, false, false>;
        default: return stdp ? (const void *)dense_kernel<8, true, false> : (const void *)dense_kernel<8, false, false>;
    }
}

cudaError_t launch_dense(const NetArgs &a, int grid, int block, cudaStream_t s) {
    (void)block;
    void *args[] = {(void *)&a};
    const size_t smem = dense_smem(a.words, a.chunk / 32);
    const bool vec = a.n % 4 == 0 && ((uintptr_t)a.W & 15u) == 0;
    const void *fn = dense_fn(a.chunk / 32, a.stdp != 0, vec);
    cudaError_t e = reset_barrier(a.ctl, s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, smem, s);
}

// Executor plan of a dense network: the smallest columns-per-lane (1, 2, 4,
// 8) whose grid of ceil(n / (32 * cpl)) blocks is co-resident; a network of
// at most 128 neurons runs as one block (no grid barrier).  force_cpl (1, 2,
// 4 or 8; 0 = choose) takes that slab width if its grid is co-resident.
cudaError_t plan_dense(int n, int *grid, int *chunk, int force_cpl) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int words = (n + 31) / 32;
    for (int cpl : {1, 2, 4, 8}) {
        if (force_cpl ? cpl != force_cpl : (n <= 128 && 32 * cpl < n)) continue;
        const size_t smem = dense_smem(words, cpl);
        int per = 1 << 30;
        for (int v = 0; v < 3; ++v) {
            const void *fn = dense_fn(cpl, v == 1, v == 2);
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int p = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, kBlock, smem);
            if (e != cudaSuccess) return e;
            per = p < per ? p : per;
        }
        const int g = (n + 32 * cpl - 1) / (32 * cpl);
        if (per > 0 && g <= per * sms) {
            *grid = g;
            *chunk = 32 * cpl;
            return cudaSuccess;
        }
    }
    *grid = 0;
    *chunk = 0;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Weights of a sparse network back in input order: out[k] = weight of input
// synapse k, whose CSR position is perm_inv[k].
__global__ void gather_weights_kernel(const uint2 *syn, const long long *perm_inv, long long m,
                                      float *out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = __uint_as_float(syn[perm_inv[k]].y);
}

// The inverse: weight of input synapse k into its CSR position.
__global__ void scatter_weights_kernel(uint2 *syn, const long long *perm_inv, long long m, const float *w) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x)
        syn[perm_inv[k]].y = __float_as_uint(w[k]);
}

cudaError_t launch_scatter_weights(uint2 *syn, const long long *perm_inv, long long m, const float *w,
                                   cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    scatter_weights_kernel<<<(int)blocks, 256, 0, s>>>(syn, perm_inv, m, w);
    return cudaGetLastError();
}

cudaError_t launch_gather_weights(const uint2 *syn, const long long *perm_inv, long long m,
                                  float *out, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    gather_weights_kernel<<<(int)blocks, 256, 0, s>>>(syn, perm_inv, m, out);
    return cudaGetLastError();
}

}  // namespace sn
