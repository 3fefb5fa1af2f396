// Pull propagation for sparse networks (Section 2.1, second step of a
// timestep: the input of neuron j is the sum over its incoming synapses of
// w * s_i(t - d); Section 2.2: a spike reaches the post-neuron d steps later).
//
// Every block keeps the spike bits of recent steps in a shared-memory window
// of hL rows of Wp = roundup(ceil(n/32), 4) words: the row of step tau sits
// at position tau - base.  Each thread owns one neuron and holds its state in
// registers; thread p of a block walks the incoming synapses of the block's
// neuron pin_perm[p] (the host orders each block's neurons by list length, so
// that a warp's 32 lists are about equally long: a warp runs to its longest)
// in descending delay, then ascending pre and input index (the oldest spikes
// first), testing the bit of pre at step t - d and adding the weight, and
// hands the sum to that neuron's thread through shared memory.  That bit lies
// y = (D - d) * Wp * 32 + pre bits after the row of step t - D, and y never
// decreases along a list.  The lists of a slice of 32 thread positions (one
// warp) are stored in one of two forms (built on the host):
//  - plain, 8 bytes a synapse: x = (y / 32) << 7 | y % 32 and the weight bits;
//    entry q of lane l sits in pair q / 2 of the slice, so that each 16-byte
//    load of a warp reads 512 contiguous bytes; a test is one shift, one
//    shared load and one funnel shift;
//  - coded, 6 bytes a synapse: groups of 8 entries, each group three 16-byte
//    loads of the lane (weights 0-3, weights 4-7, the eight 16-bit steps of y),
//    y running from the region's first offset; a step above 65535 is split
//    over filler entries of weight 0.
// Unused entries and fillers add +0 (an exact no-op: the sum starts at +0 and
// is never -0), at offsets inside the window.  In
// SN_F32 mode the sum is a float accumulation in that order, the FP32
// mirror's order, so the state does not depend on thread timing and matches
// the mirror bit for bit.
//
// One grid barrier per step, split: a block arrives once its spike words of
// step t are in the global history, then (while the other blocks finish)
// compacts its window when the next row would fall off its end and sums the
// synapses of delay >= 2 of step t + 1, which read rows up to t - 1 only; after
// the wait it copies row t into the window and adds the synapses of delay 1.
// The synapses of delay >= 2 and of delay 1 sit in two regions of the store,
// so that both loops read whole 512-byte runs per warp.  The global history
// (row of step tau in slot tau % D) holds, between runs, every spike of the
// last D steps whose deliveries are still due;
// pull_flush_kernel turns them into pending ring input when the context
// switches to push propagation.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sn_device.cuh"

namespace sn {
namespace {

constexpr int kPullUnroll = 4;      // 16-byte loads (two synapses each) per half of the double buffer
constexpr int kPullMaxBlock = 1024;

template <int MODE> struct PullAcc;
template <> struct PullAcc<SN_F32> {
    using T = float;
    static __device__ __forceinline__ T add(T acc, unsigned wbits) { return __fadd_rn(acc, __uint_as_float(wbits)); }
};
template <> struct PullAcc<SN_I32> {
    using T = long long;            // exact: int32 weights, at most 2^32 synapses
    static __device__ __forceinline__ T add(T acc, unsigned wbits) { return acc + (long long)(int)wbits; }
};

// One synapse: the bit of its pre-neuron at step t - d, from the window whose
// first row (step t - D) starts at byte `row0` of shared memory.
template <int MODE>
__device__ __forceinline__ void pull_one(typename PullAcc<MODE>::T &acc, unsigned x, unsigned wbits,
                                         const unsigned char *win, unsigned row0) {
    const unsigned word = *(const unsigned *)(win + row0 + (x >> 5));
    if (__funnelshift_r(word, word, x) & 1u) acc = PullAcc<MODE>::add(acc, wbits);
}

template <int MODE>
__device__ __forceinline__ void pull_batch(typename PullAcc<MODE>::T &acc, const uint4 (&e)[kPullUnroll],
                                           const unsigned char *win, unsigned row0) {
#pragma unroll
    for (int u = 0; u < kPullUnroll; ++u) {
        pull_one<MODE>(acc, e[u].x, e[u].y, win, row0);
        pull_one<MODE>(acc, e[u].z, e[u].w, win, row0);
    }
}

// The pairs u < valid of a unit only (valid is the same for the whole warp);
// for a region's last, partly used unit.
template <int MODE>
__device__ __forceinline__ void pull_batch_part(typename PullAcc<MODE>::T &acc, const uint4 (&e)[kPullUnroll],
                                                const unsigned char *win, unsigned row0, int valid) {
#pragma unroll
    for (int u = 0; u < kPullUnroll; ++u) {
        if (u < valid) {
            pull_one<MODE>(acc, e[u].x, e[u].y, win, row0);
            pull_one<MODE>(acc, e[u].z, e[u].w, win, row0);
        }
    }
}

__device__ __forceinline__ void pull_load(uint4 (&e)[kPullUnroll], const uint4 *ent, int p0, int np) {
#pragma unroll
    for (int u = 0; u < kPullUnroll; ++u)
        e[u] = p0 + u < np ? __ldg(ent + (size_t)(p0 + u) * 32) : make_uint4(0u, 0u, 0u, 0u);
}


// Coded store: a group of 8 synapses is three uint4s of a lane (weights 0-3,
// weights 4-7, eight 16-bit offset steps), 96 uint4s apart per group in a
// slice; y is the synapse's bit offset from the start of the window.
constexpr int kCodedBuf = 3;

__device__ __forceinline__ void coded_load(uint4 (&e)[kCodedBuf], const uint4 *ent, int g, int ng) {
    if (g < ng) {
        const uint4 *p = ent + (size_t)g * 96;
        e[0] = __ldg(p);
        e[1] = __ldg(p + 32);
        e[2] = __ldg(p + 64);
    } else {
        e[0] = e[1] = e[2] = make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int MODE>
__device__ __forceinline__ void coded_one(typename PullAcc<MODE>::T &acc, unsigned &y, unsigned step,
                                          unsigned wbits, const unsigned char *win) {
    y += step;
    const unsigned word = *(const unsigned *)(win + ((y >> 3) & ~3u));
    if (__funnelshift_r(word, word, y) & 1u) acc = PullAcc<MODE>::add(acc, wbits);
}

template <int MODE>
__device__ __forceinline__ void coded_batch(typename PullAcc<MODE>::T &acc, unsigned &y,
                                            const uint4 (&e)[kCodedBuf], const unsigned char *win) {
    coded_one<MODE>(acc, y, e[2].x & 0xffffu, e[0].x, win);
    coded_one<MODE>(acc, y, e[2].x >> 16, e[0].y, win);
    coded_one<MODE>(acc, y, e[2].y & 0xffffu, e[0].z, win);
    coded_one<MODE>(acc, y, e[2].y >> 16, e[0].w, win);
    coded_one<MODE>(acc, y, e[2].z & 0xffffu, e[1].x, win);
    coded_one<MODE>(acc, y, e[2].z >> 16, e[1].y, win);
    coded_one<MODE>(acc, y, e[2].w & 0xffffu, e[1].z, win);
    coded_one<MODE>(acc, y, e[2].w >> 16, e[1].w, win);
}

// The synapses [0, np) of one region of the plain form (np pairs per lane,
// npmax the warp's largest) added to acc; e0 holds the region's first
// kPullUnroll pairs on entry and nothing useful on exit.
template <int MODE>
__device__ __forceinline__ void pull_region(typename PullAcc<MODE>::T &acc, uint4 (&e0)[kPullUnroll],
                                            uint4 (&e1)[kPullUnroll], const uint4 *ent, int np, int npmax,
                                            const unsigned char *win, unsigned row0) {
    constexpr int P = kPullUnroll;
    int p0 = 0;
    for (; p0 + 2 * P <= npmax; p0 += 2 * P) {
        pull_load(e1, ent, p0 + P, np);
        pull_batch<MODE>(acc, e0, win, row0);
        pull_load(e0, ent, p0 + 2 * P, np);
        pull_batch<MODE>(acc, e1, win, row0);
    }
    // the last pairs, fewer than 2P: only those before the warp's longest
    // list's end are tested
    const int rem = npmax - p0;
    if (rem > P) {
        pull_load(e1, ent, p0 + P, np);
        pull_batch<MODE>(acc, e0, win, row0);
        pull_batch_part<MODE>(acc, e1, win, row0, rem - P);
    } else if (rem > 0) {
        pull_batch_part<MODE>(acc, e0, win, row0, rem);
    }
}

// The same for the coded form: ng groups (the warp's largest ngmax), the
// first entry at bit y0 after byte row0 of the window.
template <int MODE>
__device__ __forceinline__ void coded_region(typename PullAcc<MODE>::T &acc, uint4 (&e0)[kCodedBuf],
                                             uint4 (&e1)[kCodedBuf], const uint4 *ent, int ng, int ngmax,
                                             const unsigned char *win, unsigned row0, unsigned y0) {
    unsigned y = row0 * 8u + y0;
    for (int g0 = 0; g0 < ngmax; g0 += 2) {
        coded_load(e1, ent, g0 + 1, ng);
        coded_batch<MODE>(acc, y, e0, win);
        coded_load(e0, ent, g0 + 2, ng);
        coded_batch<MODE>(acc, y, e1, win);
    }
}

// The two forms behind one interface (overloads on the buffer size): the
// load of a region's first unit (four pairs or a group of 8), and the
// region's sum, one unit's loads ahead of their use.
__device__ __forceinline__ void region_start(uint4 (&e)[kPullUnroll], const uint4 *ent, int np) {
    pull_load(e, ent, 0, np);
}
__device__ __forceinline__ void region_start(uint4 (&e)[kCodedBuf], const uint4 *ent, int ng) {
    coded_load(e, ent, 0, ng);
}
template <int MODE>
__device__ __forceinline__ void region_sum(typename PullAcc<MODE>::T &acc, uint4 (&e0)[kPullUnroll],
                                           uint4 (&e1)[kPullUnroll], const uint4 *ent, int np, int npmax,
                                           const unsigned char *win, unsigned row0, unsigned) {
    pull_region<MODE>(acc, e0, e1, ent, np, npmax, win, row0);
}
template <int MODE>
__device__ __forceinline__ void region_sum(typename PullAcc<MODE>::T &acc, uint4 (&e0)[kCodedBuf],
                                           uint4 (&e1)[kCodedBuf], const uint4 *ent, int ng, int ngmax,
                                           const unsigned char *win, unsigned row0, unsigned y0) {
    coded_region<MODE>(acc, e0, e1, ent, ng, ngmax, win, row0, y0);
}

template <int MODE, bool CODED>
__global__ void __launch_bounds__(kPullMaxBlock, 1) sparse_pull_kernel(NetArgs a) {
    using V = typename Tr<MODE>::V;
    using Acc = typename PullAcc<MODE>::T;
    extern __shared__ uint4 s_win4[];                 // [hL][Wp] words
    unsigned *s_win = (unsigned *)s_win4;
    const unsigned char *win = (const unsigned char *)s_win4;
    __shared__ int s_ok, s_stop;
    const int D = a.hD, W = a.words, Wp = (a.words + 3) & ~3, L = a.hL;
    const int lane = threadIdx.x & 31;
    int base = a.t0 - D;                              // step of window row 0
    for (int i = threadIdx.x; i < D * Wp; i += blockDim.x) {
        const int tau = base + i / Wp, w = i % Wp;
        s_win[i] = (tau >= 0 && w < W) ? __ldcg(a.hist + (size_t)(tau % D) * W + w) : 0u;
    }

    const int j = a.j_first + blockIdx.x * a.chunk + threadIdx.x;
    const bool mine = j < a.j_end;
    // this thread sums the lists of neuron pj (the store orders each block's
    // neurons by list length) and hands the sum to pj's own thread through
    // s_acc, which follows the window in shared memory
    const int bfirst = a.j_first + blockIdx.x * a.chunk;
    const int pj = mine ? a.pin_perm[j] : j;
    Acc *s_acc = (Acc *)(s_win + (size_t)L * Wp);
    const int wbase = j - lane;                       // first neuron of this warp's slice
    V v = 0, th = 0, lk = 0, rs = 0, amp = 0;
    int rr = 0, R = 0, npA = 0, npB = 0;
    unsigned thr = 0, yA = 0, yB = 0;
    unsigned long long outdeg = 0;
    const uint4 *ent = a.pin;
    if (mine) {
        v = ((const V *)a.V)[j];
        rr = a.r[j];
        th = ((const V *)a.th)[j];
        lk = ((const V *)a.lk)[j];
        rs = ((const V *)a.rs)[j];
        R = a.R[j];
        thr = a.prate[j];
        amp = ((const V *)a.pamp)[j];
        // units of the store per region: pairs (plain) or groups of 8 (coded)
        npA = CODED ? (a.pin_len[j] + 7) >> 3 : (a.pin_len[j] + 1) >> 1;
        npB = CODED ? (a.pin_len1[j] + 7) >> 3 : (a.pin_len1[j] + 1) >> 1;
        if (CODED) {
            yA = a.pin_y0[j];
            yB = a.pin_y0[(size_t)a.n + j];
        }
        outdeg = (unsigned long long)(a.rowptr[j + 1] - a.rowptr[j]);
        ent = a.pin + a.pin_off[j >> 5] + lane;
    }
    // units of the warp's longest list in each region; the delay-1 region
    // starts after the slice's delay->=2 region
    const int npAmax = __reduce_max_sync(0xffffffffu, npA);
    const int npBmax = __reduce_max_sync(0xffffffffu, npB);
    const uint4 *entB = ent + (size_t)npAmax * (CODED ? 96 : 32);
    using RA = typename Tr<MODE>::A;
    RA *ring = (RA *)a.ring;
    unsigned long long my_spikes = 0, my_events = 0;
    bool overflow = false;
    // synapse loads run one half (four pairs or a group of 8) ahead of their use
    uint4 ea[CODED ? kCodedBuf : kPullUnroll], eb[CODED ? kCodedBuf : kPullUnroll];
    region_start(ea, ent, npA);
    __syncthreads();
    // the delay >= 2 part of the first step: every row it reads is in the window
    Acc acc = 0;
    if (a.steps > 0) {
        region_sum<MODE>(acc, ea, eb, ent, npA, npAmax, win, (unsigned)((a.t0 - base - D) * Wp) * 4u, yA);
        region_start(ea, entB, npB);
    }
    for (int s = 0; s < a.steps; ++s) {
        const int t = a.t0 + s;
        const unsigned row0 = (unsigned)((t - base - D) * Wp) * 4u;
        bool fire = false;
        // the delay-1 part: row t - 1 is in the window
        region_sum<MODE>(acc, ea, eb, entB, npB, npBmax, win, row0, yB);
        if (mine) s_acc[pj - bfirst] = acc;
        __syncthreads();
        const Acc sum = mine ? s_acc[threadIdx.x] : Acc(0);
        if (mine) {
            // input still pending in the ring from an earlier push run
            V ring_in = 0;
            if (t < a.ring_until) {
                RA *slot = ring + (size_t)(t % a.D1) * a.n + j;
                ring_in = Tr<MODE>::from_acc(*slot);
                *slot = 0;
            }
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
            if constexpr (MODE == SN_F32) {
                const float in = t < a.ring_until ? __fadd_rn(sum, ring_in) : sum;
                fire = lif_update_f32(v, rr, in, ext, th, lk, rs, R);
            } else {
                // the integrated state is checked against int32 before the threshold
                const long long in = sum + (long long)ring_in;
                long long u;
                if (v > rs) { u = (long long)v - lk; u = u > rs ? u : rs; }
                else if (v < rs) { u = (long long)v + lk; u = u < rs ? u : rs; }
                else u = rs;
                u += in;
                u += ext;
                if (u > 2147483647ll || u < -2147483648ll) overflow = true;
                fire = (u > th) && (rr == 0);
                if (fire) { u = rs; rr = R; }
                else if (rr > 0) rr -= 1;
                v = (int)u;
            }
        }
        const int tD = t % D;
        const unsigned ball = __ballot_sync(0xffffffffu, fire);
        if (lane == 0 && wbase < a.j_end) {
            a.hist[(size_t)tD * W + (wbase >> 5)] = ball;
            a.raster[(size_t)(t % a.cap) * W + (wbase >> 5)] = ball;
        }
        if (fire) { my_spikes += 1; my_events += outdeg; }
        if (overflow) atomicCAS(&a.ctl->status, 0, (int)SN_EOVERFLOW);

        // grid barrier, split: arrive, do this block's independent work, wait
        __syncthreads();                              // every warp's words of step t are stored
        unsigned gen = 0;
        if (threadIdx.x == 0 && gridDim.x > 1) gen = bar_arrive_k(a.ctl, (unsigned)s);
        // a single block reads the status word now, so that the read overlaps
        // the work below (a grid reads it after the barrier)
        int stop_early = 0;
        if (threadIdx.x == 0 && gridDim.x == 1) stop_early = ld_status(a.ctl);
        // the first synapses of step t + 1 (the store is static)
        region_start(ea, ent, npA);
        int pos = t - base;                           // window position of row t
        if (pos >= L) {
            // rows t-D+1 .. t-1 move down by sh = pos - D + 1 rows to positions
            // 0 .. D-2, in chunks of at most sh rows' words: a chunk's source and
            // destination do not overlap, and the barrier between a chunk's reads
            // and writes orders them against the neighbouring chunks
            const int sh = pos - D + 1;
            const int total4 = (D - 1) * Wp / 4, shw4 = sh * Wp / 4;
            const int per = min((int)blockDim.x, shw4);
            for (int c0 = 0; c0 < total4; c0 += per) {
                const int k = c0 + (int)threadIdx.x;
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                const bool act = threadIdx.x < per && k < total4;
                if (act) val = s_win4[k + shw4];
                __syncthreads();
                if (act) s_win4[k] = val;
            }
            base = t - D + 1;
            pos = D - 1;
        }
        // a single block owns every word of row t: it puts its own words into
        // the window now, and its store keeps the delay-1 synapses at the end of
        // the first region, so the sum below is the whole step's
        if (gridDim.x == 1) {
            if (lane == 0 && wbase < a.j_end) s_win[(size_t)pos * Wp + (wbase >> 5)] = ball;
            __syncthreads();
        }
        // the delay >= 2 part of step t + 1 (rows t + 1 - d <= t - 1, all in the
        // window) while the other blocks arrive; then the first delay-1 loads
        acc = 0;
        if (s + 1 < a.steps) {
            region_sum<MODE>(acc, ea, eb, ent, npA, npAmax, win, (unsigned)((t + 1 - base - D) * Wp) * 4u, yA);
            region_start(ea, entB, npB);
        }
        if (threadIdx.x == 0) s_ok = gridDim.x > 1 ? bar_wait(a.ctl, gen) : 1;
        __syncthreads();
        if (!s_ok) break;
        // row t enters the window (a single block has put it in above); the
        // status word is read while the row's loads are in flight
        int st = stop_early;
        if (gridDim.x > 1) {
            if (threadIdx.x == 0) st = ld_status(a.ctl);
            for (int i = threadIdx.x; i < W; i += blockDim.x)
                s_win[(size_t)pos * Wp + i] = __ldcg(a.hist + (size_t)tD * W + i);
        }
        if (threadIdx.x == 0) s_stop = st;
        __syncthreads();
        if (s_stop) break;
    }
    if (mine) {
        ((V *)a.V)[j] = v;
        a.r[j] = rr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_spikes += __shfl_down_sync(0xffffffffu, my_spikes, o);
        my_events += __shfl_down_sync(0xffffffffu, my_events, o);
    }
    if (lane == 0 && my_spikes) {
        atomicAdd(&a.ctl->spikes, my_spikes);
        atomicAdd(&a.ctl->events, my_events);
    }
}

// Spikes of steps t0 - D .. t0 - 1 held in the history go into the ring for
// their arrival steps >= t0 (earlier arrivals were delivered by the pull
// kernel), so that push propagation continues the run exactly.
template <int MODE>
__global__ void pull_flush_kernel(NetArgs a, int t0) {
    using RA = typename Tr<MODE>::A;
    RA *ring = (RA *)a.ring;
    const int D = a.hD, W = a.words;
    const long long total = (long long)D * W;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int tau = t0 - (int)(q / W) - 1;
        const int w = (int)(q % W);
        if (tau < 0) continue;
        unsigned bits = a.hist[(size_t)(tau % D) * W + w];
        while (bits) {
            const int i = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            if (i >= a.n) break;
            for (long long p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) {
                const uint2 sy = a.syn[p];
                const int arrive = tau + (int)(sy.x >> kPostBits) + 1;
                if (arrive < t0) continue;
                const int post = (int)(sy.x & kPostMask);
                atomicAdd(ring + (size_t)(arrive % a.D1) * a.n + post, Tr<MODE>::to_acc(sy.y));
            }
        }
    }
}

// Spike words of the other shards of a network, rows of steps t0 .. t0 + rows - 1
// (whole-network rows of `words` words), into the history and the raster;
// the words [w0, w1) are this shard's own and are left as its kernel wrote them.
__global__ void shard_put_kernel(unsigned *hist, unsigned *raster, int D, int cap, int words, int w0, int w1,
                                 long long t0, int rows, const unsigned *src) {
    const long long total = (long long)rows * words;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(q / words), w = (int)(q % words);
        if (w >= w0 && w < w1) continue;
        const long long tau = t0 + row;
        const unsigned bits = src[q];
        hist[(size_t)(tau % D) * words + w] = bits;
        raster[(size_t)(tau % cap) * words + w] = bits;
    }
}

const void *pull_fn(int dtype, bool coded) {
    if (coded)
        return dtype == SN_F32 ? (const void *)sparse_pull_kernel<SN_F32, true>
                               : (const void *)sparse_pull_kernel<SN_I32, true>;
    return dtype == SN_F32 ? (const void *)sparse_pull_kernel<SN_F32, false>
                           : (const void *)sparse_pull_kernel<SN_I32, false>;
}

}  // namespace

// own_slices >= 0: a shard simulating that many 32-neuron slices of the
// network (its window still holds every neuron's spike bits).
cudaError_t plan_pull(int n, int D, long long m, int *grid, int *chunk, int *rows, size_t *smem, int own_slices) {
    *grid = 0;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    const long long words = (n + 31) / 32, wp = (words + 3) & ~3ll;
    // one neuron per thread, at most one block per SM; a window of at least
    // D rows must fit a block's shared memory next to the few static words
    // slices per block: spread over the SMs; a small network (at most 1024
    // neurons and 64 Ki synapses) runs as one block, without a grid barrier
    const long long sl = own_slices >= 0 ? own_slices : words;
    const long long per = (sl * 32 <= kPullMaxBlock && m <= 65536) ? sl : (sl + sms - 1) / sms;
    if (per * 32 > kPullMaxBlock) return cudaSuccess;
    // the window rows, and after them one 8-byte sum per thread
    const long long L = std::min<long long>((optin - 64 - per * 32 * 8) / (wp * 4), 1 << 14);
    if (L < D) return cudaSuccess;
    const long long bytes = L * wp * 4 + per * 32 * 8;
    const int block = (int)(per * 32);
    for (const void *fn : {pull_fn(SN_F32, false), pull_fn(SN_I32, false), pull_fn(SN_F32, true),
                           pull_fn(SN_I32, true)}) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        int p = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, block, (size_t)bytes);
        if (e != cudaSuccess) return e;
        if (p < 1) return cudaSuccess;
    }
    *chunk = (int)(per * 32);
    *grid = (int)((sl + per - 1) / per);
    *rows = (int)L;
    *smem = (size_t)bytes;
    return cudaSuccess;
}

cudaError_t launch_sparse_pull(const NetArgs &a, int dtype, bool coded, int grid, size_t smem, cudaStream_t s) {
    void *args[] = {(void *)&a};
    const void *fn = pull_fn(dtype, coded);
    // the grid barrier's arrival count starts every launch at zero
    cudaError_t e = cudaMemsetAsync(&a.ctl->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(a.chunk), args, smem, s);
}

cudaError_t launch_shard_put(unsigned *hist, unsigned *raster, int D, int cap, int words, int w0, int w1,
                             long long t0, int rows, const unsigned *src, cudaStream_t s) {
    const long long total = (long long)rows * words;
    if (total == 0) return cudaSuccess;
    const int block = 256;
    const int grid = (int)std::min<long long>((total + block - 1) / block, 2048);
    shard_put_kernel<<<grid, block, 0, s>>>(hist, raster, D, cap, words, w0, w1, t0, rows, src);
    return cudaGetLastError();
}

cudaError_t launch_pull_flush(const NetArgs &a, int dtype, int t0, cudaStream_t s) {
    const long long total = (long long)a.hD * a.words;
    const int block = 256;
    const int grid = (int)std::min<long long>((total + block - 1) / block, 4096);
    if (dtype == SN_F32) pull_flush_kernel<SN_F32><<<grid, block, 0, s>>>(a, t0);
    else pull_flush_kernel<SN_I32><<<grid, block, 0, s>>>(a, t0);
    return cudaGetLastError();
}

}  // namespace sn
