// Batched simulation: thousands of independent networks of uneven size and
// heterogeneous parameters in one persistent launch.
//
// Each network runs all requested timesteps on one executor: a whole block
// for networks larger than the warp threshold, a single warp for the small
// ones (no block-wide barrier then, eight networks per block at a time).
// Blocks take networks from two atomic work queues, largest first, so the
// long networks start early and the short ones fill the tail.  The
// timestep is the same as in the single-network kernels (Section 2.1 order,
// strict threshold, clamped constant leak; delays through a ring of D+1
// pending-input slots with fixed-point accumulation).  A network's ring is
// copied into shared memory while it runs when it fits the block's arena.

#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_device.cuh"
#include "sn_internal.h"

namespace sn {

constexpr int kWarps = kBatchBlock / 32;
constexpr int kListInts = kBatchMaxN;          // spiker list arena (ints) per block

template <int MODE>
struct BatchNet {
    using A = typename Tr<MODE>::A;
    using V = typename Tr<MODE>::V;
    int b, off, n, woff;
    unsigned long long key;
};

// Update of neuron j (local) of network nb at step t, in two halves so that a
// thread can issue the loads of several neurons before it uses any of them:
// batch_load reads the pending input, state and parameters; batch_finish
// clears the pending-input slot, adds the external input and applies the LIF
// rule (Section 2.1 order), storing the state.  Returns the spike.
template <int MODE>
struct NeuronIn {
    typename Tr<MODE>::A raw;
    typename Tr<MODE>::V v, th, lk, rs;
    int rr, R;
};

template <int MODE>
__device__ __forceinline__ void batch_load(const BatchArgs &a, const BatchNet<MODE> &nb, int j,
                                           const typename Tr<MODE>::A *slot, bool global_ring, NeuronIn<MODE> &in) {
    using V = typename Tr<MODE>::V;
    const int g = nb.off + j;
    in.raw = global_ring ? __ldcg(slot + j) : slot[j];
    in.v = ((const V *)a.V)[g];
    in.rr = a.r[g];
    in.th = __ldg((const V *)a.th + g);
    in.lk = __ldg((const V *)a.lk + g);
    in.rs = __ldg((const V *)a.rs + g);
    in.R = __ldg(a.R + g);
}

template <int MODE>
__device__ __forceinline__ bool batch_finish(const BatchArgs &a, const BatchNet<MODE> &nb, int t, int j,
                                             typename Tr<MODE>::A *slot, NeuronIn<MODE> &in, bool &overflow) {
    using V = typename Tr<MODE>::V;
    const int g = nb.off + j;
    slot[j] = 0;
    const V acc = Tr<MODE>::from_acc(in.raw);
    const V ext = external_input_at<MODE>(a.ev_off, a.ev_nsteps, a.ev_neuron, a.ev_val, a.prate, a.pamp,
                                          nb.key, t, g, j);
    bool fire;
    if constexpr (MODE == SN_F32)
        fire = lif_update_f32(in.v, in.rr, acc, ext, in.th, in.lk, in.rs, in.R);
    else
        fire = lif_update_i32(in.v, in.rr, acc, ext, in.th, in.lk, in.rs, in.R, overflow);
    ((V *)a.V)[g] = in.v;
    a.r[g] = in.rr;
    return fire;
}

// Neurons whose loads one thread issues together in the update phase.
constexpr int kUpdAhead = 8;

// Synapses of a row whose loads a lane issues together before their adds.
constexpr int kPushAhead = 8;

// Push of spiker i (local) of network nb: lanes stride the CSR row, each
// lane loading kPushAhead synapses before it issues their accumulates (the
// accumulates are fixed-point, so their order does not matter).
template <int MODE>
__device__ __forceinline__ long long batch_push(const BatchArgs &a, const BatchNet<MODE> &nb, int i, int cur,
                                                typename Tr<MODE>::A *ring, int lane) {
    const long long beg = a.rowptr[nb.off + i], end = a.rowptr[nb.off + i + 1];
    for (long long p0 = beg + lane; p0 < end; p0 += 32 * kPushAhead) {
        unsigned e[kPushAhead], w[kPushAhead];
#pragma unroll
        for (int u = 0; u < kPushAhead; ++u) {
            const long long p = p0 + 32 * u;
            e[u] = p < end ? __ldg(a.sidx + p) : 0u;
            w[u] = p < end ? __ldg(a.sw + p) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kPushAhead; ++u) {
            if (p0 + 32 * u >= end) break;
            const int post = (int)(e[u] & 0xFFFu);
            int sl = cur + (int)(e[u] >> 12) + 1;
            if (sl >= a.D1) sl -= a.D1;
            atomicAdd(ring + (size_t)sl * nb.n + post, Tr<MODE>::to_acc(w[u]));
        }
    }
    return end - beg;
}

template <int MODE>
__device__ BatchNet<MODE> load_net(const BatchArgs &a, int b) {
    BatchNet<MODE> nb;
    nb.b = b;
    nb.off = a.net_off[b];
    nb.n = a.net_off[b + 1] - nb.off;
    nb.woff = a.word_off[b];
    nb.key = a.pkey[b];
    return nb;
}

template <int MODE>
__global__ void __launch_bounds__(kBatchBlock, 2) batch_kernel(BatchArgs a) {
    using A = typename Tr<MODE>::A;
    extern __shared__ __align__(16) unsigned char smem[];
    A *arena = (A *)smem;                                  // ring arena
    int *lists = (int *)(smem + a.ring_smem);              // spiker lists
    __shared__ int s_item, s_cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long my_spikes = 0, my_events = 0;
    bool overflow = false;

    // ---- networks run by the whole block
    for (;;) {
        // thread 0 decides for the whole block (a latched status ends the work)
        if (threadIdx.x == 0)
            s_item = ld_status(a.ctl) != 0 ? a.n_cta : (int)atomicAdd(&a.ctl->queue[0], 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n_cta) break;
        const BatchNet<MODE> nb = load_net<MODE>(a, a.cta_order[item]);
        A *gring = (A *)a.ring + a.ring_off[nb.b];
        const size_t ring_elems = (size_t)a.D1 * nb.n;
        const bool in_smem = ring_elems * sizeof(A) <= (size_t)a.ring_smem;
        A *ring = in_smem ? arena : gring;
        if (in_smem)
            for (size_t q = threadIdx.x; q < ring_elems; q += blockDim.x) arena[q] = __ldcg(gring + q);
        __syncthreads();
        for (int s = 0; s < a.steps; ++s) {
            const int t = a.t0 + s;
            const int cur = t % a.D1;
            A *slot = ring + (size_t)cur * nb.n;
            unsigned *rrow = a.raster + (size_t)(t % a.cap) * a.total_words + nb.woff;
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            for (int jb0 = 0; jb0 < nb.n; jb0 += kUpdAhead * blockDim.x) {
                NeuronIn<MODE> in[kUpdAhead];
#pragma unroll
                for (int u = 0; u < kUpdAhead; ++u) {
                    const int j = jb0 + u * blockDim.x + threadIdx.x;
                    if (j < nb.n) batch_load<MODE>(a, nb, j, slot, !in_smem, in[u]);
                }
#pragma unroll
                for (int u = 0; u < kUpdAhead; ++u) {
                    const int jb = jb0 + u * blockDim.x;
                    if (jb >= nb.n) break;
                    const int j = jb + threadIdx.x;
                    const bool fire = j < nb.n && batch_finish<MODE>(a, nb, t, j, slot, in[u], overflow);
                    const unsigned ball = __ballot_sync(0xffffffffu, fire);
                    const int wb = jb + warp * 32;
                    if (lane == 0 && wb < nb.n) rrow[wb >> 5] = ball;
                    if (ball) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&s_cnt, __popc(ball));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (fire) lists[base + __popc(ball & ((1u << lane) - 1u))] = j;
                    }
                }
            }
            __syncthreads();
            const int k = s_cnt;
            if (threadIdx.x == 0) my_spikes += (unsigned long long)k;
            for (int q = warp; q < k; q += kWarps) {
                const long long len = batch_push<MODE>(a, nb, lists[q], cur, ring, lane);
                if (lane == 0) my_events += (unsigned long long)len;
            }
            __syncthreads();
        }
        if (in_smem)
            for (size_t q = threadIdx.x; q < ring_elems; q += blockDim.x) gring[q] = arena[q];
        __syncthreads();
    }

    // ---- networks run by single warps
    const int warp_ring_bytes = (a.ring_smem / kWarps) & ~15;
    A *wring_smem = (A *)(smem + (size_t)warp * warp_ring_bytes);
    int *wlist = lists + warp * (kListInts / kWarps);
    for (;;) {
        int item = 0;
        if (lane == 0) item = ld_status(a.ctl) != 0 ? a.n_warp : (int)atomicAdd(&a.ctl->queue[1], 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_warp) break;
        const BatchNet<MODE> nb = load_net<MODE>(a, a.warp_order[item]);
        A *gring = (A *)a.ring + a.ring_off[nb.b];
        const size_t ring_elems = (size_t)a.D1 * nb.n;
        const bool in_smem = ring_elems * sizeof(A) <= (size_t)warp_ring_bytes;
        A *ring = in_smem ? wring_smem : gring;
        if (in_smem)
            for (size_t q = lane; q < ring_elems; q += 32) wring_smem[q] = __ldcg(gring + q);
        __syncwarp();
        for (int s = 0; s < a.steps; ++s) {
            const int t = a.t0 + s;
            const int cur = t % a.D1;
            A *slot = ring + (size_t)cur * nb.n;
            unsigned *rrow = a.raster + (size_t)(t % a.cap) * a.total_words + nb.woff;
            int cnt = 0;
            for (int jb0 = 0; jb0 < nb.n; jb0 += kUpdAhead * 32) {
                NeuronIn<MODE> in[kUpdAhead];
#pragma unroll
                for (int u = 0; u < kUpdAhead; ++u) {
                    const int j = jb0 + u * 32 + lane;
                    if (j < nb.n) batch_load<MODE>(a, nb, j, slot, !in_smem, in[u]);
                }
#pragma unroll
                for (int u = 0; u < kUpdAhead; ++u) {
                    const int jb = jb0 + u * 32;
                    if (jb >= nb.n) break;
                    const int j = jb + lane;
                    const bool fire = j < nb.n && batch_finish<MODE>(a, nb, t, j, slot, in[u], overflow);
                    const unsigned ball = __ballot_sync(0xffffffffu, fire);
                    if (lane == 0) rrow[jb >> 5] = ball;
                    if (fire) wlist[cnt + __popc(ball & ((1u << lane) - 1u))] = j;
                    cnt += __popc(ball);
                }
            }
            __syncwarp();
            if (lane == 0) my_spikes += (unsigned long long)cnt;
            for (int q = 0; q < cnt; ++q) {
                const long long len = batch_push<MODE>(a, nb, wlist[q], cur, ring, lane);
                if (lane == 0) my_events += (unsigned long long)len;
            }
            __syncwarp();
        }
        if (in_smem)
            for (size_t q = lane; q < ring_elems; q += 32) gring[q] = wring_smem[q];
        __syncwarp();
    }
    if (MODE == SN_I32 && overflow) atomicCAS(&a.ctl->status, 0, (int)SN_EOVERFLOW);
    if (my_spikes) atomicAdd(&a.ctl->spikes, my_spikes);
    if (my_events) atomicAdd(&a.ctl->events, my_events);
}

size_t batch_smem(int ring_smem) { return (size_t)ring_smem + (size_t)kListInts * sizeof(int); }

static const void *batch_fn(int dtype) {
    return dtype == SN_F32 ? (const void *)batch_kernel<SN_F32> : (const void *)batch_kernel<SN_I32>;
}

cudaError_t batch_kernel_node(int dtype, void **fn) {
    *fn = (void *)batch_fn(dtype);
    return cudaSuccess;
}

cudaError_t max_grid_batch(int dtype, int ring_smem, int *grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = batch_smem(ring_smem);
    e = cudaFuncSetAttribute(batch_fn(dtype), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_fn(dtype), kBatchBlock, smem);
    if (e != cudaSuccess) return e;
    *grid = per * sms;
    return cudaSuccess;
}

cudaError_t launch_batch(const BatchArgs &a, int dtype, int grid, cudaStream_t s) {
    const size_t smem = batch_smem(a.ring_smem);
    cudaError_t e = cudaFuncSetAttribute(batch_fn(dtype), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(batch_fn(dtype), dim3(grid), dim3(kBatchBlock), args, smem, s);
}

}  // namespace sn
