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
                    float w = __uint_as_float(a.syn[c.y].y);
                    a.syn[c.y].y = __float_as_uint(clampf(__fadd_rn(w, dw), a.wmin, a.wmax));
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

cudaError_t launch_sparse_reg(const NetArgs &a, int dtype, int grid, cudaStream_t s) {
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel(sparse_reg_fn(dtype), dim3(grid), dim3(kRegBlock), args, 0, s);
}

cudaError_t launch_sparse(const NetArgs &a, int dtype, int grid, int block, cudaStream_t s) {
    void *args[] = {(void *)&a};
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
// Dense network: W[n][n] row-major (row = pre).  After every block's update
// of step t (barrier), work items (column tile, spike chunk) gather the rows of
// the spikers of step t, in ascending pre order within a chunk, into
// partial[chunk][column].  The next update sums the S partials of its neurons
// in chunk order into the ring slot of the arrival step, so the result does
// not depend on timing.

constexpr int kDenseCols = 4;                      // columns per thread per tile
constexpr int kTile = kBlock * kDenseCols;         // columns per tile
constexpr int kListMax = 2048;                     // spikers held in shared memory

// Spikers of step t with rank in [lo, hi) (ascending neuron order) into list.
__device__ void extract_ranks(const unsigned *rrow, const int *wpre, int words, int lo, int hi,
                              int *list) {
    // first word whose prefix count exceeds lo
    int a = 0, b = words;
    while (a < b) {
        int mid = (a + b) >> 1;
        if (wpre[mid + 1] <= lo) a = mid + 1; else b = mid;
    }
    for (int w = a + threadIdx.x; w < words && wpre[w] < hi; w += blockDim.x) {
        unsigned bits = rrow[w];
        int rank = wpre[w];
        while (bits) {
            const int bpos = __ffs(bits) - 1;
            bits &= bits - 1u;
            if (rank >= lo && rank < hi) list[rank - lo] = w * 32 + bpos;
            ++rank;
        }
    }
}

template <bool STDP>
__global__ void __launch_bounds__(kBlock) dense_kernel(NetArgs a) {
    extern __shared__ int smem[];
    int *wpre = smem;                           // [words + 1] prefix popcounts
    int *list = smem + a.words + 1;             // [kListMax]
    __shared__ int s_cnt;
    __shared__ int s_scan[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * a.chunk;
    const int j1 = min(a.n, j0 + a.chunk);
    const int n = a.n;
    const int ntile = (n + kTile - 1) / kTile;
    const int items = ntile * a.S;
    float *ring = (float *)a.ring;
    unsigned long long my_spikes = 0;

    __shared__ int s_stop;
    for (int s = 0; s < a.steps; ++s) {
        if (threadIdx.x == 0) { s_cnt = 0; s_stop = ld_status(a.ctl); }
        __syncthreads();
        if (s_stop) break;
        const int t = a.t0 + s;
        const int cur = t % a.D1;
        // U: fold the partials of step t-1 into the arrival slot, then update
        int arr = (t - 1 + a.dense_delay) % a.D1;
        phase_update<SN_F32, STDP>(a, t, j0, j1, list, &s_cnt, [&](int j) -> float {
            float sum = 0.0f;
            for (int c = 0; c < a.S; ++c) sum = __fadd_rn(sum, a.partial[(size_t)c * n + j]);
            ring[(size_t)arr * n + j] = sum;
            return ring[(size_t)cur * n + j];
        });
        __syncthreads();
        if (threadIdx.x == 0) my_spikes += (unsigned long long)s_cnt;
        if (!grid_barrier(a.ctl)) break;

        // G: prefix popcounts of the raster row of step t
        const unsigned *rrow = a.raster + (size_t)(t % a.cap) * a.words;
        {
            int run = 0;
            for (int w0 = 0; w0 < a.words; w0 += blockDim.x) {
                const int w = w0 + threadIdx.x;
                int c = w < a.words ? __popc(rrow[w]) : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) s_scan[warp] = incl;
                __syncthreads();
                if (warp == 0) {
                    int v = lane < (int)(blockDim.x >> 5) ? s_scan[lane] : 0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        int y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (lane < (int)(blockDim.x >> 5)) s_scan[lane] = v;
                }
                __syncthreads();
                const int wexcl = warp ? s_scan[warp - 1] : 0;
                if (w < a.words) wpre[w] = run + wexcl + incl - c;
                const int tot = s_scan[(blockDim.x >> 5) - 1];
                __syncthreads();
                run += tot;
            }
            if (threadIdx.x == 0) wpre[a.words] = run;
            __syncthreads();
        }
        const int k = wpre[a.words];
        const float *xo = STDP ? a.trace + (size_t)((t & 1) ^ 1) * n : nullptr;

        for (int item = blockIdx.x; item < items; item += gridDim.x) {
            const int tile = item % ntile, chunk = item / ntile;
            const int lo = (int)((long long)chunk * k / a.S);
            const int hi = (int)((long long)(chunk + 1) * k / a.S);
            const int c0 = tile * kTile + threadIdx.x;
            float acc[kDenseCols];
            float xc[kDenseCols];
            bool sc[kDenseCols];
#pragma unroll
            for (int u = 0; u < kDenseCols; ++u) {
                acc[u] = 0.0f;
                const int c = c0 + u * kBlock;
                if (STDP && c < n) { xc[u] = xo[c]; sc[u] = spiked(rrow, c); }
                else { xc[u] = 0.0f; sc[u] = false; }
            }
            for (int base = lo; base < hi; base += kListMax) {
                const int cnt = min(kListMax, hi - base);
                __syncthreads();
                extract_ranks(rrow, wpre, a.words, base, base + cnt, list);
                __syncthreads();
                int q = 0;
                if constexpr (!STDP) {
                    for (; q + 4 <= cnt; q += 4) {
                        float v[4][kDenseCols];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float *row = a.W + (size_t)list[q + r] * n;
#pragma unroll
                            for (int u = 0; u < kDenseCols; ++u) {
                                const int c = c0 + u * kBlock;
                                v[r][u] = c < n ? __ldg(row + c) : 0.0f;
                            }
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int u = 0; u < kDenseCols; ++u) acc[u] = __fadd_rn(acc[u], v[r][u]);
                    }
                }
                for (; q < cnt; ++q) {
                    const int i = list[q];
                    float *row = a.W + (size_t)i * n;
                    const float xi = STDP ? xo[i] : 0.0f;
#pragma unroll
                    for (int u = 0; u < kDenseCols; ++u) {
                        const int c = c0 + u * kBlock;
                        if (c >= n) continue;
                        float w = row[c];
                        if (STDP && c != i) {
                            float dw = sc[u] ? __fmul_rn(a.a_plus, xi) : 0.0f;
                            dw = __fsub_rn(dw, __fmul_rn(a.a_minus, xc[u]));
                            w = clampf(__fadd_rn(w, dw), a.wmin, a.wmax);
                            row[c] = w;
                        }
                        acc[u] = __fadd_rn(acc[u], w);
                    }
                }
            }
            float *part = a.partial + (size_t)chunk * n;
#pragma unroll
            for (int u = 0; u < kDenseCols; ++u) {
                const int c = c0 + u * kBlock;
                if (c < n) part[c] = acc[u];
            }
        }

        if constexpr (STDP) {
            // LTP on columns of spiking post-neurons, rows of non-spiking
            // pre-neurons (spiking rows were updated in full above).
            const int nwarp_grid = gridDim.x * (blockDim.x >> 5);
            const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
            for (int base = 0; base < k; base += kListMax) {
                const int cnt = min(kListMax, k - base);
                __syncthreads();
                extract_ranks(rrow, wpre, a.words, base, base + cnt, list);
                __syncthreads();
                for (int i = gw; i < n; i += nwarp_grid) {
                    if (spiked(rrow, i)) continue;
                    const float dw = __fmul_rn(a.a_plus, xo[i]);
                    float *row = a.W + (size_t)i * n;
                    for (int q = lane; q < cnt; q += 32) {
                        const int j = list[q];
                        row[j] = clampf(__fadd_rn(row[j], dw), a.wmin, a.wmax);
                    }
                }
            }
        }
        if (!grid_barrier(a.ctl)) break;
    }
    if (threadIdx.x == 0 && my_spikes) {
        atomicAdd(&a.ctl->spikes, my_spikes);
        atomicAdd(&a.ctl->events, my_spikes * (unsigned long long)n);
    }
}

static size_t dense_smem(int words) { return (size_t)(words + 1 + kListMax) * sizeof(int); }

cudaError_t launch_dense(const NetArgs &a, int grid, int block, cudaStream_t s) {
    void *args[] = {(void *)&a};
    const size_t smem = dense_smem(a.words);
    const void *fn = a.stdp ? (const void *)dense_kernel<true> : (const void *)dense_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t max_grid_dense(int block, int *grid, size_t *smem_for_words) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int words = (int)(*smem_for_words);
    const size_t smem = dense_smem(words);
    for (const void *fn : {(const void *)dense_kernel<true>, (const void *)dense_kernel<false>}) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    per = 1 << 30;
    for (const void *fn : {(const void *)dense_kernel<true>, (const void *)dense_kernel<false>}) {
        int p = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, block, smem);
        if (e != cudaSuccess) return e;
        per = p < per ? p : per;
    }
    *grid = per * sms;
    *smem_for_words = smem;
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

cudaError_t launch_gather_weights(const uint2 *syn, const long long *perm_inv, long long m,
                                  float *out, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    gather_weights_kernel<<<(int)blocks, 256, 0, s>>>(syn, perm_inv, m, out);
    return cudaGetLastError();
}

}  // namespace sn
