// Device helpers shared by the simulation kernels: the counter-based Poisson
// source, the LIF rule, fixed-point accumulation traits and the bounded grid
// barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sn_internal.h"

namespace sn {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool poisson_fires(unsigned long long key, unsigned t, unsigned j,
                                              unsigned thr) {
    unsigned long long ctr = ((unsigned long long)t << 32) | (unsigned long long)j;
    return (unsigned)(splitmix64(key ^ ctr) >> 32) < thr;
}

// A 4-byte load for scattered reads (one weight of a column): an L2 miss
// fetches 64 bytes instead of the default 128 (measured on random loads over
// 1 GiB: 2 sectors requested per missed sector instead of 3.8, half the DRAM
// bytes).
__device__ __forceinline__ float ld_scattered(const float *p) {
    float x;
    asm volatile("ld.global.L2::64B.f32 %0, [%1];" : "=f"(x) : "l"(p));
    return x;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_status(const Control *ctl) {
    return *(volatile const int *)&ctl->status;
}

// Grid-wide barrier for a cooperative launch, on a counter that only grows
// during a launch (the host zeroes it before every launch): thread 0 of each
// block adds one with release semantics and waits until the count reaches the
// next multiple of the grid size.  No block can arrive at barrier e + 1
// before every block has arrived at barrier e, so the count a block sees on
// arrival lies in [e * grid, (e + 1) * grid) and fixes its target.
__device__ __forceinline__ unsigned bar_arrive(Control *ctl) {
    unsigned old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(&ctl->bar.count) : "memory");
    return (old / gridDim.x + 1u) * gridDim.x;
}

// Arrival at the k-th barrier of a launch (k = 0, 1, ...): the target is
// (k + 1) * gridDim.x, so the add is issued without waiting for its return
// (one round trip fewer before the arriving block starts polling).
__device__ __forceinline__ unsigned bar_arrive_k(Control *ctl, unsigned k) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" : : "l"(&ctl->bar.count) : "memory");
    return (k + 1u) * gridDim.x;
}

// Thread 0: wait until the count reaches `target` (bounded: wall-clock limit,
// or a status latched by another block).  Returns false if it gave up.
__device__ __forceinline__ bool bar_wait(Control *ctl, unsigned target) {
    const unsigned long long t_start = global_timer_ns();
    unsigned spins = 0;
    while ((int)(ld_acquire_u32(&ctl->bar.count) - target) < 0) {
        if ((++spins & 63u) == 0) {
            if (ld_status(ctl) != 0) return false;
            if (global_timer_ns() - t_start > kBarrierTimeoutNs) {
                atomicCAS(&ctl->status, 0, (int)SN_ETIMEOUT);
                return false;
            }
        }
        __nanosleep(32);
    }
    return true;
}

// Whole-block grid barrier.  Returns false if the wait gave up (wall-clock
// limit or a status latched by another block); the caller then leaves its
// time loop.
__device__ inline bool grid_barrier(Control *ctl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (gridDim.x > 1) ok = bar_wait(ctl, bar_arrive(ctl)) ? 1 : 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int MODE> struct Tr;
template <> struct Tr<SN_F32> {
    using V = float;
    using A = unsigned long long;   // two's-complement fixed point, 2^-32 units
    static __device__ __forceinline__ A to_acc(unsigned wbits) {
        return (A)__float2ll_rn(__uint_as_float(wbits) * 4294967296.0f);
    }
    static __device__ __forceinline__ float from_acc(A a) {
        return __ll2float_rn((long long)a) * 2.3283064365386963e-10f;
    }
};
template <> struct Tr<SN_I32> {
    using V = int;
    using A = unsigned int;
    static __device__ __forceinline__ A to_acc(unsigned wbits) { return (A)wbits; }
    static __device__ __forceinline__ int from_acc(A a) { return (int)a; }
};

// External input of neuron g (index in the event / Poisson tables) at step t:
// explicit events (pre-summed per (step, neuron) on the host, in the order
// given) then the Poisson source, whose stream uses the network key and the
// neuron's index j within its network.
template <int MODE>
__device__ __forceinline__ typename Tr<MODE>::V external_input_at(
    const int *ev_off, int ev_nsteps, const int *ev_neuron, const void *ev_val, const unsigned *prate,
    const void *pamp, unsigned long long key, int t, int g, int j) {
    using V = typename Tr<MODE>::V;
    V ext = 0;
    if (t < ev_nsteps) {
        int lo = ev_off[t], hi = ev_off[t + 1];
        const int end = hi;
        while (lo < hi) {                       // binary search for neuron g
            int mid = (lo + hi) >> 1;
            if (ev_neuron[mid] < g) lo = mid + 1; else hi = mid;
        }
        if (lo < end && ev_neuron[lo] == g) ext = ((const V *)ev_val)[lo];
    }
    unsigned thr = prate[g];
    if (thr && poisson_fires(key, (unsigned)t, (unsigned)j, thr)) {
        V amp = ((const V *)pamp)[g];
        if (MODE == SN_F32) ext = __fadd_rn(ext, amp); else ext = ext + amp;
    }
    return ext;
}

template <int MODE>
__device__ __forceinline__ typename Tr<MODE>::V external_input(const NetArgs &a, int t, int j) {
    return external_input_at<MODE>(a.ev_off, a.ev_nsteps, a.ev_neuron, a.ev_val, a.prate, a.pamp, a.pkey,
                                   t, j, j);
}

// The LIF rule for one neuron.  Returns true on a spike; v and rr updated.
// Leak: constant, toward the reset state, clamped there (Section 2.1).
__device__ __forceinline__ bool lif_update_f32(float &v, int &rr, float acc, float ext, float th,
                                               float lk, float rs, int R) {
    float u;
    if (v > rs) { u = __fsub_rn(v, lk); u = u > rs ? u : rs; }
    else if (v < rs) { u = __fadd_rn(v, lk); u = u < rs ? u : rs; }
    else u = rs;
    u = __fadd_rn(u, acc);
    u = __fadd_rn(u, ext);
    bool fire = (u > th) && (rr == 0);
    if (fire) { u = rs; rr = R; }
    else if (rr > 0) rr -= 1;
    v = u;
    return fire;
}

__device__ __forceinline__ bool lif_update_i32(int &v, int &rr, int acc, int ext, int th, int lk,
                                               int rs, int R, bool &overflow) {
    long long u;
    if (v > rs) { u = (long long)v - lk; u = u > rs ? u : rs; }
    else if (v < rs) { u = (long long)v + lk; u = u < rs ? u : rs; }
    else u = rs;
    u += acc;
    u += ext;
    // the integrated state must fit int32 before it meets the threshold
    if (u > 2147483647ll || u < -2147483648ll) overflow = true;
    bool fire = (u > th) && (rr == 0);
    if (fire) { u = rs; rr = R; }
    else if (rr > 0) rr -= 1;
    v = (int)u;
    return fire;
}

__device__ __forceinline__ bool spiked(const unsigned *rrow, int j) {
    return (rrow[j >> 5] >> (j & 31)) & 1u;
}

__device__ __forceinline__ float clampf(float w, float lo, float hi) {
    w = w < lo ? lo : w;
    return w > hi ? hi : w;
}

}  // namespace sn
