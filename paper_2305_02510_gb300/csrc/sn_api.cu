// Host side of the C ABI declared in include/sn.h: argument checking, network
// construction on the device, executor sizing, launches, getters and
// checkpoints.  All device memory of a context is allocated here at creation
// (or when inputs / STDP are configured) and freed by sn_destroy; sn_run
// allocates nothing.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "sn_ctx.h"

using namespace sn;

thread_local std::string g_create_err;
namespace sn {
thread_local long long g_fault_alloc = 0;
thread_local int g_fault_depth = 0;
}  // namespace sn

namespace {

sn_status check_config(const sn_config *cfg) {
    if (!cfg) return fail(nullptr, SN_EINVAL, "cfg is NULL");
    if (cfg->dtype != SN_F32 && cfg->dtype != SN_I32) return fail(nullptr, SN_EINVAL, "bad dtype");
    if (cfg->max_delay < 1 || cfg->max_delay > SN_MAX_DELAY)
        return fail(nullptr, SN_EINVAL, "max_delay must be in 1..64");
    if (cfg->record_steps < 0) return fail(nullptr, SN_EINVAL, "record_steps < 0");
    if (cfg->flags & ~(SN_EXEC_CTA | SN_EXEC_GRID | SN_PROP_PULL | SN_DENSE_SLAB_MASK | SN_PULL_STORE_MASK))
        return fail(nullptr, SN_EINVAL, "unknown flags");
    if ((cfg->flags & SN_PULL_STORE_MASK) == SN_PULL_STORE_MASK)
        return fail(nullptr, SN_EINVAL, "SN_PULL_PLAIN and SN_PULL_CODED are exclusive");
    if ((cfg->flags & SN_EXEC_CTA) && (cfg->flags & SN_EXEC_GRID))
        return fail(nullptr, SN_EINVAL, "SN_EXEC_CTA and SN_EXEC_GRID are exclusive");
    return SN_OK;
}

sn_status size_sparse_executor(sn_ctx *c) {
    const int n = c->n;
    c->block = 256;
    const bool cta = (c->flags & SN_EXEC_CTA) || (!(c->flags & SN_EXEC_GRID) && n <= 2048);
    // register-resident executor (used without STDP): at most one neuron per
    // thread of a 512-thread block
    {
        int gr = 0;
        cudaError_t e = max_grid_sparse_reg(&gr);
        if (e != cudaSuccess) return fail(nullptr, SN_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e));
        if (cta) {
            if (n <= kSparseRegBlock) { c->reg_grid = 1; c->reg_chunk = (n + 31) / 32 * 32; }
        } else if (gr >= 1 && (long long)gr * kSparseRegBlock >= n) {
            const int g = std::min(gr, (n + 31) / 32);
            c->reg_chunk = ((n + g - 1) / g + 31) / 32 * 32;
            c->reg_grid = (n + c->reg_chunk - 1) / c->reg_chunk;
        }
    }
    if (cta) {
        c->grid = 1;
        c->chunk = (n + 31) / 32 * 32;
        if (c->chunk > 16384) return fail(nullptr, SN_EINVAL, "SN_EXEC_CTA supports n <= 16384");
        return SN_OK;
    }
    int gmax = 0;
    cudaError_t e = max_grid_sparse(c->dtype, 1, c->block, &gmax);
    if (e != cudaSuccess) return fail(nullptr, SN_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e));
    if (gmax < 1) return fail(nullptr, SN_ECUDA, "no resident blocks possible");
    int g = std::min(gmax, (n + 31) / 32);
    int chunk = ((n + g - 1) / g + 31) / 32 * 32;
    if (chunk > 1024) return fail(nullptr, SN_EUNSUPPORTED, "network too large for the grid executor");
    c->chunk = chunk;
    c->grid = (n + chunk - 1) / chunk;
    return SN_OK;
}

// Incoming synapses of every neuron in the canonical order of the float sum:
// descending delay, then ascending pre and input index (the oldest spikes
// first), laid out for the pull kernel in two regions per slice of 32 neurons
// (neurons 32s .. 32s+31): first the synapses of delay >= 2 (the ones a step
// can add before the previous step's spikes are in), then those of delay 1.
// A synapse's bit in the kernel's spike window lies y = (D - d) * Wp * 32 + pre
// bits after the row of step t - D, and y never decreases along a list.
// Two forms of the store, both in uint4 units, both padded per region to the
// slice's longest list (padding is all-zero):
//  - plain: entry q of the neuron in lane l is half q % 2 of uint4
//    start + (q / 2) * 32 + l, as {(y / 32 * 4) << 5 | y % 32, weight bits}
//    (8 bytes per synapse);
//  - coded: entries in groups of 8; group g of lane l is the uint4s
//    start + g * 96 + {0, 32, 64} + l, holding weights 0-3, weights 4-7 and the
//    eight 16-bit steps y_q - y_(q-1) (the first step is 0; the first y is
//    pin_y0[region * n + j]).  A step above 65535 is taken in filler entries
//    of step 65535 and weight 0, which add +0 (an exact no-op: the sum starts
//    at +0 and is never -0) at offsets inside the window (6 bytes per synapse
//    plus the fillers).
// The form is the plain one while its store takes at most 80 % of the L2,
// else the smaller one, unless pin_format forces one.  (At 10^5 neurons and
// delays 1..16, 100 synapses a neuron run at the same speed in both forms;
// at 125 the plain store, 124 MB, no longer stays in the L2 and the coded
// one, 96 MB, runs 1.6x faster.)  The delay->=2
// region of slice s starts at pin_off[s]; the delay-1 region follows it.  A
// network run by one block (no grid barrier to overlap) keeps every synapse
// in the first region, the delay-1 ones last.  Built from the CSR, whose rows
// keep the input order, so ties of (delay, pre) stay in input order.
sn_status build_pull_store(sn_ctx *c) {
    const int n = c->n;
    const long long m = c->m;
    if (m >= (1ll << 32)) return fail(c, SN_EUNSUPPORTED, "pull propagation supports m < 2^32");
    std::vector<uint2> syn(m > 0 ? m : 1);
    std::vector<long long> rowptr(n + 1);
    SN_CUDA(c, cudaMemcpy(syn.data(), c->syn, (size_t)(m > 0 ? m : 1) * 8, cudaMemcpyDeviceToHost));
    SN_CUDA(c, cudaMemcpy(rowptr.data(), c->rowptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost));
    // CSR positions bucketed by delay, largest delay first, stable (pre
    // ascending, input order within a pre)
    const int D = c->D;
    std::vector<long long> dstart(D + 2, 0);             // bucket k holds delay D - k
    for (long long p = 0; p < m; ++p) dstart[(D - 1 - (int)(syn[p].x >> kPostBits)) + 1]++;
    for (int k = 0; k <= D; ++k) dstart[k + 1] += dstart[k];
    std::vector<uint32_t> byd(m > 0 ? m : 1), pre_of(m > 0 ? m : 1);
    for (int i = 0; i < n; ++i)
        for (long long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            byd[dstart[D - 1 - (int)(syn[p].x >> kPostBits)]++] = (uint32_t)p;
            pre_of[p] = (uint32_t)i;
        }
    const bool one_region = c->pull_grid == 1;
    const unsigned long long wbits = (unsigned long long)((c->words + 3) & ~3) * 32;   // window row, bits
    auto region_of = [&](uint32_t p) { return ((syn[p].x >> kPostBits) == 0 && !one_region) ? 1 : 0; };
    auto y_of = [&](uint32_t p) {
        return (unsigned)((unsigned long long)(D - 1 - (int)(syn[p].x >> kPostBits)) * wbits + pre_of[p]);
    };
    // list lengths of both forms (the coded one with its fillers)
    std::vector<int> len[2] = {std::vector<int>(n, 0), std::vector<int>(n, 0)};
    std::vector<int> lenc[2] = {std::vector<int>(n, 0), std::vector<int>(n, 0)};
    std::vector<unsigned> y0(2 * (size_t)n, 0u), ylast(2 * (size_t)n, 0u);
    for (long long k = 0; k < m; ++k) {
        const uint32_t p = byd[k];
        const int j = (int)(syn[p].x & kPostMask), r = region_of(p);
        const unsigned y = y_of(p);
        if (len[r][j]++ == 0) { y0[(size_t)r * n + j] = y; lenc[r][j] = 1; }
        else lenc[r][j] += (int)std::max(1u, (y - ylast[(size_t)r * n + j] + 65534u) / 65535u);
        ylast[(size_t)r * n + j] = y;
    }
    // Positions: thread p of the launch sums the lists of neuron perm[p].
    // Within each block's range of neurons the lists are sorted longest
    // first, so that the 32 lists of a warp have about the same length (the
    // warp runs to its longest); the block hands each sum to the neuron's
    // own thread through shared memory.  Neurons outside the simulated range
    // (other shards') keep their own positions.
    std::vector<int> perm(n), pos_of(n);
    for (int j = 0; j < n; ++j) perm[j] = j;
    {
        const int j0 = c->shard_end ? c->shard_first : 0, j1 = c->shard_end ? c->shard_end : n;
        const int chunk = std::max(c->pull_chunk, 32);
        for (int b0 = j0; b0 < j1; b0 += chunk) {
            const int b1 = std::min(j1, b0 + chunk);
            std::stable_sort(perm.begin() + b0, perm.begin() + b1, [&](int x, int y) {
                return len[0][x] + len[1][x] > len[0][y] + len[1][y];
            });
            // then, within runs of two warps, by the delay-1 list (summed after
            // the barrier, on the step's critical path)
            for (int w0 = b0; w0 < b1; w0 += 64)
                std::stable_sort(perm.begin() + w0, perm.begin() + std::min(b1, w0 + 64),
                                 [&](int x, int y) { return len[1][x] > len[1][y]; });
        }
    }
    for (int q = 0; q < n; ++q) pos_of[perm[q]] = q;
    const int slices = (n + 31) / 32;
    long long total[2] = {0, 0};                          // uint4s: plain, coded
    std::vector<long long> off[2] = {std::vector<long long>(slices), std::vector<long long>(slices)};
    std::vector<long long> offB[2] = {std::vector<long long>(slices), std::vector<long long>(slices)};
    for (int sl = 0; sl < slices; ++sl) {
        int LA[2] = {0, 0}, LB[2] = {0, 0};
        for (int q = sl * 32; q < std::min(n, sl * 32 + 32); ++q) {
            const int j = perm[q];
            LA[0] = std::max(LA[0], len[0][j]);  LB[0] = std::max(LB[0], len[1][j]);
            LA[1] = std::max(LA[1], lenc[0][j]); LB[1] = std::max(LB[1], lenc[1][j]);
        }
        off[0][sl] = total[0];
        offB[0][sl] = total[0] + (long long)((LA[0] + 1) / 2) * 32;
        total[0] = offB[0][sl] + (long long)((LB[0] + 1) / 2) * 32;
        off[1][sl] = total[1];
        offB[1][sl] = total[1] + (long long)((LA[1] + 7) / 8) * 96;
        total[1] = offB[1][sl] + (long long)((LB[1] + 7) / 8) * 96;
    }
    // the library's choice: the plain form (fewer instructions a synapse)
    // while its store stays well inside the L2, which serves it every step;
    // the coded form when that keeps the store smaller
    int l2 = 0, dev = 0;
    SN_CUDA(c, cudaGetDevice(&dev));
    SN_CUDA(c, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const bool plain_fits = (double)total[0] * 16 <= 0.8 * (double)l2;
    const int f = c->pin_format == 1 ? 0 : c->pin_format == 2 ? 1 : (!plain_fits && total[1] < total[0] ? 1 : 0);
    const long long tot = std::max(total[f], 1ll);
    std::vector<uint4> pin(tot, make_uint4(0, 0, 0, 0));
    auto comp = [](uint4 &v, int i) -> unsigned & { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; };
    std::vector<int> fill[2] = {std::vector<int>(n, 0), std::vector<int>(n, 0)};
    for (long long k = 0; k < m; ++k) {
        const uint32_t p = byd[k];
        const int j = (int)(syn[p].x & kPostMask), r = region_of(p), ps = pos_of[j], l = ps & 31;
        const unsigned y = y_of(p);
        const long long start = (r ? offB[f] : off[f])[ps >> 5];
        if (f == 0) {
            const int q = fill[r][j]++;
            uint4 &u = pin[start + (long long)(q >> 1) * 32 + l];
            const unsigned x = ((y >> 5) << 7) | (y & 31u);
            if (q & 1) { u.z = x; u.w = syn[p].y; } else { u.x = x; u.y = syn[p].y; }
            continue;
        }
        unsigned step = fill[r][j] == 0 ? 0u : y - ylast[(size_t)r * n + j];
        ylast[(size_t)r * n + j] = y;
        for (;;) {
            const int q = fill[r][j]++;
            const long long g = start + (long long)(q >> 3) * 96 + l;
            const unsigned st = std::min(step, 65535u);
            comp(pin[g + 64], (q & 7) >> 1) |= (q & 1) ? st << 16 : st;
            if (step <= 65535u) {
                comp(pin[g + (q & 4 ? 32 : 0)], q & 3) = syn[p].y;
                break;
            }
            step -= 65535u;                               // a filler: weight 0
        }
    }
    sn_status s;
    const size_t bytes = (size_t)tot * 16;
    if (c->pin && c->pin_cap < bytes) { dfree(c, c->pin); c->pin = nullptr; }
    if (!c->pin) {
        if ((s = dalloc(c, &c->pin, bytes))) return s;
        c->pin_cap = bytes;
    }
    if (!c->pin_off) {
        if ((s = dalloc(c, &c->pin_off, (size_t)slices * 8)) || (s = dalloc(c, &c->pin_len, (size_t)n * 4)) ||
            (s = dalloc(c, &c->pin_len1, (size_t)n * 4)) || (s = dalloc(c, &c->pin_y0, (size_t)n * 8)) ||
            (s = dalloc(c, &c->pin_perm, (size_t)n * 4)))
            return s;
    }
    // list lengths and first offsets by position
    std::vector<int> lA(n), lB(n);
    std::vector<unsigned> y0p(2 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        const int j = perm[q];
        lA[q] = (f ? lenc[0] : len[0])[j];
        lB[q] = (f ? lenc[1] : len[1])[j];
        y0p[q] = y0[j];
        y0p[(size_t)n + q] = y0[(size_t)n + j];
    }
    SN_CUDA(c, cudaMemcpy(c->pin, pin.data(), bytes, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pin_off, off[f].data(), (size_t)slices * 8, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pin_len, lA.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pin_len1, lB.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pin_y0, y0p.data(), (size_t)n * 8, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pin_perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    c->pin_coded = f;
    c->pin_bytes = (long long)bytes;
    c->pin_entries = 0;
    for (int j = 0; j < n; ++j) c->pin_entries += (long long)lA[j] + lB[j];
    c->pin_stale = false;
    return SN_OK;
}

sn_status select_pull(sn_ctx *c) {
    if (c->stdp) return fail(c, SN_EUNSUPPORTED, "STDP runs on push propagation");
    if (c->pull_grid == 0) {
        const int own = c->shard_end ? (c->shard_end - c->shard_first + 31) / 32 : -1;
        cudaError_t e = plan_pull(c->n, c->D, c->m, &c->pull_grid, &c->pull_chunk, &c->pull_rows, &c->pull_smem, own);
        if (e != cudaSuccess) return cuda_fail(c, e, "pull executor");
        if (c->pull_grid == 0)
            return fail(c, SN_EUNSUPPORTED,
                        "pull propagation needs max_delay * ceil(n/32) spike words within a block's shared "
                        "memory and at most 1024 neurons per SM");
    }
    sn_status s;
    if ((s = quiesce(c))) return s;            // a queued push run may still read the ring
    if (!c->hist) {
        if ((s = dalloc(c, &c->hist, (size_t)c->D * c->words * 4))) return s;
        SN_CUDA(c, cudaMemset(c->hist, 0, (size_t)c->D * c->words * 4));
    }
    if (c->pin_stale && (s = build_pull_store(c))) return s;
    c->prop_pull = 1;
    return SN_OK;
}

}  // namespace

namespace sn {

// Neuron parameters to device arrays (float or int32 according to dtype).
sn_status upload_neurons(sn_ctx *c, const sn_neurons *nr) {
    const int n = c->n;
    if (!nr->threshold || !nr->leak || !nr->reset || !nr->refractory)
        return fail(nullptr, SN_EINVAL, "neuron parameter array is NULL");
    for (int j = 0; j < n; ++j) {
        const bool th_inf = std::isinf(nr->threshold[j]) && nr->threshold[j] > 0;
        if (!std::isfinite(nr->threshold[j]) && !th_inf)
            return fail(nullptr, SN_EINVAL, "threshold must not be NaN or -inf");
        if (!std::isfinite(nr->leak[j]) || nr->leak[j] < 0)
            return fail(nullptr, SN_EINVAL, "leak must be finite and >= 0");
        if (!std::isfinite(nr->reset[j])) return fail(nullptr, SN_EINVAL, "reset must be finite");
        if (nr->refractory[j] < 0) return fail(nullptr, SN_EINVAL, "refractory must be >= 0");
        if (c->dtype == SN_I32 &&
            !((th_inf || is_int_valued(nr->threshold[j])) && is_int_valued(nr->leak[j]) &&
              is_int_valued(nr->reset[j])))
            return fail(nullptr, SN_EINVAL, "SN_I32 parameters must be integers below 2^24");
    }
    const size_t vb = (size_t)n * 4;
    sn_status s;
    if ((s = dalloc(c, &c->V, vb)) || (s = dalloc(c, &c->r, vb)) || (s = dalloc(c, &c->th, vb)) ||
        (s = dalloc(c, &c->lk, vb)) || (s = dalloc(c, &c->rs, vb)) || (s = dalloc(c, &c->R, vb)) ||
        (s = dalloc(c, &c->prate, vb)) || (s = dalloc(c, &c->pamp, vb)))
        return fail(nullptr, s, "neuron arrays: " + c->err);
    // +inf thresholds in integer mode become INT32_MAX: V > INT32_MAX never holds
    auto up = [&](void *dst, const float *src) -> cudaError_t {
        if (c->dtype == SN_F32) return cudaMemcpy(dst, src, vb, cudaMemcpyHostToDevice);
        std::vector<int> tmp(n);
        for (int j = 0; j < n; ++j) tmp[j] = std::isinf(src[j]) ? 2147483647 : (int)src[j];
        return cudaMemcpy(dst, tmp.data(), vb, cudaMemcpyHostToDevice);
    };
    cudaError_t e;
    if ((e = up(c->th, nr->threshold)) || (e = up(c->lk, nr->leak)) || (e = up(c->rs, nr->reset)) ||
        (e = up(c->V, nr->reset)) ||
        (e = cudaMemcpy(c->R, nr->refractory, vb, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->r, 0, vb)) || (e = cudaMemset(c->prate, 0, vb)) ||
        (e = cudaMemset(c->pamp, 0, vb)))
        return fail(nullptr, SN_ECUDA, std::string("neuron upload: ") + cudaGetErrorString(e));
    return SN_OK;
}

sn_status alloc_common(sn_ctx *c, const sn_config *cfg) {
    c->cap = cfg->record_steps > 0 ? cfg->record_steps : 1;
    c->words = (c->n + 31) / 32;
    sn_status s;
    if ((s = dalloc(c, &c->raster, (size_t)c->cap * c->words * 4)) || (s = dalloc(c, &c->ctl, sizeof(Control))))
        return fail(nullptr, s, c->err);
    cudaError_t e;
    if ((e = cudaMemset(c->raster, 0, (size_t)c->cap * c->words * 4)) ||
        (e = cudaMemset(c->ctl, 0, sizeof(Control))))
        return fail(nullptr, SN_ECUDA, cudaGetErrorString(e));
    return SN_OK;
}

void destroy_all(sn_ctx *c) {
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
}

}  // namespace sn

extern "C" {

const char *sn_version(void) { return "sn-gb300 0.1 (sm_103a)"; }

sn_status sn_selftest_barrier_timeout(void *cuda_stream, int32_t *status) {
    if (!status) return fail(nullptr, SN_EINVAL, "status is NULL");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    Control *ctl = nullptr;
    if (cudaMalloc(&ctl, sizeof(Control)) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(nullptr, SN_ENOMEM, "device allocation of the control block failed");
    }
    Control h;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(Control), s)) || (e = launch_barrier_selftest(ctl, 4, s)) ||
        (e = cudaStreamSynchronize(s)) || (e = cudaMemcpy(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost))) {
        cudaFree(ctl);
        return fail(nullptr, SN_ECUDA, std::string("self-test: ") + cudaGetErrorString(e));
    }
    cudaFree(ctl);
    *status = h.status;
    return SN_OK;
}

const char *sn_last_error(const sn_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

sn_status sn_create(const sn_config *cfg, const sn_neurons *nr, const sn_synapses *sy, sn_ctx **out) {
    FaultScope fault_scope;
    NvtxRange nvtx("sn_create");
    sn_status s = check_config(cfg);
    if (s) return s;
    if (!nr || !sy || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    const int n = nr->n;
    if (n < 1 || n >= (1 << kPostBits)) return fail(nullptr, SN_EINVAL, "n must be in 1 .. 2^26-1");
    if (sy->m < 0) return fail(nullptr, SN_EINVAL, "m < 0");
    if (sy->m > 0 && (!sy->pre || !sy->post || !sy->weight || !sy->delay))
        return fail(nullptr, SN_EINVAL, "synapse array is NULL");
    const long long m = sy->m;
    bool all1 = true;
    for (long long k = 0; k < m; ++k) {
        if (sy->pre[k] < 0 || sy->pre[k] >= n || sy->post[k] < 0 || sy->post[k] >= n)
            return fail(nullptr, SN_EINVAL, "synapse " + std::to_string(k) + ": neuron index out of range");
        if (sy->delay[k] < 1 || sy->delay[k] > cfg->max_delay)
            return fail(nullptr, SN_EINVAL, "synapse " + std::to_string(k) + ": delay outside 1..max_delay");
        const float w = sy->weight[k];
        if (!std::isfinite(w) || std::fabs(w) > 1e9f)
            return fail(nullptr, SN_EINVAL, "synapse " + std::to_string(k) + ": weight not finite or too large");
        if (cfg->dtype == SN_I32 && !is_int_valued(w))
            return fail(nullptr, SN_EINVAL, "SN_I32 weights must be integers below 2^24");
        if (sy->delay[k] != 1) all1 = false;
    }
    sn_ctx *c = new (std::nothrow) sn_ctx();
    if (!c) return fail(nullptr, SN_ENOMEM, "host allocation failed");
    c->kind = KIND_SPARSE;
    c->dtype = cfg->dtype;
    c->n = n;
    c->D = cfg->max_delay;
    c->D1 = c->D + 1;
    c->flags = cfg->flags;
    c->pin_format = (cfg->flags & SN_PULL_CODED) ? 2 : (cfg->flags & SN_PULL_PLAIN) ? 1 : 0;
    c->m = m;
    c->all_delay_one = all1;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    auto bail = [&](sn_status st) { std::string msg = c->err.empty() ? g_create_err : c->err;
                                    destroy_all(c); delete c; g_create_err = msg; return st; };
    if ((s = upload_neurons(c, nr))) return bail(s);
    if ((s = alloc_common(c, cfg))) return bail(s);
    // CSR by pre-neuron, input order kept within a row
    std::vector<long long> rowptr(n + 1, 0);
    for (long long k = 0; k < m; ++k) rowptr[sy->pre[k] + 1]++;
    for (int i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    std::vector<uint2> syn(m > 0 ? m : 1);
    c->h_perm_inv.assign(m, 0);
    {
        std::vector<long long> fill(rowptr.begin(), rowptr.end() - 1);
        for (long long k = 0; k < m; ++k) {
            const long long p = fill[sy->pre[k]]++;
            uint2 e;
            e.x = (unsigned)sy->post[k] | ((unsigned)(sy->delay[k] - 1) << kPostBits);
            if (cfg->dtype == SN_F32) { float w = sy->weight[k]; memcpy(&e.y, &w, 4); }
            else { int w = (int)sy->weight[k]; memcpy(&e.y, &w, 4); }
            syn[p] = e;
            c->h_perm_inv[k] = p;
        }
    }
    c->ring_bytes = (size_t)c->D1 * n * (cfg->dtype == SN_F32 ? 8 : 4);
    if ((s = dalloc(c, &c->rowptr, (size_t)(n + 1) * 8)) || (s = dalloc(c, &c->syn, (size_t)(m > 0 ? m : 1) * 8)) ||
        (s = dalloc(c, &c->ring, c->ring_bytes)))
        return bail(s);
    cudaError_t e;
    if ((e = cudaMemcpy(c->rowptr, rowptr.data(), (size_t)(n + 1) * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->syn, syn.data(), (size_t)(m > 0 ? m : 1) * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->ring, 0, c->ring_bytes))) {
        c->err = std::string("upload: ") + cudaGetErrorString(e);
        return bail(SN_ECUDA);
    }
    if ((s = size_sparse_executor(c))) return bail(s);
    if ((cfg->flags & SN_PROP_PULL) && (s = select_pull(c))) return bail(s);
    *out = c;
    return SN_OK;
}

sn_status sn_create_shard(const sn_config *cfg, const sn_neurons *nr, const sn_synapses *sy, int32_t first,
                          int32_t count, sn_ctx **out) {
    FaultScope fault_scope;
    NvtxRange nvtx("sn_create");
    if (!cfg || !nr || !sy || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    const int n = nr->n;
    if (first < 0 || count < 1 || (long long)first + count > n || first % 32 != 0 ||
        (count % 32 != 0 && first + count != n))
        return fail(nullptr, SN_EINVAL,
                    "shard: first must be a multiple of 32 and [first, first + count) a range of whole 32-neuron "
                    "words of [0, n) (the last shard may end at n)");
    if (cfg->flags & (SN_EXEC_CTA | SN_EXEC_GRID))
        return fail(nullptr, SN_EINVAL, "shard: executor flags do not apply (a shard runs pull propagation)");
    int dmin = cfg->max_delay;
    for (long long k = 0; k < sy->m && sy->delay; ++k)
        if (sy->delay[k] >= 1 && sy->delay[k] < dmin) dmin = sy->delay[k];
    sn_config c2 = *cfg;
    c2.flags &= ~SN_PROP_PULL;
    sn_ctx *c = nullptr;
    sn_status s = sn_create(&c2, nr, sy, &c);
    if (s) return s;
    c->shard_first = first;
    c->shard_end = first + count;
    c->shard_dmin = dmin;
    c->shard_known = 0;
    if ((s = dalloc(c, &c->shard_stage, (size_t)c->D * c->words * 4)) || (s = select_pull(c))) {
        std::string msg = c->err;
        sn_destroy(c);
        return fail(nullptr, s, "shard: " + msg);
    }
    *out = c;
    return SN_OK;
}

sn_status sn_shard_info(const sn_ctx *c, int32_t *first, int32_t *count, int32_t *steps_per_exchange) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (!c->shard_end) return SN_ESTATE;
    if (first) *first = c->shard_first;
    if (count) *count = c->shard_end - c->shard_first;
    if (steps_per_exchange) *steps_per_exchange = c->shard_dmin;
    return SN_OK;
}

sn_status sn_shard_put_spikes(sn_ctx *c, int64_t t0, int64_t t1, const uint32_t *bits, int32_t on_device) {
    NvtxRange nvtx("sn_shard_put_spikes");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (!c->shard_end) return fail(c, SN_ESTATE, "not a shard (sn_create_shard)");
    if (c->failed) return fail(c, SN_ESTATE, "context has a latched device error");
    if (t0 != c->shard_known)
        return fail(c, SN_EINVAL, "shard: the next rows to put start at step " + std::to_string(c->shard_known));
    if (t1 < t0 || t1 > c->step)
        return fail(c, SN_EINVAL, "shard: rows can be put only for steps this shard has run");
    if (t1 - t0 > c->D) return fail(c, SN_EINVAL, "shard: at most max_delay rows per call");
    if (t1 == t0) return SN_OK;
    if (!bits) return fail(c, SN_EINVAL, "bits is NULL");
    const int rows = (int)(t1 - t0);
    const size_t bytes = (size_t)rows * c->words * 4;
    const unsigned *src = bits;
    if (!on_device) {
        // the staging rows may still be read by an earlier put queued on the stream
        if (sn_status q = quiesce(c)) return q;
        SN_CUDA(c, cudaMemcpyAsync(c->shard_stage, bits, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->shard_stage;
    }
    const int w0 = c->shard_first / 32, w1 = (c->shard_end + 31) / 32;
    cudaError_t e = launch_shard_put(c->hist, c->raster, c->D, c->cap, c->words, w0, w1, t0, rows, src, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "shard spike rows");
    if (!on_device) SN_CUDA(c, cudaStreamSynchronize(c->stream));
    c->shard_known = t1;
    return SN_OK;
}

sn_status sn_create_axonal(const sn_config *cfg, const sn_neurons *nr, const sn_synapses *sy,
                           const int32_t *axonal_delay, sn_ctx **out) {
    FaultScope fault_scope;
    NvtxRange nvtx("sn_create");
    if (!axonal_delay) return sn_create(cfg, nr, sy, out);
    sn_status s = check_config(cfg);
    if (s) return s;
    if (!nr || !sy || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    const int n = nr->n;
    if (n < 1 || n >= (1 << kPostBits)) return fail(nullptr, SN_EINVAL, "n must be in 1 .. 2^26-1");
    if (sy->m < 0) return fail(nullptr, SN_EINVAL, "m < 0");
    if (sy->m > 0 && (!sy->pre || !sy->delay)) return fail(nullptr, SN_EINVAL, "synapse array is NULL");
    for (int i = 0; i < n; ++i)
        if (axonal_delay[i] < 0 || axonal_delay[i] >= cfg->max_delay)
            return fail(nullptr, SN_EINVAL, "neuron " + std::to_string(i) + ": axonal delay outside 0..max_delay-1");
    // a spike of i at t travels the axon (axonal_delay[i] steps), then the
    // synapse (delay[k] >= 1 steps): it arrives at t + axonal_delay[i] + delay[k]
    std::vector<int32_t> eff(sy->m > 0 ? sy->m : 1);
    for (long long k = 0; k < sy->m; ++k) {
        if (sy->pre[k] < 0 || sy->pre[k] >= n)
            return fail(nullptr, SN_EINVAL, "synapse " + std::to_string(k) + ": neuron index out of range");
        if (sy->delay[k] < 1 || (long long)sy->delay[k] + axonal_delay[sy->pre[k]] > cfg->max_delay)
            return fail(nullptr, SN_EINVAL, "synapse " + std::to_string(k) +
                                                ": delay + axonal delay outside 1..max_delay");
        eff[k] = sy->delay[k] + axonal_delay[sy->pre[k]];
    }
    sn_synapses s2 = *sy;
    s2.delay = eff.data();
    return sn_create(cfg, nr, &s2, out);
}

sn_status sn_create_dense(const sn_config *cfg, const sn_neurons *nr, const float *w, int32_t delay,
                          sn_ctx **out) {
    FaultScope fault_scope;
    NvtxRange nvtx("sn_create");
    sn_status s = check_config(cfg);
    if (s) return s;
    if (!nr || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    if (cfg->dtype != SN_F32) return fail(nullptr, SN_EUNSUPPORTED, "dense networks are SN_F32 only");
    if (cfg->flags & (SN_PROP_PULL | SN_PULL_STORE_MASK))
        return fail(nullptr, SN_EUNSUPPORTED, "SN_PROP_PULL and SN_PULL_* apply to sn_create networks");
    const int n = nr->n;
    if (n < 1 || n > 200000) return fail(nullptr, SN_EINVAL, "dense n must be in 1 .. 200000");
    if (delay < 1 || delay > cfg->max_delay) return fail(nullptr, SN_EINVAL, "delay outside 1..max_delay");
    const int force_cpl = (int)((cfg->flags & SN_DENSE_SLAB_MASK) >> 8);
    if (force_cpl != 0 && force_cpl != 1 && force_cpl != 2 && force_cpl != 4 && force_cpl != 8)
        return fail(nullptr, SN_EINVAL, "SN_DENSE_SLAB(k) takes k = 1, 2, 4 or 8");
    const size_t nn = (size_t)n * n;
    for (size_t q = 0; w && q < nn; ++q)
        if (!std::isfinite(w[q]) || std::fabs(w[q]) > 1e9f) return fail(nullptr, SN_EINVAL, "weight not finite");
    sn_ctx *c = new (std::nothrow) sn_ctx();
    if (!c) return fail(nullptr, SN_ENOMEM, "host allocation failed");
    c->kind = KIND_DENSE;
    c->dtype = SN_F32;
    c->n = n;
    c->D = cfg->max_delay;
    c->D1 = c->D + 1;
    c->flags = cfg->flags;
    c->m = (long long)nn;
    c->dense_delay = delay;
    c->all_delay_one = delay == 1;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    auto bail = [&](sn_status st) { std::string msg = c->err.empty() ? g_create_err : c->err;
                                    destroy_all(c); delete c; g_create_err = msg; return st; };
    if ((s = upload_neurons(c, nr))) return bail(s);
    if ((s = alloc_common(c, cfg))) return bail(s);
    // executor: column slabs of 32 * cpl columns, one block each, co-resident
    c->block = 256;
    int grid = 0, chunk = 0;
    cudaError_t e = plan_dense(n, &grid, &chunk, force_cpl);
    if (e != cudaSuccess) { c->err = std::string("dense executor: ") + cudaGetErrorString(e); return bail(SN_ECUDA); }
    if (grid < 1) {
        c->err = force_cpl ? "the forced column slab gives no co-resident grid for this n"
                           : "dense network too large for a co-resident grid";
        return bail(SN_EUNSUPPORTED);
    }
    c->grid = grid;
    c->chunk = chunk;
    c->S = 1;
    c->ring_bytes = (size_t)c->D1 * n * 4;
    if ((s = dalloc(c, &c->W, nn * 4)) || (s = dalloc(c, &c->spk, (size_t)2 * c->words * 4)) ||
        (s = dalloc(c, &c->ring, c->ring_bytes)))
        return bail(s);
    if ((e = w ? cudaMemcpy(c->W, w, nn * 4, cudaMemcpyHostToDevice) : cudaMemset(c->W, 0, nn * 4)) ||
        (e = cudaMemset(c->spk, 0, (size_t)2 * c->words * 4)) || (e = cudaMemset(c->ring, 0, c->ring_bytes))) {
        c->err = std::string("upload: ") + cudaGetErrorString(e);
        return bail(SN_ECUDA);
    }
    *out = c;
    return SN_OK;
}

sn_status sn_set_input(sn_ctx *c, int64_t nev, const int32_t *step, const int32_t *neuron, const float *value) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE && c->kind != KIND_BATCH)
        return fail(c, SN_ESTATE, "wrong context kind");
    if (nev < 0 || (nev > 0 && (!step || !neuron || !value))) return fail(c, SN_EINVAL, "bad event arrays");
    int max_step = -1;
    for (long long e = 0; e < nev; ++e) {
        if (step[e] < 0 || step[e] >= (1 << 27)) return fail(c, SN_EINVAL, "event step outside 0 .. 2^27-1");
        if (neuron[e] < 0 || neuron[e] >= c->n) return fail(c, SN_EINVAL, "event neuron out of range");
        if (!std::isfinite(value[e])) return fail(c, SN_EINVAL, "event value not finite");
        if (c->dtype == SN_I32 && !is_int_valued(value[e])) return fail(c, SN_EINVAL, "SN_I32 event values must be integers");
        max_step = std::max(max_step, (int)step[e]);
    }
    // stable order by (step, neuron); values of one (step, neuron) summed in input order
    std::vector<long long> idx(nev);
    for (long long e = 0; e < nev; ++e) idx[e] = e;
    std::stable_sort(idx.begin(), idx.end(), [&](long long a, long long b) {
        return step[a] != step[b] ? step[a] < step[b] : neuron[a] < neuron[b];
    });
    std::vector<int> off(max_step + 2, 0), nu;
    std::vector<float> vf;
    std::vector<int> vi;
    for (long long q = 0; q < nev;) {
        long long e = idx[q];
        const int st = step[e], j = neuron[e];
        float sf = value[e];
        long long si = (long long)value[e];
        ++q;
        while (q < nev && step[idx[q]] == st && neuron[idx[q]] == j) {
            sf = sf + value[idx[q]];        // float addition in the order given
            si += (long long)value[idx[q]];
            ++q;
        }
        if (c->dtype == SN_I32 && (si > 2147483647ll || si < -2147483648ll))
            return fail(c, SN_EINVAL, "summed integer event value overflows int32");
        off[st + 1]++;
        nu.push_back(j);
        vf.push_back(sf);
        vi.push_back((int)si);
    }
    for (int t = 0; t <= max_step; ++t) off[t + 1] += off[t];
    if (sn_status q = quiesce(c)) return q;   // a queued run may read the old events
    dfree(c, c->ev_off); dfree(c, c->ev_neuron); dfree(c, c->ev_val);
    c->ev_off = c->ev_neuron = nullptr;
    c->ev_val = nullptr;
    c->ev_nsteps = 0;
    if (nev == 0) return SN_OK;
    sn_status s;
    const size_t ne = nu.size();
    if ((s = dalloc(c, &c->ev_off, off.size() * 4)) || (s = dalloc(c, &c->ev_neuron, ne * 4)) ||
        (s = dalloc(c, &c->ev_val, ne * 4)))
        return s;
    SN_CUDA(c, cudaMemcpy(c->ev_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->ev_neuron, nu.data(), ne * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->ev_val, c->dtype == SN_F32 ? (const void *)vf.data() : (const void *)vi.data(),
                          ne * 4, cudaMemcpyHostToDevice));
    c->ev_nsteps = max_step + 1;
    return SN_OK;
}

sn_status sn_set_poisson(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                         const float *amp, uint64_t seed) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE && c->kind != KIND_BATCH && c->kind != KIND_SHARED_I8)
        return fail(c, SN_ESTATE, "wrong context kind");
    if (nsrc < 0 || (nsrc > 0 && (!neuron || !rate || !amp))) return fail(c, SN_EINVAL, "bad source arrays");
    if (c->kind == KIND_BATCH) return batch_set_poisson(c, nsrc, neuron, rate, amp, seed, 0);
    if (c->kind == KIND_SHARED_I8) return shared_set_poisson(c, nsrc, neuron, rate, amp, seed, 0);
    const int n = c->n;
    std::vector<unsigned> thr(n, 0u);
    std::vector<float> af(n, 0.0f);
    std::vector<int> ai(n, 0);
    std::vector<char> used(n, 0);
    for (int k = 0; k < nsrc; ++k) {
        const int j = neuron[k];
        if (j < 0 || j >= n) return fail(c, SN_EINVAL, "source neuron out of range");
        if (used[j]) return fail(c, SN_EINVAL, "a neuron may have at most one Poisson source");
        if (!(rate[k] >= 0.0f) || !std::isfinite(rate[k])) return fail(c, SN_EINVAL, "rate must be finite and >= 0");
        if (!std::isfinite(amp[k])) return fail(c, SN_EINVAL, "amplitude not finite");
        if (c->dtype == SN_I32 && !is_int_valued(amp[k])) return fail(c, SN_EINVAL, "SN_I32 amplitudes must be integers");
        used[j] = 1;
        thr[j] = rate_threshold(rate[k]);
        af[j] = amp[k];
        ai[j] = (int)amp[k];
    }
    if (sn_status q = quiesce(c)) return q;   // a queued run may read the old sources
    SN_CUDA(c, cudaMemcpy(c->prate, thr.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pamp, c->dtype == SN_F32 ? (const void *)af.data() : (const void *)ai.data(),
                          (size_t)n * 4, cudaMemcpyHostToDevice));
    c->pkey = host_splitmix64(seed ^ host_splitmix64(0ull));
    return SN_OK;
}

sn_status sn_set_poisson_stream(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                                const float *amp, uint64_t seed, uint64_t net) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind == KIND_BATCH || c->kind == KIND_SHARED_I8) {
        if (nsrc < 0 || (nsrc > 0 && (!neuron || !rate || !amp))) return fail(c, SN_EINVAL, "bad source arrays");
        return c->kind == KIND_BATCH ? batch_set_poisson(c, nsrc, neuron, rate, amp, seed, net)
                                     : shared_set_poisson(c, nsrc, neuron, rate, amp, seed, net);
    }
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE) return fail(c, SN_ESTATE, "wrong context kind");
    sn_status s = sn_set_poisson(c, nsrc, neuron, rate, amp, seed);
    if (s) return s;
    c->pkey = host_splitmix64(seed ^ host_splitmix64(net));
    return SN_OK;
}

sn_status sn_stdp(sn_ctx *c, float decay, float a_plus, float a_minus, float wmin, float wmax, int32_t enable) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE) return fail(c, SN_EUNSUPPORTED, "STDP: single networks only");
    if (c->shard_end && enable) return fail(c, SN_EUNSUPPORTED, "STDP is not available for a shard");
    if (!enable) { c->stdp = 0; return SN_OK; }
    if (c->dtype != SN_F32) return fail(c, SN_EUNSUPPORTED, "STDP needs an SN_F32 network");
    if (!c->all_delay_one)
        return fail(c, SN_EUNSUPPORTED, "STDP needs every synaptic delay to be 1 (weights apply at emission)");
    if (!(std::isfinite(decay) && std::isfinite(a_plus) && std::isfinite(a_minus) && std::isfinite(wmin) &&
          std::isfinite(wmax) && wmin <= wmax))
        return fail(c, SN_EINVAL, "bad STDP parameters");
    if (sn_status q = quiesce(c)) return q;   // queued runs use the current rule and weights
    if (!c->trace) {
        sn_status s = dalloc(c, &c->trace, (size_t)3 * c->n * 4);
        if (s) return s;
        SN_CUDA(c, cudaMemset(c->trace, 0, (size_t)3 * c->n * 4));
    }
    if (c->kind == KIND_SPARSE && !c->csc) {
        // CSC by post: {pre, CSR position}
        const int n = c->n;
        const long long m = c->m;
        std::vector<uint2> syn(m > 0 ? m : 1);
        std::vector<long long> rowptr(n + 1);
        SN_CUDA(c, cudaMemcpy(syn.data(), c->syn, (size_t)(m > 0 ? m : 1) * 8, cudaMemcpyDeviceToHost));
        SN_CUDA(c, cudaMemcpy(rowptr.data(), c->rowptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost));
        if (m >= (1ll << 32)) return fail(c, SN_EUNSUPPORTED, "STDP supports m < 2^32");
        std::vector<long long> colptr(n + 1, 0);
        for (long long p = 0; p < m; ++p) colptr[(syn[p].x & kPostMask) + 1]++;
        for (int j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
        std::vector<uint2> csc(m > 0 ? m : 1);
        std::vector<long long> fill(colptr.begin(), colptr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (long long p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int j = (int)(syn[p].x & kPostMask);
                csc[fill[j]++] = make_uint2((unsigned)i, (unsigned)p);
            }
        sn_status s;
        if ((s = dalloc(c, &c->colptr, (size_t)(n + 1) * 8)) || (s = dalloc(c, &c->csc, (size_t)(m > 0 ? m : 1) * 8)))
            return s;
        SN_CUDA(c, cudaMemcpy(c->colptr, colptr.data(), (size_t)(n + 1) * 8, cudaMemcpyHostToDevice));
        SN_CUDA(c, cudaMemcpy(c->csc, csc.data(), (size_t)(m > 0 ? m : 1) * 8, cudaMemcpyHostToDevice));
    }
    c->stdp = 1;
    c->prop_pull = 0;                  // STDP rewrites the CSR weights: push propagation
    c->decay = decay; c->a_plus = a_plus; c->a_minus = a_minus; c->wmin = wmin; c->wmax = wmax;
    return SN_OK;
}

static sn_status read_status(sn_ctx *c) {
    Control h;
    SN_CUDA(c, cudaMemcpy(&h, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    if (h.status != 0) {
        c->failed = h.status;
        return fail(c, (sn_status)h.status, h.status == SN_ETIMEOUT ? "a grid barrier wait timed out on the device"
                                            : h.status == SN_EOVERFLOW ? "integer state overflowed int32"
                                                                       : "device status latched");
    }
    return SN_OK;
}

sn_status sn_run(sn_ctx *c, int32_t steps) {
    NvtxRange nvtx("sn_run");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->failed) return fail(c, SN_ESTATE, "context has a latched device error");
    if (steps < 0) return fail(c, SN_EINVAL, "steps < 0");
    if (steps == 0) return SN_OK;
    if (c->step + steps >= (1ll << 31)) return fail(c, SN_EINVAL, "step counter would exceed 2^31");
    if (c->kind == KIND_BATCH || c->kind == KIND_SHARED_I8) {
        sn_status st = c->kind == KIND_BATCH ? batch_run(c, steps) : shared_run(c, steps);
        if (st) return st;
        c->step += steps;
        if (c->step - c->raster_from > c->cap) c->raster_from = c->step - c->cap;
        return SN_OK;
    }
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE) return fail(c, SN_ESTATE, "wrong context kind");
    if (c->shard_end) {
        // a shard runs at most the smallest delay's worth of steps, and only
        // once the other shards' spikes of every earlier step are in
        if (c->shard_known < c->step)
            return fail(c, SN_ESTATE, "shard: the other shards' spikes of steps " + std::to_string(c->shard_known) +
                                          " .. " + std::to_string(c->step - 1) + " are not in (sn_shard_put_spikes)");
        if (steps > c->shard_dmin)
            return fail(c, SN_EINVAL, "shard: a run may take at most the smallest synaptic delay (" +
                                          std::to_string(c->shard_dmin) + ") steps between exchanges");
    }
    NetArgs a;
    memset(&a, 0, sizeof(a));
    a.n = c->n; a.D1 = c->D1; a.words = c->words; a.cap = c->cap;
    a.t0 = (int)c->step; a.steps = steps; a.chunk = c->chunk;
    a.V = c->V; a.r = c->r; a.th = c->th; a.lk = c->lk; a.rs = c->rs; a.R = c->R;
    a.prate = c->prate; a.pamp = c->pamp; a.pkey = c->pkey;
    a.ev_off = c->ev_off; a.ev_nsteps = c->ev_nsteps; a.ev_neuron = c->ev_neuron; a.ev_val = c->ev_val;
    a.rowptr = c->rowptr; a.syn = c->syn; a.colptr = c->colptr; a.csc = c->csc;
    a.ring = c->ring;
    a.W = c->W; a.partial = c->partial; a.S = c->S; a.dense_delay = c->dense_delay; a.spk = c->spk;
    a.raster = c->raster;
    a.stdp = c->stdp; a.decay = c->decay; a.a_plus = c->a_plus; a.a_minus = c->a_minus;
    a.wmin = c->wmin; a.wmax = c->wmax; a.trace = c->trace;
    a.ctl = c->ctl;
    a.hist = c->hist; a.hD = c->D;
    cudaError_t e;
    if (c->kind == KIND_SPARSE && c->prop_pull && !c->stdp) {
        if (c->pin_stale) {
            sn_status st = build_pull_store(c);
            if (st) return st;
        }
        a.pin = c->pin; a.pin_off = c->pin_off; a.pin_len = c->pin_len; a.pin_len1 = c->pin_len1;
        a.pin_y0 = c->pin_y0; a.pin_perm = c->pin_perm;
        a.ring_until = (int)std::min<long long>(c->ring_live_until, 2147483647ll);
        a.hL = c->pull_rows;
        a.chunk = c->pull_chunk;
        a.j_first = c->shard_end ? c->shard_first : 0;
        a.j_end = c->shard_end ? c->shard_end : c->n;
        e = launch_sparse_pull(a, c->dtype, c->pin_coded != 0, c->pull_grid, c->pull_smem, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "simulation launch");
        c->hist_live = true;
    } else {
        if (c->kind == KIND_SPARSE && c->hist_live) {
            // spikes of a pull run whose deliveries are still due go to the ring
            if ((e = launch_pull_flush(a, c->dtype, (int)c->step, c->stream)) != cudaSuccess ||
                (e = cudaMemsetAsync(c->hist, 0, (size_t)c->D * c->words * 4, c->stream)) != cudaSuccess)
                return cuda_fail(c, e, "pull-to-push handover");
            c->hist_live = false;
        }
        if (c->kind == KIND_SPARSE && !c->stdp && c->reg_grid > 0) {
            a.chunk = c->reg_chunk;
            e = launch_sparse_reg(a, c->dtype, c->reg_grid, c->stream);
        } else {
            e = c->kind == KIND_SPARSE ? launch_sparse(a, c->dtype, c->grid, c->block, c->stream)
                                       : launch_dense(a, c->grid, c->block, c->stream);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "simulation launch");
        c->ring_live_until = c->step + steps + c->D;
        if (c->stdp) c->pin_stale = true;
    }
    c->step += steps;
    if (c->step - c->raster_from > c->cap) c->raster_from = c->step - c->cap;
    return SN_OK;
}

sn_status sn_reset(sn_ctx *c) {
    NvtxRange nvtx("sn_reset");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind == KIND_SHARED_I8) {
        const size_t bn = (size_t)c->sh_B * c->n;
        SN_CUDA(c, cudaMemcpyAsync(c->V, c->sh_V0, bn * 4, cudaMemcpyDeviceToDevice, c->stream));
        SN_CUDA(c, cudaMemsetAsync(c->r, 0, bn * 4, c->stream));
        SN_CUDA(c, cudaMemsetAsync(c->sh_A0, 0, bn, c->stream));
        SN_CUDA(c, cudaMemsetAsync(c->sh_A1, 0, bn, c->stream));
        SN_CUDA(c, cudaMemsetAsync(c->raster, 0, (size_t)c->cap * c->words * 4, c->stream));
        SN_CUDA(c, cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->stream));
        c->step = 0;
        c->raster_from = 0;
        c->failed = 0;
        return SN_OK;
    }
    if (c->kind != KIND_SPARSE && c->kind != KIND_DENSE && c->kind != KIND_BATCH)
        return fail(c, SN_ESTATE, "wrong context kind");
    const size_t vb = (size_t)c->n * 4;
    SN_CUDA(c, cudaMemcpyAsync(c->V, c->rs, vb, cudaMemcpyDeviceToDevice, c->stream));
    SN_CUDA(c, cudaMemsetAsync(c->r, 0, vb, c->stream));
    SN_CUDA(c, cudaMemsetAsync(c->ring, 0, c->ring_bytes, c->stream));
    if (c->spk) SN_CUDA(c, cudaMemsetAsync(c->spk, 0, (size_t)2 * c->words * 4, c->stream));
    if (c->trace) SN_CUDA(c, cudaMemsetAsync(c->trace, 0, 3 * vb, c->stream));
    if (c->hist) SN_CUDA(c, cudaMemsetAsync(c->hist, 0, (size_t)c->D * c->words * 4, c->stream));
    c->hist_live = false;
    c->ring_live_until = 0;
    c->shard_known = 0;
    SN_CUDA(c, cudaMemsetAsync(c->raster, 0, (size_t)c->cap * c->words * 4, c->stream));
    SN_CUDA(c, cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->stream));
    c->step = 0;
    c->raster_from = 0;
    c->failed = 0;
    return SN_OK;
}

sn_status sn_sync(sn_ctx *c) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

static sn_status copy_out(sn_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
    if (on_device) {
        SN_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return SN_OK;
    }
    SN_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

sn_status sn_get_spikes(sn_ctx *c, int64_t t0, int64_t t1, uint32_t *bits, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (t0 < 0 || t1 < t0 || t1 > c->step) return fail(c, SN_EINVAL, "steps not yet run");
    if (t0 < c->raster_from) return fail(c, SN_EINVAL, "steps older than the raster capacity (record_steps)");
    if (t1 == t0) return SN_OK;
    if (!bits) return fail(c, SN_EINVAL, "bits is NULL");
    const size_t row = (size_t)c->words * 4;
    // rows are a ring indexed by step % cap: copy the contiguous pieces
    long long t = t0;
    while (t < t1) {
        const long long slot = t % c->cap;
        const long long len = std::min<long long>(t1 - t, c->cap - slot);
        uint8_t *dst = (uint8_t *)bits + (size_t)(t - t0) * row;
        const uint8_t *src = (const uint8_t *)c->raster + (size_t)slot * row;
        cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)len * row,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "raster copy");
        t += len;
    }
    if (on_device) return SN_OK;
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

sn_status sn_get_state(sn_ctx *c, void *v, int32_t *refr, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    sn_status s;
    if (c->kind == KIND_FF) return fail(c, SN_ESTATE, "feedforward contexts: use sn_ff_get_checkpoints");
    if (c->kind == KIND_SHARED_I8) {
        if ((s = shared_get_state(c, v, refr, on_device))) return s;
        return on_device ? SN_OK : read_status(c);
    }
    const size_t bytes = (size_t)state_elems(c) * 4;
    if (v && (s = copy_out(c, v, c->V, bytes, on_device))) return s;
    if (refr && (s = copy_out(c, refr, c->r, bytes, on_device))) return s;
    return SN_OK;
}

sn_status sn_get_trace(sn_ctx *c, float *x, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (!x) return fail(c, SN_EINVAL, "trace is NULL");
    if (!c->trace) return fail(c, SN_ESTATE, "STDP was never enabled");
    const int buf = c->kind == KIND_DENSE ? (int)((c->step + 2) % 3)
                                          : (c->step > 0 ? (int)((c->step - 1) & 1) : 1);
    return copy_out(c, x, c->trace + (size_t)buf * c->n, (size_t)c->n * 4, on_device);
}

sn_status sn_get_weights(sn_ctx *c, float *w, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (!w) return fail(c, SN_EINVAL, "w is NULL");
    if (c->kind == KIND_DENSE) return copy_out(c, w, c->W, (size_t)c->n * c->n * 4, on_device);
    if (c->kind != KIND_SPARSE) return fail(c, SN_ESTATE, "wrong context kind");
    if (c->m == 0) return SN_OK;
    if (c->dtype != SN_F32) return fail(c, SN_EUNSUPPORTED, "weights of SN_I32 networks are never changed");
    if (!c->perm_inv) {
        sn_status s = dalloc(c, &c->perm_inv, (size_t)c->m * 8);
        if (s) return s;
        SN_CUDA(c, cudaMemcpy(c->perm_inv, c->h_perm_inv.data(), (size_t)c->m * 8, cudaMemcpyHostToDevice));
    }
    float *dst = w;
    float *tmp = nullptr;
    if (!on_device) {
        sn_status s = dalloc(c, &tmp, (size_t)c->m * 4);
        if (s) return s;
        dst = tmp;
    }
    cudaError_t e = launch_gather_weights(c->syn, c->perm_inv, c->m, dst, c->stream);
    if (e != cudaSuccess) { dfree(c, tmp); return cuda_fail(c, e, "weight gather"); }
    if (!on_device) {
        e = cudaMemcpyAsync(w, tmp, (size_t)c->m * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dfree(c, tmp);
        if (e != cudaSuccess) return cuda_fail(c, e, "weight copy");
        return read_status(c);
    }
    return SN_OK;
}

// Spikes in flight (emitted at step tau < t0, arriving at tau + d >= t0) are
// delivered with the weights in place when they arrive.  After the weights
// change, the pending input is rebuilt from the spike rows of the last D
// steps (the raster): pull keeps them as its history, push re-sends them into
// a cleared ring with the new weights.
static sn_status rebuild_pending(sn_ctx *c) {
    const long long t0 = c->step;
    const int D = c->D;
    const long long first = std::max<long long>(0, t0 - D);
    if (first >= t0) return SN_OK;                      // nothing emitted yet
    if (first < c->raster_from || t0 - first > c->cap)
        return fail(c, SN_EUNSUPPORTED, "spikes in flight are older than the raster (record_steps < max_delay)");
    const size_t row = (size_t)c->words * 4;
    if (!c->hist) {
        sn_status s = dalloc(c, &c->hist, (size_t)D * row);
        if (s) return s;
    }
    SN_CUDA(c, cudaMemsetAsync(c->hist, 0, (size_t)D * row, c->stream));
    for (long long tau = first; tau < t0; ++tau)
        SN_CUDA(c, cudaMemcpyAsync((char *)c->hist + (size_t)(tau % D) * row,
                                   (const char *)c->raster + (size_t)(tau % c->cap) * row, row,
                                   cudaMemcpyDeviceToDevice, c->stream));
    SN_CUDA(c, cudaMemsetAsync(c->ring, 0, c->ring_bytes, c->stream));
    if (c->prop_pull && !c->stdp) {
        c->hist_live = true;
        c->ring_live_until = t0;
        return SN_OK;
    }
    NetArgs a;
    memset(&a, 0, sizeof(a));
    a.n = c->n; a.D1 = c->D1; a.words = c->words;
    a.rowptr = c->rowptr; a.syn = c->syn; a.ring = c->ring; a.hist = c->hist; a.hD = D;
    cudaError_t e = launch_pull_flush(a, c->dtype, (int)t0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pending input rebuild");
    SN_CUDA(c, cudaMemsetAsync(c->hist, 0, (size_t)D * row, c->stream));
    c->hist_live = false;
    c->ring_live_until = t0 + D;
    return SN_OK;
}

sn_status sn_set_weights(sn_ctx *c, const float *w, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (!w) return fail(c, SN_EINVAL, "w is NULL");
    if (c->failed) return fail(c, SN_ESTATE, "context is in an error state");
    if (c->shard_end) return fail(c, SN_EUNSUPPORTED, "the weights of a shard are fixed at creation");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->kind == KIND_DENSE) {
        if (c->step != 0)
            return fail(c, SN_ESTATE, "dense weights change only at step 0 (after creation, sn_reset or a load)");
        SN_CUDA(c, cudaMemcpyAsync(c->W, w, (size_t)c->n * c->n * 4, kind, c->stream));
        if (!on_device) SN_CUDA(c, cudaStreamSynchronize(c->stream));
        return SN_OK;
    }
    if (c->kind != KIND_SPARSE) return fail(c, SN_ESTATE, "wrong context kind");
    if (c->dtype != SN_F32) return fail(c, SN_EUNSUPPORTED, "weights of SN_I32 networks are fixed at creation");
    if (c->m == 0) return SN_OK;
    if (sn_status q = quiesce(c)) return q;    // queued runs read the current weights
    if (!c->perm_inv) {
        sn_status s = dalloc(c, &c->perm_inv, (size_t)c->m * 8);
        if (s) return s;
        SN_CUDA(c, cudaMemcpy(c->perm_inv, c->h_perm_inv.data(), (size_t)c->m * 8, cudaMemcpyHostToDevice));
    }
    const float *src = w;
    float *tmp = nullptr;
    if (!on_device) {
        for (long long k = 0; k < c->m; ++k)
            if (std::isnan(w[k])) return fail(c, SN_EINVAL, "NaN weight");
        sn_status s = dalloc(c, &tmp, (size_t)c->m * 4);
        if (s) return s;
        cudaError_t e = cudaMemcpyAsync(tmp, w, (size_t)c->m * 4, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) { dfree(c, tmp); return cuda_fail(c, e, "weight upload"); }
        src = tmp;
    }
    cudaError_t e = launch_scatter_weights(c->syn, c->perm_inv, c->m, src, c->stream);
    if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(c->stream);
    dfree(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "weight scatter");
    c->pin_stale = true;                       // the pull store holds copies of the weights
    return rebuild_pending(c);
}

sn_status sn_get_counters(sn_ctx *c, int64_t *steps, int64_t *spikes, int64_t *events) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    Control h;
    SN_CUDA(c, cudaMemcpy(&h, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    if (steps) *steps = c->step;
    if (spikes) *spikes = (int64_t)h.spikes;
    if (events) *events = (int64_t)h.events;
    return read_status(c);
}

// Checkpoint layout: header, V, r, ring, spike bits (dense), trace (if any),
// weights (sparse CSR words or dense W), spike history of a pull run (if its
// deliveries may be due), counters in the header.
struct SaveHeader {
    char magic[8];
    int kind, dtype, n, D1, S, has_trace, has_hist;
    int count;                // batched: networks; shared: input trains; else 0
    long long m, step;
    unsigned long long spikes, events;
};

static int save_count(const sn_ctx *c) {
    return c->kind == KIND_BATCH ? c->nets : c->kind == KIND_SHARED_I8 ? c->sh_B : 0;
}

// Checkpoint layout after the header, by kind:
//   sparse:  V, r, ring, synapse store, [traces], [spike history]
//   dense:   V, r, ring, spike words, W, [traces]
//   batched: V, r, ring (the synapses never change)
//   shared:  V, r ([n][trains]), both spike operands (the weights never change)
static size_t save_size(const sn_ctx *c, bool has_trace, bool has_hist) {
    if (c->kind == KIND_SHARED_I8) {
        const size_t bn = (size_t)c->sh_B * c->n;
        return sizeof(SaveHeader) + bn * 8 + bn * 2;
    }
    size_t s = sizeof(SaveHeader) + (size_t)c->n * 8 + c->ring_bytes;
    if (c->kind == KIND_DENSE) s += (size_t)2 * c->words * 4 + (size_t)c->n * c->n * 4;
    else if (c->kind == KIND_SPARSE) s += (size_t)(c->m > 0 ? c->m : 0) * 8;
    if (has_trace) s += (size_t)3 * c->n * 4;
    if (has_hist) s += (size_t)c->D * c->words * 4;
    return s;
}

static bool can_save(const sn_ctx *c) {
    return !c->shard_end &&
           (c->kind == KIND_SPARSE || c->kind == KIND_DENSE || c->kind == KIND_BATCH || c->kind == KIND_SHARED_I8);
}

sn_status sn_save(sn_ctx *c, void *buf, size_t *size) {
    NvtxRange nvtx("sn_save");
    if (!c || !size) return fail(c, SN_EINVAL, "NULL argument");
    if (!can_save(c)) return fail(c, SN_ESTATE, "wrong context kind");
    const bool has_hist = c->kind == KIND_SPARSE && c->hist_live;
    const size_t need = save_size(c, c->trace != nullptr, has_hist);
    if (!buf) { *size = need; return SN_OK; }
    if (*size < need) return fail(c, SN_EINVAL, "buffer too small");
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    sn_status st = read_status(c);
    if (st) return st;
    Control h;
    SN_CUDA(c, cudaMemcpy(&h, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    SaveHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "SNCKPT2", 8);
    hd.kind = c->kind; hd.dtype = c->dtype; hd.n = c->n; hd.D1 = c->D1; hd.S = c->S;
    hd.has_trace = c->trace != nullptr; hd.has_hist = has_hist; hd.m = c->m; hd.step = c->step;
    hd.count = save_count(c);
    hd.spikes = h.spikes; hd.events = h.events;
    uint8_t *p = (uint8_t *)buf;
    memcpy(p, &hd, sizeof(hd)); p += sizeof(hd);
    auto get = [&](const void *src, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMemcpy(p, src, bytes, cudaMemcpyDeviceToHost);
        p += bytes;
        return e;
    };
    cudaError_t e;
    if (c->kind == KIND_SHARED_I8) {
        const size_t bn = (size_t)c->sh_B * c->n;
        if ((e = get(c->V, bn * 4)) || (e = get(c->r, bn * 4)) || (e = get(c->sh_A0, bn)) || (e = get(c->sh_A1, bn)))
            return cuda_fail(c, e, "save");
        *size = need;
        return SN_OK;
    }
    if ((e = get(c->V, (size_t)c->n * 4)) || (e = get(c->r, (size_t)c->n * 4)) || (e = get(c->ring, c->ring_bytes)))
        return cuda_fail(c, e, "save");
    if (c->kind == KIND_DENSE) {
        if ((e = get(c->spk, (size_t)2 * c->words * 4)) || (e = get(c->W, (size_t)c->n * c->n * 4)))
            return cuda_fail(c, e, "save");
    } else if (c->kind == KIND_SPARSE && c->m > 0 && (e = get(c->syn, (size_t)c->m * 8))) {
        return cuda_fail(c, e, "save");
    }
    if (c->trace && (e = get(c->trace, (size_t)3 * c->n * 4))) return cuda_fail(c, e, "save");
    if (has_hist && (e = get(c->hist, (size_t)c->D * c->words * 4))) return cuda_fail(c, e, "save");
    *size = need;
    return SN_OK;
}

sn_status sn_load(sn_ctx *c, const void *buf, size_t size) {
    NvtxRange nvtx("sn_load");
    if (!c || !buf) return fail(c, SN_EINVAL, "NULL argument");
    if (size < sizeof(SaveHeader)) return fail(c, SN_EINVAL, "buffer too small");
    SaveHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "SNCKPT2", 8) != 0) return fail(c, SN_EINVAL, "not a checkpoint");
    if (!can_save(c)) return fail(c, SN_ESTATE, "wrong context kind");
    if (hd.kind != c->kind || hd.dtype != c->dtype || hd.n != c->n || hd.D1 != c->D1 || hd.m != c->m ||
        hd.S != c->S || hd.count != save_count(c) || (hd.has_hist && c->kind != KIND_SPARSE) ||
        (hd.has_trace && c->kind != KIND_SPARSE && c->kind != KIND_DENSE))
        return fail(c, SN_EINVAL, "checkpoint is of a different network");
    if (size < save_size(c, hd.has_trace != 0, hd.has_hist != 0)) return fail(c, SN_EINVAL, "checkpoint truncated");
    sn_status s;
    if (hd.has_trace && !c->trace && (s = dalloc(c, &c->trace, (size_t)3 * c->n * 4))) return s;
    if (hd.has_hist && !c->hist && (s = dalloc(c, &c->hist, (size_t)c->D * c->words * 4))) return s;
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    const uint8_t *p = (const uint8_t *)buf + sizeof(hd);
    auto put = [&](void *dst, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMemcpy(dst, p, bytes, cudaMemcpyHostToDevice);
        p += bytes;
        return e;
    };
    cudaError_t e;
    if (c->kind == KIND_SHARED_I8) {
        const size_t bn = (size_t)c->sh_B * c->n;
        if ((e = put(c->V, bn * 4)) || (e = put(c->r, bn * 4)) || (e = put(c->sh_A0, bn)) || (e = put(c->sh_A1, bn)))
            return cuda_fail(c, e, "load");
    } else {
        if ((e = put(c->V, (size_t)c->n * 4)) || (e = put(c->r, (size_t)c->n * 4)) ||
            (e = put(c->ring, c->ring_bytes)))
            return cuda_fail(c, e, "load");
    }
    if (c->kind == KIND_DENSE) {
        if ((e = put(c->spk, (size_t)2 * c->words * 4)) || (e = put(c->W, (size_t)c->n * c->n * 4)))
            return cuda_fail(c, e, "load");
    } else if (c->kind == KIND_SPARSE && c->m > 0 && (e = put(c->syn, (size_t)c->m * 8))) {
        return cuda_fail(c, e, "load");
    }
    if (hd.has_trace && (e = put(c->trace, (size_t)3 * c->n * 4))) return cuda_fail(c, e, "load");
    if (hd.has_hist) {
        if ((e = put(c->hist, (size_t)c->D * c->words * 4))) return cuda_fail(c, e, "load");
    } else if (c->hist) {
        SN_CUDA(c, cudaMemset(c->hist, 0, (size_t)c->D * c->words * 4));
    }
    if (c->kind == KIND_SPARSE) {
        c->hist_live = hd.has_hist != 0;
        c->ring_live_until = hd.step + c->D;   // the loaded ring may hold pending input
        c->pin_stale = true;                   // the loaded weights replace the CSR's
    }
    Control h;
    memset(&h, 0, sizeof(h));
    h.spikes = hd.spikes;
    h.events = hd.events;
    SN_CUDA(c, cudaMemcpy(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice));
    c->step = hd.step;
    c->raster_from = hd.step;
    c->failed = 0;
    return SN_OK;
}

// Propagation of a sparse network: push (SN_PUSH, every spike adds its
// weights to the pending input of its targets) or pull (SN_PULL).
sn_status sn_set_propagation(sn_ctx *c, int32_t mode) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_SPARSE) return fail(c, SN_EUNSUPPORTED, "propagation mode: sparse single networks only");
    if (c->shard_end && mode != SN_PULL) return fail(c, SN_EUNSUPPORTED, "a shard runs pull propagation only");
    if (mode == SN_PUSH) { c->prop_pull = 0; return SN_OK; }
    if (mode != SN_PULL) return fail(c, SN_EINVAL, "mode must be SN_PUSH or SN_PULL");
    return select_pull(c);
}

sn_status sn_get_propagation(const sn_ctx *c, int32_t *mode) {
    if (!c || !mode) return SN_EINVAL;
    *mode = (c->kind == KIND_SPARSE && c->prop_pull && !c->stdp) ? SN_PULL : SN_PUSH;
    return SN_OK;
}

sn_status sn_pull_store_info(const sn_ctx *c, int32_t *format, int64_t *bytes, int64_t *entries) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_SPARSE) return fail(nullptr, SN_EINVAL, "not a sparse network");
    const bool built = c->pin != nullptr && c->pin_bytes > 0;
    if (format) *format = !built ? 0 : c->pin_coded ? (int32_t)SN_PULL_CODED : (int32_t)SN_PULL_PLAIN;
    if (bytes) *bytes = built ? c->pin_bytes : 0;
    if (entries) *entries = built ? c->pin_entries : 0;
    return SN_OK;
}

void sn_destroy(sn_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    destroy_all(c);
    delete c;
}

}  // extern "C"

namespace sn {

// sn_autotune on a sparse network: time push and (where the network fits it)
// pull propagation on trial_steps steps from the initial state, keep the
// faster, reset.  The second of two runs of each is timed (the first also
// pays first-launch costs).
sn_status sparse_autotune(sn_ctx *c, int trial_steps, float *best_ms) {
    cudaEvent_t e0, e1;
    SN_CUDA(c, cudaEventCreate(&e0));
    SN_CUDA(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_pull = 0;
    sn_status st = SN_OK;
    for (int pull = 0; pull < 2 && st == SN_OK; ++pull) {
        if (pull) {
            if (c->stdp || select_pull(c) != SN_OK) { c->err.clear(); break; }
        } else {
            c->prop_pull = 0;
        }
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && st == SN_OK; ++rep) {
            if ((st = sn_reset(c))) break;
            cudaEventRecord(e0, c->stream);
            if ((st = sn_run(c, trial_steps))) break;
            cudaEventRecord(e1, c->stream);
            if ((st = sn_sync(c))) break;
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (st == SN_OK && ms < best) { best = ms; best_pull = pull; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    c->prop_pull = best_pull;
    if ((st = sn_reset(c))) return st;
    if (best_ms) *best_ms = best;
    return sn_sync(c);
}

}  // namespace sn
