// Host side of batched contexts: many independent networks in one context,
// simulated by one persistent kernel launch (sn_batch.cu) replayed from a
// CUDA graph, with an autotuner for the executor mapping.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "sn_ctx.h"

namespace sn {

// Queues: networks above the warp threshold run on whole blocks, the others
// on single warps; both largest first.
static sn_status batch_upload_orders(sn_ctx *c) {
    std::vector<int> big, small;
    for (int b = 0; b < c->nets; ++b) (c->h_net_n[b] > c->warp_max_n ? big : small).push_back(b);
    auto by_size = [&](int x, int y) { return c->h_net_n[x] != c->h_net_n[y] ? c->h_net_n[x] > c->h_net_n[y] : x < y; };
    std::sort(big.begin(), big.end(), by_size);
    std::sort(small.begin(), small.end(), by_size);
    c->n_cta = (int)big.size();
    c->n_warp = (int)small.size();
    if (!big.empty()) SN_CUDA(c, cudaMemcpy(c->cta_order, big.data(), big.size() * 4, cudaMemcpyHostToDevice));
    if (!small.empty()) SN_CUDA(c, cudaMemcpy(c->warp_order, small.data(), small.size() * 4, cudaMemcpyHostToDevice));
    return SN_OK;
}

static void batch_drop_graph(sn_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_kernel = nullptr;
}

static BatchArgs batch_args(sn_ctx *c, int steps) {
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.nets = c->nets; a.t0 = (int)c->step; a.steps = steps; a.cap = c->cap; a.total_words = c->words;
    a.D1 = c->D1;
    a.net_off = c->net_off; a.word_off = c->word_off; a.ring_off = c->ring_off; a.pkey = c->pkeys;
    a.cta_order = c->cta_order; a.n_cta = c->n_cta; a.warp_order = c->warp_order; a.n_warp = c->n_warp;
    a.V = c->V; a.r = c->r; a.th = c->th; a.lk = c->lk; a.rs = c->rs; a.R = c->R;
    a.prate = c->prate; a.pamp = c->pamp;
    a.ev_off = c->ev_off; a.ev_nsteps = c->ev_nsteps; a.ev_neuron = c->ev_neuron; a.ev_val = c->ev_val;
    a.rowptr = c->rowptr; a.sidx = c->sidx; a.sw = c->sw;
    a.ring = c->ring; a.raster = c->raster; a.ring_smem = c->ring_smem; a.ctl = c->ctl;
    return a;
}

// One persistent launch, replayed from a graph (queue reset + kernel); only
// the kernel's arguments (first step, step count) change between runs.
sn_status batch_run(sn_ctx *c, int steps) {
    BatchArgs a = batch_args(c, steps);
    void *fn = nullptr;
    batch_kernel_node(c->dtype, &fn);
    void *args[] = {(void *)&a};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = fn;
    kp.gridDim = dim3(c->batch_grid);
    kp.blockDim = dim3(kBatchBlock);
    kp.sharedMemBytes = (unsigned)batch_smem(c->ring_smem);
    kp.kernelParams = args;
    if (!c->graph_exec) {
        SN_CUDA(c, cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kp.sharedMemBytes));
        SN_CUDA(c, cudaGraphCreate(&c->graph, 0));
        cudaMemsetParams mp;
        memset(&mp, 0, sizeof(mp));
        mp.dst = (void *)&c->ctl->queue[0];
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 2;
        mp.height = 1;
        cudaGraphNode_t mnode;
        SN_CUDA(c, cudaGraphAddMemsetNode(&mnode, c->graph, nullptr, 0, &mp));
        SN_CUDA(c, cudaGraphAddKernelNode(&c->graph_kernel, c->graph, &mnode, 1, &kp));
        SN_CUDA(c, cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
    } else {
        SN_CUDA(c, cudaGraphExecKernelNodeSetParams(c->graph_exec, c->graph_kernel, &kp));
    }
    SN_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
    return SN_OK;
}

static sn_status batch_size_grid(sn_ctx *c) {
    int g = 0;
    cudaError_t e = max_grid_batch(c->dtype, c->ring_smem, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch occupancy");
    if (g < 1) return fail(c, SN_EUNSUPPORTED, "batched kernel cannot be resident with this shared memory");
    c->batch_grid = g;
    batch_drop_graph(c);
    return SN_OK;
}

sn_status batch_set_poisson(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                            const float *amp, uint64_t seed, uint64_t net0) {
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
    std::vector<unsigned long long> keys(c->nets);
    for (int b = 0; b < c->nets; ++b) keys[b] = host_splitmix64(seed ^ host_splitmix64(net0 + (unsigned long long)b));
    if (sn_status q = quiesce(c)) return q;   // a queued run may read the old sources
    SN_CUDA(c, cudaMemcpy(c->prate, thr.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pamp, c->dtype == SN_F32 ? (const void *)af.data() : (const void *)ai.data(),
                          (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pkeys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice));
    return SN_OK;
}

}  // namespace sn

extern "C" {

sn_status sn_create_batch(const sn_config *cfg, int32_t nets, const sn_neurons *neurons,
                          const sn_synapses *synapses, sn_ctx **out) {
    sn::FaultScope fault_scope;
    if (!cfg || !neurons || !synapses || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    if (cfg->dtype != SN_F32 && cfg->dtype != SN_I32) return fail(nullptr, SN_EINVAL, "bad dtype");
    if (cfg->max_delay < 1 || cfg->max_delay > kBatchMaxDelay)
        return fail(nullptr, SN_EINVAL, "batched contexts support max_delay 1..16");
    if (cfg->record_steps < 0) return fail(nullptr, SN_EINVAL, "record_steps < 0");
    if (nets < 1) return fail(nullptr, SN_EINVAL, "nets must be >= 1");
    long long ntot = 0, mtot = 0, wtot = 0;
    for (int b = 0; b < nets; ++b) {
        const sn_neurons &nr = neurons[b];
        const sn_synapses &sy = synapses[b];
        if (nr.n < 1 || nr.n > kBatchMaxN)
            return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": n must be in 1..4096");
        if (!nr.threshold || !nr.leak || !nr.reset || !nr.refractory)
            return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": neuron array is NULL");
        if (sy.m < 0 || (sy.m > 0 && (!sy.pre || !sy.post || !sy.weight || !sy.delay)))
            return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": bad synapse arrays");
        for (long long k = 0; k < sy.m; ++k) {
            if (sy.pre[k] < 0 || sy.pre[k] >= nr.n || sy.post[k] < 0 || sy.post[k] >= nr.n)
                return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": neuron index out of range");
            if (sy.delay[k] < 1 || sy.delay[k] > cfg->max_delay)
                return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": delay outside 1..max_delay");
            const float w = sy.weight[k];
            if (!std::isfinite(w) || std::fabs(w) > 1e9f)
                return fail(nullptr, SN_EINVAL, "network " + std::to_string(b) + ": weight not finite");
            if (cfg->dtype == SN_I32 && !is_int_valued(w))
                return fail(nullptr, SN_EINVAL, "SN_I32 weights must be integers below 2^24");
        }
        ntot += nr.n;
        mtot += sy.m;
        wtot += (nr.n + 31) / 32;
    }
    if (ntot >= (1ll << 31) || wtot >= (1ll << 31)) return fail(nullptr, SN_EINVAL, "batch too large");
    sn_ctx *c = new (std::nothrow) sn_ctx();
    if (!c) return fail(nullptr, SN_ENOMEM, "host allocation failed");
    c->kind = KIND_BATCH;
    c->dtype = cfg->dtype;
    c->n = (int)ntot;
    c->D = cfg->max_delay;
    c->D1 = c->D + 1;
    c->flags = cfg->flags;
    c->m = mtot;
    c->nets = nets;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    auto bail = [&](sn_status st) { std::string msg = c->err.empty() ? g_create_err : c->err;
                                    destroy_all(c); delete c; g_create_err = msg; return st; };
    // concatenated neuron parameters
    std::vector<float> th(ntot), lk(ntot), rs(ntot);
    std::vector<int> R(ntot);
    std::vector<int> net_off(nets + 1, 0), word_off(nets + 1, 0);
    std::vector<long long> ring_off(nets, 0);
    c->h_net_n.resize(nets);
    long long roff = 0;
    for (int b = 0; b < nets; ++b) {
        const sn_neurons &nr = neurons[b];
        memcpy(&th[net_off[b]], nr.threshold, (size_t)nr.n * 4);
        memcpy(&lk[net_off[b]], nr.leak, (size_t)nr.n * 4);
        memcpy(&rs[net_off[b]], nr.reset, (size_t)nr.n * 4);
        memcpy(&R[net_off[b]], nr.refractory, (size_t)nr.n * 4);
        net_off[b + 1] = net_off[b] + nr.n;
        word_off[b + 1] = word_off[b] + (nr.n + 31) / 32;
        ring_off[b] = roff;
        roff += (long long)c->D1 * nr.n;
        c->h_net_n[b] = nr.n;
    }
    sn_neurons all;
    all.n = (int)ntot;
    all.threshold = th.data(); all.leak = lk.data(); all.reset = rs.data(); all.refractory = R.data();
    sn_status s;
    if ((s = upload_neurons(c, &all))) return bail(s);
    c->words = (int)wtot;
    c->cap = cfg->record_steps > 0 ? cfg->record_steps : 1;
    if ((s = dalloc(c, &c->raster, (size_t)c->cap * c->words * 4)) || (s = dalloc(c, &c->ctl, sizeof(Control))))
        return bail(s);
    // CSR per network over local indices, one global row pointer
    std::vector<long long> rowptr(ntot + 1, 0);
    for (int b = 0; b < nets; ++b)
        for (long long k = 0; k < synapses[b].m; ++k) rowptr[net_off[b] + synapses[b].pre[k] + 1]++;
    for (long long g = 0; g < ntot; ++g) rowptr[g + 1] += rowptr[g];
    std::vector<unsigned short> sidx(mtot > 0 ? mtot : 1);
    std::vector<unsigned> sw(mtot > 0 ? mtot : 1);
    {
        std::vector<long long> fill(rowptr.begin(), rowptr.end() - 1);
        for (int b = 0; b < nets; ++b) {
            const sn_synapses &sy = synapses[b];
            for (long long k = 0; k < sy.m; ++k) {
                const long long p = fill[net_off[b] + sy.pre[k]]++;
                sidx[p] = (unsigned short)(sy.post[k] | ((sy.delay[k] - 1) << 12));
                if (cfg->dtype == SN_F32) memcpy(&sw[p], &sy.weight[k], 4);
                else { int w = (int)sy.weight[k]; memcpy(&sw[p], &w, 4); }
            }
        }
    }
    const size_t acc_bytes = cfg->dtype == SN_F32 ? 8 : 4;
    c->ring_bytes = (size_t)roff * acc_bytes;
    std::vector<unsigned long long> keys(nets);
    for (int b = 0; b < nets; ++b) keys[b] = host_splitmix64(0ull ^ host_splitmix64((unsigned long long)b));
    if ((s = dalloc(c, &c->net_off, (size_t)(nets + 1) * 4)) || (s = dalloc(c, &c->word_off, (size_t)(nets + 1) * 4)) ||
        (s = dalloc(c, &c->ring_off, (size_t)nets * 8)) || (s = dalloc(c, &c->pkeys, (size_t)nets * 8)) ||
        (s = dalloc(c, &c->cta_order, (size_t)nets * 4)) || (s = dalloc(c, &c->warp_order, (size_t)nets * 4)) ||
        (s = dalloc(c, &c->rowptr, (size_t)(ntot + 1) * 8)) || (s = dalloc(c, &c->sidx, sidx.size() * 2)) ||
        (s = dalloc(c, &c->sw, sw.size() * 4)) || (s = dalloc(c, &c->ring, c->ring_bytes)))
        return bail(s);
    cudaError_t e;
    if ((e = cudaMemcpy(c->net_off, net_off.data(), (size_t)(nets + 1) * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->word_off, word_off.data(), (size_t)(nets + 1) * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ring_off, ring_off.data(), (size_t)nets * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->pkeys, keys.data(), (size_t)nets * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->rowptr, rowptr.data(), (size_t)(ntot + 1) * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->sidx, sidx.data(), sidx.size() * 2, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->sw, sw.data(), sw.size() * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->ring, 0, c->ring_bytes)) ||
        (e = cudaMemset(c->raster, 0, (size_t)c->cap * c->words * 4)) || (e = cudaMemset(c->ctl, 0, sizeof(Control)))) {
        c->err = std::string("upload: ") + cudaGetErrorString(e);
        return bail(SN_ECUDA);
    }
    if ((s = batch_upload_orders(c)) || (s = batch_size_grid(c))) return bail(s);
    *out = c;
    return SN_OK;
}

sn_status sn_autotune(sn_ctx *c, int32_t trial_steps, float *best_ms) {
    NvtxRange nvtx("sn_autotune");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_BATCH && c->kind != KIND_SPARSE)
        return fail(c, SN_EUNSUPPORTED, "autotuning applies to batched and sparse contexts");
    if (c->shard_end) return fail(c, SN_EUNSUPPORTED, "a shard runs pull propagation only: nothing to tune");
    if (c->failed) return fail(c, SN_ESTATE, "context has a latched device error");
    if (trial_steps < 1) return fail(c, SN_EINVAL, "trial_steps must be >= 1");
    if (c->kind == KIND_SPARSE) return sparse_autotune(c, trial_steps, best_ms);
    const int warp_opts[] = {0, 64, 128, 256, 512};
    const int smem_opts[] = {32 * 1024, 64 * 1024, 112 * 1024, 176 * 1024};
    cudaEvent_t e0, e1;
    SN_CUDA(c, cudaEventCreate(&e0));
    SN_CUDA(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int bw = c->warp_max_n, bs = c->ring_smem;
    sn_status st = SN_OK;
    for (int w : warp_opts) {
        for (int sm : smem_opts) {
            c->warp_max_n = w;
            c->ring_smem = sm;
            if ((st = batch_upload_orders(c)) || (st = batch_size_grid(c))) { c->err += " (autotune)"; break; }
            float ms_sum = 0.0f;
            for (int rep = 0; rep < 2 && st == SN_OK; ++rep) {
                if ((st = sn_reset(c))) break;
                cudaEventRecord(e0, c->stream);
                if ((st = batch_run(c, trial_steps))) break;
                c->step += trial_steps;
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) ms_sum = ms;   // the first run also pays first-launch costs
            }
            if (st) break;
            if (ms_sum < best) { best = ms_sum; bw = w; bs = sm; }
        }
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    c->warp_max_n = bw;
    c->ring_smem = bs;
    sn_status s2;
    if ((s2 = batch_upload_orders(c)) || (s2 = batch_size_grid(c)) || (s2 = sn_reset(c))) return s2;
    if (best_ms) *best_ms = best;
    return sn_sync(c);
}

sn_status sn_batch_config(sn_ctx *c, int32_t warp_max_n, int32_t ring_smem_bytes) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_BATCH) return fail(c, SN_EUNSUPPORTED, "batched contexts only");
    if (warp_max_n < 0 || warp_max_n > 512) return fail(c, SN_EINVAL, "warp_max_n must be in 0..512");
    if (ring_smem_bytes < 0 || ring_smem_bytes > 192 * 1024 || ring_smem_bytes % 1024)
        return fail(c, SN_EINVAL, "ring_smem_bytes must be a multiple of 1024 in 0..196608");
    if (sn_status q = quiesce(c)) return q;   // a queued run reads the work queues
    c->warp_max_n = warp_max_n;
    c->ring_smem = ring_smem_bytes;
    sn_status s;
    if ((s = batch_upload_orders(c)) || (s = batch_size_grid(c))) return s;
    return SN_OK;
}

}  // extern "C"
