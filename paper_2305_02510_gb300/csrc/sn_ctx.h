// Host-side context of the C ABI and helpers shared by the host translation
// units (sn_api.cu, sn_batch_api.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sn_internal.h"

using namespace sn;

struct sn_ctx {
    int kind = KIND_SPARSE;
    int dtype = SN_F32;
    int n = 0;
    int D = 1, D1 = 2;
    unsigned flags = 0;
    int cap = 1, words = 1;
    cudaStream_t stream = nullptr;
    long long step = 0;            // steps run so far (absolute step of the next run)
    long long raster_from = 0;     // first step whose raster row is valid
    long long m = 0;
    bool all_delay_one = true;
    int dense_delay = 1;
    // executor
    int grid = 1, block = 256, chunk = 32, S = 1;
    int reg_grid = 0, reg_chunk = 0;   // register-resident sparse executor (0: not usable)
    // pull propagation of sparse networks (sn_pull.cu)
    int prop_pull = 0;                 // 1: sparse runs use pull propagation
    int pull_grid = 0, pull_chunk = 0, pull_rows = 0;
    size_t pull_smem = 0;
    uint4 *pin = nullptr;              // incoming synapses in 32-neuron slices
    long long *pin_off = nullptr;
    int *pin_len = nullptr;            // entries of delay >= 2 of each thread position's list
    int *pin_len1 = nullptr;           // entries of delay 1 of each thread position's list
    unsigned *pin_y0 = nullptr;        // coded store: [2][n] bit offset of each region's first entry
    int *pin_perm = nullptr;           // [n] the neuron whose lists thread position p sums
    size_t pin_cap = 0;                // bytes allocated for pin
    int pin_coded = 0;                 // 1: the store holds 16-bit offset steps (coded form)
    int pin_format = 0;                // 0 = the smaller of the two forms, 1 = plain, 2 = coded
    long long pin_bytes = 0, pin_entries = 0;   // store size; entries incl. padding and gap fillers
    bool pin_stale = true;             // the pull store must be (re)built from the CSR
    unsigned *hist = nullptr;          // [D][words] spike bits whose deliveries may be due
    bool hist_live = false;            // hist may hold spikes not yet delivered
    long long ring_live_until = 0;     // the ring may hold pending input for steps before this
    // device memory
    void *V = nullptr;
    int *r = nullptr;
    void *th = nullptr, *lk = nullptr, *rs = nullptr;
    int *R = nullptr;
    unsigned *prate = nullptr;
    void *pamp = nullptr;
    unsigned long long pkey = 0;
    int *ev_off = nullptr, *ev_neuron = nullptr;
    void *ev_val = nullptr;
    int ev_nsteps = 0;
    long long *rowptr = nullptr;
    uint2 *syn = nullptr;
    long long *colptr = nullptr;
    uint2 *csc = nullptr;
    long long *perm_inv = nullptr;  // input index -> CSR position (device)
    void *ring = nullptr;
    size_t ring_bytes = 0;
    float *W = nullptr, *partial = nullptr;
    unsigned *spk = nullptr;          // dense: spike bits of the last two steps [2][words]
    unsigned *raster = nullptr;
    float *trace = nullptr;
    Control *ctl = nullptr;
    // host copies
    std::vector<long long> h_perm_inv;
    // STDP
    int stdp = 0;
    float decay = 0, a_plus = 0, a_minus = 0, wmin = 0, wmax = 0;
    // batched networks
    int nets = 0;
    std::vector<int> h_net_n;          // neurons of each network
    int *net_off = nullptr, *word_off = nullptr, *cta_order = nullptr, *warp_order = nullptr;
    long long *ring_off = nullptr;
    unsigned long long *pkeys = nullptr;
    unsigned short *sidx = nullptr;
    unsigned *sw = nullptr;
    int n_cta = 0, n_warp = 0;
    int warp_max_n = 128, ring_smem = 96 * 1024, batch_grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphNode_t graph_kernel = nullptr;
    // feedforward network trained by BPTT
    int ff_layers = 0, ff_batch = 0, ff_steps = 0, ff_k = 10, ff_splits = 1, ff_refr = 0;
    size_t ff_part_elems = 0;          // floats of the weight gradient's partial-sum buffer
    float ff_theta = 1, ff_leak = 0, ff_reset = 0, ff_slope = 10;
    std::vector<int> ff_sizes;
    std::vector<uint8_t *> ff_D;       // device delays per layer
    std::vector<void *> ff_DM;         // device delay bit masks per layer
    std::vector<unsigned *> ff_S;      // device spike bits per layer (0 = input)
    std::vector<float *> ff_vck;
    std::vector<float *> ff_Ik;        // per layer: the forward's synaptic input (empty: recompute)
    std::vector<int *> ff_rck;
    float *ff_I = nullptr, *ff_gI = nullptr, *ff_gS = nullptr, *ff_part = nullptr;
    std::vector<const float *> ff_w;   // weights of the last forward (caller's device memory)
    bool ff_have_forward = false;
    // tensor-core contractions (sn_ff_tc.cu): engine choice and BF16 operands
    int ff_engine = 0;                 // SN_FF_AUTO, SN_FF_SIMT or SN_FF_TENSOR
    bool ff_tc_ok = false;             // the shapes fit the tensor-core path
    bool ff_fwd_tc = false;            // the last forward ran on the tensor cores
    void *ff_Sbf = nullptr, *ff_ST = nullptr, *ff_G = nullptr, *ff_GT = nullptr;
    std::vector<void *> ff_Wf, ff_Wb;  // forward and backward weight parts per layer
    void *ff_encode = nullptr;         // the driver's cuTensorMapEncodeTiled
    // shared dense network driven by many trains (tensor cores)
    int sh_B = 0, sh_grid = 0;
    unsigned char *sh_A0 = nullptr, *sh_A1 = nullptr, *sh_WT = nullptr;
    int *sh_V0 = nullptr;
    alignas(64) unsigned char sh_tmaps[3 * 128];
    // shard of a sparse network (sn_create_shard): neurons [shard_first,
    // shard_end) simulated here, the other shards' spikes put in by the caller
    int shard_first = 0, shard_end = 0;  // shard_end == 0: not a shard
    int shard_dmin = 1;                  // smallest synaptic delay of the network
    long long shard_known = 0;           // every spike row before this step is complete
    unsigned *shard_stage = nullptr;     // [max_delay][words] staging of host rows
    int failed = 0;                // sticky device failure seen
    std::string err;
    std::vector<void *> allocs;
};

extern thread_local std::string g_create_err;

namespace sn {

inline sn_status fail(sn_ctx *c, sn_status s, const std::string &msg) {
    if (c) c->err = msg; else g_create_err = msg;
    return s;
}

inline sn_status cuda_fail(sn_ctx *c, cudaError_t e, const char *what) {
    return fail(c, SN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Wait for the work queued on the context's stream.  Host calls that rewrite
// device buffers with blocking copies (setters, mode switches) call this
// first: a blocking cudaMemcpy orders itself after the legacy default stream
// but not after a cudaStreamNonBlocking stream, where a queued run may still
// be reading the buffer.
inline sn_status quiesce(sn_ctx *c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "waiting for the context's queued work");
}

#define SN_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
    } while (0)

// An NVTX range over one library call (visible to profilers that record
// NVTX; free when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side fault injection for tests of the failure paths: while a create
// call runs with the environment variable SN_FAULT_ALLOC_AT = k (k >= 1), its
// k-th device allocation fails with SN_ENOMEM (no allocation is made).
extern thread_local long long g_fault_alloc;   // allocations left before the injected failure; 0 = off
extern thread_local int g_fault_depth;

struct FaultScope {
    FaultScope() {
        if (g_fault_depth++ == 0) {
            const char *e = std::getenv("SN_FAULT_ALLOC_AT");
            g_fault_alloc = e ? std::atoll(e) : 0;
            if (g_fault_alloc < 0) g_fault_alloc = 0;
        }
    }
    ~FaultScope() {
        if (--g_fault_depth == 0) g_fault_alloc = 0;
    }
};

template <typename T>
inline sn_status dalloc(sn_ctx *c, T **p, size_t bytes) {
    void *q = nullptr;
    if (bytes == 0) bytes = 16;
    if (g_fault_alloc > 0 && --g_fault_alloc == 0)
        return fail(c, SN_ENOMEM, "injected device allocation failure (SN_FAULT_ALLOC_AT)");
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, SN_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    c->allocs.push_back(q);
    *p = (T *)q;
    return SN_OK;
}

inline void dfree(sn_ctx *c, void *p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
}

inline bool is_int_valued(float x) { return std::isfinite(x) && std::floor(x) == x && std::fabs(x) < 16777216.0f; }

inline unsigned long long host_splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline unsigned rate_threshold(float rate) {
    double r = std::floor((double)rate * 4294967296.0);
    if (!(r > 0)) return 0u;
    if (r > 4294967295.0) return 4294967295u;
    return (unsigned)r;
}

// shared by sn_api.cu and sn_batch_api.cu
sn_status upload_neurons(sn_ctx *c, const sn_neurons *nr);
sn_status alloc_common(sn_ctx *c, const sn_config *cfg);
void destroy_all(sn_ctx *c);
sn_status batch_run(sn_ctx *c, int steps);
sn_status sparse_autotune(sn_ctx *c, int trial_steps, float *best_ms);
sn_status shared_run(sn_ctx *c, int steps);
sn_status shared_get_state(sn_ctx *c, void *v, int32_t *refr, int32_t on_device);
sn_status shared_set_poisson(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                             const float *amp, uint64_t seed, uint64_t net0);
inline long long state_elems(const sn_ctx *c) { return c->kind == KIND_SHARED_I8 ? (long long)c->sh_B * c->n : c->n; }
sn_status batch_set_poisson(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                            const float *amp, uint64_t seed, uint64_t net0);

}  // namespace sn
