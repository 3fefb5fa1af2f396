// sn_run_dense_noalloc: the dense simulation for callers that cannot allocate
// device memory (an application whose device memory is all owned by its own
// pool allocator, or a plug-in whose host forbids it to allocate).  It launches
// the same dense kernel as sn_run on a dense context, but every buffer comes
// from the caller except the kernel's scratch (spike bits of the last two
// steps, pending-input ring, zero Poisson table, control block), which lives
// in one fixed file-scope device array.  No cudaMalloc, cudaFree or
// allocating library routine is called on this path.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "sn_ctx.h"
#include "sn_internal.h"

namespace {

constexpr size_t kScratchBytes = SN_NOALLOC_SCRATCH_BYTES;

// The shared scratch: every call on a device uses it, and it keeps the last
// call's contents (cleared below where a call needs zeros).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch for each device, looked up once per device with
// that device current.  In host code `g_scratch` names a host-side shadow,
// not device memory, so only this address may be handed to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];

sn_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return SN_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return SN_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SN_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of scratch a network of n neurons with synaptic delay `delay` needs:
// control | spike bits [2][words] | ring [delay + 1][n] | zero Poisson table [n].
struct ScratchLayout {
    size_t off_spk, off_ring, off_zero, need;
};

ScratchLayout scratch_layout(int n, int delay) {
    const size_t words = ((size_t)n + 31) / 32;
    ScratchLayout L;
    L.off_spk = align256(sizeof(sn::Control));
    L.off_ring = L.off_spk + align256(2 * words * 4);
    L.off_zero = L.off_ring + align256((size_t)(delay + 1) * n * 4);
    L.need = L.off_zero + align256((size_t)n * 4);
    return L;
}

}  // namespace

extern "C" sn_status sn_run_dense_noalloc(const sn_dense_noalloc_args *p) {
    using namespace sn;
    if (!p) return fail(nullptr, SN_EINVAL, "sn_run_dense_noalloc: NULL arguments");
    const int n = p->n;
    if (n < 1 || n > 200000) return fail(nullptr, SN_EINVAL, "sn_run_dense_noalloc: n outside 1..200000");
    if (p->steps < 0) return fail(nullptr, SN_EINVAL, "sn_run_dense_noalloc: steps < 0");
    if (p->delay < 1 || p->delay > SN_MAX_DELAY)
        return fail(nullptr, SN_EINVAL, "sn_run_dense_noalloc: delay outside 1..64");
    if (!p->w || !p->threshold || !p->leak || !p->reset || !p->refractory || !p->v || !p->r ||
        (p->steps > 0 && !p->raster))
        return fail(nullptr, SN_EINVAL, "sn_run_dense_noalloc: a required pointer is NULL");
    if ((p->poisson_threshold == nullptr) != (p->poisson_amplitude == nullptr))
        return fail(nullptr, SN_EINVAL,
                    "sn_run_dense_noalloc: poisson_threshold and poisson_amplitude must both be given or both NULL");
    // the scratch check needs only n and delay, so it comes before any CUDA call
    const ScratchLayout lay = scratch_layout(n, p->delay);
    if (lay.need > kScratchBytes)
        return fail(nullptr, SN_EINVAL,
                    "sn_run_dense_noalloc: the network needs " + std::to_string(lay.need) +
                        " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes));
    if (p->steps == 0) return SN_OK;
    cudaStream_t stream = (cudaStream_t)p->cuda_stream;

    // executor sizing, the same rule as a dense context
    const int words = (n + 31) / 32;
    int grid = 0, chunk = 0;
    cudaError_t ce = plan_dense(n, &grid, &chunk);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "sn_run_dense_noalloc: executor sizing");
    if (grid < 1) return fail(nullptr, SN_EUNSUPPORTED, "sn_run_dense_noalloc: no co-resident grid for this n");
    const int D1 = p->delay + 1;
    const size_t off_spk = lay.off_spk, off_ring = lay.off_ring, off_zero = lay.off_zero, need = lay.need;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SN_ECUDA;
    void *base = nullptr;
    sn_status st = scratch_address(dev, &base);
    if (st != SN_OK) return fail(nullptr, st, "sn_run_dense_noalloc: scratch address lookup failed");
    unsigned char *b = (unsigned char *)base;

    // zero what must start at zero: control block, spike bits, ring, table
    ce = cudaMemsetAsync(b, 0, need, stream);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "sn_run_dense_noalloc: clearing the scratch");

    NetArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n; a.D1 = D1; a.words = words; a.cap = p->steps;
    a.t0 = 0; a.steps = p->steps; a.chunk = chunk;
    a.V = p->v; a.r = p->r;
    a.th = p->threshold; a.lk = p->leak; a.rs = p->reset; a.R = p->refractory;
    a.prate = p->poisson_threshold ? p->poisson_threshold : (const unsigned *)(b + off_zero);
    a.pamp = p->poisson_amplitude ? (const void *)p->poisson_amplitude : (const void *)(b + off_zero);
    {
        // the same key derivation as sn_set_poisson for network 0
        auto sm = [](unsigned long long x) {
            unsigned long long z = x + 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        a.pkey = sm(p->seed ^ sm(0ull));
    }
    a.W = (float *)p->w;
    a.spk = (unsigned *)(b + off_spk);
    a.S = 1;
    a.dense_delay = p->delay;
    a.ring = b + off_ring;
    a.raster = p->raster;
    a.ctl = (Control *)b;
    ce = launch_dense(a, grid, 256, stream);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "sn_run_dense_noalloc: launch");

    // wait, then read the device status word (no allocation involved)
    ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "sn_run_dense_noalloc: synchronize");
    int status = 0;
    ce = cudaMemcpy(&status, b, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "sn_run_dense_noalloc: status read");
    if (status != SN_OK) return fail(nullptr, (sn_status)status, "sn_run_dense_noalloc: the kernel latched a failure");
    return SN_OK;
}
