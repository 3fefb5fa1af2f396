// Internal declarations shared by the host API (sn_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sn.h"

namespace sn {

enum Kind { KIND_SPARSE = 0, KIND_DENSE = 1, KIND_BATCH = 2, KIND_SHARED_I8 = 3, KIND_FF = 4 };

// Grid barrier state (one per context): the arrival count of the running
// launch, zeroed before every launch that uses it.
struct GridBarrier {
    unsigned int count;
    unsigned int pad;
};

// Device-side control block: latched status word and run counters.
struct Control {
    int status;                       // 0 or an sn_status latched by a kernel
    int pad;
    unsigned long long spikes;        // total spikes
    unsigned long long events;        // total synaptic events
    GridBarrier bar;
    unsigned queue[2];                // batched work queues: next block item, next warp item
};

// Wall-clock limit of one grid-barrier wait before the kernel gives up and
// latches SN_ETIMEOUT (nanoseconds of %globaltimer).
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

// Packed synapse of the CSR (pre-major) store: x = post | (delay-1) << 26,
// y = weight bits (float in SN_F32 mode, int32 in SN_I32 mode).
constexpr int kPostBits = 26;
constexpr unsigned kPostMask = (1u << kPostBits) - 1u;

// Arguments of the single-network kernels (sparse push and dense gather).
struct NetArgs {
    int n, D1, words, cap;            // neurons, ring slots (D+1), raster words/row, raster rows
    int t0, steps;                    // first absolute step, steps to run
    int chunk;                        // neurons owned per block (multiple of 32)
    // neuron state and parameters (float or int32 according to the mode)
    void *V;
    int *r;
    const void *th, *lk, *rs;
    const int *R;
    const unsigned *prate;            // Poisson threshold per neuron (0: no source)
    const void *pamp;                 // Poisson amplitude per neuron
    unsigned long long pkey;          // Poisson stream key of the network
    // explicit events, deduplicated per (step, neuron), sorted by neuron per step
    const int *ev_off;                // [ev_nsteps + 1] offsets by absolute step
    int ev_nsteps;
    const int *ev_neuron;
    const void *ev_val;
    // sparse store (CSR by pre)
    const long long *rowptr;
    uint2 *syn;                       // weights are rewritten in place by STDP
    const long long *colptr;          // CSC by post (STDP only)
    const uint2 *csc;                 // {pre, CSR position}
    void *ring;                       // [D1][n] pending input (int64 fixed point / int32 / float)
    // sparse store for pull propagation (sn_pull.cu): incoming synapses of
    // 32-neuron slices, plain ({bit offset, weight bits} pairs) or coded
    // (groups of 8 weights and 16-bit offset steps)
    const uint4 *pin;
    const long long *pin_off;         // [slices] first uint4 of each slice
    const int *pin_len;               // [n] entries of delay >= 2 of each position's list
    const int *pin_len1;              // [n] entries of delay 1 (the region after them)
    const unsigned *pin_y0;           // coded store: [2][n] window bit offset of each region's first entry
    const int *pin_perm;              // [n] the neuron whose lists thread position p sums (the store,
                                      // pin_len, pin_len1 and pin_y0 are indexed by position)
    unsigned *hist;                   // [hD][words] spike bits of step tau in row tau % hD
    int hD;                           // history depth (the maximum delay D)
    int hL;                           // rows of the pull kernel's shared-memory window
    int ring_until;                   // the ring may hold pending input for steps < ring_until
    int j_first, j_end;               // pull: the neurons [j_first, j_end) this launch simulates
                                      // (a shard of the network; 0 and n otherwise)
    // dense store
    float *W;                         // [n][n]
    float *partial;                   // [S][n] gather partial sums
    int S, dense_delay;
    // spikes
    unsigned *raster;                 // [cap][words]
    unsigned *spk;                    // [2][words] spike bits of the last two steps (dense)
    // STDP
    int stdp;
    float decay, a_plus, a_minus, wmin, wmax;
    float *trace;                     // [3][n]: sparse kernels use buffer t & 1, dense t % 3
    Control *ctl;
};

// Arguments of the batched kernel: many independent networks, each run for
// all steps by one block or one warp.
struct BatchArgs {
    int nets, t0, steps, cap, total_words, D1;
    const int *net_off;               // [nets + 1] first neuron of each network
    const int *word_off;              // [nets + 1] first raster word of each network
    const long long *ring_off;        // [nets] first ring element of each network (D1 * n_b)
    const unsigned long long *pkey;   // [nets] Poisson stream key
    const int *cta_order;             // networks run by whole blocks, largest first
    int n_cta;
    const int *warp_order;            // networks run by single warps
    int n_warp;
    void *V;
    int *r;
    const void *th, *lk, *rs;
    const int *R;
    const unsigned *prate;
    const void *pamp;
    const int *ev_off;
    int ev_nsteps;
    const int *ev_neuron;
    const void *ev_val;
    const long long *rowptr;          // [sum n + 1] over global neuron index
    const unsigned short *sidx;       // post (12 bits) | (delay-1) << 12
    const unsigned *sw;               // weight bits
    void *ring;                       // all networks' pending-input rings
    unsigned *raster;                 // [cap][total_words]
    int ring_smem;                    // bytes of shared ring arena per block
    Control *ctl;
};

constexpr int kBatchBlock = 256;
constexpr int kBatchMaxN = 4096;      // largest network of a batched context
constexpr int kBatchMaxDelay = 16;

cudaError_t launch_batch(const BatchArgs &a, int dtype, int grid, cudaStream_t s);
cudaError_t batch_kernel_node(int dtype, void **fn);
cudaError_t max_grid_batch(int dtype, int ring_smem, int *grid);
size_t batch_smem(int ring_smem);

// Shared dense network on tensor cores, sn_shared.cu
struct SharedHostArgs {
    int n, B, t0, steps, cap;
    unsigned char *A0, *A1;
    int *V, *r;
    const int *th, *lk, *rs, *R;
    const unsigned *prate;
    const int *pamp;
    const unsigned long long *pkey;
    unsigned *raster;
    Control *ctl;
};
cudaError_t launch_shared(const void *tmaps, const SharedHostArgs &h, int grid, cudaStream_t s);
cudaError_t max_grid_shared(int *grid);
size_t shared_smem_bytes();
cudaError_t launch_shared_transpose(const int *src, int *dst, int n, int B, cudaStream_t s);

// Feedforward (BPTT) kernels, sn_ff.cu
// sbf (may be null): the spikes also as BF16 rows of ldbf elements
cudaError_t ff_pack(const uint8_t *in, int rows, int n, int words, unsigned *out, void *sbf, int ldbf,
                    cudaStream_t s);
cudaError_t ff_delay_fwd(const unsigned *sprev, int words_in, const float *W, const void *dm, int n_in,
                         int n_out, int B, int row0, int rows, float *I, cudaStream_t s);
cudaError_t ff_scan_fwd(const float *I, int n, int B, int T, int k, float theta, float leak, float reset,
                        int refractory, unsigned *S, float *vck, int *rck, float *counts, void *sbf, int ldbf,
                        cudaStream_t s);
cudaError_t ff_scan_bwd(const float *I, int n, int B, int T, int k, float theta, float leak, float reset,
                        int refractory, float slope, const float *vck, const int *rck, const float *gs,
                        const float *gc, float *gI, cudaStream_t s);
cudaError_t ff_bwd_data(const float *gI, const float *W, const uint8_t *D, int n_in, int n_out, int B, int T,
                        float *gsp, cudaStream_t s);
cudaError_t ff_dw(const float *gI, const unsigned *sprev, int words_in, const uint8_t *D, int n_in, int n_out,
                  int B, int T, int splits, float *part, float *dW, cudaStream_t s);

// Tensor-core contractions of the feedforward network (sn_ff_tc.cu).  A pass
// is a K loop over `kblocks` 64-element blocks: A tile rows a_y + 128 * tm,
// K a_x + 64 * kb of map amap; B tile rows b_y + 128 * tn, K b_x + 64 * kb of
// map bmap (and, with nb = 2, a second B tile from bmap2 at rows b_y2 + 128 *
// tn, multiplying the same A tile); into accumulator acc.  mode 0: C[m][n] = acc 0; mode 1: C[m][n] =
// acc (D[m][n] - 1) (delay-selected weight gradient).  With ksplit > 1 the
// work item of split ks covers its share of every pass's K blocks and writes
// C + ks * cstride.
constexpr int kFfTcMaxMaps = 4;
constexpr int kFfTcMaxPasses = 16;
struct FfTcMaps {
    CUtensorMap m[kFfTcMaxMaps];
};
struct FfTcPass {
    int amap, bmap, a_y, a_x, b_y, b_x, kblocks, acc;
    int nb, bmap2, b_y2;              // B tiles per stage (1, or 2: the second from bmap2 at rows b_y2)
};
struct FfTcArgs {
    int M, N, tiles_m, tiles_n, ksplit, npass, nacc, mode;
    int part_stride;                  // forward kernel: rows between the B parts of a pass
    FfTcPass pass[kFfTcMaxPasses];
    float *C;
    long long ldc, cstride;
    const uint8_t *D;
    Control *ctl;
};
cudaError_t ff_tc_gemm(const FfTcMaps &maps, const FfTcArgs &args, cudaStream_t s);
cudaError_t ff_tc_forward(const FfTcMaps &maps, const FfTcArgs &args, cudaStream_t s);
cudaError_t ff_tc_weights(const float *W, const uint8_t *D, int n_in, int n_out, int nout_p, int rows_in,
                          void *Wb, int nin_p, int rows_out, void *Wf, cudaStream_t s);
cudaError_t ff_tc_spikes(const unsigned *bits, int rows, int n_in, int words, int nin_p, int rows_p, void *S,
                         void *ST, cudaStream_t s);
cudaError_t ff_tc_gsplit(const float *g, int rows, int n_out, int nout_p, int rows_p, void *G, void *GT,
                         cudaStream_t s);
cudaError_t ff_dw_reduce(const float *part, int splits, long long count, float *dW, cudaStream_t s);

// Launchers (kernels live in sn_kernels.cu).  Return a CUDA error code.
cudaError_t launch_sparse(const NetArgs &a, int dtype, int grid, int block, cudaStream_t s);
cudaError_t launch_dense(const NetArgs &a, int grid, int block, cudaStream_t s);
cudaError_t max_grid_sparse(int dtype, int stdp, int block, int *grid);
cudaError_t max_grid_sparse_reg(int *grid);
cudaError_t launch_sparse_reg(const NetArgs &a, int dtype, int grid, cudaStream_t s);
constexpr int kSparseRegBlock = 512;
cudaError_t plan_dense(int n, int *grid, int *chunk, int force_cpl = 0);
// Pull propagation (sn_pull.cu).  plan_pull sets *grid = 0 when the network
// does not fit the executor (a window of max_delay spike rows above a block's
// shared memory, or more than one neuron per thread).  Synapse words of the
// pull store: x = ((D - d) * Wp + pre / 32) << 7 | (pre & 31),
// Wp = roundup(ceil(n/32), 4).
cudaError_t plan_pull(int n, int D, long long m, int *grid, int *chunk, int *rows, size_t *smem,
                      int own_slices = -1);
cudaError_t launch_shard_put(unsigned *hist, unsigned *raster, int D, int cap, int words, int w0, int w1,
                             long long t0, int rows, const unsigned *src, cudaStream_t s);
cudaError_t launch_sparse_pull(const NetArgs &a, int dtype, bool coded, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_pull_flush(const NetArgs &a, int dtype, int t0, cudaStream_t s);
cudaError_t launch_gather_weights(const uint2 *syn, const long long *perm_inv, long long m,
                                  float *out, cudaStream_t s);
cudaError_t launch_scatter_weights(uint2 *syn, const long long *perm_inv, long long m, const float *w,
                                   cudaStream_t s);
cudaError_t launch_barrier_selftest(Control *ctl, int blocks, cudaStream_t s);

}  // namespace sn
