/*
 * sn.h - C ABI of the GB300 spiking-network simulator (libsn.so).
 *
 * The library simulates networks of leaky integrate-and-fire (LIF) neurons
 * joined by synapses that carry a weight and an integer delay, driven by
 * external input spikes, optionally with pair-based STDP, on one GPU
 * (sm_103a).  The rules follow SuperNeuro (arXiv 2305.02510):
 *
 *   Section 2.1, "The MAT Mode": four neuron parameters (threshold, leak,
 *     reset state, refractory period); a constant leak that moves the state
 *     toward the reset state; synapses with a weight and a delay; the order of
 *     one timestep: leak, add previous spikes times weights, add external
 *     spikes, compare with the threshold, zero the spikes of refractory
 *     neurons; built-in STDP.
 *   Section 2.2, "The ABM Mode": the spike condition is "greater than" the
 *     threshold; delay registers deliver a spike to the post-neuron after the
 *     synaptic delay.
 *
 * Semantics of one timestep t for neuron j (the library's reading of those
 * passages, identical to the CPU oracle):
 *   V_j <- L(V_j) + sum_{synapses i->j, delay d} w * s_i(t - d) + ext_j(t)
 *   L(V) = max(V - leak, reset) if V > reset; min(V + leak, reset) if V < reset
 *   s_j(t) = [V_j > threshold_j] and (refractory countdown r_j == 0)
 *   on a spike: V_j <- reset_j, r_j <- refractory_j; otherwise r_j <- max(r_j - 1, 0)
 * A spike at step t arrives at t + d (d >= 1).  A neuron that spiked at t
 * cannot spike at t+1 .. t+refractory.  Initial state: V = reset, r = 0, no
 * spikes before step 0.  ext_j(t) = (explicit events of (t, j) summed in the
 * order given) + (amplitude of j's Poisson source if it fires at t).
 *
 * Conventions for every entry point:
 *   - All input arrays are caller-owned host memory and are copied before
 *     the call returns, unless a parameter says it is a device pointer.
 *   - The context owns all device memory it allocates; sn_destroy frees it.
 *   - Work is issued on the context's CUDA stream (sn_config.cuda_stream, or
 *     the legacy default stream when NULL).  sn_run returns once the work is
 *     queued; sn_sync waits for it.  Host-buffer getters synchronise.  Calls
 *     that replace device-side inputs or tables (sn_set_input,
 *     sn_set_poisson, sn_stdp, sn_set_propagation, sn_set_weights of a
 *     sparse network, sn_batch_config) first wait for the work queued on the
 *     context's stream, so a run already queued (also on a
 *     cudaStreamNonBlocking stream) sees the old values and the next run the
 *     new ones.
 *   - No exception crosses the ABI.  Each call returns an sn_status;
 *     sn_last_error gives a message for the last failure of a context.
 *     Device-side failures (a timed-out grid barrier, an integer overflow)
 *     latch in a device status word and are reported by the next sn_sync or
 *     getter; after that the context refuses further runs (SN_ESTATE).
 */
#ifndef SN_H
#define SN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_ctx sn_ctx;

typedef enum {
    SN_OK = 0,
    SN_EINVAL = 1,        /* an argument is out of range or inconsistent       */
    SN_ENOMEM = 2,        /* a device or host allocation failed                */
    SN_ECUDA = 3,         /* a CUDA runtime call failed                        */
    SN_ESTATE = 4,        /* the context is in an error state or wrong kind    */
    SN_ETIMEOUT = 5,      /* a device-side wait gave up (bounded spin)         */
    SN_EUNSUPPORTED = 6,  /* valid request this build or context cannot serve  */
    SN_EOVERFLOW = 7      /* an integer-mode state left the int32 range        */
} sn_status;

/* Arithmetic of the membrane state. */
typedef enum {
    SN_F32 = 0,  /* float state.  Push propagation sums the synaptic input
                    exactly in fixed point (2^-32) and rounds it once to
                    float; pull propagation adds the weights in float,
                    the oldest spikes first (descending delay, then
                    ascending pre and input index).  Neither depends on
                    thread timing.                                           */
    SN_I32 = 1   /* exact integer state; parameters and weights must be
                    integral (checked)                                       */
} sn_dtype;

/* sn_config.flags */
#define SN_AUTO 0u          /* the library picks the executor                      */
#define SN_EXEC_CTA 1u      /* force the one-block executor (small networks)       */
#define SN_EXEC_GRID 2u     /* force the grid-wide persistent executor             */
#define SN_PROP_PULL 4u     /* sn_create only: start with pull propagation (see
                               sn_set_propagation); SN_EUNSUPPORTED if the
                               network does not fit it                             */
#define SN_FF_RECOMPUTE 8u  /* sn_create_ff only: sn_backward recomputes each
                               layer's synaptic input instead of keeping it from
                               the forward (saves steps * batch * sum(sizes[1..])
                               floats of device memory)                            */

#define SN_DENSE_SLAB(k) ((uint32_t)(k) << 8)
                            /* sn_create_dense only: each block owns a slab of
                               32 * k weight columns, k = 1, 2, 4 or 8, instead
                               of the narrowest slab whose grid is co-resident
                               (k = 1 up to about 19,000 neurons).  k changes
                               only the order of the float additions of each
                               neuron's synaptic input; it lets a small network
                               run the wide-slab code of large ones (tests,
                               tuning).  SN_EUNSUPPORTED if that grid is not
                               co-resident                                        */
#define SN_DENSE_SLAB_MASK 0xF00u
#define SN_PULL_PLAIN 0x1000u
#define SN_PULL_CODED 0x2000u
                            /* sn_create only: the form of the pull store (see
                               sn_pull_store_info).  Without either flag the
                               library builds the plain form while it takes at
                               most 80 % of the L2 cache, else the smaller
                               form.  The two forms
                               hold the same synapses in the same order, so
                               the results are identical; the flags let tests
                               and tuning run either                          */
#define SN_PULL_STORE_MASK 0x3000u

#define SN_MAX_DELAY 64     /* largest supported synaptic delay                    */

typedef struct {
    int32_t dtype;          /* sn_dtype                                            */
    int32_t max_delay;      /* D: every synaptic delay lies in 1..D, D <= 64       */
    uint32_t flags;         /* SN_AUTO or one SN_EXEC_* value, optionally with
                               SN_PROP_PULL, one SN_PULL_* form or
                               SN_DENSE_SLAB(k)                                    */
    int32_t record_steps;   /* spike-raster capacity in steps (a ring); sn_get_spikes
                               can return any of the last record_steps steps; 0
                               means 1                                              */
    void *cuda_stream;      /* cudaStream_t for all work, NULL = default stream    */
} sn_config;

/* Neuron parameters, each an array of n values (Section 2.1: threshold, leak,
 * reset state, refractory period).  In SN_I32 mode the float values must be
 * integers of magnitude below 2^24.  leak >= 0 and refractory >= 0. */
typedef struct {
    int32_t n;
    const float *threshold;
    const float *leak;
    const float *reset;
    const int32_t *refractory;
} sn_neurons;

/* Synapse list (Section 2.1: each synapse has a weight and a delay; the
 * weight matrix has the pre-neuron as row and the post-neuron as column).
 * Synapse k joins pre[k] -> post[k] with weight[k] and delay[k] in 1..D.
 * Duplicated pairs are allowed and act as separate synapses.  Neuron
 * indices must lie in [0, n). */
typedef struct {
    int64_t m;
    const int32_t *pre;
    const int32_t *post;
    const float *weight;
    const int32_t *delay;
} sn_synapses;

/* Create a network from a synapse list.  The synapses are stored grouped by
 * pre-neuron (CSR) for event-driven propagation.  Returns SN_EINVAL for an
 * index, delay or parameter out of range (n < 1, n >= 2^26, D outside 1..64,
 * non-integral values in SN_I32 mode, NaN weights).  *out is set only on
 * success. */
sn_status sn_create(const sn_config *cfg, const sn_neurons *neurons,
                    const sn_synapses *synapses, sn_ctx **out);

/* sn_create with axonal delays (Section 2.2 lists the axonal delay among the
 * neuron parameters; the benchmark of Section 3 sets it to 0).  Neuron i has
 * axonal_delay[i] >= 0 (n values; NULL = all 0): its spike at step t reaches
 * the post-neuron of synapse k (pre[k] = i) at t + axonal_delay[i] + delay[k].
 * Every such sum must lie in 1..cfg->max_delay (SN_EINVAL otherwise).  The
 * context is then an sn_create context whose synapse delays are those sums
 * (checkpoints, propagation modes and getters as for sn_create; STDP needs
 * every sum to be 1). */
sn_status sn_create_axonal(const sn_config *cfg, const sn_neurons *neurons, const sn_synapses *synapses,
                           const int32_t *axonal_delay, sn_ctx **out);

/* One shard of a sparse network run on several GPUs (Section 4 motivates
 * networks larger than one device; one context per GPU, one rank per
 * context).  The network is given whole (all n neurons' parameters, every
 * synapse); this context simulates the neurons [first, first + count) with
 * pull propagation and keeps every neuron's spike bits of the last max_delay
 * steps.  first is a multiple of 32 and count a multiple of 32 unless the
 * shard ends at n, so that every 32-neuron raster word belongs to one shard.
 * The shards exchange spike rows: sn_run may advance at most
 * steps_per_exchange steps (the network's smallest synaptic delay: a spike
 * of step t reaches no neuron before t + that delay), and only once the
 * other shards' spikes of every earlier step have been put in with
 * sn_shard_put_spikes (SN_ESTATE otherwise).  A run of all shards with their
 * rows exchanged after every sn_run equals the single context's run bit for
 * bit.  Inputs (sn_set_input, sn_set_poisson) take global neuron indices;
 * sn_get_state returns n values of which the shard's own are meaningful;
 * sn_get_spikes returns whole rows (own words from this shard, the others as
 * put in); the counters count this shard's spikes and their synaptic events.
 * STDP, push propagation, sn_set_weights, sn_autotune and checkpoints are
 * not available for shards (SN_EUNSUPPORTED / SN_ESTATE). */
sn_status sn_create_shard(const sn_config *cfg, const sn_neurons *neurons, const sn_synapses *synapses,
                          int32_t first, int32_t count, sn_ctx **out);

/* The shard's range and the largest number of steps one sn_run may advance
 * between exchanges (any pointer may be NULL); SN_ESTATE for a context that
 * is not a shard. */
sn_status sn_shard_info(const sn_ctx *ctx, int32_t *first, int32_t *count, int32_t *steps_per_exchange);

/* The other shards' spikes of steps [t0, t1): rows of ceil(n/32) words of the
 * whole network (the words of this shard's own neurons are ignored), into
 * the history and the raster.  t0 must be the first step whose rows are not
 * in yet, t1 at most the current step, t1 - t0 <= max_delay.  on_device = 1:
 * `bits` is a device pointer read on the context's stream; 0: host memory,
 * copied before the call returns. */
sn_status sn_shard_put_spikes(sn_ctx *ctx, int64_t t0, int64_t t1, const uint32_t *bits, int32_t on_device);

/* Create an all-to-all network from a dense row-major n x n weight matrix
 * (w[i*n + j] is the weight of i -> j, Section 2.1).  Every synapse has delay
 * `delay` (1..cfg->max_delay).  The diagonal takes part in propagation like
 * any entry (pass zeros for no self-synapses) but is never changed by STDP.
 * w = NULL starts every weight at zero (install them with sn_set_weights,
 * e.g. from device memory, without an n x n host copy).  Only SN_F32 is
 * supported (SN_EUNSUPPORTED otherwise). */
sn_status sn_create_dense(const sn_config *cfg, const sn_neurons *neurons,
                          const float *w, int32_t delay, sn_ctx **out);

/* Create a batched context: `nets` independent networks (neurons[b],
 * synapses[b] as for sn_create, indices local to each network) simulated
 * together, each with its own parameters.  Every network has 1..4096
 * neurons; cfg->max_delay <= 16.  The context's neuron index space is the
 * concatenation of the networks (network b's neuron j is global index
 * offset_b + j); sn_set_input and sn_set_poisson take global indices (the
 * Poisson stream of network b uses net = b and the local index j);
 * sn_get_state concatenates the states, and every raster row holds each
 * network's ceil(n_b/32) words in network order.  sn_run advances all
 * networks by the same number of steps in one persistent kernel launch,
 * replayed from a CUDA graph.  STDP and weight access are not available
 * for batched contexts (SN_EUNSUPPORTED / SN_ESTATE); sn_save / sn_load
 * are. */
sn_status sn_create_batch(const sn_config *cfg, int32_t nets, const sn_neurons *neurons,
                          const sn_synapses *synapses, sn_ctx **out);

/* Create one shared dense integer network driven by `trains` independent
 * input trains: every train has its own state, spikes and Poisson stream
 * (net = train index), and all share the weights w (row-major n x n int8,
 * w[i*n + j] = weight of i -> j, values -8..8; the diagonal acts like any
 * entry) and the neuron parameters (integers).  cfg->dtype must be SN_I32,
 * cfg->max_delay 1; n and trains multiples of 128.  Each step's synaptic
 * input of all trains is one tensor-core GEMM of the previous spikes with w
 * (Section 2.1: previous spike vector times the weight matrix), exact in
 * integers.  State (sn_get_state) is [trains][n]; every raster row holds
 * each train's n/32 words in train order; sn_set_poisson takes neuron
 * indices 0..n-1 and drives that neuron in every train.  Explicit events
 * and STDP are not available; sn_save / sn_load are. */
sn_status sn_create_shared_dense_i8(const sn_config *cfg, const sn_neurons *neurons, const int8_t *w,
                                    int32_t trains, sn_ctx **out);

/* Executor mapping of a batched context: networks with at most warp_max_n
 * neurons (0..512) run on a single warp, larger ones on a whole block; a
 * network's pending-input ring is held in shared memory while it runs when
 * it fits ring_smem_bytes (per block; a warp gets an eighth).  Results do
 * not depend on the mapping. */
sn_status sn_batch_config(sn_ctx *ctx, int32_t warp_max_n, int32_t ring_smem_bytes);

/* Time every mapping of a fixed candidate set on `trial_steps` steps of the
 * context's own networks and inputs, keep the fastest, then reset the
 * dynamic state (as sn_reset).  *best_ms (may be NULL) receives the time of
 * the chosen mapping.  Batched contexts: the warp/block split and the
 * shared-memory ring size.  Sparse contexts (sn_create): push or pull
 * propagation (pull only where it fits, never with STDP on). */
sn_status sn_autotune(sn_ctx *ctx, int32_t trial_steps, float *best_ms);

/* Replace the explicit external input (Section 2.1, third step of a
 * timestep): event e adds value[e] to neuron[e] at absolute step step[e] >= 0.
 * Events of one (step, neuron) are summed in the order given.  nev = 0 clears
 * the input.  SN_I32 contexts require integral values. */
sn_status sn_set_input(sn_ctx *ctx, int64_t nev, const int32_t *step,
                       const int32_t *neuron, const float *value);

/* Replace the Poisson sources.  Source k drives neuron[k] (each neuron at most
 * once): at absolute step t it adds amplitude[k] when
 *   u = SplitMix64(key ^ ((t << 32) | j)) >> 32  <  floor(rate[k] * 2^32)
 * with key = SplitMix64(seed ^ SplitMix64(net)), j the neuron index within its
 * network and net the network's index (0 for a single network, the train or
 * network index in batched contexts).  SplitMix64(x) is the published mixer:
 * z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
 * z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31.  rate is clamped to
 * [0, 1).  nsrc = 0 clears the sources. */
sn_status sn_set_poisson(sn_ctx *ctx, int32_t nsrc, const int32_t *neuron,
                         const float *rate, const float *amplitude, uint64_t seed);

/* sn_set_poisson with the stream's network index given explicitly.  A single
 * network uses key = SplitMix64(seed ^ SplitMix64(net)), so a single context
 * can reproduce network `net` of a batched context.  A batched or shared
 * dense context takes `net` as the global index of its first network or
 * train: network (train) b uses net + b.  A context holding networks
 * [k, k + nets) of a larger family (one shard of it, on one GPU of several)
 * then draws exactly the input those networks get in a context holding the
 * whole family.  Feedforward contexts: SN_ESTATE. */
sn_status sn_set_poisson_stream(sn_ctx *ctx, int32_t nsrc, const int32_t *neuron, const float *rate,
                                const float *amplitude, uint64_t seed, uint64_t net);

/* Enable (enable = 1) or disable pair-based STDP (Section 2.1 names STDP but
 * gives no formula; this is the trace form).  Each neuron keeps a trace
 * x <- decay * x + s after every step.  When i or j spikes at step t, the
 * weight of every synapse i -> j changes once, from the traces before the
 * step:  w <- clip(w + A+ * x_i * s_j(t) - A- * x_j * s_i(t), wmin, wmax).
 * Spike times are emission times (delays do not enter).  The new weight is
 * used from step t + 1.  Supported for SN_F32 networks (sparse and dense). */
sn_status sn_stdp(sn_ctx *ctx, float decay, float a_plus, float a_minus,
                  float wmin, float wmax, int32_t enable);

/* Propagation of a sparse network (sn_create), SN_PUSH or SN_PULL.
 *   push: each spike of step t adds its weights to the pending input of its
 *     targets for steps t + d (event-driven; work grows with the spike count).
 *   pull: each neuron sums, over its incoming synapses in descending delay,
 *     then ascending pre and input index, the weights whose pre-neuron spiked
 *     at t - d
 *     (Section 2.1's "spikes of the previous step times the weights", with
 *     delays); work is the synapse count every step, independent of activity.
 *     In SN_F32 mode this is exactly the FP32 mirror's order of additions.
 *     It needs max_delay * ceil(n/32) * 4 bytes of spike history in one
 *     block's shared memory (about 220 KiB) and n <= 1024 per SM; otherwise,
 *     or with STDP on, SN_EUNSUPPORTED.
 * The mode may change between any two sn_run calls: input already pending is
 * carried over exactly.  Enabling STDP selects push. */
#define SN_PUSH 0
#define SN_PULL 1
sn_status sn_set_propagation(sn_ctx *ctx, int32_t mode);
sn_status sn_get_propagation(const sn_ctx *ctx, int32_t *mode);

/* The pull store of a sparse context, built on the first pull run (or by
 * SN_PROP_PULL / sn_set_propagation).  Every synapse is one entry; the store
 * pads each region of a 32-neuron slice to the slice's longest list.
 *   *format  (may be NULL): 0 = not built yet, SN_PULL_PLAIN = 8 bytes per
 *            entry (bit offset, weight), SN_PULL_CODED = 6 bytes per entry
 *            (weight and the 16-bit step of the bit offset from the previous
 *            entry; a larger step takes filler entries of weight 0);
 *   *bytes   (may be NULL): device bytes of the store, padding included;
 *   *entries (may be NULL): entries of all lists, fillers included
 *            (m when there are none).
 * SN_EINVAL for a context that is not a sparse network. */
sn_status sn_pull_store_info(const sn_ctx *ctx, int32_t *format, int64_t *bytes, int64_t *entries);

/* Advance `steps` timesteps (steps >= 0) from the current step.  Queued on the
 * context's stream; a step counter makes repeated calls continue the run. */
sn_status sn_run(sn_ctx *ctx, int32_t steps);

/* Return the dynamic state to that of a new context: step 0, V = reset,
 * r = 0, no pending synaptic input, zero STDP traces, zero counters, empty
 * raster.  Weights and inputs are kept (weights changed by STDP stay
 * changed).  Queued on the stream; allocates nothing. */
sn_status sn_reset(sn_ctx *ctx);

/* Wait for queued work; report a latched device status (SN_ETIMEOUT,
 * SN_EOVERFLOW) if any. */
sn_status sn_sync(sn_ctx *ctx);

/* Spike raster of steps [t0, t1): row k holds ceil(n/32) 32-bit words for
 * step t0 + k; bit (j % 32) of word (j / 32) is s_j.  Batched contexts lay
 * out each network's (or train's) words one after another in every row.
 * The steps must have been run and lie within the last record_steps steps.
 * on_device = 1: `bits` is a device pointer and the copy is queued on the
 * stream; 0: host memory, the call synchronises. */
sn_status sn_get_spikes(sn_ctx *ctx, int64_t t0, int64_t t1, uint32_t *bits,
                        int32_t on_device);

/* Current state: v (float, or int32 in SN_I32 mode) and the refractory
 * countdown r, n values each (batched: concatenated).  Either pointer may be
 * NULL. */
sn_status sn_get_state(sn_ctx *ctx, void *v, int32_t *refractory, int32_t on_device);

/* STDP traces x (n floats). */
sn_status sn_get_trace(sn_ctx *ctx, float *trace, int32_t on_device);

/* Current weights: m floats in the order the synapses were given to
 * sn_create, or n*n floats row-major for a dense network. */
sn_status sn_get_weights(sn_ctx *ctx, float *w, int32_t on_device);

/* Replace the weights (the inverse of sn_get_weights, same layout: m floats
 * in input order, or n*n floats row-major for a dense network; Section 2.1's
 * synapse weights).  on_device = 1: `w` is a device pointer, copied on the
 * stream without validation; 0: host memory (NaN rejected with SN_EINVAL),
 * copied before the call returns.  Delays and the state are kept.  A spike
 * delivered at step t uses the weight in place at t (Section 2.2's delay
 * registers carry the spike; the weight applies on delivery): for a sparse
 * context the call rebuilds the input of
 * spikes still in flight from the raster, which must then hold the last
 * max_delay steps (record_steps >= max_delay, else SN_EUNSUPPORTED); a dense
 * context accepts new weights only at step 0 (after creation, sn_reset or an
 * sn_load of a step-0 checkpoint; SN_ESTATE otherwise).  Dense contexts and
 * SN_F32 sparse contexts (SN_EUNSUPPORTED for SN_I32, SN_ESTATE for other
 * kinds). */
sn_status sn_set_weights(sn_ctx *ctx, const float *w, int32_t on_device);

/* Steps run so far, total spikes and total synaptic events (one event = one
 * spike delivered along one synapse), counted on the device. */
sn_status sn_get_counters(sn_ctx *ctx, int64_t *steps, int64_t *spikes, int64_t *events);

/* Checkpoint: sn_save with buf == NULL stores the needed size in *size;
 * otherwise it writes the full dynamic state (step counter, V, refractory
 * countdowns, pending synaptic input and the recent spikes whose deliveries
 * are due, STDP traces, weights, counters) into
 * buf.  sn_load restores it into a context created with the same network.
 * A run of T steps equals a run of T1 steps, save, load into a fresh
 * context, and a run of T - T1 steps.  Single sparse and dense networks,
 * batched networks (state and pending input of every network; the synapses
 * never change) and the shared dense network (every train's state and the
 * previous step's spikes); feedforward contexts return SN_ESTATE.  sn_load
 * returns SN_EINVAL for a checkpoint of another kind, dtype, size, synapse
 * count, delay range, network count or train count. */
sn_status sn_save(sn_ctx *ctx, void *buf, size_t *size);
sn_status sn_load(sn_ctx *ctx, const void *buf, size_t size);

/* Message for the last failure of ctx (or of the last failed create call
 * when ctx is NULL).  Valid until the next call on the same context. */
const char *sn_last_error(const sn_ctx *ctx);

/* Free the context and its device memory (NULL is ignored). */
void sn_destroy(sn_ctx *ctx);

/* ------------------------------------------------------------------------
 * Feedforward spiking network trained by backpropagation through time.  The
 * paper names SNN training only as a use (Section 1); the forward pass is the
 * simulator's timestep (Section 2.1 order and rules) applied layer by layer.
 *
 * Layer l = 1..L maps sizes[l-1] inputs to sizes[l] LIF neurons; synapse
 * i -> j has weight W_l[i][j] (row-major [sizes[l-1]][sizes[l]]) and delay
 * D_l[i][j] in 1..4, so a spike of layer l-1 at step t reaches layer l at
 * t + D.  Layer 0 is the input spike train.  The output is the spike count
 * of each neuron of layer L.  All neurons share the parameters in
 * sn_ff_params.  Gradients use the fast-sigmoid surrogate
 * ds/du = 1 / (1 + slope |u - threshold|)^2 (u = state compared with the
 * threshold), a detached reset, a constant refractory mask and the clamped
 * leak's derivative [|V - reset| > leak]; delays get no gradient.  The
 * forward keeps every spike (as bits) and the membrane state every
 * checkpoint_every steps; the backward recomputes each segment's states from
 * its checkpoint.  Results do not depend on thread timing.
 * ------------------------------------------------------------------------ */
typedef struct {
    float threshold, leak, reset;
    int32_t refractory;
    float surrogate_slope;
    int32_t checkpoint_every;       /* 1, 2, 5, 10 or 20                          */
} sn_ff_params;

/* delays[l] (host, [sizes[l]][sizes[l+1]] bytes for layer l+1) are copied.
 * batch >= 1, steps >= 1; every size in 1..65536.  By default the forward
 * keeps every layer's synaptic input [steps * batch][sizes[l]] for the
 * backward; with SN_FF_RECOMPUTE in cfg->flags (or when that memory cannot
 * be allocated) the backward recomputes it with the forward's own kernel.
 * Both give identical results. */
sn_status sn_create_ff(const sn_config *cfg, int32_t layers, const int32_t *sizes,
                       const uint8_t *const *delays, const sn_ff_params *params, int32_t batch,
                       int32_t steps, sn_ctx **out);

/* Forward pass.  input: device [steps][batch][sizes[0]] bytes (nonzero =
 * spike); w: host array of `layers` device pointers to the weights (kept
 * unchanged until the matching sn_backward); counts: device
 * [batch][sizes[L]] floats out. */
sn_status sn_ff_forward(sn_ctx *ctx, const uint8_t *input, const float *const *w, float *counts);

/* Backward pass of the last forward: grad_counts = dLoss/dcounts (device
 * [batch][sizes[L]]); grad_w: host array of `layers` device pointers that
 * receive dLoss/dW_l.  on_device must be 1. */
sn_status sn_backward(sn_ctx *ctx, const float *grad_counts, float *const *grad_w, int32_t on_device);

/* Engine of the contractions (synaptic input, weight gradient, spike
 * gradient): SN_FF_SIMT (CUDA-core FP32; exploits spike sparsity) or
 * SN_FF_TENSOR (tcgen05 BF16 tensor cores: one GEMM per delay with the
 * weights of that delay).  On the tensor cores the forward multiplies 0/1
 * spikes by an exact three-part BF16 split of every weight and adds the
 * partial sums of each 64-input block in FP32 (so forward states differ from
 * the SIMT engine's only in the order of FP32 additions); the backward uses
 * two-part BF16 splits of weights and gradients (about 16 significant bits
 * per factor, relative error near 2^-16 per product).  SN_FF_AUTO (the
 * default) takes the tensor cores where the shapes allow (batch a multiple
 * of 8); SN_FF_TENSOR on shapes that do not fit returns SN_EUNSUPPORTED.
 * sn_backward always uses the engine of the forward it differentiates. */
#define SN_FF_AUTO 0
#define SN_FF_SIMT 1
#define SN_FF_TENSOR 2
sn_status sn_ff_set_engine(sn_ctx *ctx, int32_t engine);

/* Spikes of layer l (0 = input) of the last forward: [steps][batch][ceil(n_l/32)]
 * words.  Membrane checkpoints of layer l >= 1: [steps/k][batch][n_l] floats,
 * entry c = state after step (c+1)k - 1. */
sn_status sn_ff_get_spikes(sn_ctx *ctx, int32_t layer, uint32_t *bits, int32_t on_device);
sn_status sn_ff_get_checkpoints(sn_ctx *ctx, int32_t layer, float *v, int32_t on_device);

/* ------------------------------------------------------------------------
 * Dense run without allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, for example a
 * host application whose device memory is all reserved by its own pool
 * allocator, or a plug-in whose host process does not let it allocate.
 *
 * It simulates `steps` timesteps (steps 0 .. steps-1) of an all-to-all
 * network exactly as sn_create_dense + sn_run would (bit for bit), on buffers
 * the caller owns, starting from the caller's state with no synaptic input
 * pending and no explicit events.  Every pointer below is a device pointer:
 *   w                  [n*n] row-major weights (row = pre), read only
 *   threshold, leak, reset [n] float; refractory [n] int32
 *   poisson_threshold  [n] uint32 = floor(rate * 2^32) per neuron (0: none),
 *                      poisson_amplitude [n] float; both NULL for no input;
 *                      the stream key is derived from seed as in
 *                      sn_set_poisson with net = 0
 *   v, r               [n] state in/out (start: v = reset, r = 0)
 *   raster             [steps * ceil(n/32)] uint32 out, row k = step k
 * The kernel's scratch (spike bits of the last two steps, pending-input
 * ring, control block) lives in one static device array of
 * SN_NOALLOC_SCRATCH_BYTES, held by every device that loads the library until
 * the process exits.  A network needs
 *   256 + 256-rounded(8 * ceil(n/32)) + 256-rounded(4 * (delay + 1) * n)
 *       + 256-rounded(4 * n) bytes
 * of it (so every network up to the 200,000-neuron dense limit fits while
 * delay <= 18); a larger need is rejected with SN_EINVAL before any CUDA
 * call, with the sizes in sn_last_error(NULL).  The first call on a device
 * looks up the array's device address with that device current.  Every call
 * shares the array and clears it first, so calls whose work overlaps on the
 * GPU (two streams, two threads) race and must not be issued.  The call
 * waits for its work to finish and returns the device status (SN_ETIMEOUT if
 * a grid barrier gave up); messages of failures go to sn_last_error(NULL).
 * ------------------------------------------------------------------------ */
#define SN_NOALLOC_SCRATCH_BYTES (16u << 20)

typedef struct {
    int32_t n;
    int32_t delay;                  /* 1 .. SN_MAX_DELAY                         */
    int32_t steps;
    int32_t pad;
    const float *w;
    const float *threshold;
    const float *leak;
    const float *reset;
    const int32_t *refractory;
    const uint32_t *poisson_threshold;
    const float *poisson_amplitude;
    uint64_t seed;
    float *v;
    int32_t *r;
    uint32_t *raster;
    void *cuda_stream;              /* cudaStream_t, NULL = default stream       */
} sn_dense_noalloc_args;

sn_status sn_run_dense_noalloc(const sn_dense_noalloc_args *args);

/* Failure-detection self-test.  Launches on cuda_stream (NULL = default
 * stream) a kernel of four blocks whose grid barrier one block never
 * reaches, so that the other blocks' bounded wait runs out (after about 2 s
 * of wall-clock time); *status receives the status the kernel latched:
 * SN_ETIMEOUT when the bound works.  Nothing faults or traps, and the CUDA
 * context stays usable.  Returns SN_OK when the self-test ran, SN_EINVAL for
 * a NULL status, SN_ENOMEM or SN_ECUDA when it could not run. */
sn_status sn_selftest_barrier_timeout(void *cuda_stream, int32_t *status);

/* Library version string. */
const char *sn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SN_H */
