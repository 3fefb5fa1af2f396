/*
 * Plain CPU oracle for the time-stepped LIF spiking-network simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the simulator computes.  It is used by the tests, by the
 * benchmark's CPU-baseline leg and by the smoke check; the library never calls,
 * links or includes it, and it shares no code with the CUDA path.
 *
 * Source of each rule (SuperNeuro, arXiv 2305.02510):
 *   - LIF neuron with four parameters: threshold, leak, reset state and
 *     refractory period (Section 2.1 "The MAT Mode"; Section 2.2).
 *   - Constant leak that moves the state toward the reset state; it is
 *     clamped at the reset state (our reading; see the leak rule below).
 *   - Per timestep, in this order (Section 2.1): apply the leak; add the
 *     previous spikes times the weight matrix; add the external spikes of the
 *     current step; compare with the thresholds; zero the spikes of neurons in
 *     their refractory period.
 *   - A spike crosses the threshold strictly ("greater than", Section 2.2).
 *   - Synaptic delays: a spike emitted at step t reaches the post-neuron at
 *     t + d (delay registers, Section 2.2; proxy chains of unit-delay hops,
 *     Section 2.1).
 *   - STDP exists in the paper without a formula (Section 2.1); the pair-based
 *     rule here is the trace form given in the function stdp_apply below.
 *
 * Precision modes.  Every value is held in a double.
 *   ORC_F64: double arithmetic throughout (the reference trajectory).
 *   ORC_F32: after every arithmetic operation the result is rounded to float.
 *            For +, -, * of float operands, rounding the exact double result
 *            to float gives the correctly rounded float result, so this is
 *            float arithmetic in the canonical order stated below.
 *   ORC_INT: integer values; all operations are exact in double while the
 *            magnitudes stay below 2^53 (checked: the state compared with
 *            the threshold must stay below 2^31 in magnitude).
 * Canonical order of the synaptic sum for post-neuron j at step t (the paper
 * fixes none: Section 2.1 writes the input as the spikes times the weights,
 * Section 2.2 as the deliveries of the delay registers): the arrivals are
 * added oldest spike first, i.e.
 *   acc = 0; for each incoming synapse in descending delay, then ascending
 *   pre and input index: if pre spiked at t - delay: acc = acc + w.
 * Then V = (L(V) + acc) + ext.
 * External input of (t, j): the explicit events of (t, j) in the order given,
 * then the Poisson source of j (if any), summed into ext starting from 0.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fused
 * multiply-add).  The per-neuron loop of a step may run on several threads
 * (orc_set_threads; 1 by default): each neuron's sum, update and spike depend
 * only on earlier steps and on its own state, so the result is the same bit
 * for bit on any number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { ORC_F64 = 0, ORC_F32 = 1, ORC_INT = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EOVERFLOW = 3 };

/* A network and its inputs, as plain arrays (all caller-owned). */
typedef struct {
    int32_t mode;            /* ORC_F64 / ORC_F32 / ORC_INT                  */
    int32_t n;               /* neurons                                      */
    int32_t max_delay;       /* D >= 1; history kept for D steps              */
    int32_t dense;           /* 1: all-to-all matrix form                    */
    const double *threshold, *leak, *reset;   /* [n]                        */
    const int32_t *refractory;                /* [n]                        */
    /* sparse form: synapse k is pre[k] -> post[k], weight[k], delay[k]      */
    int64_t m;
    const int32_t *pre, *post, *delay;
    double *weight;          /* [m], updated in place by STDP                */
    /* dense form: w_dense[i*n + j] is the weight of i -> j (i == j included) */
    double *w_dense;         /* [n*n], updated in place by STDP              */
    int32_t dense_delay;
    /* explicit external events (absolute steps)                            */
    int64_t nev;
    const int32_t *ev_step, *ev_neuron;
    const double *ev_value;
    /* counter-hash Poisson sources                                          */
    int32_t nsrc;
    const int32_t *src_neuron;
    const uint32_t *src_rate_u32;
    const double *src_amp;
    uint64_t seed;
    uint64_t net;
    /* STDP (pair-based, nearest-trace form)                                 */
    int32_t stdp;
    double decay, a_plus, a_minus, wmin, wmax;
} orc_net;

/* ---------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), in the form of its public-domain reference
 * implementation: advance the state by the golden gamma, then mix.          */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

/* 32-bit uniform of (seed, net, t, j): the counter-based Poisson stream. */
uint32_t orc_poisson_u32(uint64_t seed, uint64_t net, uint32_t t, uint32_t j)
{
    uint64_t key = splitmix64(seed ^ splitmix64(net));
    uint64_t ctr = ((uint64_t)t << 32) | (uint64_t)j;
    return (uint32_t)(splitmix64(key ^ ctr) >> 32);
}

/* ---------------------------------------------------------------------- */
static int g_mode;
static int g_threads = 1;

/* Threads for the per-neuron loop of each step (k >= 1); returns the count. */
int orc_set_threads(int k)
{
    g_threads = k < 1 ? 1 : k;
    return g_threads;
}

static double R(double x)
{
    return g_mode == ORC_F32 ? (double)(float)x : x;
}

/* Constant leak toward the reset state, clamped at it (Section 2.1). */
static double leak_toward_reset(double v, double leak, double reset)
{
    if (v > reset) {
        double u = R(v - leak);
        return u > reset ? u : reset;
    }
    if (v < reset) {
        double u = R(v + leak);
        return u < reset ? u : reset;
    }
    return reset;
}

typedef struct { int32_t d, pre; int64_t k; } inc_key;

static int cmp_inc(const void *a, const void *b)
{
    const inc_key *x = (const inc_key *)a, *y = (const inc_key *)b;
    if (x->d != y->d) return x->d > y->d ? -1 : 1;      /* oldest spike (largest delay) first */
    if (x->pre != y->pre) return x->pre < y->pre ? -1 : 1;
    return x->k < y->k ? -1 : (x->k > y->k);
}

/* Pair-based STDP for the spikes s of one step.  x holds each neuron's trace
 * before this step.  For every existing synapse i -> j (diagonal excluded in
 * the dense form): dw = A+ * x_i * s_j - A- * x_j * s_i, applied once, then
 * w = clip(w + dw, wmin, wmax).  Spike times are emission times. */
static void stdp_apply(const orc_net *net, const uint8_t *s, const double *x)
{
    const int n = net->n;
    if (net->dense) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j || !(s[i] || s[j])) continue;
                double dw = 0.0;
                if (s[j]) dw = R(dw + R(net->a_plus * x[i]));
                if (s[i]) dw = R(dw - R(net->a_minus * x[j]));
                double w = R(net->w_dense[(int64_t)i * n + j] + dw);
                if (w < net->wmin) w = net->wmin;
                if (w > net->wmax) w = net->wmax;
                net->w_dense[(int64_t)i * n + j] = w;
            }
    } else {
        for (int64_t k = 0; k < net->m; ++k) {
            int i = net->pre[k], j = net->post[k];
            if (!(s[i] || s[j])) continue;
            double dw = 0.0;
            if (s[j]) dw = R(dw + R(net->a_plus * x[i]));
            if (s[i]) dw = R(dw - R(net->a_minus * x[j]));
            double w = R(net->weight[k] + dw);
            if (w < net->wmin) w = net->wmin;
            if (w > net->wmax) w = net->wmax;
            net->weight[k] = w;
        }
    }
}

/*
 * Run `steps` timesteps starting at absolute step t0.
 *
 * State (in/out):
 *   v[n]          internal state (membrane potential)
 *   r[n]          refractory countdown: a spike at t blocks t+1 .. t+R
 *   hist[D*n]     spikes of steps t0-D .. t0-1, row k = step t0-D+k
 *   trace[n]      STDP trace (used when net->stdp)
 * Outputs (optional, may be NULL):
 *   raster[steps*n]  spikes of each step
 *   vtrace[steps*n]  state after each step
 *   ctrace[steps*n]  state compared with the threshold in each step (after
 *                    input, before reset)
 * Returns ORC_OK or an error code.
 */
int orc_run(const orc_net *net, int64_t t0, int32_t steps,
            double *v, int32_t *r, uint8_t *hist, double *trace,
            uint8_t *raster, double *vtrace, double *ctrace)
{
    const int n = net->n, D = net->max_delay;
    if (n < 0 || D < 1 || steps < 0) return ORC_EINVAL;
    g_mode = net->mode;

    /* incoming synapses of each post-neuron, in canonical order */
    int64_t *inc_ptr = NULL, *inc = NULL;
    if (!net->dense) {
        inc_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        inc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(net->m > 0 ? net->m : 1));
        inc_key *keys = (inc_key *)malloc(sizeof(inc_key) * (size_t)(net->m > 0 ? net->m : 1));
        int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        if (!inc_ptr || !inc || !keys || !fill) return ORC_ENOMEM;
        for (int64_t k = 0; k < net->m; ++k) {
            if (net->pre[k] < 0 || net->pre[k] >= n || net->post[k] < 0 ||
                net->post[k] >= n || net->delay[k] < 1 || net->delay[k] > D)
                return ORC_EINVAL;
            inc_ptr[net->post[k] + 1]++;
        }
        for (int j = 0; j < n; ++j) inc_ptr[j + 1] += inc_ptr[j];
        for (int64_t k = 0; k < net->m; ++k) {
            int j = net->post[k];
            inc_key *e = &keys[inc_ptr[j] + fill[j]++];
            e->d = net->delay[k]; e->pre = net->pre[k]; e->k = k;
        }
        for (int j = 0; j < n; ++j)
            qsort(keys + inc_ptr[j], (size_t)(inc_ptr[j + 1] - inc_ptr[j]),
                  sizeof(inc_key), cmp_inc);
        for (int64_t k = 0; k < net->m; ++k) inc[k] = keys[k].k;
        free(keys); free(fill);
    } else if (net->dense_delay < 1 || net->dense_delay > D) {
        return ORC_EINVAL;
    }

    /* spike history: rows for steps t0-D .. t0+steps-1 */
    uint8_t *sp = (uint8_t *)calloc((size_t)(D + steps) * (size_t)(n > 0 ? n : 1), 1);
    double *ext = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int32_t *src_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *xold = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!sp || !ext || !src_of || !xold) return ORC_ENOMEM;
    memcpy(sp, hist, (size_t)D * n);
    for (int j = 0; j < n; ++j) src_of[j] = -1;
    for (int k = 0; k < net->nsrc; ++k) src_of[net->src_neuron[k]] = k;

    int status = ORC_OK;
    for (int32_t s = 0; s < steps; ++s) {
        const int64_t t = t0 + s;
        const uint8_t *cur_prev = sp;          /* row index base: step t0-D */
        uint8_t *cur = sp + (size_t)(D + s) * n;

        /* external input of step t */
        for (int j = 0; j < n; ++j) ext[j] = 0.0;
        for (int64_t e = 0; e < net->nev; ++e)
            if (net->ev_step[e] == t) {
                int j = net->ev_neuron[e];
                ext[j] = R(ext[j] + net->ev_value[e]);
            }
        for (int j = 0; j < n; ++j)
            if (src_of[j] >= 0) {
                int k = src_of[j];
                uint32_t u = orc_poisson_u32(net->seed, net->net, (uint32_t)t, (uint32_t)j);
                if (u < net->src_rate_u32[k]) ext[j] = R(ext[j] + net->src_amp[k]);
            }

        int overflow = 0;
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(| : overflow)
        for (int j = 0; j < n; ++j) {
            /* synaptic input: spikes of t-d reach j at t */
            double acc = 0.0;
            if (net->dense) {
                const int d = net->dense_delay;
                const uint8_t *row = cur_prev + (size_t)(D + s - d) * n;
                for (int i = 0; i < n; ++i)
                    if (row[i]) acc = R(acc + net->w_dense[(int64_t)i * n + j]);
            } else {
                for (int64_t q = inc_ptr[j]; q < inc_ptr[j + 1]; ++q) {
                    int64_t k = inc[q];
                    int d = net->delay[k];
                    if (cur_prev[(size_t)(D + s - d) * n + net->pre[k]])
                        acc = R(acc + net->weight[k]);
                }
            }
            double vj = leak_toward_reset(v[j], net->leak[j], net->reset[j]);
            vj = R(vj + acc);
            vj = R(vj + ext[j]);
            if (ctrace) ctrace[(size_t)s * n + j] = vj;
            /* integer mode: the integrated state must fit int32 */
            if (net->mode == ORC_INT && fabs(vj) >= 2147483648.0) overflow = 1;
            /* threshold (strict), refractory mask, reset */
            int fire = (vj > net->threshold[j]) && (r[j] == 0);
            if (fire) {
                vj = net->reset[j];
                r[j] = net->refractory[j];
            } else if (r[j] > 0) {
                r[j] -= 1;
            }
            v[j] = vj;
            cur[j] = (uint8_t)fire;
        }
        if (overflow) status = ORC_EOVERFLOW;

        if (net->stdp) {
            for (int j = 0; j < n; ++j) xold[j] = trace[j];
            stdp_apply(net, cur, xold);
            for (int j = 0; j < n; ++j)
                trace[j] = R(R(net->decay * trace[j]) + (double)cur[j]);
        }
        if (raster) memcpy(raster + (size_t)s * n, cur, (size_t)n);
        if (vtrace) memcpy(vtrace + (size_t)s * n, v, sizeof(double) * (size_t)n);
    }
    memcpy(hist, sp + (size_t)steps * n, (size_t)D * n);
    free(sp); free(ext); free(src_of); free(xold);
    free(inc_ptr); free(inc);
    return status;
}
