// Host side of the feedforward (BPTT) context: buffers, the delay bit masks,
// and the launch sequences of the forward and backward passes (sn_ff.cu).

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sn_ctx.h"

extern "C" {

sn_status sn_create_ff(const sn_config *cfg, int32_t layers, const int32_t *sizes, const uint8_t *const *delays,
                       const sn_ff_params *p, int32_t batch, int32_t steps, sn_ctx **out) {
    if (!cfg || !sizes || !delays || !p || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    if (layers < 1 || layers > 16) return fail(nullptr, SN_EINVAL, "layers must be in 1..16");
    if (batch < 1 || steps < 1) return fail(nullptr, SN_EINVAL, "batch and steps must be >= 1");
    const int k = p->checkpoint_every;
    if (!(k == 1 || k == 2 || k == 5 || k == 10 || k == 20))
        return fail(nullptr, SN_EINVAL, "checkpoint_every must be 1, 2, 5, 10 or 20");
    if (!std::isfinite(p->threshold) || !std::isfinite(p->leak) || p->leak < 0 || !std::isfinite(p->reset) ||
        p->refractory < 0 || !std::isfinite(p->surrogate_slope) || p->surrogate_slope < 0)
        return fail(nullptr, SN_EINVAL, "bad neuron or surrogate parameters");
    for (int l = 0; l <= layers; ++l)
        if (sizes[l] < 1 || sizes[l] > 65536) return fail(nullptr, SN_EINVAL, "sizes must be in 1..65536");
    if ((long long)steps * batch * std::max(1, *std::max_element(sizes, sizes + layers + 1)) >= (1ll << 33))
        return fail(nullptr, SN_EINVAL, "steps * batch * size too large");
    for (int l = 0; l < layers; ++l) {
        if (!delays[l]) return fail(nullptr, SN_EINVAL, "delay array is NULL");
        const size_t cnt = (size_t)sizes[l] * sizes[l + 1];
        for (size_t q = 0; q < cnt; ++q)
            if (delays[l][q] < 1 || delays[l][q] > 4) return fail(nullptr, SN_EINVAL, "delays must be in 1..4");
    }
    sn_ctx *c = new (std::nothrow) sn_ctx();
    if (!c) return fail(nullptr, SN_ENOMEM, "host allocation failed");
    c->kind = KIND_FF;
    c->dtype = SN_F32;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    c->ff_layers = layers;
    c->ff_sizes.assign(sizes, sizes + layers + 1);
    c->ff_batch = batch;
    c->ff_steps = steps;
    c->ff_k = k;
    c->ff_theta = p->threshold; c->ff_leak = p->leak; c->ff_reset = p->reset;
    c->ff_refr = p->refractory; c->ff_slope = p->surrogate_slope;
    c->n = sizes[layers];
    auto bail = [&](sn_status st) { std::string msg = c->err.empty() ? g_create_err : c->err;
                                    destroy_all(c); delete c; g_create_err = msg; return st; };
    const long long rows = (long long)steps * batch;
    const int nmax = *std::max_element(sizes, sizes + layers + 1);
    int nin_max = 0, nout_max = 0;
    c->ff_D.assign(layers, nullptr);
    c->ff_DM.assign(layers, nullptr);
    c->ff_S.assign(layers + 1, nullptr);
    c->ff_vck.assign(layers + 1, nullptr);
    c->ff_rck.assign(layers + 1, nullptr);
    sn_status s;
    const int C = steps / k;
    for (int l = 0; l <= layers; ++l) {
        const int words = (sizes[l] + 31) / 32;
        if ((s = dalloc(c, &c->ff_S[l], (size_t)rows * words * 4))) return bail(s);
        if (l >= 1) {
            if ((s = dalloc(c, &c->ff_vck[l], (size_t)std::max(C, 1) * batch * sizes[l] * 4)) ||
                (s = dalloc(c, &c->ff_rck[l], (size_t)std::max(C, 1) * batch * sizes[l] * 4)))
                return bail(s);
        }
    }
    for (int l = 0; l < layers; ++l) {
        const int nin = sizes[l], nout = sizes[l + 1];
        nin_max = std::max(nin_max, nin);
        nout_max = std::max(nout_max, nout);
        const size_t cnt = (size_t)nin * nout;
        const int chunks = (nin + 31) / 32;
        // per 32-input chunk and output column: one bit mask per delay
        std::vector<unsigned> dm((size_t)chunks * nout * 4, 0u);
        for (int i = 0; i < nin; ++i)
            for (int j = 0; j < nout; ++j) {
                const int d = delays[l][(size_t)i * nout + j];
                dm[((size_t)(i / 32) * nout + j) * 4 + (d - 1)] |= 1u << (i % 32);
            }
        if ((s = dalloc(c, &c->ff_D[l], cnt)) || (s = dalloc(c, &c->ff_DM[l], dm.size() * 4))) return bail(s);
        cudaError_t e;
        if ((e = cudaMemcpy(c->ff_D[l], delays[l], cnt, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->ff_DM[l], dm.data(), dm.size() * 4, cudaMemcpyHostToDevice))) {
            c->err = std::string("upload: ") + cudaGetErrorString(e);
            return bail(SN_ECUDA);
        }
    }
    // weight-gradient splits over the (t, b) rows: enough blocks to fill the GPU
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long base_blocks = (long long)((nout_max + 255) / 256) * ((nin_max + 31) / 32);
    c->ff_splits = (int)std::max(1LL, std::min<long long>(64, (4LL * sms + base_blocks - 1) / std::max(1LL, base_blocks)));
    if ((s = dalloc(c, &c->ff_I, (size_t)rows * nmax * 4)) || (s = dalloc(c, &c->ff_gI, (size_t)rows * nmax * 4)) ||
        (s = dalloc(c, &c->ff_gS, (size_t)rows * nmax * 4)) ||
        (s = dalloc(c, &c->ff_part, (size_t)c->ff_splits * nin_max * nout_max * 4)) ||
        (s = dalloc(c, &c->ctl, sizeof(Control))))
        return bail(s);
    if (cudaMemset(c->ctl, 0, sizeof(Control)) != cudaSuccess) return bail(SN_ECUDA);
    c->ff_w.assign(layers, nullptr);
    *out = c;
    return SN_OK;
}

sn_status sn_ff_forward(sn_ctx *c, const uint8_t *input, const float *const *w, float *counts) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (!input || !w || !counts) return fail(c, SN_EINVAL, "NULL argument");
    for (int l = 0; l < c->ff_layers; ++l)
        if (!w[l]) return fail(c, SN_EINVAL, "weight pointer is NULL");
    const int B = c->ff_batch, T = c->ff_steps, L = c->ff_layers;
    const int rows = B * T;
    cudaError_t e = ff_pack(input, rows, c->ff_sizes[0], (c->ff_sizes[0] + 31) / 32, c->ff_S[0], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "input pack");
    for (int l = 1; l <= L; ++l) {
        const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
        c->ff_w[l - 1] = w[l - 1];
        if ((e = ff_delay_fwd(c->ff_S[l - 1], (nin + 31) / 32, w[l - 1], c->ff_DM[l - 1], nin, nout, B, 0, rows,
                              c->ff_I, c->stream)))
            return cuda_fail(c, e, "forward synaptic input");
        if ((e = ff_scan_fwd(c->ff_I, nout, B, T, c->ff_k, c->ff_theta, c->ff_leak, c->ff_reset, c->ff_refr,
                             c->ff_S[l], c->ff_vck[l], c->ff_rck[l], l == L ? counts : nullptr, c->stream)))
            return cuda_fail(c, e, "forward recurrence");
    }
    c->ff_have_forward = true;
    return SN_OK;
}

sn_status sn_backward(sn_ctx *c, const float *grad_counts, float *const *grad_w, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (!on_device) return fail(c, SN_EUNSUPPORTED, "sn_backward takes device buffers (on_device = 1)");
    if (!c->ff_have_forward) return fail(c, SN_ESTATE, "no forward pass to differentiate");
    if (!grad_counts || !grad_w) return fail(c, SN_EINVAL, "NULL argument");
    const int B = c->ff_batch, T = c->ff_steps, L = c->ff_layers;
    const int rows = B * T;
    cudaError_t e;
    for (int l = L; l >= 1; --l) {
        const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
        const int words_in = (nin + 31) / 32;
        if (!grad_w[l - 1]) return fail(c, SN_EINVAL, "gradient pointer is NULL");
        // recompute the synaptic input (the forward kept only spikes and checkpoints)
        if ((e = ff_delay_fwd(c->ff_S[l - 1], words_in, c->ff_w[l - 1], c->ff_DM[l - 1], nin, nout, B, 0, rows,
                              c->ff_I, c->stream)))
            return cuda_fail(c, e, "recompute synaptic input");
        if ((e = ff_scan_bwd(c->ff_I, nout, B, T, c->ff_k, c->ff_theta, c->ff_leak, c->ff_reset, c->ff_refr,
                             c->ff_slope, c->ff_vck[l], c->ff_rck[l], l == L ? nullptr : c->ff_gS,
                             l == L ? grad_counts : nullptr, c->ff_gI, c->stream)))
            return cuda_fail(c, e, "adjoint recurrence");
        if ((e = ff_dw(c->ff_gI, c->ff_S[l - 1], words_in, c->ff_D[l - 1], nin, nout, B, T, c->ff_splits,
                       c->ff_part, grad_w[l - 1], c->stream)))
            return cuda_fail(c, e, "weight gradient");
        if (l > 1 && (e = ff_bwd_data(c->ff_gI, c->ff_w[l - 1], c->ff_D[l - 1], nin, nout, B, T, c->ff_gS,
                                      c->stream)))
            return cuda_fail(c, e, "spike gradient");
    }
    return SN_OK;
}

sn_status sn_ff_get_spikes(sn_ctx *c, int32_t layer, uint32_t *bits, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (layer < 0 || layer > c->ff_layers || !bits) return fail(c, SN_EINVAL, "bad layer or buffer");
    const size_t bytes = (size_t)c->ff_steps * c->ff_batch * ((c->ff_sizes[layer] + 31) / 32) * 4;
    SN_CUDA(c, cudaMemcpyAsync(bits, c->ff_S[layer], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
    if (!on_device) SN_CUDA(c, cudaStreamSynchronize(c->stream));
    return SN_OK;
}

sn_status sn_ff_get_checkpoints(sn_ctx *c, int32_t layer, float *v, int32_t on_device) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (layer < 1 || layer > c->ff_layers || !v) return fail(c, SN_EINVAL, "bad layer or buffer");
    const size_t bytes = (size_t)(c->ff_steps / c->ff_k) * c->ff_batch * c->ff_sizes[layer] * 4;
    if (bytes == 0) return SN_OK;
    SN_CUDA(c, cudaMemcpyAsync(v, c->ff_vck[layer], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               c->stream));
    if (!on_device) SN_CUDA(c, cudaStreamSynchronize(c->stream));
    return SN_OK;
}

}  // extern "C"
