// Host side of the feedforward (BPTT) context: buffers, the delay bit masks,
// and the launch sequences of the forward and backward passes (sn_ff.cu).

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "sn_ctx.h"

namespace sn {
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline int up(int x, int m) { return (x + m - 1) / m * m; }

// Row-major BF16 [rows][cols] (cols a multiple of 64), boxes of 128 rows x 64
// columns, 128-byte swizzle; coordinates outside the tensor read as zero.
sn_status bf16_map(sn_ctx *c, CUtensorMap *out, const void *base, long long rows, long long cols) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, 128};
    cuuint32_t es[2] = {1, 1};
    CUresult r = ((EncodeTiledFn)c->ff_encode)(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides,
                                               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, SN_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SN_OK;
}

bool use_tc(const sn_ctx *c) { return c->ff_tc_ok && c->ff_engine != SN_FF_SIMT; }

// Synaptic input of layer l for all rows, I[r][j] = sum_d sum_i S[r - dB][i] W_d[i][j]:
// 4 delays x 3 exact BF16 weight parts (4 passes of 3 parts each), accumulated
// block by block (ff_tc_forward).  Unpacks the previous layer's spikes, and their transpose
// when the weight gradient will need it.
sn_status tc_forward(sn_ctx *c, int l, bool want_st, float *I, bool sbf_ready = false) {
    const int B = c->ff_batch, rows = B * c->ff_steps;
    const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
    const int nin_p = up(nin, 64), rows_out = up(nout, 128), rows_p = up(rows, 64);
    cudaError_t e = cudaSuccess;
    if (!sbf_ready || want_st)
        e = ff_tc_spikes(c->ff_S[l - 1], rows, nin, (nin + 31) / 32, nin_p, rows_p, sbf_ready ? nullptr : c->ff_Sbf,
                         want_st ? c->ff_ST : nullptr, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "spike operands");
    FfTcMaps maps;
    FfTcArgs a;
    memset(&maps, 0, sizeof(maps));
    memset(&a, 0, sizeof(a));
    sn_status s;
    if ((s = bf16_map(c, &maps.m[0], c->ff_Sbf, rows, nin_p)) ||
        (s = bf16_map(c, &maps.m[1], c->ff_Wf[l - 1], 12LL * rows_out, nin_p)))
        return s;
    // one pass per delay; the kernel multiplies its spike tile by the three
    // weight parts, rows_out apart in the map
    for (int d = 1; d <= 4; ++d) {
        FfTcPass &ps = a.pass[a.npass++];
        ps.amap = 0; ps.a_y = -d * B; ps.a_x = 0;
        ps.bmap = 1; ps.b_y = (d - 1) * 3 * rows_out; ps.b_x = 0;
        ps.kblocks = nin_p / 64; ps.acc = 0;
    }
    a.part_stride = rows_out;
    a.M = rows; a.N = nout;
    a.tiles_m = (rows + 127) / 128; a.tiles_n = (nout + 127) / 128; a.ksplit = 1;
    a.nacc = 1; a.mode = 0; a.C = I; a.ldc = nout; a.cstride = 0; a.ctl = c->ctl;
    if ((e = ff_tc_forward(maps, a, c->stream)) != cudaSuccess) return cuda_fail(c, e, "tensor-core synaptic input");
    return SN_OK;
}

// Weight gradient of layer l from gI (already split and transposed into GT)
// and the transposed spikes ST: 4 delays x 2 gradient parts, one accumulator
// per delay, split over K (the rows) to fill the GPU, then reduced in order.
sn_status tc_weight_grad(sn_ctx *c, int l, float *dW) {
    const int B = c->ff_batch, rows = B * c->ff_steps;
    const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
    const int rows_p = up(rows, 64);
    FfTcMaps maps;
    FfTcArgs a;
    memset(&maps, 0, sizeof(maps));
    memset(&a, 0, sizeof(a));
    sn_status s;
    const __nv_bfloat16 *GT = (const __nv_bfloat16 *)c->ff_GT;
    if ((s = bf16_map(c, &maps.m[0], c->ff_ST, nin, rows_p)) ||
        (s = bf16_map(c, &maps.m[1], GT, nout, rows_p)) ||
        (s = bf16_map(c, &maps.m[2], GT + (size_t)nout * rows_p, nout, rows_p)))
        return s;
    // one pass per delay: the shifted spike tile times both gradient parts
    for (int d = 1; d <= 4; ++d) {
        FfTcPass &ps = a.pass[a.npass++];
        ps.amap = 0; ps.a_y = 0; ps.a_x = -d * B;
        ps.bmap = 1; ps.b_y = 0; ps.b_x = 0;
        ps.nb = 2; ps.bmap2 = 2; ps.b_y2 = 0;
        ps.kblocks = rows_p / 64; ps.acc = d - 1;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    a.M = nin; a.N = nout;
    a.tiles_m = (nin + 127) / 128; a.tiles_n = (nout + 127) / 128;
    const int tiles = a.tiles_m * a.tiles_n;
    // K (the T * B rows) split over enough blocks to fill the GPU, as far as
    // the partial-sum buffer holds the splits (a narrow output layer has few
    // tiles and takes many splits)
    const long long cap = (long long)(c->ff_part_elems / ((size_t)nin * nout));
    int ks = (int)std::max(1LL, std::min<long long>({(long long)(sms / std::max(1, tiles)), cap,
                                                     (long long)(rows_p / 64 / 8)}));
    a.ksplit = ks;
    a.nacc = 4; a.mode = 1; a.D = c->ff_D[l - 1]; a.ldc = nout; a.ctl = c->ctl;
    const long long count = (long long)nin * nout;
    a.C = ks == 1 ? dW : c->ff_part;
    a.cstride = count;
    cudaError_t e = ff_tc_gemm(maps, a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core weight gradient");
    if (ks > 1 && (e = ff_dw_reduce(c->ff_part, ks, count, dW, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "weight gradient reduction");
    return SN_OK;
}

// Gradient of the spikes of layer l-1: gS[r][i] = sum_d sum_j gI[r + dB][j] W_d[i][j],
// with the two-part splits hi*hi + hi*mid + mid*hi: 12 passes.
sn_status tc_spike_grad(sn_ctx *c, int l) {
    const int B = c->ff_batch, rows = B * c->ff_steps;
    const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
    const int nout_p = up(nout, 64), rows_in = up(nin, 128);
    FfTcMaps maps;
    FfTcArgs a;
    memset(&maps, 0, sizeof(maps));
    memset(&a, 0, sizeof(a));
    sn_status s;
    const __nv_bfloat16 *G = (const __nv_bfloat16 *)c->ff_G;
    if ((s = bf16_map(c, &maps.m[0], G, rows, nout_p)) ||
        (s = bf16_map(c, &maps.m[1], G + (size_t)rows * nout_p, rows, nout_p)) ||
        (s = bf16_map(c, &maps.m[2], c->ff_Wb[l - 1], 8LL * rows_in, nout_p)))
        return s;
    // per delay: hi gradient part times both weight parts, mid part times hi
    for (int d = 1; d <= 4; ++d) {
        FfTcPass &ps = a.pass[a.npass++];
        ps.amap = 0; ps.a_y = d * B; ps.a_x = 0;
        ps.bmap = 2; ps.b_y = (d - 1) * 2 * rows_in; ps.b_x = 0;
        ps.nb = 2; ps.bmap2 = 2; ps.b_y2 = ((d - 1) * 2 + 1) * rows_in;
        ps.kblocks = nout_p / 64; ps.acc = 0;
        FfTcPass &pl = a.pass[a.npass++];
        pl.amap = 1; pl.a_y = d * B; pl.a_x = 0;
        pl.bmap = 2; pl.b_y = (d - 1) * 2 * rows_in; pl.b_x = 0;
        pl.nb = 1;
        pl.kblocks = nout_p / 64; pl.acc = 0;
    }
    a.M = rows; a.N = nin;
    a.tiles_m = (rows + 127) / 128; a.tiles_n = (nin + 127) / 128; a.ksplit = 1;
    a.nacc = 1; a.mode = 0; a.C = c->ff_gS; a.ldc = nin; a.cstride = 0; a.ctl = c->ctl;
    cudaError_t e = ff_tc_gemm(maps, a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core spike gradient");
    return SN_OK;
}

// Allocate the BF16 operand buffers and look up the tensor-map encoder; on
// any failure the context keeps the SIMT engine only.
void tc_setup(sn_ctx *c) {
    const int L = c->ff_layers, B = c->ff_batch, rows = B * c->ff_steps;
    if (B % 8 != 0) return;                    // delay shifts of d * B rows must stay 16-byte aligned in K
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return;
    c->ff_encode = fn;
    const int rows_p = up(rows, 64);
    size_t s_elems = 0, st_elems = 0, g_elems = 0, gt_elems = 0;
    c->ff_Wf.assign(L, nullptr);
    c->ff_Wb.assign(L, nullptr);
    for (int l = 1; l <= L; ++l) {
        const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
        s_elems = std::max(s_elems, (size_t)rows * up(nin, 64));
        st_elems = std::max(st_elems, (size_t)nin * rows_p);
        g_elems = std::max(g_elems, (size_t)2 * rows * up(nout, 64));
        gt_elems = std::max(gt_elems, (size_t)2 * nout * rows_p);
        const size_t wf = (size_t)12 * up(nout, 128) * up(nin, 64) * 2, wb = (size_t)8 * up(nin, 128) * up(nout, 64) * 2;
        if (dalloc(c, &c->ff_Wf[l - 1], wf) || dalloc(c, &c->ff_Wb[l - 1], wb))
            return;
        // the weight parts of the other three delays and the padding stay
        // zero for the context's lifetime (each forward rewrites only every
        // weight's own delay slot)
        if (cudaMemset(c->ff_Wf[l - 1], 0, wf) || cudaMemset(c->ff_Wb[l - 1], 0, wb)) return;
    }
    if (dalloc(c, &c->ff_Sbf, s_elems * 2) || dalloc(c, &c->ff_ST, st_elems * 2) || dalloc(c, &c->ff_G, g_elems * 2) ||
        dalloc(c, &c->ff_GT, gt_elems * 2))
        return;
    // padding columns and rows of the operands stay zero from here on (the
    // spike rows' padding may later hold 0/1 values of a wider layer, which
    // meet zero weight columns)
    if (cudaMemset(c->ff_Sbf, 0, s_elems * 2) || cudaMemset(c->ff_ST, 0, st_elems * 2) ||
        cudaMemset(c->ff_G, 0, g_elems * 2) || cudaMemset(c->ff_GT, 0, gt_elems * 2))
        return;
    c->ff_tc_ok = true;
}

}  // namespace
}  // namespace sn

extern "C" {

sn_status sn_ff_set_engine(sn_ctx *c, int32_t engine) {
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (engine != SN_FF_AUTO && engine != SN_FF_SIMT && engine != SN_FF_TENSOR)
        return fail(c, SN_EINVAL, "unknown engine");
    if (engine == SN_FF_TENSOR && !c->ff_tc_ok)
        return fail(c, SN_EUNSUPPORTED, "the tensor-core engine needs a batch that is a multiple of 8");
    c->ff_engine = engine;
    return SN_OK;
}

sn_status sn_create_ff(const sn_config *cfg, int32_t layers, const int32_t *sizes, const uint8_t *const *delays,
                       const sn_ff_params *p, int32_t batch, int32_t steps, sn_ctx **out) {
    sn::FaultScope fault_scope;
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
    c->ff_part_elems = (size_t)c->ff_splits * nin_max * nout_max;
    // every layer's synaptic input kept for the backward, unless asked not to
    // or the memory is not there (then the backward recomputes it)
    if (!(cfg->flags & SN_FF_RECOMPUTE)) {
        c->ff_Ik.assign(layers + 1, nullptr);
        for (int l = 1; l <= layers; ++l) {
            void *q = nullptr;
            if (cudaMalloc(&q, (size_t)rows * sizes[l] * 4) != cudaSuccess) {
                (void)cudaGetLastError();
                for (int u = 1; u < l; ++u) cudaFree(c->ff_Ik[u]);
                c->ff_Ik.clear();
                break;
            }
            c->ff_Ik[l] = (float *)q;
        }
        for (float *q : c->ff_Ik)
            if (q) c->allocs.push_back(q);
    }
    c->ff_w.assign(layers, nullptr);
    tc_setup(c);
    c->err.clear();
    *out = c;
    return SN_OK;
}

sn_status sn_ff_forward(sn_ctx *c, const uint8_t *input, const float *const *w, float *counts) {
    NvtxRange nvtx("sn_ff_forward");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (!input || !w || !counts) return fail(c, SN_EINVAL, "NULL argument");
    for (int l = 0; l < c->ff_layers; ++l)
        if (!w[l]) return fail(c, SN_EINVAL, "weight pointer is NULL");
    const int B = c->ff_batch, T = c->ff_steps, L = c->ff_layers;
    const int rows = B * T;
    const bool tc = use_tc(c);
    c->ff_fwd_tc = tc;
    // with the tensor cores, the input packing and each layer's recurrence
    // also write the spikes as the next contraction's BF16 operand
    cudaError_t e = ff_pack(input, rows, c->ff_sizes[0], (c->ff_sizes[0] + 31) / 32, c->ff_S[0],
                            tc ? c->ff_Sbf : nullptr, up(c->ff_sizes[0], 64), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "input pack");
    for (int l = 1; l <= L; ++l) {
        const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
        float *I = c->ff_Ik.empty() ? c->ff_I : c->ff_Ik[l];
        c->ff_w[l - 1] = w[l - 1];
        if (tc) {
            // weight parts for this forward and the matching backward
            if ((e = ff_tc_weights(w[l - 1], c->ff_D[l - 1], nin, nout, (nout + 63) / 64 * 64, (nin + 127) / 128 * 128,
                                   l > 1 ? c->ff_Wb[l - 1] : nullptr, (nin + 63) / 64 * 64, (nout + 127) / 128 * 128,
                                   c->ff_Wf[l - 1], c->stream)))
                return cuda_fail(c, e, "weight parts");
            sn_status st = tc_forward(c, l, false, I, true);
            if (st) return st;
        } else if ((e = ff_delay_fwd(c->ff_S[l - 1], (nin + 31) / 32, w[l - 1], c->ff_DM[l - 1], nin, nout, B, 0,
                                     rows, I, c->stream))) {
            return cuda_fail(c, e, "forward synaptic input");
        }
        if ((e = ff_scan_fwd(I, nout, B, T, c->ff_k, c->ff_theta, c->ff_leak, c->ff_reset, c->ff_refr,
                             c->ff_S[l], c->ff_vck[l], c->ff_rck[l], l == L ? counts : nullptr,
                             tc && l < L ? c->ff_Sbf : nullptr, up(nout, 64), c->stream)))
            return cuda_fail(c, e, "forward recurrence");
    }
    c->ff_have_forward = true;
    return SN_OK;
}

sn_status sn_backward(sn_ctx *c, const float *grad_counts, float *const *grad_w, int32_t on_device) {
    NvtxRange nvtx("sn_backward");
    if (!c) return fail(nullptr, SN_EINVAL, "ctx is NULL");
    if (c->kind != KIND_FF) return fail(c, SN_ESTATE, "not a feedforward context");
    if (!on_device) return fail(c, SN_EUNSUPPORTED, "sn_backward takes device buffers (on_device = 1)");
    if (!c->ff_have_forward) return fail(c, SN_ESTATE, "no forward pass to differentiate");
    if (!grad_counts || !grad_w) return fail(c, SN_EINVAL, "NULL argument");
    const int B = c->ff_batch, T = c->ff_steps, L = c->ff_layers;
    const int rows = B * T;
    cudaError_t e;
    for (int l = 1; l <= L; ++l)
        if (!grad_w[l - 1]) return fail(c, SN_EINVAL, "gradient pointer is NULL");
    const bool tc = c->ff_fwd_tc;              // the engine of the forward being differentiated
    for (int l = L; l >= 1; --l) {
        const int nin = c->ff_sizes[l - 1], nout = c->ff_sizes[l];
        const int words_in = (nin + 31) / 32;
        // the forward's synaptic input: kept, or recomputed with the
        // forward's own kernel so that the states match; the tensor-core
        // weight gradient also takes the transposed input spikes
        float *I = c->ff_I;
        if (!c->ff_Ik.empty()) {
            I = c->ff_Ik[l];
            if (tc && (e = ff_tc_spikes(c->ff_S[l - 1], rows, nin, words_in, up(nin, 64), up(rows, 64), nullptr,
                                        c->ff_ST, c->stream)))
                return cuda_fail(c, e, "spike operands");
        } else if (tc) {
            sn_status st = tc_forward(c, l, true, I);
            if (st) return st;
        } else if ((e = ff_delay_fwd(c->ff_S[l - 1], words_in, c->ff_w[l - 1], c->ff_DM[l - 1], nin, nout, B, 0,
                                     rows, I, c->stream))) {
            return cuda_fail(c, e, "recompute synaptic input");
        }
        if ((e = ff_scan_bwd(I, nout, B, T, c->ff_k, c->ff_theta, c->ff_leak, c->ff_reset, c->ff_refr,
                             c->ff_slope, c->ff_vck[l], c->ff_rck[l], l == L ? nullptr : c->ff_gS,
                             l == L ? grad_counts : nullptr, c->ff_gI, c->stream)))
            return cuda_fail(c, e, "adjoint recurrence");
        if (tc) {
            const int nout_p = (nout + 63) / 64 * 64, rows_p = (rows + 63) / 64 * 64;
            if ((e = ff_tc_gsplit(c->ff_gI, rows, nout, nout_p, rows_p, l > 1 ? c->ff_G : nullptr, c->ff_GT,
                                  c->stream)))
                return cuda_fail(c, e, "gradient parts");
            sn_status st = tc_weight_grad(c, l, grad_w[l - 1]);
            if (st) return st;
            if (l > 1 && (st = tc_spike_grad(c, l))) return st;
            continue;
        }
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
