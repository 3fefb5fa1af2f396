// Host side of the shared dense network driven by many input trains
// (sn_shared.cu): FP8 E4M3 encoding of the integer weights, TMA tensor maps,
// state and launches.

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "sn_ctx.h"

namespace sn {

// E4M3 byte of an integer in [-8, 8] (exact): sign, 4 exponent bits with
// bias 7, 3 mantissa bits.
static uint8_t e4m3_of_int(int v) {
    if (v == 0) return 0;
    const uint8_t sign = v < 0 ? 0x80 : 0x00;
    int a = v < 0 ? -v : v;
    int e = 0;
    while ((2 << e) <= a) ++e;                   // 2^e <= a < 2^(e+1)
    const int mant = ((a - (1 << e)) * 8) >> e;  // exact for a <= 8
    return (uint8_t)(sign | ((e + 7) << 3) | mant);
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Row-major bytes [rows][cols], boxes of 128 rows x 128 bytes, 128B swizzle.
static sn_status encode_map(sn_ctx *c, EncodeTiled fn, void *out, void *base, long long rows, long long cols) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols};
    cuuint32_t box[2] = {128, 128};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn((CUtensorMap *)out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, SN_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SN_OK;
}

sn_status shared_run(sn_ctx *c, int steps) {
    SharedHostArgs h;
    h.n = c->n; h.B = c->sh_B; h.t0 = (int)c->step; h.steps = steps; h.cap = c->cap;
    h.A0 = c->sh_A0; h.A1 = c->sh_A1; h.V = (int *)c->V; h.r = c->r;
    h.th = (const int *)c->th; h.lk = (const int *)c->lk; h.rs = (const int *)c->rs; h.R = c->R;
    h.prate = c->prate; h.pamp = (const int *)c->pamp; h.pkey = c->pkeys; h.raster = c->raster; h.ctl = c->ctl;
    cudaError_t e = launch_shared(c->sh_tmaps, h, c->sh_grid, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "shared dense launch");
    return SN_OK;
}

// State in the ABI's order [trains][n] from the kernel's [n][trains].
sn_status shared_get_state(sn_ctx *c, void *v, int32_t *refr, int32_t on_device) {
    const size_t bn = (size_t)c->sh_B * c->n;
    int *tmp = nullptr;
    sn_status s = SN_OK;
    if (!on_device && (s = dalloc(c, &tmp, bn * 4))) return s;
    void *outs[2] = {v, refr};
    const int *src[2] = {(const int *)c->V, c->r};
    for (int k = 0; k < 2 && s == SN_OK; ++k) {
        if (!outs[k]) continue;
        int *dst = on_device ? (int *)outs[k] : tmp;
        cudaError_t e = launch_shared_transpose(src[k], dst, c->n, c->sh_B, c->stream);
        if (e == cudaSuccess && !on_device) {
            e = cudaMemcpyAsync(outs[k], tmp, bn * 4, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        }
        if (e != cudaSuccess) s = cuda_fail(c, e, "state transpose");
    }
    dfree(c, tmp);
    return s;
}

sn_status shared_set_poisson(sn_ctx *c, int32_t nsrc, const int32_t *neuron, const float *rate,
                             const float *amp, uint64_t seed, uint64_t net0) {
    const int n = c->n;
    std::vector<unsigned> thr(n, 0u);
    std::vector<int> ai(n, 0);
    std::vector<char> used(n, 0);
    for (int k = 0; k < nsrc; ++k) {
        const int j = neuron[k];
        if (j < 0 || j >= n) return fail(c, SN_EINVAL, "source neuron out of range (0 .. n-1 of one train)");
        if (used[j]) return fail(c, SN_EINVAL, "a neuron may have at most one Poisson source");
        if (!(rate[k] >= 0.0f) || !std::isfinite(rate[k])) return fail(c, SN_EINVAL, "rate must be finite and >= 0");
        if (!is_int_valued(amp[k])) return fail(c, SN_EINVAL, "amplitudes must be integers");
        used[j] = 1;
        thr[j] = rate_threshold(rate[k]);
        ai[j] = (int)amp[k];
    }
    std::vector<unsigned long long> keys(c->sh_B);
    for (int b = 0; b < c->sh_B; ++b) keys[b] = host_splitmix64(seed ^ host_splitmix64(net0 + (unsigned long long)b));
    if (sn_status q = quiesce(c)) return q;   // a queued run may read the old sources
    SN_CUDA(c, cudaMemcpy(c->prate, thr.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pamp, ai.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->pkeys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice));
    return SN_OK;
}

}  // namespace sn

extern "C" sn_status sn_create_shared_dense_i8(const sn_config *cfg, const sn_neurons *nr, const int8_t *w,
                                               int32_t trains, sn_ctx **out) {
    sn::FaultScope fault_scope;
    if (!cfg || !nr || !w || !out) return fail(nullptr, SN_EINVAL, "NULL argument");
    if (cfg->dtype != SN_I32) return fail(nullptr, SN_EINVAL, "the shared dense network is integer (SN_I32)");
    if (cfg->max_delay != 1) return fail(nullptr, SN_EINVAL, "the shared dense network has delay 1 (max_delay = 1)");
    if (cfg->record_steps < 0) return fail(nullptr, SN_EINVAL, "record_steps < 0");
    const int n = nr->n;
    if (n < 128 || n % 128 != 0 || n > (1 << 21)) return fail(nullptr, SN_EINVAL, "n must be a multiple of 128 in 128 .. 2^21");
    if (trains < 128 || trains % 128 != 0 || (long long)trains * n >= (1ll << 31))
        return fail(nullptr, SN_EINVAL, "trains must be a multiple of 128 with trains * n < 2^31");
    const size_t nn = (size_t)n * n;
    for (size_t q = 0; q < nn; ++q)
        if (w[q] < -8 || w[q] > 8) return fail(nullptr, SN_EINVAL, "weights must lie in -8 .. 8");
    sn_ctx *c = new (std::nothrow) sn_ctx();
    if (!c) return fail(nullptr, SN_ENOMEM, "host allocation failed");
    c->kind = KIND_SHARED_I8;
    c->dtype = SN_I32;
    c->n = n;
    c->D = 1;
    c->D1 = 2;
    c->sh_B = trains;
    c->m = (long long)nn;
    c->stream = (cudaStream_t)cfg->cuda_stream;
    auto bail = [&](sn_status st) { std::string msg = c->err.empty() ? g_create_err : c->err;
                                    destroy_all(c); delete c; g_create_err = msg; return st; };
    sn_status s;
    if ((s = upload_neurons(c, nr))) return bail(s);
    const size_t bn = (size_t)trains * n;
    c->words = (int)(bn / 32);
    c->cap = cfg->record_steps > 0 ? cfg->record_steps : 1;
    int *V = nullptr, *r = nullptr;
    if ((s = dalloc(c, &V, bn * 4)) || (s = dalloc(c, &r, bn * 4)) || (s = dalloc(c, &c->sh_V0, bn * 4)) ||
        (s = dalloc(c, &c->sh_A0, bn)) || (s = dalloc(c, &c->sh_A1, bn)) || (s = dalloc(c, &c->sh_WT, nn)) ||
        (s = dalloc(c, &c->pkeys, (size_t)trains * 8)) ||
        (s = dalloc(c, &c->raster, (size_t)c->cap * c->words * 4)) || (s = dalloc(c, &c->ctl, sizeof(Control))))
        return bail(s);
    c->V = V;
    c->r = r;
    {
        // weights transposed (K = pre index contiguous per post row) as E4M3
        std::vector<uint8_t> wt(nn);
        uint8_t lut[17];
        for (int v = -8; v <= 8; ++v) lut[v + 8] = e4m3_of_int(v);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) wt[(size_t)j * n + i] = lut[w[(size_t)i * n + j] + 8];
        // the kernel keeps the state neuron-major, [n][trains]
        std::vector<int> v0(bn);
        for (int j = 0; j < n; ++j)
            for (int b = 0; b < trains; ++b) v0[(size_t)j * trains + b] = (int)nr->reset[j];
        std::vector<unsigned long long> keys(trains);
        for (int b = 0; b < trains; ++b) keys[b] = host_splitmix64(0ull ^ host_splitmix64((unsigned long long)b));
        cudaError_t e;
        if ((e = cudaMemcpy(c->sh_WT, wt.data(), nn, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->sh_V0, v0.data(), bn * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->V, v0.data(), bn * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemset(c->r, 0, bn * 4)) || (e = cudaMemset(c->sh_A0, 0, bn)) || (e = cudaMemset(c->sh_A1, 0, bn)) ||
            (e = cudaMemcpy(c->pkeys, keys.data(), (size_t)trains * 8, cudaMemcpyHostToDevice)) ||
            (e = cudaMemset(c->raster, 0, (size_t)c->cap * c->words * 4)) || (e = cudaMemset(c->ctl, 0, sizeof(Control)))) {
            c->err = std::string("upload: ") + cudaGetErrorString(e);
            return bail(SN_ECUDA);
        }
    }
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        c->err = "cuTensorMapEncodeTiled is not available from the driver";
        return bail(SN_EUNSUPPORTED);
    }
    if ((s = encode_map(c, (EncodeTiled)fn, c->sh_tmaps + 0, c->sh_A0, trains, n)) ||
        (s = encode_map(c, (EncodeTiled)fn, c->sh_tmaps + 128, c->sh_A1, trains, n)) ||
        (s = encode_map(c, (EncodeTiled)fn, c->sh_tmaps + 256, c->sh_WT, n, n)))
        return bail(s);
    cudaError_t e = max_grid_shared(&c->sh_grid);
    if (e != cudaSuccess || c->sh_grid < 1) {
        c->err = std::string("shared dense occupancy: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "no resident block");
        return bail(SN_EUNSUPPORTED);
    }
    *out = c;
    return SN_OK;
}
