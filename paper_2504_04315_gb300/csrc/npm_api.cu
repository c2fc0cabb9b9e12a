// npm_api.cu -- the C ABI of include/npm.h: handle lifetime, argument checks,
// parameter management and dispatch to the kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "npm.h"
#include "npm_handle.h"
#include "npm_kernels.h"

namespace npm {

#ifdef NPM_DEBUG_BOUNDS
__device__ unsigned long long g_bounds_violations = 0;
#endif

CallRange::CallRange(const char* name) { nvtxRangePushA(name); }
CallRange::~CallRange() { nvtxRangePop(); }

namespace {
thread_local int t_alloc_count = 0;  // allocations of the current npm_create
thread_local int t_alloc_fail = 0;   // which one fails (0: none)
std::atomic<long long> g_launch_count{0};
}  // namespace

cudaError_t device_alloc(void** p, size_t bytes) {
    if (t_alloc_fail > 0 && ++t_alloc_count == t_alloc_fail) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

bool inject_launch_failure() {
    static std::atomic<long long> target{-2};
    long long t = target.load(std::memory_order_relaxed);
    if (t == -2) {
        const char* e = getenv("NPM_TEST_FAIL_LAUNCH");
        t = (e && *e) ? atoll(e) : 0;
        target.store(t, std::memory_order_relaxed);
    }
    return t > 0 && g_launch_count.fetch_add(1, std::memory_order_relaxed) + 1 == t;
}

}  // namespace npm

namespace {

thread_local std::string g_last_error;

npm_status fail(npm_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

npm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(NPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NPM_CUDA(call, what)                            \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int pad_np(int v) { return v <= 16 ? 16 : v <= 32 ? 32 : v <= 64 ? 64 : 128; }

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// SplitMix64 output function; the library's own seeded initialisation.
uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double init_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t s0 = mix64(mix64(seed) ^ stream);
    return (double)(mix64(s0 + (i + 1) * 0x9E3779B97F4A7C15ull) >> 40) * (1.0 / 16777216.0);
}

npm_status validate(const npm_config* c) {
    if (!c) return fail(NPM_ERR_INVALID_ARG, "config is NULL");
    if (c->mode != NPM_RADIANCE && c->mode != NPM_PRODUCT)
        return fail(NPM_ERR_INVALID_ARG, "mode must be NPM_RADIANCE or NPM_PRODUCT");
    if (c->n_levels < 1 || c->n_levels > NPM_MAX_LEVELS)
        return fail(NPM_ERR_INVALID_ARG, "n_levels out of range [1, 32]");
    if (c->feat_per_level < 1 || c->feat_per_level > 8)
        return fail(NPM_ERR_INVALID_ARG, "feat_per_level out of range [1, 8]");
    if (c->log2_table < 1 || c->log2_table > 24)
        return fail(NPM_ERR_INVALID_ARG, "log2_table out of range [1, 24]");
    for (int l = 0; l < c->n_levels; ++l)
        if (c->level_res[l] < 2 || c->level_res[l] > 4096)
            return fail(NPM_ERR_INVALID_ARG, "level_res out of range [2, 4096]");
    if (c->n_layers < 1 || c->n_layers > NPM_MAX_LAYERS)
        return fail(NPM_ERR_INVALID_ARG, "n_layers out of range [1, 8]");
    for (int i = 0; i <= c->n_layers; ++i)
        if (c->widths[i] < 4 || c->widths[i] > NPM_MAX_WIDTH || c->widths[i] % 4)
            return fail(NPM_ERR_INVALID_ARG, "every width must be a multiple of 4 in [4, 128]");
    if (c->K < 1 || c->K > NPM_MAX_LOBES)
        return fail(NPM_ERR_INVALID_ARG, "K out of range [1, 16]");
    if (c->widths[c->n_layers] != 4 * c->K)
        return fail(NPM_ERR_INVALID_ARG, "last width must equal 4K");
    int need = c->n_levels * c->feat_per_level + (c->mode == NPM_PRODUCT ? 21 : 0);
    if (c->widths[0] < need)
        return fail(NPM_ERR_INVALID_ARG, "widths[0] smaller than the encoding width");
    if (c->kappa_act != NPM_SOFTPLUS && c->kappa_act != NPM_EXP)
        return fail(NPM_ERR_INVALID_ARG, "kappa_act must be NPM_SOFTPLUS or NPM_EXP");
    if (c->precision != NPM_FP32 && c->precision != NPM_BF16 && c->precision != NPM_BF16X3 &&
        c->precision != NPM_FP16 && c->precision != NPM_FP32_TC)
        return fail(NPM_ERR_INVALID_ARG,
                    "precision must be NPM_FP32, NPM_BF16, NPM_BF16X3, NPM_FP16 or NPM_FP32_TC");
    if (c->max_batch < 0 || c->max_batch > ((int64_t)1 << 31))
        return fail(NPM_ERR_INVALID_ARG, "max_batch out of range [0, 2^31]");
    if (!(c->lr >= 0.0f) || !(c->beta1 >= 0.0f && c->beta1 < 1.0f) ||
        !(c->beta2 >= 0.0f && c->beta2 < 1.0f) || !(c->eps > 0.0f))
        return fail(NPM_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    return NPM_OK;
}

template <typename T>
npm_status dalloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = npm::device_alloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(NPM_ERR_OOM, std::string("cudaMalloc failed for ") + what);
    }
    return NPM_OK;
}

npm_status check_call(npm_handle* h, int64_t n, int64_t ld, const void* pos, const void* aux) {
    if (!h) return fail(NPM_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(NPM_ERR_INVALID_ARG, "n < 0");
    if (n > h->cfg.max_batch) return fail(NPM_ERR_CAPACITY, "n exceeds max_batch");
    if (ld < n) return fail(NPM_ERR_INVALID_ARG, "ld < n");
    if (n > 0 && !pos) return fail(NPM_ERR_INVALID_ARG, "pos is NULL");
    if (n > 0 && h->cfg.mode == NPM_PRODUCT && !aux)
        return fail(NPM_ERR_INVALID_ARG, "product mode needs aux [7][ld]");
    return NPM_OK;
}

// Device-side count of completed Adam steps (scalars[16]).
int* step_dev(npm_handle* h) { return reinterpret_cast<int*>(h->scalars + 16); }

// Padded FP32 forward weights of the moving average (inference).
npm_status arrange_inference_weights(npm_handle* h, cudaStream_t st) {
    if (h->ema)
        NPM_CUDA(npm::launch_arrange_weights(h->dc, h->ema + h->mlp_off, h->wfwd_inf, nullptr, st),
                 "arrange ema weights");
    return NPM_OK;
}

// Every copy derived from the parameters: the FP32 kernels' padded weights,
// the FP16 grid and the tensor-core weights (of the moving average too,
// when inference evaluates it).
npm_status refresh_derived(npm_handle* h, cudaStream_t st) {
    NPM_CUDA(npm::launch_arrange_weights(h->dc, h->params + h->mlp_off, h->wfwd, h->wbwd, st),
             "arrange weights");
    npm_status s = arrange_inference_weights(h, st);
    if (s != NPM_OK) return s;
    if (h->grid_h) NPM_CUDA(npm::launch_to_half(h->ng, inf_params(h), h->grid_h, st), "grid fp16 copy");
    if (h->tc) NPM_CUDA(npm::tc_refresh_weights(h, st), "bf16 weight copy");
    return NPM_OK;
}

}  // namespace

namespace npm {

npm_status make_devcfg(const npm_config* cfg, DevCfg* out, int64_t* ng, int64_t* nmlp) {
    npm_status s = validate(cfg);
    if (s != NPM_OK) return s;
    DevCfg& d = *out;
    memset(&d, 0, sizeof(d));
    d.mode = cfg->mode;
    d.n_levels = cfg->n_levels;
    d.feat = cfg->feat_per_level;
    d.K = cfg->K;
    d.kappa_act = cfg->kappa_act;
    d.n_layers = cfg->n_layers;
    d.grid_feats = cfg->n_levels * cfg->feat_per_level;
    d.table_mask = (uint32_t)((1ull << cfg->log2_table) - 1);
    uint64_t T = 1ull << cfg->log2_table, off = 0;
    for (int l = 0; l < cfg->n_levels; ++l) {
        uint64_t D = (uint64_t)cfg->level_res[l];
        d.level_res[l] = (int)D;
        d.level_off[l] = (uint32_t)off;
        if (D * D * D <= T) {
            d.dense_mask |= 1u << l;
            off += D * D * D;
        } else {
            off += T;
        }
        if (off * (uint64_t)cfg->feat_per_level >= (1ull << 32))
            return fail(NPM_ERR_INVALID_ARG, "grid larger than 2^32 values");
    }
    *ng = (int64_t)off * cfg->feat_per_level;
    int maxw = 0, of = 0, ob = 0;
    *nmlp = 0;
    for (int l = 0; l <= cfg->n_layers; ++l) {
        d.widths[l] = cfg->widths[l];
        maxw = cfg->widths[l] > maxw ? cfg->widths[l] : maxw;
    }
    for (int l = 0; l < cfg->n_layers; ++l) {
        const int K = cfg->widths[l], N = cfg->widths[l + 1];
        d.np_fwd[l] = pad_np(N);
        d.np_bwd[l] = pad_np(K);
        d.off_fwd[l] = of;
        d.off_bwd[l] = ob;
        of += K * d.np_fwd[l];
        ob += N * d.np_bwd[l];
        *nmlp += (int64_t)K * N;
    }
    d.fwd_floats = of;
    d.bwd_floats = ob;
    d.max_width = maxw;
    if (fwd_smem_bytes(d) > 227 * 1024)
        return fail(NPM_ERR_UNSUPPORTED, "MLP weights do not fit in shared memory");
    return NPM_OK;
}

npm_status set_error(npm_status s, const char* msg) { return fail(s, msg); }

}  // namespace npm

extern "C" {

const char* npm_last_error(void) { return g_last_error.c_str(); }

npm_status npm_create(const npm_config* cfg, npm_handle** out) {
    npm::CallRange range("npm_create");
    if (!out) return fail(NPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    // Test-only: NPM_TEST_FAIL_ALLOC=N fails the N-th allocation of this
    // call; the guard switches the injection off again on every return.
    struct AllocInjection {
        AllocInjection() {
            const char* e = getenv("NPM_TEST_FAIL_ALLOC");
            npm::t_alloc_fail = (e && *e) ? atoi(e) : 0;
            npm::t_alloc_count = 0;
        }
        ~AllocInjection() { npm::t_alloc_fail = 0; }
    } injection;
    npm_status s = validate(cfg);
    if (s != NPM_OK) return s;
    npm_handle* h = new npm_handle();
    h->cfg = *cfg;
    cudaGetDevice(&h->device);
    if ((s = npm::make_devcfg(cfg, &h->dc, &h->ng, &h->nmlp)) != NPM_OK) {
        delete h;
        return s;
    }
    const npm::DevCfg& d = h->dc;
    const int of = d.fwd_floats, ob = d.bwd_floats;
    h->mlp_off = round_up(h->ng, 64);
    h->n_int = round_up(h->mlp_off + h->nmlp, 64);
    h->fwd_smem = npm::fwd_smem_bytes(d);
    h->train_smem = npm::train_smem_bytes(d);

    size_t nb = (size_t)(cfg->max_batch > 0 ? cfg->max_batch : 1);
    if ((s = dalloc(&h->params, h->n_int, "params")) != NPM_OK ||
        (s = dalloc(&h->grads, h->n_int, "grads")) != NPM_OK ||
        (s = dalloc(&h->adam_m, h->n_int, "adam m")) != NPM_OK ||
        (s = dalloc(&h->adam_v, h->n_int, "adam v")) != NPM_OK ||
        (s = dalloc(&h->wfwd, (size_t)of, "forward weights")) != NPM_OK ||
        (s = dalloc(&h->wbwd, (size_t)ob, "backward weights")) != NPM_OK ||
        (s = dalloc(&h->scalars, 64, "scalars")) != NPM_OK ||
        (s = dalloc(&h->stage, nb * (3 + 7 + 4 + 3 + 1), "host staging")) != NPM_OK) {
        npm_destroy(h);
        return s;
    }
    for (int i = 0; i < 2; ++i)
        if (cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking) != cudaSuccess) {
            npm_destroy(h);
            return fail(NPM_ERR_CUDA, "cannot create internal streams");
        }
    for (int i = 0; i < 3; ++i)
        if (cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming) != cudaSuccess) {
            npm_destroy(h);
            return fail(NPM_ERR_CUDA, "cannot create internal events");
        }
    if (cfg->precision != NPM_FP32) {
        if ((s = dalloc(&h->grid_h, (size_t)h->ng, "grid fp16")) != NPM_OK) {
            npm_destroy(h);
            return s;
        }
        if ((s = npm::tc_create(h)) != NPM_OK) {
            npm_destroy(h);
            return s;
        }
    }
    cudaMemset(h->grads, 0, h->n_int * sizeof(float));
    cudaMemset(h->adam_m, 0, h->n_int * sizeof(float));
    cudaMemset(h->adam_v, 0, h->n_int * sizeof(float));
    cudaMemset(h->scalars, 0, 64 * sizeof(float));
    // Seeded initialisation: grid U[-1e-4, 1e-4], MLP Glorot-uniform.
    std::vector<float> init(h->n_int, 0.0f);
    for (int64_t i = 0; i < h->ng; ++i)
        init[i] = (float)((init_uniform(cfg->seed, 5, (uint64_t)i) * 2.0 - 1.0) * 1e-4);
    int64_t o = h->mlp_off, c = 0;
    for (int l = 0; l < cfg->n_layers; ++l) {
        const int K = cfg->widths[l], N = cfg->widths[l + 1];
        const double a = sqrt(6.0 / (K + N));
        for (int64_t i = 0; i < (int64_t)K * N; ++i, ++c)
            init[o + i] = (float)((init_uniform(cfg->seed, 6, (uint64_t)c) * 2.0 - 1.0) * a);
        o += (int64_t)K * N;
    }
    cudaError_t e = cudaMemcpy(h->params, init.data(), h->n_int * sizeof(float),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        npm_destroy(h);
        return cuda_fail(e, "upload initial parameters");
    }
    if ((s = refresh_derived(h, 0)) != NPM_OK) {
        npm_destroy(h);
        return s;
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        npm_destroy(h);
        return cuda_fail(e, "npm_create");
    }
    *out = h;
    return NPM_OK;
}

npm_status npm_destroy(npm_handle* h) {
    npm::CallRange range("npm_destroy");
    if (!h) return NPM_OK;
    cudaDeviceSynchronize();
    if (h->tc) npm::tc_destroy(h);
    void* ptrs[] = {h->params, h->grads, h->adam_m, h->adam_v,   h->wfwd,  h->wbwd,
                    h->scalars, h->stage, h->grid_h, h->ema, h->wfwd_inf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < 2; ++i)
        if (h->side[i]) cudaStreamDestroy(h->side[i]);
    for (int i = 0; i < 3; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    delete h;
    return NPM_OK;
}

int64_t npm_num_params(const npm_handle* h) { return h ? h->ng + h->nmlp : -1; }

float* npm_params_device(npm_handle* h) { return h ? h->params : nullptr; }
float* npm_grads_device(npm_handle* h) { return h ? h->grads : nullptr; }

static npm_status copy_public(npm_handle* h, float* dev, float* host, int64_t count, bool to_dev) {
    if (!h || !host) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    if (count != h->ng + h->nmlp) return fail(NPM_ERR_INVALID_ARG, "count != npm_num_params");
    cudaMemcpyKind k = to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    NPM_CUDA(cudaDeviceSynchronize(), "synchronise");
    if (to_dev) {
        NPM_CUDA(cudaMemcpy(dev, host, h->ng * sizeof(float), k), "copy grid");
        NPM_CUDA(cudaMemcpy(dev + h->mlp_off, host + h->ng, h->nmlp * sizeof(float), k), "copy mlp");
    } else {
        NPM_CUDA(cudaMemcpy(host, dev, h->ng * sizeof(float), k), "copy grid");
        NPM_CUDA(cudaMemcpy(host + h->ng, dev + h->mlp_off, h->nmlp * sizeof(float), k), "copy mlp");
    }
    return NPM_OK;
}

npm_status npm_set_params(npm_handle* h, const float* host, int64_t count) {
    npm::CallRange range("npm_set_params");
    npm_status s = copy_public(h, h ? h->params : nullptr, const_cast<float*>(host), count, true);
    if (s != NPM_OK) return s;
    if (h->ema)  // the average restarts from the new parameters
        NPM_CUDA(cudaMemcpy(h->ema, h->params, h->n_int * sizeof(float), cudaMemcpyDeviceToDevice),
                 "reset ema");
    if ((s = refresh_derived(h, 0)) != NPM_OK) return s;
    NPM_CUDA(cudaDeviceSynchronize(), "npm_set_params");
    return NPM_OK;
}

npm_status npm_get_params(npm_handle* h, float* host, int64_t count) {
    npm::CallRange range("npm_get_params");
    return copy_public(h, h ? h->params : nullptr, host, count, false);
}

npm_status npm_set_params_device(npm_handle* h, const float* dev, int64_t count, void* stream) {
    npm::CallRange range("npm_set_params_device");
    if (!h || !dev) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    if (count != h->ng + h->nmlp) return fail(NPM_ERR_INVALID_ARG, "count != npm_num_params");
    cudaStream_t st = (cudaStream_t)stream;
    NPM_CUDA(cudaMemcpyAsync(h->params, dev, h->ng * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy grid");
    NPM_CUDA(cudaMemcpyAsync(h->params + h->mlp_off, dev + h->ng, h->nmlp * sizeof(float),
                             cudaMemcpyDeviceToDevice, st),
             "copy mlp");
    if (h->ema)
        NPM_CUDA(cudaMemcpyAsync(h->ema, h->params, h->n_int * sizeof(float), cudaMemcpyDeviceToDevice, st),
                 "reset ema");
    return refresh_derived(h, st);
}

npm_status npm_get_grads_device(npm_handle* h, float* dev, int64_t count, void* stream) {
    npm::CallRange range("npm_get_grads_device");
    if (!h || !dev) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    if (count != h->ng + h->nmlp) return fail(NPM_ERR_INVALID_ARG, "count != npm_num_params");
    cudaStream_t st = (cudaStream_t)stream;
    NPM_CUDA(cudaMemcpyAsync(dev, h->grads, h->ng * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy grid");
    NPM_CUDA(cudaMemcpyAsync(dev + h->ng, h->grads + h->mlp_off, h->nmlp * sizeof(float),
                             cudaMemcpyDeviceToDevice, st),
             "copy mlp");
    return NPM_OK;
}

npm_status npm_set_ema(npm_handle* h, float decay, void* stream) {
    npm::CallRange range("npm_set_ema");
    if (!h) return fail(NPM_ERR_INVALID_ARG, "handle is NULL");
    if (!(decay >= 0.0f && decay < 1.0f)) return fail(NPM_ERR_INVALID_ARG, "decay must be in [0, 1)");
    cudaStream_t st = (cudaStream_t)stream;
    if (decay == 0.0f) {
        if (h->ema) {
            NPM_CUDA(cudaStreamSynchronize(st), "synchronise");
            cudaFree(h->ema);
            cudaFree(h->wfwd_inf);
            h->ema = h->wfwd_inf = nullptr;
        }
        h->ema_decay = 0.0f;
        npm_status s = refresh_derived(h, st);
        if (s != NPM_OK) return s;
        NPM_CUDA(cudaStreamSynchronize(st), "npm_set_ema");
        return NPM_OK;
    }
    if (!h->ema) {
        npm_status s;
        if ((s = dalloc(&h->ema, h->n_int, "ema")) != NPM_OK) return s;
        if ((s = dalloc(&h->wfwd_inf, (size_t)h->dc.fwd_floats, "ema forward weights")) != NPM_OK) {
            cudaFree(h->ema);
            h->ema = nullptr;
            return s;
        }
        NPM_CUDA(cudaMemcpyAsync(h->ema, h->params, h->n_int * sizeof(float), cudaMemcpyDeviceToDevice, st),
                 "start ema");
    }
    h->ema_decay = decay;
    npm_status s = refresh_derived(h, st);
    if (s != NPM_OK) return s;
    NPM_CUDA(cudaStreamSynchronize(st), "npm_set_ema");
    return NPM_OK;
}

npm_status npm_get_ema_params(npm_handle* h, float* host, int64_t count) {
    if (h && !h->ema) return fail(NPM_ERR_INVALID_ARG, "the moving average is off (npm_set_ema)");
    return copy_public(h, h ? h->ema : nullptr, host, count, false);
}

npm_status npm_get_grads(npm_handle* h, float* host, int64_t count) {
    return copy_public(h, h ? h->grads : nullptr, host, count, false);
}

npm_status npm_get_adam(npm_handle* h, int* step, float* m_host, float* v_host) {
    if (!h || !step) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    NPM_CUDA(cudaDeviceSynchronize(), "synchronise");
    NPM_CUDA(cudaMemcpy(&h->step, step_dev(h), sizeof(int), cudaMemcpyDeviceToHost), "read step");
    *step = h->step;
    npm_status s = NPM_OK;
    if (m_host && (s = copy_public(h, h->adam_m, m_host, h->ng + h->nmlp, false)) != NPM_OK) return s;
    if (v_host && (s = copy_public(h, h->adam_v, v_host, h->ng + h->nmlp, false)) != NPM_OK) return s;
    return NPM_OK;
}

npm_status npm_set_adam(npm_handle* h, int step, const float* m_host, const float* v_host) {
    if (!h || step < 0) return fail(NPM_ERR_INVALID_ARG, "bad argument");
    npm_status s = NPM_OK;
    if (m_host &&
        (s = copy_public(h, h->adam_m, const_cast<float*>(m_host), h->ng + h->nmlp, true)) != NPM_OK)
        return s;
    if (v_host &&
        (s = copy_public(h, h->adam_v, const_cast<float*>(v_host), h->ng + h->nmlp, true)) != NPM_OK)
        return s;
    h->step = step;
    NPM_CUDA(cudaMemcpy(step_dev(h), &step, sizeof(int), cudaMemcpyHostToDevice), "write step");
    return NPM_OK;
}

npm_status npm_query_sample(npm_handle* h, int64_t n, const float* pos, const float* aux,
                            const float* u, int64_t ld, float uniform_frac, float* dir_out,
                            float* pdf_out, float* mix_out, void* stream) {
    npm::CallRange range("npm_query_sample");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (!(uniform_frac >= 0.0f && uniform_frac <= 1.0f))
        return fail(NPM_ERR_INVALID_ARG, "uniform_frac outside [0, 1]");
    if (n > 0 && (!u || !dir_out || !pdf_out))
        return fail(NPM_ERR_INVALID_ARG, "u, dir_out and pdf_out are required");
    if (n == 0) return NPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->tc) return npm::tc_query(h, n, ld, pos, aux, u, uniform_frac, true, dir_out, pdf_out, mix_out, st);
    NPM_CUDA(npm::launch_forward_fp32(h->dc, inf_params(h), inf_wfwd(h), n, ld, pos, aux, u, uniform_frac,
                                      true, dir_out, pdf_out, mix_out, st, status_word(h), h->wait_limit),
             "query_sample launch");
    return NPM_OK;
}

npm_status npm_query_sample_host(npm_handle* h, int64_t n, const float* pos, const float* aux,
                                 const float* u, int64_t ld, float uniform_frac, float* dir_out,
                                 float* pdf_out, void* stream) {
    npm::CallRange range("npm_query_sample_host");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (!(uniform_frac >= 0.0f && uniform_frac <= 1.0f))
        return fail(NPM_ERR_INVALID_ARG, "uniform_frac outside [0, 1]");
    if (n > 0 && (!u || !dir_out || !pdf_out))
        return fail(NPM_ERR_INVALID_ARG, "u, dir_out and pdf_out are required");
    if (n == 0) return NPM_OK;
    cudaStream_t user = (cudaStream_t)stream;
    const int64_t mb = h->cfg.max_batch;
    float* dpos = h->stage;
    float* daux = dpos + 3 * mb;
    float* du = daux + 7 * mb;
    float* ddir = du + 4 * mb;
    float* dpdf = ddir + 3 * mb;
    const int urows = uniform_frac > 0.0f ? 4 : 3;
    const int arows = h->cfg.mode == NPM_PRODUCT ? 7 : 0;
    // Chunks of at least 2^16 queries, four of them by default (measured
    // best for 2^20 queries: fewer expose more of the first and last copies,
    // more pay more kernel ramp-up and tail); NPM_HOST_CHUNKS overrides.
    static std::atomic<int> env_chunks{INT32_MIN + 1};
    const int nch = npm::env_override("NPM_HOST_CHUNKS", env_chunks);
    int64_t chunk = n / (nch >= 1 && nch <= 64 ? nch : 4);
    if (chunk < 65536) chunk = 65536;
    NPM_CUDA(cudaEventRecord(h->ev[0], user), "record");
    for (int i = 0; i < 2; ++i) NPM_CUDA(cudaStreamWaitEvent(h->side[i], h->ev[0], 0), "wait");
    int c = 0;
    for (int64_t c0 = 0; c0 < n; c0 += chunk, ++c) {
        const int64_t cn = n - c0 < chunk ? n - c0 : chunk;
        cudaStream_t st = h->side[c & 1];
        const size_t bytes = (size_t)cn * sizeof(float);
        const size_t hp = (size_t)ld * sizeof(float), dp = (size_t)mb * sizeof(float);  // row pitches
        // One strided copy per [rows][chunk] block (rows are ld apart on the
        // host, mb apart on the device).
        NPM_CUDA(cudaMemcpy2DAsync(dpos + c0, dp, pos + c0, hp, bytes, 3, cudaMemcpyHostToDevice, st),
                 "copy pos");
        if (arows)
            NPM_CUDA(cudaMemcpy2DAsync(daux + c0, dp, aux + c0, hp, bytes, arows, cudaMemcpyHostToDevice, st),
                     "copy aux");
        NPM_CUDA(cudaMemcpy2DAsync(du + c0, dp, u + c0, hp, bytes, urows, cudaMemcpyHostToDevice, st),
                 "copy u");
        s = npm_query_sample(h, cn, dpos + c0, arows ? daux + c0 : nullptr, du + c0, mb,
                             uniform_frac, ddir + c0, dpdf + c0, nullptr, st);
        if (s != NPM_OK) return s;
        NPM_CUDA(cudaMemcpy2DAsync(dir_out + c0, hp, ddir + c0, dp, bytes, 3, cudaMemcpyDeviceToHost, st),
                 "copy dir");
        NPM_CUDA(cudaMemcpyAsync(pdf_out + c0, dpdf + c0, bytes, cudaMemcpyDeviceToHost, st),
                 "copy pdf");
    }
    for (int i = 0; i < 2; ++i) {
        NPM_CUDA(cudaEventRecord(h->ev[1 + i], h->side[i]), "record");
        NPM_CUDA(cudaStreamWaitEvent(user, h->ev[1 + i], 0), "wait");
    }
    NPM_CUDA(cudaStreamSynchronize(user), "npm_query_sample_host");
    return NPM_OK;
}

npm_status npm_eval_pdf(npm_handle* h, int64_t n, const float* pos, const float* aux,
                        const float* dir, int64_t ld, float* pdf_out, void* stream) {
    npm::CallRange range("npm_eval_pdf");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (n > 0 && (!dir || !pdf_out)) return fail(NPM_ERR_INVALID_ARG, "dir and pdf_out are required");
    if (n == 0) return NPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->tc) return npm::tc_query(h, n, ld, pos, aux, dir, 0.0f, false, nullptr, pdf_out, nullptr, st);
    NPM_CUDA(npm::launch_forward_fp32(h->dc, inf_params(h), inf_wfwd(h), n, ld, pos, aux, dir, 0.0f, false,
                                      nullptr, pdf_out, nullptr, st, status_word(h), h->wait_limit),
             "eval_pdf launch");
    return NPM_OK;
}

npm_status npm_eval_log_pdf(npm_handle* h, int64_t n, const float* pos, const float* aux,
                            const float* dir, int64_t ld, float* logpdf_out, void* stream) {
    npm::CallRange range("npm_eval_log_pdf");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (n > 0 && (!dir || !logpdf_out)) return fail(NPM_ERR_INVALID_ARG, "dir and logpdf_out are required");
    if (n == 0) return NPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->tc) return npm::tc_query(h, n, ld, pos, aux, dir, 0.0f, false, nullptr, logpdf_out, nullptr, st, true);
    NPM_CUDA(npm::launch_forward_fp32(h->dc, inf_params(h), inf_wfwd(h), n, ld, pos, aux, dir, 0.0f, false,
                                      nullptr, logpdf_out, nullptr, st, status_word(h), h->wait_limit, false,
                                      true),
             "eval_log_pdf launch");
    return NPM_OK;
}

static npm_status backward_impl(npm_handle* h, int64_t n, const float* pos, const float* aux,
                                const float* dir, const float* rad, const float* spdf,
                                const float* dlogv, int64_t ld, cudaStream_t st) {
    if (!npm::tc_can_train(h) && h->train_smem > 227 * 1024)
        return fail(NPM_ERR_UNSUPPORTED, "training activations do not fit in shared memory");
    float* loss_acc = h->scalars;
    NPM_CUDA(cudaMemsetAsync(loss_acc, 0, sizeof(float), st), "clear loss");
    if (n == 0) return NPM_OK;
    if (npm::tc_can_train(h)) {
        NPM_CUDA(npm::tc_train(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss_acc, st), "train launch");
        return NPM_OK;
    }
    NPM_CUDA(npm::launch_train_fp32(h->dc, h->params, h->mlp_off, h->wfwd, h->wbwd, n, ld, pos, aux,
                                    dir, rad, spdf, dlogv, h->grads, loss_acc, st),
             "train launch");
    return NPM_OK;
}

static npm_status adam_impl(npm_handle* h, const float* loss, cudaStream_t st) {
    h->step += 1;
    int* status = reinterpret_cast<int*>(h->scalars + 8);
    NPM_CUDA(npm::launch_adam(h->n_int, h->params, h->grads, h->adam_m, h->adam_v, h->cfg.lr,
                              h->cfg.beta1, h->cfg.beta2, h->cfg.eps, step_dev(h), loss, status,
                              h->grid_h, h->grid_h ? h->ng : 0, h->ema, h->ema_decay, st),
             "adam launch");
    // The FP32 kernels' padded weights: needed unless the tensor-core
    // kernels serve both inference and training.
    if (!(h->tc && npm::tc_can_train(h))) {
        NPM_CUDA(npm::launch_arrange_weights(h->dc, h->params + h->mlp_off, h->wfwd, h->wbwd, st),
                 "arrange weights");
        npm_status s = arrange_inference_weights(h, st);
        if (s != NPM_OK) return s;
    }
    if (h->tc) NPM_CUDA(npm::tc_refresh_weights(h, st), "bf16 weight copy");
    return NPM_OK;
}

npm_status npm_train_step(npm_handle* h, int64_t n, const float* pos, const float* aux,
                          const float* dir, const float* radiance, const float* sample_pdf,
                          int64_t ld, float* loss_out, void* stream) {
    npm::CallRange range("npm_train_step");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (n > 0 && (!dir || !radiance || !sample_pdf))
        return fail(NPM_ERR_INVALID_ARG, "dir, radiance and sample_pdf are required");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = backward_impl(h, n, pos, aux, dir, radiance, sample_pdf, nullptr, ld, st)) != NPM_OK)
        return s;
    if ((s = adam_impl(h, h->scalars, st)) != NPM_OK) return s;
    if (loss_out) NPM_CUDA(npm::launch_copy_loss(h->scalars, loss_out, st), "copy loss");
    return NPM_OK;
}

npm_status npm_backward(npm_handle* h, int64_t n, const float* pos, const float* aux,
                        const float* dir, const float* dlogv, int64_t ld, void* stream) {
    npm::CallRange range("npm_backward");
    npm_status s = check_call(h, n, ld, pos, aux);
    if (s != NPM_OK) return s;
    if (npm::inject_launch_failure()) return fail(NPM_ERR_CUDA, "injected launch failure (test)");
    if (n > 0 && (!dir || !dlogv)) return fail(NPM_ERR_INVALID_ARG, "dir and dlogv are required");
    cudaStream_t st = (cudaStream_t)stream;
    NPM_CUDA(cudaMemsetAsync(h->grads, 0, h->n_int * sizeof(float), st), "clear grads");
    return backward_impl(h, n, pos, aux, dir, nullptr, nullptr, dlogv, ld, st);
}

npm_status npm_adam_step(npm_handle* h, void* stream) {
    npm::CallRange range("npm_adam_step");
    if (!h) return fail(NPM_ERR_INVALID_ARG, "handle is NULL");
    return adam_impl(h, nullptr, (cudaStream_t)stream);
}

npm_status npm_grid_indices(npm_handle* h, int64_t n, const float* pos, int64_t ld, int32_t* out,
                            void* stream) {
    npm::CallRange range("npm_grid_indices");
    npm_status s = check_call(h, n, ld, pos, nullptr);
    if (s != NPM_OK && s != NPM_ERR_INVALID_ARG) return s;
    if (!h) return s;
    if (n < 0 || ld < n) return fail(NPM_ERR_INVALID_ARG, "bad n or ld");
    if (n > 0 && (!pos || !out)) return fail(NPM_ERR_INVALID_ARG, "pos and out are required");
    if (n == 0) return NPM_OK;
    NPM_CUDA(npm::launch_grid_indices(h->dc, n, ld, pos, out, (cudaStream_t)stream),
             "grid indices launch");
    return NPM_OK;
}

npm_status npm_check_device_status(npm_handle* h, void* stream) {
    npm::CallRange range("npm_check_device_status");
    if (!h) return fail(NPM_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int word = 0;
    int* status = reinterpret_cast<int*>(h->scalars + 8);
    NPM_CUDA(cudaMemcpyAsync(&word, status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
    NPM_CUDA(cudaStreamSynchronize(st), "synchronise");
    NPM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st), "clear status");
    NPM_CUDA(cudaStreamSynchronize(st), "synchronise");
    if (word & npm::kStatusTimeout) return fail(NPM_ERR_TIMEOUT, "a device-side wait timed out");
    if (word & npm::kStatusNumeric) return fail(NPM_ERR_NUMERIC, "non-finite loss; Adam step skipped");
    return NPM_OK;
}

int64_t npm_debug_bounds_violations(void) {
#ifdef NPM_DEBUG_BOUNDS
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, npm::g_bounds_violations, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    return (int64_t)v;
#else
    return -1;
#endif
}

npm_status npm_set_wait_limit(npm_handle* h, int64_t cycles) {
    if (!h) return fail(NPM_ERR_INVALID_ARG, "handle is NULL");
    h->wait_limit = cycles;
    return NPM_OK;
}

// ------------------------------------------------------------ checkpoint

static const char kMagic[8] = {'N', 'P', 'M', 'C', 'K', 'P', 'T', '1'};

npm_status npm_save(npm_handle* h, const char* path) {
    npm::CallRange range("npm_save");
    if (!h || !path) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    const int64_t np = h->ng + h->nmlp;
    std::vector<float> p(np), m(np), v(np);
    npm_status s;
    int step = 0;
    if ((s = npm_get_adam(h, &step, nullptr, nullptr)) != NPM_OK) return s;
    if ((s = npm_get_params(h, p.data(), np)) != NPM_OK) return s;
    if ((s = copy_public(h, h->adam_m, m.data(), np, false)) != NPM_OK) return s;
    if ((s = copy_public(h, h->adam_v, v.data(), np, false)) != NPM_OK) return s;
    FILE* f = fopen(path, "wb");
    if (!f) return fail(NPM_ERR_IO, std::string("cannot open ") + path);
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&h->cfg, sizeof(npm_config), 1, f) == 1 &&
              fwrite(&h->step, sizeof(int), 1, f) == 1 && fwrite(&np, sizeof(int64_t), 1, f) == 1 &&
              fwrite(p.data(), sizeof(float), np, f) == (size_t)np &&
              fwrite(m.data(), sizeof(float), np, f) == (size_t)np &&
              fwrite(v.data(), sizeof(float), np, f) == (size_t)np;
    ok = (fclose(f) == 0) && ok;
    return ok ? NPM_OK : fail(NPM_ERR_IO, std::string("write failed: ") + path);
}

npm_status npm_load(npm_handle* h, const char* path) {
    npm::CallRange range("npm_load");
    if (!h || !path) return fail(NPM_ERR_INVALID_ARG, "NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(NPM_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    npm_config c;
    int step = 0;
    int64_t np = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(&c, sizeof(npm_config), 1, f) == 1 && fread(&step, sizeof(int), 1, f) == 1 &&
              fread(&np, sizeof(int64_t), 1, f) == 1;
    if (!ok || np != h->ng + h->nmlp) {
        fclose(f);
        return fail(NPM_ERR_IO, "not a checkpoint of this configuration");
    }
    // The shape-defining fields must match (hyper-parameters may differ).
    if (c.mode != h->cfg.mode || c.n_levels != h->cfg.n_levels ||
        c.feat_per_level != h->cfg.feat_per_level || c.log2_table != h->cfg.log2_table ||
        c.n_layers != h->cfg.n_layers || c.K != h->cfg.K || c.kappa_act != h->cfg.kappa_act ||
        memcmp(c.level_res, h->cfg.level_res, sizeof(int) * h->cfg.n_levels) != 0 ||
        memcmp(c.widths, h->cfg.widths, sizeof(int) * (h->cfg.n_layers + 1)) != 0) {
        fclose(f);
        return fail(NPM_ERR_IO, "checkpoint configuration differs");
    }
    std::vector<float> p(np), m(np), v(np);
    ok = fread(p.data(), sizeof(float), np, f) == (size_t)np &&
         fread(m.data(), sizeof(float), np, f) == (size_t)np &&
         fread(v.data(), sizeof(float), np, f) == (size_t)np;
    fclose(f);
    if (!ok) return fail(NPM_ERR_IO, "truncated checkpoint");
    npm_status s;
    if ((s = npm_set_params(h, p.data(), np)) != NPM_OK) return s;
    return npm_set_adam(h, step, m.data(), v.data());
}

}  // extern "C"
