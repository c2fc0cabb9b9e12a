// npm_handle.h -- the library-side state behind an npm_handle (internal).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "npm.h"
#include "npm_device.cuh"

namespace npm {
struct TcState;
}

struct npm_handle {
    npm_config cfg;
    npm::DevCfg dc;
    int device = 0;
    // Internal parameter blob: grid [0, ng), MLP weights at mlp_off (aligned
    // to 64 floats), total n_int (a multiple of 64). The public layout packs
    // the MLP right after the grid.
    int64_t ng = 0, nmlp = 0, mlp_off = 0, n_int = 0;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* wfwd = nullptr;     // padded W^T blobs for the FP32 kernels
    float* wbwd = nullptr;     // padded W blobs (backward)
    __half* grid_h = nullptr;  // FP16 grid copy (BF16 precision)
    float* scalars = nullptr;  // [0] loss accumulator, [8] status word
    float* stage = nullptr;    // device staging for the _host entry points
    cudaStream_t side[2] = {nullptr, nullptr};  // internal streams (host staging)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    size_t fwd_smem = 0, train_smem = 0;
    int step = 0;
    npm::TcState* tc = nullptr;  // tensor-core (BF16) path state
    // Exponential moving average of the parameters (Sec. 5.3), evaluated by
    // inference when enabled: ema (n_int, internal layout) and its padded
    // forward weights; the FP16 grid copy and the tensor-core inference
    // weights are then derived from ema too.
    float* ema = nullptr;
    float* wfwd_inf = nullptr;
    float ema_decay = 0.0f;
    // Bound of the FP32 forward kernel's internal waits (npm_set_wait_limit).
    long long wait_limit = 1ll << 31;
};

// Parameters and FP32 forward weights that inference evaluates.
inline const float* inf_params(const npm_handle* h) { return h->ema ? h->ema : h->params; }
inline const float* inf_wfwd(const npm_handle* h) { return h->ema ? h->wfwd_inf : h->wfwd; }
// Device status word (kStatus* bits, read by npm_check_device_status).
inline int* status_word(npm_handle* h) { return reinterpret_cast<int*>(h->scalars + 8); }

namespace npm {
// NVTX range named after an entry point for the lifetime of the object, so
// that a profiler's timeline groups the kernels of each call (a few
// nanoseconds when no tool is attached).
struct CallRange {
    explicit CallRange(const char* name);
    ~CallRange();
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

// Test-only host-side fault injection, off unless the environment sets it:
// NPM_TEST_FAIL_ALLOC=N makes the N-th device allocation of each npm_create
// fail (NPM_ERR_OOM); NPM_TEST_FAIL_LAUNCH=N makes the N-th hot call of the
// process report a failed launch (NPM_ERR_CUDA) without launching anything.
cudaError_t device_alloc(void** p, size_t bytes);
bool inject_launch_failure();

// Validates cfg and derives the kernels' view of it; ng / nmlp receive the
// grid and MLP parameter counts (npm_api.cu).
npm_status make_devcfg(const npm_config* cfg, DevCfg* out, int64_t* ng, int64_t* nmlp);
// Records msg as the thread's last error and returns s.
npm_status set_error(npm_status s, const char* msg);

// Tensor-core (tcgen05, BF16) path, npm_tc.cu.
npm_status tc_create(npm_handle* h);
void tc_destroy(npm_handle* h);
cudaError_t tc_refresh_weights(npm_handle* h, cudaStream_t st);
// pdl: the small networks' kernel may be launched as a programmatic
// dependent of the stream's previous kernel, which must then not write the
// model's weights or grid (other kernels launch as usual).
cudaError_t tc_query_batch(npm_handle* h, QueryBatch& qb, int64_t max_n, cudaStream_t st, bool pdl = false);
// Training step kernels on tensor cores (split BF16 operands).
bool tc_can_train(npm_handle* h);
cudaError_t tc_train(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux, const float* dir,
                     const float* rad, const float* spdf, const float* dlogv, float* loss, cudaStream_t st);
// log_pdf (evaluation only): pdf_out receives log V instead of V.
npm_status tc_query(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux,
                    const float* uin, float ufrac, bool sample, float* dir_out, float* pdf_out,
                    float* mix_out, cudaStream_t st, bool log_pdf = false);
}  // namespace npm
