// npm_kernels.h -- host-side launchers of the NPM kernels (internal).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>

#include "npm_device.cuh"

namespace npm {

// Dynamic shared-memory limit and L1/shared carveout of a kernel, set only
// when (device, size, carveout) differs from the last call for that kernel
// (`last` is the caller's per-kernel cache): the attribute calls cost host
// time that small, latency-bound launches would otherwise pay every time.
template <typename KernelT>
inline cudaError_t set_smem_attrs(KernelT kern, size_t smem, int carveout_pct, std::atomic<uint64_t>& last) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t key = ((uint64_t)(unsigned)dev << 40) | ((uint64_t)(unsigned)carveout_pct << 32) | (uint64_t)smem;
    if (last.load(std::memory_order_relaxed) == key) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_pct);
    if (e != cudaSuccess) return e;
    last.store(key, std::memory_order_relaxed);
    return cudaSuccess;
}

// Launch of kern<<<grid, block, smem, st>>>(args...), with programmatic
// stream serialization when pdl is set: the kernel may then be scheduled
// before the stream's previous kernel completes, and must call
// grid_dep_wait() before it reads anything that kernel writes.
template <typename... Params, typename... Args>
inline cudaError_t launch_maybe_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    bool pdl, Args&&... args) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&lc, kern, static_cast<Args&&>(args)...);
}

// Integer tuning override from the environment, read once per process
// (`cache` holds it; INT32_MIN when unset or not a number).
inline int env_override(const char* name, std::atomic<int>& cache) {
    int v = cache.load(std::memory_order_relaxed);
    if (v == INT32_MIN + 1) {
        const char* s = getenv(name);
        v = (s && *s) ? atoi(s) : INT32_MIN;
        cache.store(v, std::memory_order_relaxed);
    }
    return v;
}

// Default bound of a kernel-internal wait: 2^31 SM clock cycles (about a
// second at 2 GHz).
constexpr long long kDefaultWaitLimit = 1ll << 31;

size_t fwd_smem_bytes(const DevCfg& c);
// Shared-memory carveout (percent of the maximum) that holds `bytes`.
int carveout_percent(size_t bytes);
size_t train_smem_bytes(const DevCfg& c);

// wait_free: use only the tile-group kernel, which has no kernel-internal
// waits (no mailbox hand-offs), so no launch can end early on a timeout.
// log_pdf (evaluation only): pdf_out receives log V instead of V.
cudaError_t launch_forward_fp32(const DevCfg& cfg, const float* grid, const float* wfwd, int64_t n,
                                int64_t ld, const float* pos, const float* aux, const float* uin,
                                float ufrac, bool sample, float* dir_out, float* pdf_out,
                                float* mix_out, cudaStream_t st, int* status = nullptr,
                                long long wait_limit = kDefaultWaitLimit, bool wait_free = false,
                                bool log_pdf = false);

// Several requests in one launch (segment table; tile offsets filled in
// here). max_n bounds the device-side count when qb.n_dev is set. status
// (device word, or NULL) receives kStatusTimeout if a kernel-internal
// hand-off gives up after wait_limit SM clock cycles (<= 0: one
// non-blocking test per wait).
cudaError_t launch_forward_fp32_batch(const DevCfg& cfg, const float* grid, const float* wfwd,
                                      QueryBatch& qb, int64_t max_n, cudaStream_t st,
                                      int* status = nullptr, long long wait_limit = kDefaultWaitLimit,
                                      bool wait_free = false);

cudaError_t launch_train_fp32(const DevCfg& cfg, const float* params, int64_t mlp_off,
                              const float* wfwd, const float* wbwd, int64_t n, int64_t ld,
                              const float* pos, const float* aux, const float* dir,
                              const float* rad, const float* spdf, const float* dlogv,
                              float* grad, float* loss, cudaStream_t st);

cudaError_t launch_arrange_weights(const DevCfg& cfg, const float* mlp, float* wfwd, float* wbwd,
                                   cudaStream_t st);

// Adam at step *steps + 1 (device counter, advanced on the stream after the
// update). ema (or NULL): moving average updated with ema_decay; the FP16
// copy is then taken from it.
cudaError_t launch_adam(int64_t n, float* p, float* g, float* m, float* v, float lr, float b1,
                        float b2, float eps, int* steps, const float* loss, int* status,
                        __half* half_copy, int64_t n_half, float* ema, float ema_decay,
                        cudaStream_t st);

cudaError_t launch_grid_indices(const DevCfg& cfg, int64_t n, int64_t ld, const float* pos,
                                int32_t* out, cudaStream_t st);

cudaError_t launch_to_half(int64_t n, const float* src, __half* dst, cudaStream_t st);

cudaError_t launch_copy_loss(const float* acc, float* out, cudaStream_t st);

}  // namespace npm
