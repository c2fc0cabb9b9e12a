// npm_noalloc.cu -- npm_eval_pdf_noalloc: the mixture-density evaluation of
// the FP32 path for callers that cannot allocate device memory.
//
// The FP32 forward kernel reads its weights from a padded, transposed copy of
// the MLP weights (scratch derived from the parameters). npm_eval_pdf keeps
// that copy in handle-owned memory; this variant builds it instead in a
// fixed, file-scope device array, so the call needs no handle and performs
// no allocation. The array is loaded with the library on every GPU that uses
// it and stays resident until the process exits.
#include "npm_handle.h"
#include "npm_kernels.h"

namespace {

// Scratch for the padded forward weights (W^T per layer). Its size is the
// NPM_NOALLOC_MAX_WEIGHT_FLOATS limit of include/npm.h.
static __device__ __align__(256) float g_noalloc_weights[NPM_NOALLOC_MAX_WEIGHT_FLOATS];

// The device address of the scratch array on the current device. In host
// code the array's name is only a host-side stand-in, so the address comes
// from cudaGetSymbolAddress with the device current. It is looked up on
// every call (a table lookup once the module is loaded; it allocates
// nothing), so a context that was reset and re-created gets its own address.
npm_status scratch_for_current_device(float** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_weights);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return npm::set_error(NPM_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    *out = static_cast<float*>(p);
    return NPM_OK;
}

// Forward blob only (W^T [in][np] per layer, zero padded): every float of
// [0, fwd_floats) is written, so no stale value from an earlier call survives.
__global__ void k_noalloc_arrange(npm::DevCfg cfg, const float* __restrict__ mlp,
                                  float* __restrict__ wfwd) {
    int64_t woff = 0;
    for (int l = 0; l < cfg.n_layers; ++l) {
        const int K = cfg.widths[l], N = cfg.widths[l + 1], npf = cfg.np_fwd[l];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * npf; i += gridDim.x * blockDim.x) {
            const int k = i / npf, nn = i % npf;
            wfwd[cfg.off_fwd[l] + i] = nn < N ? mlp[woff + (int64_t)nn * K + k] : 0.0f;
        }
        woff += (int64_t)K * N;
    }
}

}  // namespace

extern "C" npm_status npm_eval_pdf_noalloc(const npm_config* cfg, const float* params, int64_t n,
                                           const float* pos, const float* aux, const float* dir,
                                           int64_t ld, float* pdf_out, void* stream) {
    npm::CallRange range("npm_eval_pdf_noalloc");
    npm::DevCfg dc;
    int64_t ng = 0, nmlp = 0;
    npm_status s = npm::make_devcfg(cfg, &dc, &ng, &nmlp);
    if (s != NPM_OK) return s;
    if (dc.fwd_floats > NPM_NOALLOC_MAX_WEIGHT_FLOATS)
        return npm::set_error(NPM_ERR_CAPACITY,
                              "npm_eval_pdf_noalloc: padded MLP weights exceed "
                              "NPM_NOALLOC_MAX_WEIGHT_FLOATS floats of static scratch");
    if (n < 0 || ld < n) return npm::set_error(NPM_ERR_INVALID_ARG, "bad n or ld");
    if (n > 0 && (!params || !pos || !dir || !pdf_out))
        return npm::set_error(NPM_ERR_INVALID_ARG, "params, pos, dir and pdf_out are required");
    if (n > 0 && cfg->mode == NPM_PRODUCT && !aux)
        return npm::set_error(NPM_ERR_INVALID_ARG, "product mode needs aux [7][ld]");
    if (n > 0 && (reinterpret_cast<uintptr_t>(params) & 15u))
        return npm::set_error(NPM_ERR_INVALID_ARG, "params must be 16-byte aligned");
    float* scratch = nullptr;
    if ((s = scratch_for_current_device(&scratch)) != NPM_OK) return s;
    if (n == 0) return NPM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_arrange<<<8, 256, 0, st>>>(dc, params + ng, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
    // The tile-group kernel only: it has no kernel-internal waits, so no
    // launch can give up part-way, and with no status word to report such
    // an outcome every pdf_out value is written when the call succeeds.
    e = npm::launch_forward_fp32(dc, params, scratch, n, ld, pos, aux, dir, 0.0f, false, nullptr,
                                 pdf_out, nullptr, st, nullptr, npm::kDefaultWaitLimit, true);
    if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
    return NPM_OK;
}
