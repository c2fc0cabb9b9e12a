// npm_validate.cu -- validation reduction on the GPU: the integral of the
// model's mixture density over the sphere, by a caller-given quadrature,
// accumulated in FP64 (Eq. 3-4 define V as a density, so the integral is
// 1). The density values come from npm_eval_pdf, the hot path itself; FP64
// is used only in this reduction.
#include <string.h>

#include "npm_handle.h"
#include "npm_kernels.h"

namespace {

// Queries p * n_dir + k of a chunk: position p (and its auxiliary inputs)
// with quadrature direction k; [c][m] layout with row stride mb.
__global__ void k_replicate(int64_t m, int64_t n_dir, int64_t ld, int64_t p0, const float* __restrict__ pos,
                            const float* __restrict__ aux, int arows, const float* __restrict__ dirs,
                            int64_t mb, float* __restrict__ qpos, float* __restrict__ qaux,
                            float* __restrict__ qdir) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + q / n_dir, k = q % n_dir;
        for (int r = 0; r < 3; ++r) {
            qpos[r * mb + q] = pos[r * ld + p];
            qdir[r * mb + q] = dirs[r * n_dir + k];
        }
        for (int r = 0; r < arows; ++r) qaux[r * mb + q] = aux[r * ld + p];
    }
}

// out[p] = sum_k w[k] pdf[p * n_dir + k] in FP64, one block per position.
__global__ void k_weighted_sum_f64(const float* __restrict__ pdf, const double* __restrict__ w, int64_t n_dir,
                                   double* __restrict__ out) {
    __shared__ double part[256];
    const int64_t p = blockIdx.x;
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n_dir; k += blockDim.x) s += w[k] * (double)pdf[p * n_dir + k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = part[0];
}

}  // namespace

npm_status npm_pdf_integral(npm_handle* h, int64_t n_pos, const float* pos, const float* aux, int64_t ld,
                            int64_t n_dir, const float* dirs, const double* weights, double* out,
                            void* stream) {
    npm::CallRange range("npm_pdf_integral");
    if (!h) return npm::set_error(NPM_ERR_INVALID_ARG, "handle is NULL");
    if (n_pos < 0 || n_dir < 1 || ld < n_pos) return npm::set_error(NPM_ERR_INVALID_ARG, "bad sizes");
    if (n_pos > 0 && (!pos || !dirs || !weights || !out))
        return npm::set_error(NPM_ERR_INVALID_ARG, "pos, dirs, weights and out are required");
    if (h->cfg.mode == NPM_PRODUCT && n_pos > 0 && !aux)
        return npm::set_error(NPM_ERR_INVALID_ARG, "product mode needs aux");
    const int64_t mb = h->cfg.max_batch;
    if (n_dir > mb) return npm::set_error(NPM_ERR_CAPACITY, "n_dir exceeds max_batch");
    if (n_pos == 0) return NPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // The staging buffers of the host-buffer entry points: positions [3],
    // auxiliary inputs [7], directions [3] (in the uniforms' rows), density.
    float* qpos = h->stage;
    float* qaux = qpos + 3 * mb;
    float* qdir = qaux + 7 * mb;
    float* qpdf = qdir + 7 * mb;
    const int arows = h->cfg.mode == NPM_PRODUCT ? 7 : 0;
    const int64_t per = mb / n_dir;  // positions per chunk
    for (int64_t p0 = 0; p0 < n_pos; p0 += per) {
        const int64_t np = n_pos - p0 < per ? n_pos - p0 : per;
        const int64_t m = np * n_dir;
        int64_t g = (m + 255) / 256;
        if (g > 4096) g = 4096;
        k_replicate<<<(int)g, 256, 0, st>>>(m, n_dir, ld, p0, pos, aux, arows, dirs, mb, qpos, qaux, qdir);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
        npm_status s = npm_eval_pdf(h, m, qpos, arows ? qaux : nullptr, qdir, mb, qpdf, stream);
        if (s != NPM_OK) return s;
        k_weighted_sum_f64<<<(int)np, 256, 0, st>>>(qpdf, weights, n_dir, out + p0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
    }
    return NPM_OK;
}
