// npm_scene.cu -- synthetic stand-in for the paper's renderer and scenes:
// seeded inputs and an analytic radiance target, generated on the device so
// that training loops and the wavefront frame driver stay on the GPU.
//
// Random numbers: SplitMix64 (Steele, Lea, Flood 2014) at state
// s0 + (i + 1) * 0x9E3779B97F4A7C15 with s0 = mix(mix(seed) ^ stream); a
// uniform is (bits >> 40) * 2^-24, an exact float in [0, 1). Element (r, j)
// of an [rows][n] block uses counter r * n + j. Positions, sampling uniforms
// and noise are therefore bit-identical to the host generator of the tests.
//
// Target: L(x, w) = sum_m a_m k_m exp(k_m (mu_m(x).w - 1)) / (2 pi (1 -
// e^{-2 k_m})), three lobes with a = (0.5, 0.3, 0.2), means
// normalize(e_m + 0.5 (sin(2 pi x_y + m), sin(2 pi x_z + 2m), sin(2 pi x_x + 3m)))
// and sharpness 1 + 49 (1/2 + 1/2 sin(2 pi (m+1)(x_x + x_y + x_z) / 3 + m)).
// Product mode multiplies max(0, n.w) (0.3 + 0.7 D(n.h) / D(1)), D the GGX
// distribution with alpha = roughness^2 and h = normalize(w + wo).
#include <math.h>

#include "npm_handle.h"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr float kTwoPi = 6.28318530717958647692f;

enum : uint64_t { S_POS = 1, S_U = 2, S_DIR = 3, S_NOISE = 4, S_AUX = 7 };

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t stream_key(uint64_t seed, uint64_t stream) { return mix64(mix64(seed) ^ stream); }

__device__ __forceinline__ float uni(uint64_t s0, uint64_t i) {
    return (float)(mix64(s0 + (i + 1) * kGamma) >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ void sphere_dir(float u1, float u2, float* d) {
    const float z = 1.0f - 2.0f * u1;
    const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float s, c;
    sincosf(kTwoPi * u2, &s, &c);
    d[0] = r * c;
    d[1] = r * s;
    d[2] = z;
}

__global__ void k_scene_generate(int64_t n, int64_t ld, uint64_t k_pos, uint64_t k_aux, uint64_t k_u,
                                 int urows, float* __restrict__ pos, float* __restrict__ aux,
                                 float* __restrict__ u) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        for (int r = 0; r < 3; ++r) pos[r * ld + j] = uni(k_pos, (uint64_t)(r * n + j));
        for (int r = 0; r < urows; ++r) u[r * ld + j] = uni(k_u, (uint64_t)(r * n + j));
        if (aux) {
            float a[5];
            for (int r = 0; r < 5; ++r) a[r] = uni(k_aux, (uint64_t)(r * n + j));
            float nrm[3], wo[3];
            sphere_dir(a[0], a[1], nrm);
            sphere_dir(a[2], a[3], wo);
            if (nrm[0] * wo[0] + nrm[1] * wo[1] + nrm[2] * wo[2] < 0.0f)
                for (int c = 0; c < 3; ++c) wo[c] = -wo[c];
            for (int c = 0; c < 3; ++c) {
                aux[c * ld + j] = wo[c];
                aux[(3 + c) * ld + j] = nrm[c];
            }
            aux[6 * ld + j] = 0.05f + 0.95f * a[4];
        }
    }
}

__device__ float field(const float* x, const float* w) {
    const float amp[3] = {0.5f, 0.3f, 0.2f};
    const float e[3][3] = {{0.0f, 0.0f, 1.0f}, {1.0f, 0.0f, 0.0f},
                           {-0.57735026918962584f, -0.57735026918962584f, 0.57735026918962584f}};
    float L = 0.0f;
    for (int m = 0; m < 3; ++m) {
        float v[3] = {e[m][0] + 0.5f * sinf(kTwoPi * x[1] + m), e[m][1] + 0.5f * sinf(kTwoPi * x[2] + 2 * m),
                      e[m][2] + 0.5f * sinf(kTwoPi * x[0] + 3 * m)};
        const float inv = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const float d = (v[0] * w[0] + v[1] * w[1] + v[2] * w[2]) * inv;
        const float k = 1.0f + 49.0f * (0.5f + 0.5f * sinf(kTwoPi * (m + 1) * (x[0] + x[1] + x[2]) / 3.0f + m));
        L += amp[m] * k * expf(k * (d - 1.0f)) / (kTwoPi * (-expm1f(-2.0f * k)));
    }
    return L;
}

__device__ float glossy(const float* w, const float* aux) {
    const float* wo = aux;
    const float* nn = aux + 3;
    const float r = aux[6];
    const float cos_i = fmaxf(0.0f, nn[0] * w[0] + nn[1] * w[1] + nn[2] * w[2]);
    float h[3] = {w[0] + wo[0], w[1] + wo[1], w[2] + wo[2]};
    const float hl = sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    float ratio = 0.0f;
    if (hl > 1e-9f) {
        const float ch = fminf(1.0f, fmaxf(-1.0f, (nn[0] * h[0] + nn[1] * h[1] + nn[2] * h[2]) / hl));
        if (ch > 0.0f) {
            const float a2 = (r * r) * (r * r);
            const float den = ch * ch * (a2 - 1.0f) + 1.0f;
            ratio = a2 * a2 / (den * den);
        }
    }
    return cos_i * (0.3f + 0.7f * ratio);
}

__global__ void k_scene_radiance(int64_t n, int64_t ld, int product, uint64_t k_noise,
                                 const float* __restrict__ pos, const float* __restrict__ aux,
                                 const float* __restrict__ dir, float* __restrict__ clean,
                                 float* __restrict__ noisy) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float x[3] = {pos[j], pos[ld + j], pos[2 * ld + j]};
        const float w[3] = {dir[j], dir[ld + j], dir[2 * ld + j]};
        float L = field(x, w);
        if (product) {
            float a[7];
            for (int c = 0; c < 7; ++c) a[c] = aux[c * ld + j];
            L *= glossy(w, a);
        }
        if (clean) clean[j] = L;
        if (noisy) noisy[j] = L * -log1pf(-uni(k_noise, (uint64_t)j));
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g > 8192 ? 8192 : g < 1 ? 1 : g);
}

}  // namespace

extern "C" {

npm_status npm_scene_generate(uint64_t seed, int64_t n, int product, float* pos, float* aux,
                              float* u, int urows, int64_t ld, void* stream) {
    if (n < 0 || ld < n || (n > 0 && (!pos || !u || (product && !aux))) || urows < 0 || urows > 4)
        return npm::set_error(NPM_ERR_INVALID_ARG, "bad scene_generate arguments");
    if (n == 0) return NPM_OK;
    k_scene_generate<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        n, ld, stream_key(seed, S_POS), stream_key(seed, S_AUX), stream_key(seed, S_U), urows, pos,
        product ? aux : nullptr, u);
    return cudaGetLastError() == cudaSuccess ? NPM_OK : npm::set_error(NPM_ERR_CUDA, "scene_generate launch");
}

npm_status npm_scene_radiance(int product, uint64_t noise_seed, int64_t n, const float* pos,
                              const float* aux, const float* dir, int64_t ld, float* clean_out,
                              float* noisy_out, void* stream) {
    if (n < 0 || ld < n || (n > 0 && (!pos || !dir || (product && !aux) || (!clean_out && !noisy_out))))
        return npm::set_error(NPM_ERR_INVALID_ARG, "bad scene_radiance arguments");
    if (n == 0) return NPM_OK;
    k_scene_radiance<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        n, ld, product, stream_key(noise_seed, S_NOISE), pos, aux, dir, clean_out, noisy_out);
    return cudaGetLastError() == cudaSuccess ? NPM_OK : npm::set_error(NPM_ERR_CUDA, "scene_radiance launch");
}

}  // extern "C"
