// npm_device.cuh -- device-side configuration and per-query math of the NPM
// hot path: grid lattice index and trilinear weights (Sec. 5.1, Eq. 11),
// spherical-harmonics encoding (Sec. 4.3), the Table 1 output mapping, the vMF
// mixture density (Eq. 3-4) and vMF sampling (Sec. 5.3).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "npm.h"

namespace npm {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInv4Pi = 0.0795774715459476679f;

// Everything a kernel needs to know about the model, passed by value.
struct DevCfg {
    int mode;        // NPM_RADIANCE / NPM_PRODUCT
    int n_levels;
    int feat;        // F
    int K;           // lobes
    int kappa_act;   // NPM_SOFTPLUS / NPM_EXP
    int n_layers;
    int grid_feats;  // n_levels * feat
    uint32_t table_mask;  // T - 1
    uint32_t dense_mask;  // bit l: level l is stored densely
    int widths[NPM_MAX_LAYERS + 1];
    int level_res[NPM_MAX_LEVELS];
    uint32_t level_off[NPM_MAX_LEVELS];  // first entry of each level
    // FP32 fused kernels: per layer, padded output count (multiple of 16)
    // and float offsets of the pre-arranged weight blobs.
    int np_fwd[NPM_MAX_LAYERS];   // padded N of W^T [K][np] (forward)
    int np_bwd[NPM_MAX_LAYERS];   // padded K of W [N][np] (backward)
    int off_fwd[NPM_MAX_LAYERS];
    int off_bwd[NPM_MAX_LAYERS];
    int fwd_floats, bwd_floats;
    int max_width;
};

// ------------------------------------------------------ debug bounds

// With NPM_DEBUG_BOUNDS defined (a separate debug build of the library),
// bounded_index checks a grid-entry or queue-slot index against its limit
// before the access: an index at or beyond the limit is counted in
// g_bounds_violations and replaced by 0, so the access stays inside the
// buffer and the kernel carries on (no trap). npm_debug_bounds_violations
// reads the count. In the normal build the check compiles away.

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is still
// running; grid_dep_wait() returns once that predecessor has completed and
// its writes are visible (at once for a kernel launched without it).
// grid_dep_launch() lets the stream's next such kernel be scheduled.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

#ifdef NPM_DEBUG_BOUNDS
extern __device__ unsigned long long g_bounds_violations;
__device__ __forceinline__ uint32_t bounded_index(uint32_t idx, uint32_t limit) {
    if (idx >= limit) {
        atomicAdd(&g_bounds_violations, 1ull);
        return 0u;
    }
    return idx;
}
__device__ __forceinline__ int64_t bounded_slot(int64_t j, int64_t limit) {
    if (j < 0 || j >= limit) {
        atomicAdd(&g_bounds_violations, 1ull);
        return 0;
    }
    return j;
}
#else
__device__ __forceinline__ uint32_t bounded_index(uint32_t idx, uint32_t) { return idx; }
__device__ __forceinline__ int64_t bounded_slot(int64_t j, int64_t) { return j; }
#endif

// ------------------------------------------------------ lattice (Eq. 11)

// Cell and fraction along one axis: x clamped to [0,1] (NaN -> 0),
// p = x * (D - 1) with one round-to-nearest multiply, cell = min(floor p, D-2).
__device__ __forceinline__ void lattice_axis(float x, int D, uint32_t& cell, float& frac) {
    float xa = fminf(fmaxf(x, 0.0f), 1.0f);
    float p = __fmul_rn(xa, (float)(D - 1));
    int c = (int)floorf(p);
    c = c > D - 2 ? D - 2 : c;
    cell = (uint32_t)c;
    frac = __fsub_rn(p, (float)c);
}

// Cell of a point at one level: lower lattice point and fractions.
struct Cell {
    uint32_t c[3];
    float f[3];
};

__device__ __forceinline__ Cell make_cell(float x, float y, float z, int D) {
    Cell cl;
    lattice_axis(x, D, cl.c[0], cl.f[0]);
    lattice_axis(y, D, cl.c[1], cl.f[1]);
    lattice_axis(z, D, cl.c[2], cl.f[2]);
    return cl;
}

// The 8 corners of a cell at level l (corner c: bit0 = +x, bit1 = +y,
// bit2 = +z), Eq. 11: entry indices and trilinear weights
// (wx * wy) * wz with w = f or 1 - f per axis. Lattice point (i, j, k) is
// entry i + D (j + D k) of a dense level (D^3 <= T) and
// (i ^ j * 2654435761 ^ k * 805459861) mod T of a hashed one (the
// Instant-NGP spatial hash; uint32 arithmetic). The per-axis terms are
// shared: dense corners are b + dx + D dy + D^2 dz with b = i + D (j + D k),
// hashed ones use (j + 1) * P = j * P + P (mod 2^32). corner_idx8 and
// corner_w8 compute the two halves separately, so that callers can issue
// the loads before forming the weights.
__device__ __forceinline__ void corner_idx8(const DevCfg& cfg, int l, const Cell& cl, uint32_t (&idx)[8]) {
    if ((cfg.dense_mask >> l) & 1u) {
        const uint32_t D = (uint32_t)cfg.level_res[l];
        const uint32_t b = cl.c[0] + D * (cl.c[1] + D * cl.c[2]);
        const uint32_t dy = D, dz = D * D;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            idx[c] = bounded_index(b + (c & 1) + ((c & 2) ? dy : 0u) + ((c & 4) ? dz : 0u), D * D * D);
    } else {
        const uint32_t hx[2] = {cl.c[0], cl.c[0] + 1u};
        const uint32_t hy0 = cl.c[1] * 2654435761u, hz0 = cl.c[2] * 805459861u;
        const uint32_t hy[2] = {hy0, hy0 + 2654435761u};
        const uint32_t hz[2] = {hz0, hz0 + 805459861u};
#pragma unroll
        for (int c = 0; c < 8; ++c) idx[c] = (hx[c & 1] ^ hy[(c >> 1) & 1] ^ hz[(c >> 2) & 1]) & cfg.table_mask;
    }
}

__device__ __forceinline__ void corner_w8(const Cell& cl, float (&w)[8]) {
    const float wx[2] = {1.0f - cl.f[0], cl.f[0]};
    const float wy[2] = {1.0f - cl.f[1], cl.f[1]};
    const float wz[2] = {1.0f - cl.f[2], cl.f[2]};
    float wxy[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) wxy[c] = wx[c & 1] * wy[(c >> 1) & 1];
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = wxy[c & 3] * wz[(c >> 2) & 1];
}

__device__ __forceinline__ void corners8(const DevCfg& cfg, int l, const Cell& cl, uint32_t (&idx)[8],
                                         float (&w)[8]) {
    corner_idx8(cfg, l, cl, idx);
    corner_w8(cl, w);
}

// Features of two x-adjacent corners (entries a, b of a 2-feature level
// starting at entry level_off; gl points at the level): one 16-byte load
// (FP32) or 8-byte load (FP16) when the two entries form an aligned pair,
// else one load each. Random gathers cost the L1 a wavefront per lane and
// load, so the paired lanes halve their share.
__device__ __forceinline__ void gather_pair2(const float* gl, uint32_t level_off, uint32_t a, uint32_t b,
                                             float2& va, float2& vb) {
    const uint32_t lo = a < b ? a : b;
    if ((a > b ? a - b : b - a) == 1u && ((level_off + lo) & 1u) == 0u) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(gl + (size_t)lo * 2));
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
        va = a < b ? v0 : v1;
        vb = a < b ? v1 : v0;
    } else {
        va = __ldg(reinterpret_cast<const float2*>(gl) + a);
        vb = __ldg(reinterpret_cast<const float2*>(gl) + b);
    }
}
__device__ __forceinline__ void gather_pair2(const __half* gl, uint32_t level_off, uint32_t a, uint32_t b,
                                             float2& va, float2& vb) {
    const uint32_t lo = a < b ? a : b;
    if ((a > b ? a - b : b - a) == 1u && ((level_off + lo) & 1u) == 0u) {
        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(gl + (size_t)lo * 2));
        const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
        const float2 v1 = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
        va = a < b ? v0 : v1;
        vb = a < b ? v1 : v0;
    } else {
        const unsigned int ra = __ldg(reinterpret_cast<const unsigned int*>(gl) + a);
        const unsigned int rb = __ldg(reinterpret_cast<const unsigned int*>(gl) + b);
        va = __half22float2(*reinterpret_cast<const __half2*>(&ra));
        vb = __half22float2(*reinterpret_cast<const __half2*>(&rb));
    }
}

// Grid-gradient scatter of two x-adjacent corners (entries a, b of a level
// starting at entry level_off, 2 features each; gl points at the level):
// when the two entries form one 16-byte aligned pair, one 4-wide atomic add
// serves both (the L2 atomic units are limited by operations, not bytes).
__device__ __forceinline__ void scatter_pair2(float* gl, uint32_t level_off, uint32_t a, uint32_t b, float wa,
                                              float wb, float d0, float d1) {
    const uint32_t lo = a < b ? a : b;
    if ((a > b ? a - b : b - a) == 1u && ((level_off + lo) & 1u) == 0u) {
        const float4 v = a < b ? make_float4(wa * d0, wa * d1, wb * d0, wb * d1)
                               : make_float4(wb * d0, wb * d1, wa * d0, wa * d1);
        atomicAdd(reinterpret_cast<float4*>(gl + (size_t)lo * 2), v);
    } else {
        atomicAdd(reinterpret_cast<float2*>(gl + (size_t)a * 2), make_float2(wa * d0, wa * d1));
        atomicAdd(reinterpret_cast<float2*>(gl + (size_t)b * 2), make_float2(wb * d0, wb * d1));
    }
}

// ------------------------------------------ spherical harmonics (Sec. 4.3)

// Real orthonormal SH, bands 0..3 (16 values), in the order
// l=0; l=1: y, z, x; l=2: xy, yz, 3z^2-1, xz, x^2-y^2; l=3: m=-3..3.
__device__ __forceinline__ void sh_band4(float x, float y, float z, float* o) {
    const float c0 = 0.28209479177387814f;
    const float c1 = 0.48860251190291992f;
    const float c2a = 1.09254843059207907f;   // sqrt(15/pi)/2
    const float c2b = 0.31539156525252001f;   // sqrt(5/pi)/4
    const float c2c = 0.54627421529603959f;   // sqrt(15/pi)/4
    const float c3a = 0.59004358992664352f;   // sqrt(35/(2pi))/4
    const float c3b = 2.89061144264055405f;   // sqrt(105/pi)/2
    const float c3c = 0.45704579946446573f;   // sqrt(21/(2pi))/4
    const float c3d = 0.37317633259011539f;   // sqrt(7/pi)/4
    const float c3e = 1.44530572132027702f;   // sqrt(105/pi)/4
    float xx = x * x, yy = y * y, zz = z * z;
    o[0] = c0;
    o[1] = c1 * y;
    o[2] = c1 * z;
    o[3] = c1 * x;
    o[4] = c2a * x * y;
    o[5] = c2a * y * z;
    o[6] = c2b * (3.0f * zz - 1.0f);
    o[7] = c2a * x * z;
    o[8] = c2c * (xx - yy);
    o[9] = c3a * y * (3.0f * xx - yy);
    o[10] = c3b * x * y * z;
    o[11] = c3c * y * (5.0f * zz - 1.0f);
    o[12] = c3d * z * (5.0f * zz - 3.0f);
    o[13] = c3c * x * (5.0f * zz - 1.0f);
    o[14] = c3e * z * (xx - yy);
    o[15] = c3a * x * (xx - 3.0f * yy);
}

__device__ __forceinline__ void sh_band2(float x, float y, float z, float* o) {
    o[0] = 0.28209479177387814f;
    o[1] = 0.48860251190291992f * y;
    o[2] = 0.48860251190291992f * z;
    o[3] = 0.48860251190291992f * x;
}

// ------------------------------------------------ Table 1 output mapping

__device__ __forceinline__ float logistic(float t) { return 1.0f / (1.0f + expf(-t)); }

__device__ __forceinline__ float softplus(float t) {
    return t > 0.0f ? t + log1pf(expf(-t)) : log1pf(expf(t));
}

struct Lobe {
    float lam, kap, mu[3];
};

// kappa and mean direction of one lobe from its raw outputs
// (kappa', theta', phi'); theta = pi s(theta'), phi = 2 pi s(phi').
__device__ __forceinline__ void decode_lobe(int kappa_act, float rk, float rt, float rp, Lobe& L,
                                            float* theta, float* phi) {
    L.kap = kappa_act == NPM_EXP ? expf(rk) : softplus(rk);
    float th = kPi * logistic(rt);
    float ph = 2.0f * kPi * logistic(rp);
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    L.mu[0] = st * cp;
    L.mu[1] = st * sp;
    L.mu[2] = ct;
    if (theta) *theta = th;
    if (phi) *phi = ph;
}

// Forward-path variant of decode_lobe on the hardware approximations
// (__expf, __logf, __sincosf, __fdividef). Arguments stay where those are
// accurate: sine/cosine arguments in [-pi, pi] (absolute error < 4e-7);
// exponentials of arguments |x| <~ 100 (relative error ~|x| 2^-24).
// phi = 2 pi s(phi') is evaluated as pi + pi (2 s - 1), so that
// (sin, cos)(phi) = -(sin, cos)(pi (2 s - 1)).
__device__ __forceinline__ float logistic_fast(float t) {
    return __fdividef(1.0f, 1.0f + __expf(-t));
}

__device__ __forceinline__ float softplus_fast(float t) {
    // max(t, 0) + log1p(e^{-|t|}); the log of 1 + e loses only absolute
    // accuracy (~6e-8), which kappa tolerates at every scale.
    return fmaxf(t, 0.0f) + __logf(1.0f + __expf(-fabsf(t)));
}

__device__ __forceinline__ void decode_lobe_fast(int kappa_act, float rk, float rt, float rp, Lobe& L,
                                                 float* theta, float* phi) {
    L.kap = kappa_act == NPM_EXP ? __expf(rk) : softplus_fast(rk);
    const float st = logistic_fast(rt), sp = logistic_fast(rp);
    const float th = kPi * st;
    const float ph_c = kPi * (2.0f * sp - 1.0f);  // phi - pi, in [-pi, pi]
    float sth, cth, sph, cph;
    __sincosf(th - 0.5f * kPi, &cth, &sth);       // sin(th) = cos(th - pi/2), cos(th) = -sin(th - pi/2)
    cth = -cth;
    __sincosf(ph_c, &sph, &cph);
    sph = -sph;
    cph = -cph;
    L.mu[0] = sth * cph;
    L.mu[1] = sth * sph;
    L.mu[2] = cth;
    if (theta) *theta = th;
    if (phi) *phi = ph_c + kPi;
}

// ------------------------------------------------------ vMF (Eq. 3-4)

// kappa / (4 pi sinh kappa) * e^kappa, written kappa / (2 pi (1 - e^{-2 kappa}))
// so that it pairs with exp(kappa (mu.w - 1)) without overflow.
__device__ __forceinline__ float vmf_scaled_norm(float k) {
    if (k < 1e-6f) return (1.0f + k) * kInv4Pi;
    return k / (2.0f * kPi * (-expm1f(-2.0f * k)));
}

__device__ __forceinline__ float vmf_eval(const Lobe& L, float cn, float wx, float wy, float wz) {
    float d = L.mu[0] * wx + L.mu[1] * wy + L.mu[2] * wz;
    return cn * expf(L.kap * (d - 1.0f));
}

// Forward-path variants: 1 - e^{-2k} by its series below k = 0.05 (truncation
// < 3e-8 relative), by the hardware exponential above; the lobe value by the
// hardware exponential of kappa (mu.w - 1) <= 0.
__device__ __forceinline__ float vmf_scaled_norm_fast(float k) {
    // Both forms are evaluated and selected (no divergent branch per lobe).
    const float series = k * (2.0f + k * (-2.0f + k * (4.0f / 3.0f + k * (-2.0f / 3.0f + k * (4.0f / 15.0f)))));
    const float em = k < 0.05f ? series : 1.0f - __expf(-2.0f * k);
    const float c = __fdividef(k, 2.0f * kPi * em);
    return k < 1e-6f ? (1.0f + k) * kInv4Pi : c;
}

__device__ __forceinline__ float vmf_eval_fast(const Lobe& L, float cn, float wx, float wy, float wz) {
    const float d = L.mu[0] * wx + L.mu[1] * wy + L.mu[2] * wz;
    return cn * __expf(L.kap * (d - 1.0f));
}

// One minus the cosine to the mean, t = 1 - W, by inversion of the vMF
// cosine CDF in the stable log1p / expm1 form (Jakob 2012). Returning t
// rather than W keeps sin(angle) = sqrt(t (2 - t)) accurate for samples very
// close to the mean.
__device__ __forceinline__ float vmf_sample_t(float k, float u1) {
    if (!(k > 1e-20f)) return 2.0f * u1;
    // the quotient is at most 2 and k far below 2^126: the fast divide is
    // within 2 ulp
    float t = __fdividef(-log1pf(u1 * expm1f(-2.0f * k)), k);
    return fminf(fmaxf(t, 0.0f), 2.0f);
}

// Orthonormal basis (t, b) completing unit vector n (Duff et al. 2017).
__device__ __forceinline__ void frame(const float n[3], float t[3], float b[3]) {
    float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
    float a = -__fdividef(1.0f, sg + n[2]);  // |sg + n_z| in [1, 2]
    float bb = n[0] * n[1] * a;
    t[0] = 1.0f + sg * n[0] * n[0] * a;
    t[1] = sg * bb;
    t[2] = -sg * n[0];
    b[0] = bb;
    b[1] = sg + n[1] * n[1] * a;
    b[2] = -n[1];
}

__device__ __forceinline__ void vmf_sample(const Lobe& L, float u1, float u2, float out[3]) {
    const float t1 = vmf_sample_t(L.kap, u1);
    const float W = 1.0f - t1;
    const float s = sqrtf(t1 * (2.0f - t1));
    // azimuth 2 pi u2 = pi + 2 pi (u2 - 1/2): hardware sine/cosine on [-pi, pi)
    float sp, cp;
    __sincosf(2.0f * kPi * (u2 - 0.5f), &sp, &cp);
    sp = -sp;
    cp = -cp;
    float lx = s * cp, ly = s * sp;
    float t[3], b[3];
    frame(L.mu, t, b);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = lx * t[a] + ly * b[a] + W * L.mu[a];
}

__device__ __forceinline__ void uniform_sphere(float u1, float u2, float out[3]) {
    float z = 1.0f - 2.0f * u1;
    float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    __sincosf(2.0f * kPi * (u2 - 0.5f), &sp, &cp);
    sp = -sp;
    cp = -cp;
    out[0] = r * cp;
    out[1] = r * sp;
    out[2] = z;
}

// 1/k - coth k (derivative of log(k / sinh k)). Below 0.25 its Laurent series
// -k/3 + k^3/45 - 2k^5/945 + k^7/4725 avoids the cancellation of the direct
// form (truncation < 1e-10 there).
__device__ __forceinline__ float inv_minus_coth(float k) {
    if (k < 0.25f) {
        float k2 = k * k;
        return k * (-1.0f / 3.0f + k2 * (1.0f / 45.0f + k2 * (-2.0f / 945.0f + k2 * (1.0f / 4725.0f))));
    }
    // coth k = 1 + 2 / (e^{2k} - 1)
    return 1.0f / k - 1.0f - 2.0f / expm1f(2.0f * k);
}

// A batch of query requests served by one launch of a forward kernel: the
// kernel's tiles are numbered across segments; segment s owns tiles
// [tile0, tile0 + ceil(n / tile size)). When n_dev is set (one segment),
// the query count is read from device memory at kernel start (graph replay
// with device-side batch sizes).
struct QuerySeg {
    int64_t n, ld, tile0;
    const float* pos;
    const float* aux;
    const float* uin;  // u [3 or 4][ld] when sampling, dir [3][ld] when evaluating
    float* dir;
    float* pdf;
    float* mix;
    float ufrac;
    int pad_;
};

constexpr int kMaxSegs = 16;

struct QueryBatch {
    int nseg;
    int sample;
    int log_pdf;  // evaluation only: pdf receives log V (log-sum-exp form)
    int64_t total_tiles;
    const int64_t* n_dev;
    QuerySeg seg[kMaxSegs];
};

// Device status word bits (read and cleared by npm_check_device_status).
enum : int { kStatusNumeric = 1, kStatusTimeout = 2 };

}  // namespace npm
