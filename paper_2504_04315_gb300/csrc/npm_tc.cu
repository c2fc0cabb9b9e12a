// npm_tc.cu -- tensor-core path of the NPM forward pass on sm_103a.
//
// One persistent CTA of 128 threads walks 128-query tiles; thread t owns query
// t of the tile, which is row t of every MMA and lane t of tensor memory.
// Per tile:
//   encode : thread t gathers the 8 corners of every level from the FP16
//            grid copy, blends in FP32 (Sec. 5.1, Eq. 11), appends the
//            product-mode SH encodings (Sec. 4.3), and writes its row of the
//            BF16 activation tile A (shared memory, UMMA K-major layout).
//   layers : one elected thread issues tcgen05.mma kind::f16 (BF16 x BF16 ->
//            FP32 in TMEM), M = 128, N = layer width, K in steps of 16, and
//            commits to an mbarrier; every thread then reads its accumulator
//            row with tcgen05.ld, applies ReLU and writes the next A row.
//   decode : the last accumulator row (4K FP32 raw outputs) stays in
//            registers; the thread maps it (Table 1), samples a lobe and a
//            direction (Sec. 5.3) and evaluates the mixture (Eq. 4) in FP32.
// Weights (BF16, pre-arranged in the UMMA layout) arrive once per CTA by a
// bulk asynchronous copy. Every wait on an mbarrier is bounded: on timeout
// the kernel records NPM_ERR_TIMEOUT in the status word, releases its tensor
// memory and returns.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "npm_handle.h"
#include "npm_kernels.h"
#include "npm_tc.cuh"

namespace npm {

using namespace tc;

namespace {

// --------------------------------------------------------------- encode

// Thread t writes row t of A (BF16, kp columns) for its query.
// Table entry loads: FP16 copy (inference) or FP32 master (training).
__device__ __forceinline__ float2 load_feat2(const __half* g, uint32_t idx) {
    const uint32_t raw = __ldg(reinterpret_cast<const unsigned int*>(g) + idx);
    return __half22float2(*reinterpret_cast<const __half2*>(&raw));
}
__device__ __forceinline__ float2 load_feat2(const float* g, uint32_t idx) {
    return __ldg(reinterpret_cast<const float2*>(g) + idx);
}
// Features 4h .. 4h+3 of entry idx of a table with F = 4 or 8 features: the
// raw 8-byte FP16 or 16-byte FP32 vector, widened to float4 at use.
__device__ __forceinline__ uint2 load_raw4(const __half* g, uint32_t idx, int F, int h) {
    return __ldg(reinterpret_cast<const uint2*>(g) + (size_t)idx * (F >> 2) + h);
}
__device__ __forceinline__ float4 load_raw4(const float* g, uint32_t idx, int F, int h) {
    return __ldg(reinterpret_cast<const float4*>(g) + (size_t)idx * (F >> 2) + h);
}
__device__ __forceinline__ float4 widen4(uint2 raw) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 widen4(float4 v) { return v; }
__device__ __forceinline__ float load_feat(const __half* e, int f) { return __half2float(e[f]); }
__device__ __forceinline__ float load_feat(const float* e, int f) { return __ldg(e + f); }

// Entry index of corner c of a cell (the corner_idx8 formula for one
// corner). The two-level gather below issues each corner's load as soon as
// its index is formed, which schedules better there than forming all 16
// indices first.
__device__ __forceinline__ uint32_t corner_idx1(const DevCfg& cfg, int l, const Cell& cl, int c) {
    const uint32_t i = cl.c[0] + (c & 1), j = cl.c[1] + ((c >> 1) & 1), k = cl.c[2] + ((c >> 2) & 1);
    if ((cfg.dense_mask >> l) & 1u) {
        const uint32_t D = (uint32_t)cfg.level_res[l];
        return bounded_index(i + D * (j + D * k), D * D * D);
    }
    return (i ^ (j * 2654435761u) ^ (k * 805459861u)) & cfg.table_mask;
}

// F2: the grid has 2 features per level (compile-time), so two levels' 16
// corner loads can be in flight before blending; other grids take the
// generic per-level path (fewer registers).
// Levels [lbeg, lend) are encoded; tail: also the product-mode inputs and
// the zero padding. lo: byte offset of the residual tile (0 without split).
// pad_all: write zeros up to kp; otherwise only up to the next 8-column
// chunk (the caller keeps the all-zero chunks beyond it written).
template <bool F2, typename GT>
__device__ __forceinline__ void tc_encode(const TcCfg& tc, const GT* __restrict__ grid_h,
                                          int64_t j, bool valid, int64_t ld,
                                          const float* __restrict__ pos,
                                          const float* __restrict__ aux, uint8_t* sA, int row,
                                          uint32_t lo, bool pad_all, int lbeg, int lend, bool tail) {
    const DevCfg& cfg = tc.base;
    const int kp = tc.layer[0].Kp;
    const bool f16 = tc.f16 != 0;
    float x = 0.0f, y = 0.0f, z = 0.0f;
    if (valid) {
        x = pos[j];
        y = pos[ld + j];
        z = pos[2 * ld + j];
    }
    const int F = F2 ? 2 : cfg.feat;
    int l = lbeg;
    if (!F2 && (F == 4 || F == 8) && lbeg == 0 && lend == 1 && tail && cfg.mode != NPM_PRODUCT) {
        // A single level of 4 or 8 features fills the first 8-column chunk
        // (features, then zeros): one 16-byte store (and one for residuals);
        // with pad_all, zero chunks follow up to kp.
        const Cell cl = make_cell(x, y, z, cfg.level_res[0]);
        uint32_t idx[8];
        corner_idx8(cfg, 0, cl, idx);
        float ws[8];
        corner_w8(cl, ws);
        float e[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (h == 0 || F == 8) {
                decltype(load_raw4(grid_h, 0u, F, 0)) raw[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) raw[c] = load_raw4(grid_h, idx[c], F, h);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 v = widen4(raw[c]);
                    acc.x = fmaf(ws[c], v.x, acc.x);
                    acc.y = fmaf(ws[c], v.y, acc.y);
                    acc.z = fmaf(ws[c], v.z, acc.z);
                    acc.w = fmaf(ws[c], v.w, acc.w);
                }
            }
            e[4 * h] = acc.x;
            e[4 * h + 1] = acc.y;
            e[4 * h + 2] = acc.z;
            e[4 * h + 3] = acc.w;
        }
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (f16) {
                hw[i] = pack_f16_sat(e[2 * i], e[2 * i + 1]);
                lw[i] = lo ? f16_residual(hw[i], e[2 * i], e[2 * i + 1]) : 0u;
            } else {
                __nv_bfloat162 hb = __floats2bfloat162_rn(e[2 * i], e[2 * i + 1]);
                hw[i] = *reinterpret_cast<uint32_t*>(&hb);
                const float2 hf = __bfloat1622float2(hb);
                lw[i] = pack_bf16(e[2 * i] - hf.x, e[2 * i + 1] - hf.y);
            }
        }
        const uint32_t off = tile_off(row, 0, kp);
        *reinterpret_cast<uint4*>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if (lo) *reinterpret_cast<uint4*>(sA + lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        if (pad_all)
            for (int c = 8; c < kp; c += 8) {
                const uint32_t oz = tile_off(row, c, kp);
                *reinterpret_cast<uint4*>(sA + oz) = make_uint4(0u, 0u, 0u, 0u);
                if (lo) *reinterpret_cast<uint4*>(sA + lo + oz) = make_uint4(0u, 0u, 0u, 0u);
            }
        return;
    }
    if constexpr (F2) {
        for (; l + 1 < lend; l += 2) {
            const Cell c0 = make_cell(x, y, z, cfg.level_res[l]);
            const Cell c1 = make_cell(x, y, z, cfg.level_res[l + 1]);
            const GT* g0 = grid_h + (size_t)cfg.level_off[l] * 2;
            const GT* g1 = grid_h + (size_t)cfg.level_off[l + 1] * 2;
            float2 v0[8], v1[8];
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                gather_pair2(g0, cfg.level_off[l], corner_idx1(cfg, l, c0, c), corner_idx1(cfg, l, c0, c + 1),
                             v0[c], v0[c + 1]);
                gather_pair2(g1, cfg.level_off[l + 1], corner_idx1(cfg, l + 1, c1, c),
                             corner_idx1(cfg, l + 1, c1, c + 1), v1[c], v1[c + 1]);
            }
            float w0s[8], w1s[8];
            corner_w8(c0, w0s);
            corner_w8(c1, w1s);
            float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float w0 = w0s[c], w1 = w1s[c];
                a0 = fmaf(w0, v0[c].x, a0);
                a1 = fmaf(w0, v0[c].y, a1);
                b0 = fmaf(w1, v1[c].x, b0);
                b1 = fmaf(w1, v1[c].y, b1);
            }
            store_pair(sA, tile_off(row, 2 * l, kp), a0, a1, lo, f16);
            store_pair(sA, tile_off(row, 2 * l + 2, kp), b0, b1, lo, f16);
        }
    }
    for (; l < lend; ++l) {
        const Cell cl = make_cell(x, y, z, cfg.level_res[l]);
        const GT* gl = grid_h + (size_t)cfg.level_off[l] * F;
        if (F2) {  // F = 2 (F2 kernels serve exactly the 2-feature grids)
            float s0 = 0.0f, s1 = 0.0f;
            uint32_t idx[8];
            corner_idx8(cfg, l, cl, idx);
            float2 v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = load_feat2(gl, idx[c]);
            float ws[8];
            corner_w8(cl, ws);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float w = ws[c];
                s0 = fmaf(w, v[c].x, s0);
                s1 = fmaf(w, v[c].y, s1);
            }
            store_pair(sA, tile_off(row, 2 * l, kp), s0, s1, lo, f16);
        } else if (F == 4 || F == 8) {
            // One vector load per corner and group of 4 features.
            uint32_t idx[8];
            corner_idx8(cfg, l, cl, idx);
            float ws[8];
            corner_w8(cl, ws);
            for (int h = 0; h < (F >> 2); ++h) {
                decltype(load_raw4(gl, 0u, F, 0)) raw[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) raw[c] = load_raw4(gl, idx[c], F, h);
                float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float w = ws[c];
                    const float4 v = widen4(raw[c]);
                    acc.x = fmaf(w, v.x, acc.x);
                    acc.y = fmaf(w, v.y, acc.y);
                    acc.z = fmaf(w, v.z, acc.z);
                    acc.w = fmaf(w, v.w, acc.w);
                }
                const int k = l * F + 4 * h;
                store_pair(sA, tile_off(row, k, kp), acc.x, acc.y, lo, f16);
                store_pair(sA, tile_off(row, k + 2, kp), acc.z, acc.w, lo, f16);
            }
        } else {
            // F = 1
            float s = 0.0f;
            uint32_t idx[8];
            float ws[8];
            corners8(cfg, l, cl, idx, ws);
#pragma unroll
            for (int c = 0; c < 8; ++c) s = fmaf(ws[c], load_feat(gl + idx[c], 0), s);
            store_one(sA, tile_off(row, l, kp), s, lo, f16);
        }
    }
    if (!tail) return;
    int k = cfg.grid_feats;
    if (cfg.mode == NPM_PRODUCT) {
        float e[21];
        float wo[3] = {0.0f, 0.0f, 1.0f}, nn[3] = {0.0f, 0.0f, 1.0f}, r = 0.0f;
        if (valid) {
            wo[0] = aux[j];
            wo[1] = aux[ld + j];
            wo[2] = aux[2 * ld + j];
            nn[0] = aux[3 * ld + j];
            nn[1] = aux[4 * ld + j];
            nn[2] = aux[5 * ld + j];
            r = aux[6 * ld + j];
        }
        sh_band4(wo[0], wo[1], wo[2], e);
        sh_band2(nn[0], nn[1], nn[2], e + 16);
        e[20] = r;
#pragma unroll
        for (int i = 0; i < 21; ++i) store_one(sA, tile_off(row, k + i, kp), e[i], lo, f16);
        k += 21;
    }
    const int kend = pad_all ? kp : min(kp, (k + 7) & ~7);
    for (; k < kend; ++k) store_one(sA, tile_off(row, k, kp), 0.0f, lo);
}

// --------------------------------------------------------------- decode

// KEXACT: the model has exactly KMAX lobes (no per-lobe bound checks).
template <int KMAX, bool KEXACT>
__device__ __forceinline__ void tc_decode(const TcCfg& tc, const float (&raw)[4 * KMAX], int64_t j,
                                          bool valid, int64_t ld, const float* __restrict__ uin,
                                          float ufrac, bool sample, float* __restrict__ dir_out,
                                          float* __restrict__ pdf_out,
                                          float* __restrict__ mix_out, bool log_pdf) {
    const DevCfg& cfg = tc.base;
    const int K = KEXACT ? KMAX : cfg.K;
    Lobe lob[KMAX];
    float cn[KMAX];
    float mx = -INFINITY;
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
        if (i < K) mx = fmaxf(mx, raw[4 * i]);
    float ssum = 0.0f;
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
        if (i < K) {
            lob[i].lam = __expf(raw[4 * i] - mx);
            ssum += lob[i].lam;
        }
    const float inv = __fdividef(1.0f, ssum);  // ssum in [1, K]
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
        if (i < K) {
            lob[i].lam *= inv;
            float th, ph;
            decode_lobe_fast(cfg.kappa_act, raw[4 * i + 1], raw[4 * i + 2], raw[4 * i + 3], lob[i], &th, &ph);
            cn[i] = vmf_scaled_norm_fast(lob[i].kap);
            if (mix_out && valid) {
                mix_out[(4 * i + 0) * ld + j] = lob[i].lam;
                mix_out[(4 * i + 1) * ld + j] = lob[i].kap;
                mix_out[(4 * i + 2) * ld + j] = th;
                mix_out[(4 * i + 3) * ld + j] = ph;
            }
        }
    float w[3] = {0.0f, 0.0f, 1.0f};
    bool uni = false;
    if (sample) {
        float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
        if (valid) {
            u0 = uin[j];
            u1 = uin[ld + j];
            u2 = uin[2 * ld + j];
            uni = ufrac > 0.0f && uin[3 * ld + j] < ufrac;
        }
        if (uni) {
            uniform_sphere(u1, u2, w);
        } else {
            // Smallest lobe i with u0 < lambda_0 + ... + lambda_i (last if none).
            int sel = K - 1;
            float cum = 0.0f;
            bool found = false;
#pragma unroll
            for (int i = 0; i < KMAX; ++i)
                if (i < K) {
                    cum += lob[i].lam;
                    if (!found && u0 < cum) {
                        sel = i;
                        found = true;
                    }
                }
            Lobe sl = lob[0];
#pragma unroll
            for (int i = 1; i < KMAX; ++i)
                if (i == sel) sl = lob[i];
            if (tc.fp32) vmf_sample(sl, u1, u2, w);  // the FP32 path's sampler
            else vmf_sample_rp(sl, u1, u2, w);
        }
    } else if (valid) {
        w[0] = uin[j];
        w[1] = uin[ld + j];
        w[2] = uin[2 * ld + j];
    }
    float pv = 0.0f;
    if (!sample && log_pdf) {
        // log V (Eq. 4 in log-sum-exp form), the weights' logs taken from
        // the logits so that they stay finite where lambda_i underflows.
        const float lnorm = mx + __logf(ssum);
        float a[KMAX];
        float m = -INFINITY;
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < K) {
                const float d = lob[i].mu[0] * w[0] + lob[i].mu[1] * w[1] + lob[i].mu[2] * w[2];
                a[i] = (raw[4 * i] - lnorm) + __logf(cn[i]) + lob[i].kap * (d - 1.0f);
                m = fmaxf(m, a[i]);
            }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < K) s += __expf(a[i] - m);
        pv = m + __logf(s);
    } else {
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < K) pv += lob[i].lam * vmf_eval_fast(lob[i], cn[i], w[0], w[1], w[2]);
        if (sample && ufrac > 0.0f) pv = ufrac * kInv4Pi + (1.0f - ufrac) * pv;
    }
    if (valid) {
        if (sample) {
            dir_out[j] = w[0];
            dir_out[ld + j] = w[1];
            dir_out[2 * ld + j] = w[2];
        }
        pdf_out[j] = pv;
    }
}

// Warp-per-query form of the decode, sample and density (Table 1, Sec. 5.3,
// Eq. 4): lane l of a warp owns lobe l mod KMAX of one query, so a warp
// serves 32 / KMAX queries per pass and KMAX passes cover its 32 rows. The
// raw outputs of the tile are staged in shared memory (row stride 4 KMAX + 4
// floats keeps both the row writes and the lobe reads free of bank
// conflicts). Softmax and density are reductions over the query's lanes;
// the lobe choice takes the running sum of the weights in lobe order (a
// serial scan, the same rounding as the thread-per-row form) and a ballot;
// every lane samples its own lobe and the chosen lane's direction is
// broadcast. Measured against tc_decode (one thread per query).
template <int KMAX>
__device__ __forceinline__ void tc_decode_warp(const TcCfg& tc, const float* __restrict__ sRaw, int warp, int lane,
                                               int64_t j0, int64_t n, int64_t ld, const float* __restrict__ uin,
                                               float ufrac, bool sample, float* __restrict__ dir_out,
                                               float* __restrict__ pdf_out, float* __restrict__ mix_out,
                                               bool log_pdf) {
    constexpr int RS = 4 * KMAX + 4;
    constexpr int QP = 32 / KMAX;  // queries per pass
    constexpr unsigned kAll = 0xffffffffu;
    const DevCfg& cfg = tc.base;
    const int K = cfg.K;
    const int i = lane & (KMAX - 1);
    const int qsub = lane / KMAX;
    const unsigned seg = KMAX == 32 ? kAll : (((1u << KMAX) - 1u) << (qsub * KMAX));
    const bool act = i < K;
#pragma unroll 1
    for (int p = 0; p < KMAX; ++p) {
        const int r = warp * 32 + p * QP + qsub;
        const int64_t j = j0 + r;
        const bool valid = j < n;
        const float4 rv = *reinterpret_cast<const float4*>(sRaw + r * RS + 4 * i);
        float mx = act ? rv.x : -INFINITY;
#pragma unroll
        for (int o = 1; o < KMAX; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kAll, mx, o));
        const float e = act ? __expf(rv.x - mx) : 0.0f;
        float ssum = e;
#pragma unroll
        for (int o = 1; o < KMAX; o <<= 1) ssum += __shfl_xor_sync(kAll, ssum, o);
        Lobe L;
        L.lam = e * __fdividef(1.0f, ssum);
        float th, ph;
        decode_lobe_fast(cfg.kappa_act, rv.y, rv.z, rv.w, L, &th, &ph);
        const float cn = vmf_scaled_norm_fast(L.kap);
        if (mix_out && valid && act) {
            mix_out[(4 * i + 0) * ld + j] = L.lam;
            mix_out[(4 * i + 1) * ld + j] = L.kap;
            mix_out[(4 * i + 2) * ld + j] = th;
            mix_out[(4 * i + 3) * ld + j] = ph;
        }
        float w[3] = {0.0f, 0.0f, 1.0f};
        bool uni = false;
        if (sample) {
            float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
            if (valid) {
                u0 = uin[j];
                u1 = uin[ld + j];
                u2 = uin[2 * ld + j];
                uni = ufrac > 0.0f && uin[3 * ld + j] < ufrac;
            }
            // Running sum of the weights in lobe order.
            float cum = i == 0 ? L.lam : 0.0f;
#pragma unroll
            for (int k = 1; k < KMAX; ++k) {
                const float prev = __shfl_up_sync(kAll, cum, 1);
                if (i == k) cum = prev + L.lam;
            }
            const unsigned hit = __ballot_sync(kAll, act && u0 < cum) & seg;
            const int sel = hit ? __ffs(hit) - 1 - qsub * KMAX : K - 1;
            float d[3];
            if (uni) uniform_sphere(u1, u2, d);
            else vmf_sample_rp(L, u1, u2, d);
#pragma unroll
            for (int a = 0; a < 3; ++a) w[a] = __shfl_sync(kAll, d[a], qsub * KMAX + sel);
        } else if (valid) {
            w[0] = uin[j];
            w[1] = uin[ld + j];
            w[2] = uin[2 * ld + j];
        }
        float pv;
        if (!sample && log_pdf) {
            const float dd = L.mu[0] * w[0] + L.mu[1] * w[1] + L.mu[2] * w[2];
            const float a = act ? (rv.x - mx) - __logf(ssum) + __logf(cn) + L.kap * (dd - 1.0f) : -INFINITY;
            float m = a;
#pragma unroll
            for (int o = 1; o < KMAX; o <<= 1) m = fmaxf(m, __shfl_xor_sync(kAll, m, o));
            float sx = act ? __expf(a - m) : 0.0f;
#pragma unroll
            for (int o = 1; o < KMAX; o <<= 1) sx += __shfl_xor_sync(kAll, sx, o);
            pv = m + __logf(sx);
        } else {
            pv = act ? L.lam * vmf_eval_fast(L, cn, w[0], w[1], w[2]) : 0.0f;
#pragma unroll
            for (int o = 1; o < KMAX; o <<= 1) pv += __shfl_xor_sync(kAll, pv, o);
            if (sample && ufrac > 0.0f) pv = ufrac * kInv4Pi + (1.0f - ufrac) * pv;
        }
        if (valid && i == 0) {
            if (sample) {
                dir_out[j] = w[0];
                dir_out[ld + j] = w[1];
                dir_out[2 * ld + j] = w[2];
            }
            pdf_out[j] = pv;
        }
    }
}

// --------------------------------------------------------------- kernel

// NL > 0: the network has exactly NL layers and KMAX lobes (loops over
// layers, output chunks and lobes unrolled at compile time); NL = 0: any
// layer count and K <= KMAX. WARPDEC: the warp-per-query decode
// (tc_decode_warp) instead of one thread per query. G32: the grid table is
// the FP32 master table (the FP32-accuracy mode). G: tile groups per CTA.
// Grid table type of the forward kernel: the FP16 copy, or the FP32 master
// table (inference weights) in the FP32-accuracy mode.
template <bool G32>
using GridT = typename std::conditional<G32, float, __half>::type;

// A CTA of G tile groups (128 threads each) holds one copy of the weights;
// each group has its own activation tiles, tensor-memory columns, MMA
// barrier and named barrier, and walks its own tiles. Such a CTA runs alone
// on its SM; single-group CTAs are compiled for as many per SM as the
// shapes that use them fit.
__host__ __device__ constexpr int tc_min_blocks(int kmax, bool f2, int nl, int g) {
    return g > 1 ? 1 : (kmax == 4 && !f2) ? (nl == 3 ? 8 : 6) : (kmax == 8 ? 3 : 1);
}

template <int KMAX, bool F2, int NL, bool WARPDEC = false, bool G32 = false, int G = 1>
__global__ void __launch_bounds__(kThreads * G, tc_min_blocks(KMAX, F2, NL, G)) k_forward_tc(const __grid_constant__ TcCfg tc,
                                                         const GridT<G32>* __restrict__ grid_h,
                                                         const uint8_t* __restrict__ wblob,
                                                         const __grid_constant__ QueryBatch qb,
                                                         int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int nsplit = tc.split ? 2 : 1;               // activation tiles (hi, residual)
    const int nw = (tc.split || tc.f16) ? 2 : 1;       // weight blobs (hi, residual)
    const int g = G > 1 ? (int)(threadIdx.x >> 7) : 0;  // tile group
    const int t = G > 1 ? (int)(threadIdx.x & 127) : (int)threadIdx.x;  // row of the group's tile
    const int warp = t >> 5;                            // warp of the group (its TMEM lane quarter)
    const uint32_t gbytes = nsplit * (tc.a0_bytes + tc.a_bytes);  // activation tiles of a group
    uint8_t* sW = smem;
    uint8_t* sG0 = smem + nw * tc.w_bytes;
    uint8_t* sA = sG0 + g * gbytes + nsplit * tc.a0_bytes;  // inputs of layers >= 1
    uint8_t* sA0 = tc.a0_bytes ? sG0 + g * gbytes : sA;    // layer-0 input (encoding)
    const uint32_t a0_lo = tc.a0_bytes ? tc.a0_bytes : tc.a_bytes;  // its residual tile
    uint64_t* bars = reinterpret_cast<uint64_t*>(sG0 + G * gbytes);  // [0] weights, [1 + g] mma
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 1 + G);
    const uint32_t bar_mma = smem_u32(&bars[1 + g]);
    const uint32_t bar_w = smem_u32(&bars[0]);
    // Tensor-memory columns of the CTA (a power of two: the groups' columns
    // rounded up).
    uint32_t cta_cols = 32;
    while (cta_cols < (uint32_t)G * tc.tmem_cols) cta_cols <<= 1;

    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(cta_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i <= G; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot + (uint32_t)g * tc.tmem_cols;

    // Weights: one bulk asynchronous copy global -> shared.
    if (threadIdx.x == 0) {
        const uint32_t wb = (uint32_t)nw * tc.w_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w), "r"(wb)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sW)),
            "l"(wblob), "r"(wb), "r"(bar_w)
            : "memory");
    }
    // The all-zero 8-column chunks of the encoding are written once: the
    // layer-0 buffer holds nothing else.
    if (tc.a0_bytes) {
        const int kp0 = tc.layer[0].Kp;
        for (int c = (tc.enc_width + 7) >> 3; c < (kp0 >> 3); ++c) {
            *reinterpret_cast<uint4*>(sA0 + tile_off(t, 8 * c, kp0)) = make_uint4(0u, 0u, 0u, 0u);
            if (tc.split)
                *reinterpret_cast<uint4*>(sA0 + a0_lo + tile_off(t, 8 * c, kp0)) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    bool ok = !__syncthreads_or(threadIdx.x < 32 && !mbar_wait_bounded(bar_w, 0));
    uint32_t phase = 0;
    const uint32_t sA_addr = smem_u32(sA), sA0_addr = smem_u32(sA0);
    const uint32_t sW_addr = smem_u32(sW);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int L = NL > 0 ? NL : tc.base.n_layers;
    constexpr int kUnrollL = NL > 0 ? NL : 1;
    constexpr int kUnrollC = NL > 0 ? NPM_MAX_WIDTH / 16 : 1;

    int64_t ntiles = qb.total_tiles, n0 = qb.seg[0].n;
    if (qb.n_dev) {
        n0 = *qb.n_dev;
        ntiles = (n0 + kTile - 1) / kTile;
    }
    const int64_t stride = (int64_t)gridDim.x * G;
    for (int64_t tile = (int64_t)blockIdx.x * G + g; ok && tile < ntiles; tile += stride) {
        int sg = 0;
        while (sg + 1 < qb.nseg && tile >= qb.seg[sg + 1].tile0) ++sg;
        const QuerySeg& S = qb.seg[sg];
        const int64_t n = (sg == 0 && qb.n_dev) ? n0 : S.n;
        const int64_t ld = S.ld;
        const int64_t j = (tile - S.tile0) * kTile + t;
        const bool valid = j < n;
        // Into L2 while this tile is encoded and run through the MLP: its
        // uniforms (or directions), which the decode reads last, and the
        // next tile's positions. Lane l of warp 3 takes row l >> 2 (0-3:
        // uniforms, 4-6: next positions), quarter l & 3 (128 bytes) of the
        // 512-byte rows.
        if (warp == 3) {
            const int lane = t & 31, r = lane >> 2;
            const int64_t b0 = (tile - S.tile0) * kTile + 32 * (lane & 3);
            if (r < 4) {
                if ((r < 3 || S.ufrac > 0.0f) && b0 < n)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(S.uin + r * ld + b0));
            } else if (r < 7) {
                const int64_t nt = tile + stride;
                if (nt < ntiles) {
                    int s2 = sg;
                    while (s2 + 1 < qb.nseg && nt >= qb.seg[s2 + 1].tile0) ++s2;
                    const QuerySeg& S2 = qb.seg[s2];
                    const int64_t b2 = (nt - S2.tile0) * kTile + 32 * (lane & 3);
                    const int64_t n2 = (s2 == 0 && qb.n_dev) ? n0 : S2.n;
                    if (b2 < n2) asm volatile("prefetch.global.L2 [%0];" ::"l"(S2.pos + (r - 4) * S2.ld + b2));
                }
            }
        }
        // Without a layer-0 buffer of its own the encoding also rewrites
        // the zero chunks (the hidden layers reuse the buffer).
        tc_encode<F2>(tc, grid_h, j, valid, ld, S.pos, S.aux, sA0, t, tc.split ? a0_lo : 0u, tc.a0_bytes == 0, 0,
                      tc.base.n_levels, true);
        fence_async_smem();
        tc_fence_before();
        tc_group_sync(g);
        uint32_t raw[4 * KMAX / 16][16];
#pragma unroll kUnrollL
        for (int l = 0; l < L; ++l) {
            const TcLayer& ly = tc.layer[l];
            if (t == 0) {
                tc_fence_after();
                const uint32_t sbo = (uint32_t)(ly.Kp >> 3) * 128u;
                const uint32_t a_addr = l == 0 ? sA0_addr : sA_addr;
                const uint32_t a_lo = l == 0 ? a0_lo : tc.a_bytes;
                for (int s = 0; s < (ly.Kp >> 4); ++s) {
                    const uint64_t ad = umma_desc(a_addr + s * 256u, 128u, sbo);
                    const uint64_t bd = umma_desc(sW_addr + ly.w_off + s * 256u, 128u, sbo);
                    mma_bf16(tmem, ad, bd, ly.idesc, s > 0 ? 1u : 0u);
                    if (tc.split || tc.f16) {
                        // hi*lo (the weights' residual) and, when split,
                        // lo*hi (the activations' residual)
                        const uint64_t bdl = umma_desc(sW_addr + tc.w_bytes + ly.w_off + s * 256u, 128u, sbo);
                        mma_bf16(tmem, ad, bdl, ly.idesc, 1u);
                        if (tc.split) {
                            const uint64_t adl = umma_desc(a_addr + a_lo + s * 256u, 128u, sbo);
                            mma_bf16(tmem, adl, bd, ly.idesc, 1u);
                        }
                    }
                }
                mma_commit(bar_mma);
            }
            // Warp 0 (which holds the issuing thread) waits on the MMA's
            // barrier; the other warps wait in the group barrier, issuing
            // nothing, and see the accumulators after its fence.
            const bool done = warp != 0 || mbar_wait_bounded(bar_mma, phase);
            phase ^= 1u;
            ok = !tc_group_sync_or(g, !done);
            if (!ok) break;
            tc_fence_after();
            if (l < L - 1) {
                const int kp_next = tc.layer[l + 1].Kp;
#pragma unroll kUnrollC
                for (int c0 = 0; c0 < ly.Np; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
                    tmem_wait16(r);
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(__uint_as_float(r[i]), 0.0f);
                    store16_fwd(sA, tile_off(t, c0, kp_next), tile_off(t, c0 + 8, kp_next), v,
                                tc.split ? tc.a_bytes : 0u, tc.f16 != 0);
                }
                fence_async_smem();
                tc_fence_before();
                tc_group_sync(g);
            } else {
#pragma unroll
                for (int c = 0; c < 4 * KMAX / 16; ++c)
                    if (c * 16 < ly.Np) tmem_ld16(tmem + lane_base + (uint32_t)(c * 16), raw[c]);
#pragma unroll
                for (int c = 0; c < 4 * KMAX / 16; ++c)
                    if (c * 16 < ly.Np) tmem_wait16(raw[c]);
                tc_fence_before();
            }
        }
        if (!ok) break;
        if constexpr (WARPDEC) {
            // Stage the raw outputs in the activation buffer (free until the
            // next tile's encode), then decode a query per 32 / KMAX lanes.
            constexpr int RS = 4 * KMAX + 4;
            float* sRaw = reinterpret_cast<float*>(sA);
#pragma unroll
            for (int c = 0; c < 4 * KMAX / 16; ++c)
                if (c * 16 < tc.layer[L - 1].Np)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4*>(sRaw + t * RS + 16 * c + 4 * q) =
                            make_uint4(raw[c][4 * q], raw[c][4 * q + 1], raw[c][4 * q + 2], raw[c][4 * q + 3]);
            tc_group_sync(g);
            tc_decode_warp<KMAX>(tc, sRaw, warp, t & 31, (tile - S.tile0) * kTile, n, ld, S.uin, S.ufrac,
                                 qb.sample != 0, S.dir, S.pdf, S.mix, qb.log_pdf != 0);
            tc_group_sync(g);
        } else {
            float rawf[4 * KMAX];
#pragma unroll
            for (int c = 0; c < 4 * KMAX / 16; ++c)
#pragma unroll
                for (int i = 0; i < 16; ++i) rawf[c * 16 + i] = __uint_as_float(raw[c][i]);
            tc_decode<KMAX, (NL > 0)>(tc, rawf, j, valid, ld, S.uin, S.ufrac, qb.sample != 0, S.dir, S.pdf, S.mix,
                                      qb.log_pdf != 0);
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(status, kStatusTimeout);
        // Before the tensor memory is released: wait again, bounded, for this
        // group's own asynchronous work that may still be in flight (the
        // weights' bulk copy; the MMA batch whose wait gave up, the phase
        // before `phase`).
        if (warp == 0) {
            (void)mbar_wait_bounded(bar_w, 0);
            (void)mbar_wait_bounded(bar_mma, phase ^ 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(cta_cols)
                     : "memory");
    }
}

// Master FP32 weights (packed [out][in] per layer) -> BF16 blob in the UMMA
// K-major layout, zero padded to Np x Kp per layer.
__global__ void k_tc_weights(TcCfg tc, const float* __restrict__ mlp, uint8_t* __restrict__ blob) {
    int64_t woff = 0;
    for (int l = 0; l < tc.base.n_layers; ++l) {
        const TcLayer& ly = tc.layer[l];
        const int total = ly.Np * ly.Kp;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
            const int nn = i / ly.Kp, k = i % ly.Kp;
            const float v = (nn < ly.N && k < ly.K) ? mlp[woff + (int64_t)nn * ly.K + k] : 0.0f;
            if (tc.f16) {
                // FP16 high part and FP16 residual (the weights to ~22 bits)
                const __half hh = __float2half_rn(v);
                *reinterpret_cast<__half*>(blob + ly.w_off + tile_off(nn, k, ly.Kp)) = hh;
                *reinterpret_cast<__half*>(blob + tc.w_bytes + ly.w_off + tile_off(nn, k, ly.Kp)) =
                    __float2half_rn(v - __half2float(hh));
                continue;
            }
            const __nv_bfloat16 hb = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(blob + ly.w_off + tile_off(nn, k, ly.Kp)) = hb;
            if (tc.split)
                *reinterpret_cast<__nv_bfloat16*>(blob + tc.w_bytes + ly.w_off + tile_off(nn, k, ly.Kp)) =
                    __float2bfloat16_rn(v - __bfloat162float(hb));
        }
        woff += (int64_t)ly.K * ly.N;
    }
}

// ----------------------------------------------------------- training

// Training layout: per layer the input activation tile H_l (BF16, K-major,
// 128 x Kp_l) at h_off, the delta tile D (BF16, K-major, 128 samples x
// d_cols, the widest layer) at d_off; TMEM columns [0, c0) hold the forward / input-gradient
// accumulator and [dw_col_l, dw_col_l + Kp_l) the weight gradient of
// layer l, accumulated over all tiles of the CTA.
struct TcTrain {
    uint32_t h_off[NPM_MAX_LAYERS];
    uint32_t dw_col[NPM_MAX_LAYERS];
    uint32_t idesc_dw[NPM_MAX_LAYERS];  // A MN-major, B MN-major, N = Kp_l
    uint32_t idesc_dx[NPM_MAX_LAYERS];  // A K-major,  B MN-major, N = Kp_l
    uint32_t d_off, x_off, bar_off, smem, tmem_cols;
    uint32_t d_cols;                    // columns of the delta tile
    int64_t woff[NPM_MAX_LAYERS];       // packed offset of W_l in the MLP region
    int split;                          // BF16 residual operands (three MMAs per K step)
    uint32_t hlo_off;                   // residual of the current layer's input tile
    uint32_t dlo_off;                   // residual of the delta tile
};

// Training runs two threads per sample row: thread t serves row t & 127 and
// half t >> 7 of the row's work (grid levels, epilogue column chunks,
// lobes). Warps w and w + 4 read the same TMEM lane quarter.
constexpr int kTrainThreads = 2 * kTile;

// Half h of the lobes of one sample, lobes i = h KMAX/2 + q. Pass 1 forms
// each lobe's terms and the half's partial log-sum-exps of the softmax
// logits (m1, s1) and of the unnormalised log lobe values
// a'_i = raw_i + log c(kappa_i) + kappa_i (mu_i.w - 1) (m2, s2); the caller
// combines both halves' partials (log V = LSE(a') - LSE(raw)).
template <int KMAX>
struct GradHalf {
    static constexpr int KH = KMAX / 2;
    float r0[KH], ap[KH], kap[KH], md[KH], wdt[KH], wdp[KH], sk[KH], st[KH], sp[KH];
    bool act[KH];

    __device__ __forceinline__ float4 pass1(const DevCfg& cfg, int h, const float (&raw)[4 * KH], const float w[3]) {
        float m1 = -INFINITY, m2 = -INFINITY;
#pragma unroll
        for (int q = 0; q < KH; ++q) {
            act[q] = h * KH + q < cfg.K;
            r0[q] = raw[4 * q];
            const float rk = raw[4 * q + 1];
            if (cfg.kappa_act == NPM_EXP) {
                kap[q] = __expf(rk);
                sk[q] = kap[q];
            } else {
                // softplus and its derivative, the logistic, from one e^{-|rk|}
                const float e = __expf(-fabsf(rk));
                const float r1 = __fdividef(1.0f, 1.0f + e);
                kap[q] = fmaxf(rk, 0.0f) + __logf(1.0f + e);
                sk[q] = rk >= 0.0f ? r1 : e * r1;
            }
            st[q] = logistic_fast(raw[4 * q + 2]);
            sp[q] = logistic_fast(raw[4 * q + 3]);
            // theta = pi st, phi = pi + pi (2 sp - 1): sine/cosine on [-pi, pi]
            float sth, cth, sph, cph;
            __sincosf(kPi * st[q] - 0.5f * kPi, &cth, &sth);
            cth = -cth;
            __sincosf(kPi * (2.0f * sp[q] - 1.0f), &sph, &cph);
            sph = -sph;
            cph = -cph;
            md[q] = sth * cph * w[0] + sth * sph * w[1] + cth * w[2];
            wdt[q] = cth * cph * w[0] + cth * sph * w[1] - sth * w[2];
            wdp[q] = -sth * sph * w[0] + sth * cph * w[1];
            ap[q] = r0[q] + __logf(vmf_scaled_norm_fast(kap[q])) + kap[q] * (md[q] - 1.0f);
            if (act[q]) {
                m1 = fmaxf(m1, r0[q]);
                m2 = fmaxf(m2, ap[q]);
            }
        }
        float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int q = 0; q < KH; ++q)
            if (act[q]) {
                s1 += __expf(r0[q] - m1);
                s2 += __expf(ap[q] - m2);
            }
        return make_float4(m1, s1, m2, s2);
    }

    // s d log V / d raw of this half's lobes (zero for lobes beyond K).
    __device__ __forceinline__ void pass2(float lse, float lsa, float s, float (&d)[4 * KH]) const {
#pragma unroll
        for (int q = 0; q < KH; ++q) {
            if (act[q]) {
                const float r = __expf(ap[q] - lsa);   // posterior of lobe q
                const float lam = __expf(r0[q] - lse); // its mixture weight
                const float sr = s * r;
                d[4 * q + 0] = s * (r - lam);
                d[4 * q + 1] = sr * (inv_minus_coth(kap[q]) + md[q]) * sk[q];
                d[4 * q + 2] = sr * kap[q] * wdt[q] * kPi * st[q] * (1.0f - st[q]);
                d[4 * q + 3] = sr * kap[q] * wdp[q] * 2.0f * kPi * sp[q] * (1.0f - sp[q]);
            } else {
                d[4 * q + 0] = d[4 * q + 1] = d[4 * q + 2] = d[4 * q + 3] = 0.0f;
            }
        }
    }
};

// log(e^{m_a} s_a + e^{m_b} s_b) for partial sums that may be empty (s = 0).
__device__ __forceinline__ float lse_combine(float ma, float sa, float mb, float sb) {
    const float m = fmaxf(ma, mb);
    float t = 0.0f;
    if (sa > 0.0f) t += sa * __expf(ma - m);
    if (sb > 0.0f) t += sb * __expf(mb - m);
    return m + __logf(t);
}

// NC (a multiple of 8) values as BF16 at row t, columns c0 .. c0+NC of a
// K-major tile, with their residuals lo_off bytes on when lo_off != 0.
template <int NC>
__device__ __forceinline__ void store_cols(uint8_t* base, int t, int c0, int kp, const float* v, uint32_t lo_off) {
#pragma unroll
    for (int c = 0; c < NC; c += 8) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 hb = __floats2bfloat162_rn(v[c + 2 * i], v[c + 2 * i + 1]);
            hw[i] = *reinterpret_cast<uint32_t*>(&hb);
            const float2 hf = __bfloat1622float2(hb);
            lw[i] = pack_bf16(v[c + 2 * i] - hf.x, v[c + 2 * i + 1] - hf.y);
        }
        const uint32_t off = tile_off(t, c0 + c, kp);
        *reinterpret_cast<uint4*>(base + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if (lo_off) *reinterpret_cast<uint4*>(base + lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// Encoder-gradient scatter (Eq. 11 transposed) of levels lbeg .. lbeg+NLV
// with FF features per level; dg holds their 16 columns.
template <int FF, int NLV>
__device__ __forceinline__ void scatter_levels(const DevCfg& cfg, float* __restrict__ grad, float x, float y,
                                               float z, int lbeg, const float (&dg)[16]) {
#pragma unroll
    for (int q = 0; q < NLV; ++q) {
        const int l = lbeg + q;
        if (l < cfg.n_levels) {
            const Cell cl = make_cell(x, y, z, cfg.level_res[l]);
            float* gl = grad + (size_t)cfg.level_off[l] * FF;
            uint32_t idx[8];
            float ws[8];
            corners8(cfg, l, cl, idx, ws);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float wc = ws[c];
                float* e = gl + (size_t)idx[c] * FF;
                if constexpr (FF == 1) {
                    atomicAdd(e, wc * dg[q]);
                } else if constexpr (FF == 2) {
                    if (c & 1) continue;  // corners c, c + 1 (along x) together
                    scatter_pair2(gl, cfg.level_off[l], idx[c], idx[c + 1], ws[c], ws[c + 1], dg[2 * q],
                                  dg[2 * q + 1]);
                } else {
#pragma unroll
                    for (int f = 0; f < FF; f += 4)
                        atomicAdd(reinterpret_cast<float4*>(e + f),
                                  make_float4(wc * dg[FF * q + f], wc * dg[FF * q + f + 1], wc * dg[FF * q + f + 2],
                                              wc * dg[FF * q + f + 3]));
                }
            }
        }
    }
}

// Grid features of a training batch for 2-feature grids (Sec. 5.1, Eq. 11):
// enc[j][2l + f] = sum_corners w_c V_l[corner][f] from the FP32 master
// table, in the FP32 arithmetic of tc_encode (same corners, weights and FMA
// order). One thread per (sample, group of LPT levels), all of a group's
// corner loads in flight; a full-occupancy kernel without shared memory
// keeps the whole L1 and many warps for these random L2 reads, which the
// training kernel (one CTA per SM holding most of the shared memory) cannot.
template <int LPT>
__global__ void __launch_bounds__(256) k_train_encode(const __grid_constant__ DevCfg cfg,
                                                      const float* __restrict__ grid32, int64_t n,
                                                      int64_t ld, const float* __restrict__ pos,
                                                      float* __restrict__ enc) {
    const int ng = (cfg.n_levels + LPT - 1) / LPT;
    const int G = cfg.grid_feats;
    const int64_t total = n * ng;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / ng;
        const int l0 = (int)(i - j * ng) * LPT;
        const float x = pos[j], y = pos[ld + j], z = pos[2 * ld + j];
        Cell cs[LPT];
        float2 v[LPT][8];
#pragma unroll
        for (int r = 0; r < LPT; ++r) {
            const int l = l0 + r;
            if (l < cfg.n_levels) {
                cs[r] = make_cell(x, y, z, cfg.level_res[l]);
                const float* gr = grid32 + (size_t)cfg.level_off[l] * 2;
#pragma unroll
                for (int c = 0; c < 8; c += 2)
                    gather_pair2(gr, cfg.level_off[l], corner_idx1(cfg, l, cs[r], c), corner_idx1(cfg, l, cs[r], c + 1),
                                 v[r][c], v[r][c + 1]);
            }
        }
#pragma unroll
        for (int r = 0; r < LPT; ++r) {
            const int l = l0 + r;
            if (l < cfg.n_levels) {
                float ws[8];
                corner_w8(cs[r], ws);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    a0 = fmaf(ws[c], v[r][c].x, a0);
                    a1 = fmaf(ws[c], v[r][c].y, a1);
                }
                *reinterpret_cast<float2*>(enc + j * G + 2 * l) = make_float2(a0, a1);
            }
        }
    }
}

// The small four-lobe instance (single-level grids) is compiled for three
// CTAs per SM (80 registers without spills; its delta tiles are only as
// wide as its layers, 53 KB a CTA): its tile chain of MMA round trips is
// latency-bound, and the other CTAs overlap it. (Four CTAs at 64 registers
// measured slower.)
__host__ __device__ constexpr int train_ctas_per_sm(int kmax, bool f2) { return (kmax == 4 && !f2) ? 3 : 1; }

template <int KMAX, bool F2>
__global__ void __launch_bounds__(kTrainThreads, train_ctas_per_sm(KMAX, F2)) k_train_tc(
    const __grid_constant__ TcCfg tc, const __grid_constant__ TcTrain tt, const float* __restrict__ grid32,
    const uint8_t* __restrict__ wblob, int64_t n, int64_t ld, const float* __restrict__ pos,
    const float* __restrict__ aux, const float* __restrict__ dir, const float* __restrict__ rad,
    const float* __restrict__ spdf, const float* __restrict__ dlogv, float inv_n, float* __restrict__ grad,
    int64_t mlp_off, float* __restrict__ loss, int* __restrict__ status, const float* __restrict__ enc) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int KH = KMAX / 2;
    uint8_t* sW = smem;
    uint8_t* sD = smem + tt.d_off;
    float4* xch = reinterpret_cast<float4*>(smem + tt.x_off);  // [2][kTile] partial log-sum-exps
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tt.bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    const int t = threadIdx.x, warp = t >> 5;
    const int row = t & (kTile - 1), half = t >> 7;
    const uint32_t bar_mma = smem_u32(&bars[0]), bar_w = smem_u32(&bars[1]);
    const DevCfg& cfg = tc.base;
    const int L = cfg.n_layers;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(tt.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_w, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t wbytes = (tt.split ? 2u : 1u) * tc.w_bytes;
    if (t == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w), "r"(wbytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(sW)),
                     "l"(wblob), "r"(wbytes), "r"(bar_w)
                     : "memory");
    }
    bool ok = !__syncthreads_or(warp == 0 && !mbar_wait_bounded(bar_w, 0));
    uint32_t phase = 0;
    const uint32_t sW_addr = smem_u32(sW), sD_addr = smem_u32(sD), base_addr = smem_u32(smem);
    const uint32_t wlo = tc.w_bytes;                      // residual weights follow the high parts
    const uint32_t hlo_addr = base_addr + tt.hlo_off, dlo_addr = base_addr + tt.dlo_off;
    const uint32_t drg = tt.d_cols * 16u;  // bytes per 8-sample row group of the delta tile
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    // Grid levels of this half: [lv0, lv1); the second half also encodes the
    // product-mode inputs and the padding.
    const int nl0 = (cfg.n_levels + 1) / 2;
    const int lv0 = half ? nl0 : 0, lv1 = half ? cfg.n_levels : nl0;
    float lacc = 0.0f;
    bool first = true;
    // Deferred grid scatter (2-feature grids): a tile's encoder gradient of
    // this thread's eight levels (pdg, two columns per level, the next
    // level's first) and the sample position wait for the next tile, whose
    // eight MMA waits each issue one level's atomics: the L2 atomics then
    // overlap the tensor-core work instead of following it.
    float pdg[16];
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    bool pend = false;
    int pq = 0;  // pending levels already issued
    auto scatter_next = [&]() {
        if (F2 && pend && pq < 8) {
            const int l = 8 * half + pq;
            if (l < cfg.n_levels) {
                const Cell cl = make_cell(px, py, pz, cfg.level_res[l]);
                float* gl = grad + (size_t)cfg.level_off[l] * 2;
                uint32_t idx[8];
                float ws[8];
                corners8(cfg, l, cl, idx, ws);
#pragma unroll
                for (int c = 0; c < 8; c += 2)
                    scatter_pair2(gl, cfg.level_off[l], idx[c], idx[c + 1], ws[c], ws[c + 1], pdg[0], pdg[1]);
            }
#pragma unroll
            for (int i = 0; i < 14; ++i) pdg[i] = pdg[i + 2];
            ++pq;
        }
    };
    const int64_t ntiles = (n + kTile - 1) / kTile;
    // This half's grid features (two per level, at most 8 levels) of row
    // `row` of tile tl from k_train_encode, loaded one tile ahead.
    float2 ev[8];
    auto load_enc = [&](int64_t tl) {
        const int64_t jj = tl * kTile + row;
        const bool v = tl < ntiles && jj < n;
        const float* er = enc + (v ? jj : 0) * (int64_t)cfg.grid_feats;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            ev[q] = (v && lv0 + q < lv1) ? __ldg(reinterpret_cast<const float2*>(er + 2 * (lv0 + q)))
                                         : make_float2(0.0f, 0.0f);
    };
    if (F2 && enc) load_enc(blockIdx.x);
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int64_t j = tile * kTile + row;
        const bool valid = j < n;
        if (F2 && enc) {
            // This half's grid features, then the product-mode inputs and
            // the padding; the next tile's features are loaded meanwhile.
            const int kp0 = tc.layer[0].Kp;
            const uint32_t lo = tc.split ? tc.a_bytes : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (lv0 + q < lv1) store_pair(smem + tt.h_off[0], tile_off(row, 2 * (lv0 + q), kp0), ev[q].x, ev[q].y, lo);
            load_enc(tile + gridDim.x);
            tc_encode<F2>(tc, grid32, j, valid, ld, pos, aux, smem + tt.h_off[0], row, lo, true, lv1, lv1,
                          half == 1);
        } else {
            tc_encode<F2>(tc, grid32, j, valid, ld, pos, aux, smem + tt.h_off[0], row, tc.split ? tc.a_bytes : 0u,
                          true, lv0, lv1, half == 1);
        }
        // The loss inputs of this row, loaded now so that their latency
        // passes during the forward layers' tensor-core round trips.
        float w[3] = {0.0f, 0.0f, 1.0f}, sc = 0.0f;
        if (valid) {
            w[0] = dir[j];
            w[1] = dir[ld + j];
            w[2] = dir[2 * ld + j];
            sc = dlogv ? dlogv[j] : -(rad[j] / spdf[j]) * inv_n;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        float raw[4 * KH];
        // Forward, keeping every layer's input tile.
        for (int l = 0; l < L && ok; ++l) {
            const TcLayer& ly = tc.layer[l];
            if (t == 0) {
                tc_fence_after();
                // The descriptors of K step s are those of step 0 with the
                // start address 256 bytes (16 units) further.
                const uint32_t sbo = (uint32_t)(ly.Kp >> 3) * 128u;
                const uint64_t ad0 = umma_desc(base_addr + tt.h_off[l], 128u, sbo);
                const uint64_t bd0 = umma_desc(sW_addr + ly.w_off, 128u, sbo);
                const uint64_t bl0 = umma_desc(sW_addr + wlo + ly.w_off, 128u, sbo);
                const uint64_t al0 = umma_desc(hlo_addr, 128u, sbo);
                for (int s = 0; s < (ly.Kp >> 4); ++s) {
                    const uint64_t o = (uint64_t)(16 * s);
                    mma_bf16(tmem, ad0 + o, bd0 + o, ly.idesc, s > 0 ? 1u : 0u);
                    if (tt.split) {
                        mma_bf16(tmem, ad0 + o, bl0 + o, ly.idesc, 1u);
                        mma_bf16(tmem, al0 + o, bd0 + o, ly.idesc, 1u);
                    }
                }
                mma_commit(bar_mma);
            }
            scatter_next();  // the previous tile's grid gradient, one level
            // Warp 0 spins on the barrier; the others sleep at the CTA
            // barrier, which then orders their TMEM reads after completion.
            const bool done = warp != 0 || mbar_wait_bounded(bar_mma, phase);
            phase ^= 1u;
            ok = !__syncthreads_or(!done);
            if (!ok) break;
            tc_fence_after();
            if (l < L - 1) {
                uint8_t* hn = smem + tt.h_off[l + 1];
                const int kpn = tc.layer[l + 1].Kp;
                const uint32_t lo = tt.split ? tt.hlo_off - tt.h_off[l + 1] : 0u;
                for (int c0 = 16 * half; c0 < ly.Np; c0 += 32) {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
                    tmem_wait16(r);
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(__uint_as_float(r[i]), 0.0f);
                    store16(hn, tile_off(row, c0, kpn), tile_off(row, c0 + 8, kpn), v, lo);
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
            } else {
                // This half's lobes: columns [half * 4 KH, (half + 1) * 4 KH).
                if constexpr (4 * KH >= 16) {
#pragma unroll
                    for (int c = 0; c < 4 * KH / 16; ++c) {
                        uint32_t r[16];
                        tmem_ld16(tmem + lane_base + (uint32_t)(half * 4 * KH + 16 * c), r);
                        tmem_wait16(r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) raw[16 * c + i] = __uint_as_float(r[i]);
                    }
                } else {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base, r);
                    tmem_wait16(r);
#pragma unroll
                    for (int i = 0; i < 4 * KH; ++i) raw[i] = __uint_as_float(half ? r[4 * KH + i] : r[i]);
                }
            }
        }
        if (!ok) break;
        // Loss and d loss / d raw (zero for rows beyond n).
        GradHalf<KMAX> gh;
        const float4 part = gh.pass1(cfg, half, raw, w);
        xch[half * kTile + row] = part;
        __syncthreads();
        const float4 oth = xch[(half ^ 1) * kTile + row];
        const float lse = lse_combine(part.x, part.y, oth.x, oth.y);
        const float lsa = lse_combine(part.z, part.w, oth.z, oth.w);
        if (valid && half == 0) lacc += sc * (lsa - lse);
        float dr[4 * KH];
        gh.pass2(lse, lsa, sc, dr);
        const uint32_t dlo = tt.split ? tt.dlo_off - tt.d_off : 0u;
        store_cols<4 * KH>(sD, row, half * 4 * KH, (int)tt.d_cols, dr, dlo);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // Backward, top layer first.
        for (int l = L - 1; l >= 0 && ok; --l) {
            const TcLayer& ly = tc.layer[l];
            if (t == 0) {
                tc_fence_after();
                const uint32_t hk = (uint32_t)(ly.Kp >> 3) * 128u;  // K step of an H_l / W_l tile
                // Step-0 descriptors; step s adds its byte offset >> 4 to the
                // start address field.
                // dW_l += D^T H_l: M = 128 (outputs), N = Kp_l, K = 128 samples.
                const uint64_t bh0 = umma_desc(base_addr + tt.h_off[l], hk, 128u);
                const uint64_t dw0 = umma_desc(sD_addr, drg, 128u), dwl0 = umma_desc(dlo_addr, drg, 128u);
                const uint64_t bstep = (uint64_t)((2u * hk) >> 4), dstep = (uint64_t)((2u * drg) >> 4);
                for (int s = 0; s < 8; ++s) {
                    const uint64_t bh = bh0 + s * bstep;
                    mma_bf16(tmem + tt.dw_col[l], dw0 + s * dstep, bh, tt.idesc_dw[l], (first && s == 0) ? 0u : 1u);
                    if (tt.split) mma_bf16(tmem + tt.dw_col[l], dwl0 + s * dstep, bh, tt.idesc_dw[l], 1u);
                }
                // D W_l: M = 128 samples, N = Kp_l, K = Np_l outputs.
                const uint64_t ad0 = umma_desc(sD_addr, 128u, drg), al0 = umma_desc(dlo_addr, 128u, drg);
                const uint64_t bd0 = umma_desc(sW_addr + ly.w_off, hk, 128u);
                const uint64_t bl0 = umma_desc(sW_addr + wlo + ly.w_off, hk, 128u);
                for (int s = 0; s < (ly.Np >> 4); ++s) {
                    const uint64_t o = (uint64_t)(16 * s), ob = s * bstep;
                    mma_bf16(tmem, ad0 + o, bd0 + ob, tt.idesc_dx[l], s > 0 ? 1u : 0u);
                    if (tt.split) {
                        mma_bf16(tmem, ad0 + o, bl0 + ob, tt.idesc_dx[l], 1u);
                        mma_bf16(tmem, al0 + o, bd0 + ob, tt.idesc_dx[l], 1u);
                    }
                }
                mma_commit(bar_mma);
            }
            scatter_next();
            const bool done = warp != 0 || mbar_wait_bounded(bar_mma, phase);
            phase ^= 1u;
            ok = !__syncthreads_or(!done);
            if (!ok) break;
            tc_fence_after();
            const uint8_t* hl = smem + tt.h_off[l];
            if (l > 0) {
                // delta_{l-1} = (D W_l) masked by ReLU'(z_{l-1}) (H_l > 0).
                for (int c0 = 16 * half; c0 < ly.Kp; c0 += 32) {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
                    tmem_wait16(r);
                    const uint4 m0 = *reinterpret_cast<const uint4*>(hl + tile_off(row, c0, ly.Kp));
                    const uint4 m1 = *reinterpret_cast<const uint4*>(hl + tile_off(row, c0 + 8, ly.Kp));
                    const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float2 hv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&mw[i]));
                        v[2 * i] = hv.x > 0.0f ? __uint_as_float(r[2 * i]) : 0.0f;
                        v[2 * i + 1] = hv.y > 0.0f ? __uint_as_float(r[2 * i + 1]) : 0.0f;
                    }
                    store16(sD, tile_off(row, c0, (int)tt.d_cols), tile_off(row, c0 + 8, (int)tt.d_cols), v, dlo);
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
            } else if (16 * half < cfg.grid_feats) {
                // Encoder gradient of this half's 16 grid-feature columns ->
                // grid scatter.
                float dg[16];
                {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(16 * half), r);
                    tmem_wait16(r);
#pragma unroll
                    for (int i = 0; i < 16; ++i) dg[i] = __uint_as_float(r[i]);
                }
                tc_fence_before();
                if constexpr (F2) {
                    while (pend && pq < 8) scatter_next();  // networks with fewer than 4 layers
                    pend = valid;
                    pq = 0;
                    if (valid) {
                        px = pos[j];
                        py = pos[ld + j];
                        pz = pos[2 * ld + j];
#pragma unroll
                        for (int i = 0; i < 16; ++i) pdg[i] = dg[i];
                    }
                } else if (valid) {
                    const float x = pos[j], y = pos[ld + j], z = pos[2 * ld + j];
                    const int F = cfg.feat;
                    if (F == 2) scatter_levels<2, 8>(cfg, grad, x, y, z, 8 * half, dg);
                    else if (F == 4) scatter_levels<4, 4>(cfg, grad, x, y, z, 4 * half, dg);
                    else if (F == 8) scatter_levels<8, 2>(cfg, grad, x, y, z, 2 * half, dg);
                    else scatter_levels<1, 16>(cfg, grad, x, y, z, 16 * half, dg);
                }
            } else {
                tc_fence_before();
            }
        }
        first = false;
    }
    while (pend && pq < 8) scatter_next();  // the last tile's grid gradient
    // Loss: one atomic per warp.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
    if ((t & 31) == 0 && lacc != 0.0f) atomicAdd(loss, lacc);
    // Weight gradients: lane o of layer l's TMEM region holds dW_l[o][*].
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ok && !first) {
        for (int l = 0; l < L; ++l) {
            const TcLayer& ly = tc.layer[l];
            float* gW = grad + mlp_off + tt.woff[l];
            for (int c0 = 16 * half; c0 < ly.Kp; c0 += 32) {
                uint32_t r[16];
                tmem_ld16(tmem + lane_base + tt.dw_col[l] + (uint32_t)c0, r);
                tmem_wait16(r);
                if (row < ly.N)
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < ly.K) atomicAdd(gW + (int64_t)row * ly.K + c0 + i, __uint_as_float(r[i]));
            }
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(status, kStatusTimeout);
        // As in the forward kernel: drain this CTA's in-flight weight copy and
        // MMA batch (bounded) before the tensor memory is released.
        if (warp == 0) {
            (void)mbar_wait_bounded(bar_w, 0);
            (void)mbar_wait_bounded(bar_mma, phase ^ 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tt.tmem_cols) : "memory");
    }
}

}  // namespace

struct TcState {
    TcCfg cfg;
    uint8_t* wblob = nullptr;      // BF16 weights of the training parameters
    // Training always multiplies split operands (BF16 high part and
    // residual): with single-pass BF16 inference (NPM_BF16) this is a second
    // blob in the split layout; otherwise training reads wblob.
    uint8_t* wblob_train = nullptr;
    uint8_t* wblob_inf = nullptr;  // of the moving average, when inference uses it
    size_t smem = 0;
    int grid = 0;
    TcCfg train_cfg;     // copy of cfg for training (split operands)
    TcTrain train;
    bool can_train = false;
    // Grid features of a training batch (max_batch x grid_feats FP32) for
    // 2-feature grids, written by k_train_encode; NULL: the training kernel
    // gathers them itself.
    float* enc = nullptr;
};

static int pad16(int v) { return (v + 15) / 16 * 16; }

npm_status tc_create(npm_handle* h) {
    const npm_config& c = h->cfg;
    if (c.feat_per_level != 1 && c.feat_per_level != 2 && c.feat_per_level != 4 &&
        c.feat_per_level != 8)
        return NPM_ERR_UNSUPPORTED;
    TcState* s = new TcState();
    TcCfg& t = s->cfg;
    memset(&t, 0, sizeof(t));
    t.base = h->dc;
    uint32_t off = 0;
    int maxnp = 0;
    for (int l = 0; l < c.n_layers; ++l) {
        TcLayer& ly = t.layer[l];
        ly.K = c.widths[l];
        ly.N = c.widths[l + 1];
        ly.Kp = pad16(ly.K);
        ly.Np = pad16(ly.N);
        ly.w_off = off;
        off += (uint32_t)(ly.Np * ly.Kp * 2);
        // kind::f16 descriptor: D FP32 (bit 4), A and B BF16 (bits 7, 10;
        // zero for FP16 operands), both K-major, N >> 3 at bit 17, M >> 4 at
        // bit 24.
        const bool f16ops = c.precision == NPM_FP16 || c.precision == NPM_FP32_TC;
        const uint32_t ab = f16ops ? 0u : (1u << 7) | (1u << 10);
        ly.idesc = (1u << 4) | ab | ((uint32_t)(ly.Np >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
        maxnp = ly.Np > maxnp ? ly.Np : maxnp;
    }
    t.w_bytes = (off + 127u) / 128u * 128u;
    // Layer 0 gets its own input buffer only when the encoding leaves whole
    // zero chunks to write once; otherwise it shares the buffer of the
    // hidden layers (less shared memory, more L1 for the grid gathers).
    const int enc_width = c.n_levels * c.feat_per_level + (c.mode == NPM_PRODUCT ? 21 : 0);
    // A single small grid level (the tiny models) shares the buffer anyway:
    // its zero chunk costs one store per tile, and the smaller CTA lets eight
    // of them share an SM instead of six.
    const bool single_small = c.n_levels == 1 && c.feat_per_level <= 8 && c.mode != NPM_PRODUCT;
    const bool sep0 = (enc_width + 7) / 8 * 8 < t.layer[0].Kp && !single_small;
    int maxkp1 = 16;  // widest input of the layers sharing the buffer
    for (int l = sep0 ? 1 : 0; l < c.n_layers; ++l) maxkp1 = std::max(maxkp1, t.layer[l].Kp);
    t.a_bytes = (uint32_t)(kTile * maxkp1 * 2);
    t.a0_bytes = sep0 ? (uint32_t)(kTile * t.layer[0].Kp * 2) : 0u;
    t.split = (c.precision == NPM_BF16X3 || c.precision == NPM_FP32_TC) ? 1 : 0;
    t.f16 = (c.precision == NPM_FP16 || c.precision == NPM_FP32_TC) ? 1 : 0;
    t.fp32 = c.precision == NPM_FP32_TC ? 1 : 0;
    const uint32_t nsplit = t.split ? 2u : 1u;
    const uint32_t nw = (t.split || t.f16) ? 2u : 1u;
    uint32_t cols = 32;
    while ((int)cols < maxnp) cols <<= 1;
    t.tmem_cols = cols;
    t.enc_width = enc_width;
    s->smem = nw * t.w_bytes + nsplit * (t.a0_bytes + t.a_bytes) + 64;
    if (s->smem > 200 * 1024 || c.K > 16) {
        delete s;
        return NPM_ERR_UNSUPPORTED;
    }
    // Training layout. Gradients take split BF16 operands in both
    // reduced-precision modes: single-pass BF16 compounds its rounding down
    // the layers and through the cancelling grid sums (per-tensor gradient
    // errors of tens of percent), so only inference offers the plain form.
    {
        TcTrain& tr = s->train;
        memset(&tr, 0, sizeof(tr));
        s->train_cfg = t;
        // Training multiplies BF16 operands whatever the inference format.
        s->train_cfg.f16 = 0;
        for (int l = 0; l < c.n_layers; ++l) s->train_cfg.layer[l].idesc |= (1u << 7) | (1u << 10);
        uint32_t off = 2u * t.w_bytes, col0 = 0, cols = 0;
        int64_t wo = 0;
        bool fits = c.K * 4 <= 64 && c.n_levels * c.feat_per_level <= 32;
        for (int l = 0; l < c.n_layers; ++l) {
            const TcLayer& ly = t.layer[l];
            tr.h_off[l] = off;
            off += (uint32_t)(kTile * ly.Kp * 2);
            col0 = (uint32_t)std::max<int>((int)col0, std::max(ly.Kp, ly.Np));
            tr.woff[l] = wo;
            wo += (int64_t)ly.K * ly.N;
            if (ly.Np > 128 || ly.Kp > 128) fits = false;
            // dW: A = delta^T (MN-major), B = H_l (MN-major), M = 128, N = Kp_l.
            tr.idesc_dw[l] = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(ly.Kp >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
            // dX: A = delta (K-major), B = W_l read MN-major, M = 128, N = Kp_l.
            tr.idesc_dx[l] = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) |
                             ((uint32_t)(ly.Kp >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
        }
        tr.split = 1;
        int maxkp = 0;
        for (int l = 0; l < c.n_layers; ++l) maxkp = std::max(maxkp, t.layer[l].Kp);
        col0 = (col0 + 15) / 16 * 16;
        cols = col0;
        for (int l = 0; l < c.n_layers; ++l) {
            tr.dw_col[l] = cols;
            cols += (uint32_t)t.layer[l].Kp;
        }
        uint32_t pw = 32;
        while (pw < cols) pw <<= 1;
        tr.tmem_cols = pw;
        // Delta tile: as wide as the widest layer (inputs or outputs). The
        // weight-gradient MMA reads it transposed with M = 128 output rows:
        // rows beyond the layer's outputs come from the next row groups and,
        // past the last one, up to 2 KB beyond the tile (the residual tile
        // that follows); they land in weight-gradient rows that are never
        // read.
        uint32_t dcols = 16;
        for (int l = 0; l < c.n_layers; ++l)
            dcols = std::max<uint32_t>(dcols, (uint32_t)std::max(t.layer[l].Kp, t.layer[l].Np));
        tr.d_cols = dcols;
        tr.d_off = (off + 127u) / 128u * 128u;
        tr.dlo_off = tr.d_off + kTile * dcols * 2;
        // One residual activation tile, reused layer by layer; the loss
        // step's exchange of partial log-sum-exps reuses it too (the forward
        // has finished with it, and the next tile's encode rewrites it after
        // the backward).
        tr.hlo_off = tr.dlo_off + kTile * dcols * 2;
        const uint32_t hlo_bytes = (uint32_t)(kTile * maxkp * 2);
        // (Kp >= 16, so the tile has at least 4 KB: the exchange buffer's
        // 2 x kTile float4 and the over-read's 2 KB.)
        tr.x_off = tr.hlo_off;
        tr.bar_off = tr.hlo_off + hlo_bytes;
        tr.smem = tr.bar_off + 64;
        // The encoder writes its residual at (tile + a_bytes): point that at
        // the shared residual tile.
        s->train_cfg.split = tr.split;
        s->train_cfg.a_bytes = tr.hlo_off - tr.h_off[0];
        // The FP32-accuracy mode trains with the FP32 kernels.
        s->can_train = fits && pw <= 512 && tr.smem <= 220 * 1024 && !t.fp32;
    }
    if (device_alloc((void**)&s->wblob, nw * t.w_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return NPM_ERR_OOM;
    }
    cudaMemset(s->wblob, 0, nw * t.w_bytes);
    if (s->can_train && !t.split) {
        if (device_alloc((void**)&s->wblob_train, 2u * t.w_bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(s->wblob);
            delete s;
            return NPM_ERR_OOM;
        }
        cudaMemset(s->wblob_train, 0, 2u * t.w_bytes);
    }
    if (s->can_train && c.feat_per_level == 2) {
        // Optional: without it the training kernel encodes in place.
        if (device_alloc((void**)&s->enc, sizeof(float) * (size_t)c.max_batch * h->dc.grid_feats) != cudaSuccess) {
            cudaGetLastError();
            s->enc = nullptr;
        }
    }
    h->tc = s;
    return NPM_OK;
}

void tc_destroy(npm_handle* h) {
    if (!h->tc) return;
    if (h->tc->wblob) cudaFree(h->tc->wblob);
    if (h->tc->wblob_inf) cudaFree(h->tc->wblob_inf);
    if (h->tc->wblob_train) cudaFree(h->tc->wblob_train);
    if (h->tc->enc) cudaFree(h->tc->enc);
    delete h->tc;
    h->tc = nullptr;
}

cudaError_t tc_refresh_weights(npm_handle* h, cudaStream_t st) {
    TcState* s = h->tc;
    k_tc_weights<<<16, 256, 0, st>>>(s->cfg, h->params + h->mlp_off, s->wblob);
    if (s->wblob_train) k_tc_weights<<<16, 256, 0, st>>>(s->train_cfg, h->params + h->mlp_off, s->wblob_train);
    if (h->ema) {
        if (!s->wblob_inf) {
            const size_t bytes = ((s->cfg.split || s->cfg.f16) ? 2u : 1u) * (size_t)s->cfg.w_bytes;
            cudaError_t e = cudaMalloc(&s->wblob_inf, bytes);
            if (e != cudaSuccess) return e;
            cudaMemsetAsync(s->wblob_inf, 0, bytes, st);
        }
        k_tc_weights<<<16, 256, 0, st>>>(s->cfg, h->ema + h->mlp_off, s->wblob_inf);
    }
    return cudaGetLastError();
}

// Shared memory of a k_forward_tc CTA of G tile groups: the weight blobs,
// each group's activation tiles, the barriers and the tensor-memory slot.
static size_t tc_group_smem(const TcState* s, int G) {
    const TcCfg& c = s->cfg;
    const size_t nw = (c.split || c.f16) ? 2 : 1, nsplit = c.split ? 2 : 1;
    return nw * c.w_bytes + (size_t)G * nsplit * (c.a0_bytes + c.a_bytes) + 8 * (1 + G) + 16;
}

// Whether a CTA of G tile groups fits one SM (shared and tensor memory).
static bool tc_groups_fit(const TcState* s, int G) {
    uint32_t cols = 32;
    while (cols < (uint32_t)G * s->cfg.tmem_cols) cols <<= 1;
    return cols <= 512u && tc_group_smem(s, G) + 1024 <= 227 * 1024;
}

// Whether a group's activation tiles hold the raw outputs of a 128-row tile
// staged for the warp-per-query decode (row stride 4 KMAX + 4 floats).
static bool tc_stage_fits(const TcState* s, int kmax) {
    return (size_t)(s->cfg.split ? 2 : 1) * s->cfg.a_bytes >= (size_t)kTile * (4 * kmax + 4) * sizeof(float);
}

template <int KMAX, bool F2, int NL, bool WARPDEC = false, bool G32 = false, int G = 1>
static cudaError_t launch_tc(npm_handle* h, QueryBatch& qb, int64_t max_n, cudaStream_t st) {
    TcState* s = h->tc;
    if (WARPDEC && !tc_stage_fits(s, KMAX)) return cudaErrorInvalidValue;  // the dispatch checks this
    auto kern = k_forward_tc<KMAX, F2, NL, WARPDEC, G32, G>;
    // CTAs per SM from registers (the instance's count, queried once) and
    // tensor memory; then carve out just the shared memory they need so the
    // rest stays L1 for the grid gathers.
    static std::atomic<int> regs{-1};
    int nregs = regs.load(std::memory_order_relaxed);
    if (nregs < 0) {
        cudaFuncAttributes fa;
        cudaError_t ea = cudaFuncGetAttributes(&fa, kern);
        if (ea != cudaSuccess) return ea;
        nregs = fa.numRegs;
        regs.store(nregs, std::memory_order_relaxed);
    }
    const int regs_cta = ((nregs + 7) / 8 * 8) * kThreads;
    int per_sm = regs_cta > 0 ? 65536 / regs_cta : 1;
    const int tmem_cap = (int)(512u / s->cfg.tmem_cols);
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm > 16) per_sm = 16;
    while (per_sm > 1 && (size_t)per_sm * (s->smem + 1024) > 227 * 1024) --per_sm;
    static std::atomic<int> env_ctas{INT32_MIN + 1};
    const int v = env_override("NPM_TC_CTAS_PER_SM", env_ctas);
    if (v >= 1 && v < per_sm) per_sm = v;
    if (per_sm < 1) per_sm = 1;
    const size_t smem = G > 1 ? tc_group_smem(s, G) : s->smem;
    if (G > 1) per_sm = 1;  // one CTA of G groups per SM
    static std::atomic<uint64_t> attrs{~0ull};
    cudaError_t e = set_smem_attrs(kern, smem, carveout_percent((size_t)per_sm * (smem + 1024)), attrs);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t t0 = 0;
    for (int i = 0; i < qb.nseg; ++i) {
        qb.seg[i].tile0 = t0;
        t0 += (qb.seg[i].n + kTile - 1) / kTile;
    }
    qb.total_tiles = t0;
    const int64_t hint = (qb.n_dev ? (max_n + kTile - 1) / kTile : t0 + G - 1) / G;
    int64_t g = (int64_t)per_sm * sms;
    if (g > hint) g = hint < 1 ? 1 : hint;
    int* status = reinterpret_cast<int*>(h->scalars + 8);
    const uint8_t* wb = h->ema ? s->wblob_inf : s->wblob;  // inference weights
    const GridT<G32>* grid;
    if constexpr (G32) grid = h->ema ? h->ema : h->params;  // the inference parameters
    else grid = h->grid_h;
    kern<<<(int)g, kThreads * G, smem, st>>>(s->cfg, grid, wb, qb, status);
    return cudaGetLastError();
}

template <int KMAX, bool F2>
static cudaError_t launch_train_tc(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux,
                                   const float* dir, const float* rad, const float* spdf, const float* dlogv,
                                   float* loss, cudaStream_t st) {
    TcState* s = h->tc;
    auto kern = k_train_tc<KMAX, F2>;
    // CTAs per SM: the instance's register budget, if shared and tensor
    // memory hold that many.
    int per_sm = train_ctas_per_sm(KMAX, F2);
    while (per_sm > 1 && ((size_t)per_sm * (s->train.smem + 1024) > 227 * 1024 ||
                          (uint32_t)per_sm * s->train.tmem_cols > 512u))
        --per_sm;
    static std::atomic<uint64_t> attrs{~0ull};
    cudaError_t e =
        set_smem_attrs(kern, s->train.smem, carveout_percent((size_t)per_sm * (s->train.smem + 1024)), attrs);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t slots = (int64_t)per_sm * sms;
    const int g = (int)(ntiles < slots ? ntiles : slots);
    int* status = reinterpret_cast<int*>(h->scalars + 8);
    const float* enc = nullptr;
    if (F2 && s->enc && n <= h->cfg.max_batch) {
        // Levels per thread: two (64 registers, more warps) measured a little
        // faster than four; tuning override NPM_ENC_LPT (2 or 4).
        static std::atomic<int> env_lpt{INT32_MIN + 1};
        const int lpt = env_override("NPM_ENC_LPT", env_lpt) == 4 ? 4 : 2;
        const int64_t items = n * ((h->dc.n_levels + lpt - 1) / lpt);
        int64_t eg = (items + 255) / 256;
        if (eg > (int64_t)sms * 16) eg = (int64_t)sms * 16;
        if (lpt == 2) k_train_encode<2><<<(int)eg, 256, 0, st>>>(h->dc, h->params, n, ld, pos, s->enc);
        else k_train_encode<4><<<(int)eg, 256, 0, st>>>(h->dc, h->params, n, ld, pos, s->enc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        enc = s->enc;
    }
    const uint8_t* wb = s->wblob_train ? s->wblob_train : s->wblob;
    kern<<<g < 1 ? 1 : g, kTrainThreads, s->train.smem, st>>>(s->train_cfg, s->train, h->params, wb, n, ld, pos,
                                                         aux, dir, rad, spdf, dlogv, 1.0f / (float)n, h->grads,
                                                         h->mlp_off, loss, status, enc);
    return cudaGetLastError();
}

bool tc_can_train(npm_handle* h) { return h->tc && h->tc->can_train; }

cudaError_t tc_train(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux, const float* dir,
                     const float* rad, const float* spdf, const float* dlogv, float* loss, cudaStream_t st) {
    const int K = h->cfg.K;
    const bool f2 = h->cfg.feat_per_level == 2;
    if (K <= 4)
        return f2 ? launch_train_tc<4, true>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st)
                  : launch_train_tc<4, false>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st);
    if (K <= 8)
        return f2 ? launch_train_tc<8, true>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st)
                  : launch_train_tc<8, false>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st);
    return f2 ? launch_train_tc<16, true>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st)
              : launch_train_tc<16, false>(h, n, ld, pos, aux, dir, rad, spdf, dlogv, loss, st);
}

cudaError_t tc_query_batch(npm_handle* h, QueryBatch& qb, int64_t max_n, cudaStream_t st, bool pdl) {
    const int K = h->cfg.K, L = h->cfg.n_layers;
    const bool f2 = h->cfg.feat_per_level == 2;
    // The FP32-accuracy mode gathers from the FP32 table.
    // Up to eight lobes it runs three tile groups per CTA sharing one copy
    // of the weights where they fit (more tiles in flight per SM for the
    // gathers' latency than separate CTAs, whose weight copies fill the
    // shared memory).
    if (h->tc->cfg.fp32) {
        const bool grp = tc_groups_fit(h->tc, 3);
        if (K <= 4) {
            if (grp) return f2 ? launch_tc<4, true, 0, false, true, 3>(h, qb, max_n, st)
                               : launch_tc<4, false, 0, false, true, 3>(h, qb, max_n, st);
            return f2 ? launch_tc<4, true, 0, false, true>(h, qb, max_n, st)
                      : launch_tc<4, false, 0, false, true>(h, qb, max_n, st);
        }
        if (K <= 8) {
            if (grp) return f2 ? launch_tc<8, true, 0, false, true, 3>(h, qb, max_n, st)
                               : launch_tc<8, false, 0, false, true, 3>(h, qb, max_n, st);
            return f2 ? launch_tc<8, true, 0, false, true>(h, qb, max_n, st)
                      : launch_tc<8, false, 0, false, true>(h, qb, max_n, st);
        }
        return f2 ? launch_tc<16, true, 0, false, true>(h, qb, max_n, st)
                  : launch_tc<16, false, 0, false, true>(h, qb, max_n, st);
    }
    // The small serving networks get their own kernel (npm_tc_tiny.cu);
    // tuning override NPM_TC_TINY=0 selects the general kernel instead.
    static std::atomic<int> env_tiny{INT32_MIN + 1};
    if (tiny_qualifies(h->tc->cfg) && env_override("NPM_TC_TINY", env_tiny) != 0) {
        const uint8_t* wb = h->ema ? h->tc->wblob_inf : h->tc->wblob;
        return launch_tiny(h->tc->cfg, h->tc->smem, h->grid_h, wb, qb, max_n, reinterpret_cast<int*>(h->scalars + 8), st,
                           pdl);
    }
    // Tuning override NPM_TC_DECODE=1: the warp-per-query decode in the
    // general kernel (built for the four- and eight-lobe instances; it stages
    // the raw outputs in the activation buffers, which must hold them).
    static std::atomic<int> env_dec{INT32_MIN + 1};
    const TcCfg& c = h->tc->cfg;
    const int kmax = K <= 4 ? 4 : 8;
    const bool fits = tc_stage_fits(h->tc, kmax);
    if (env_override("NPM_TC_DECODE", env_dec) == 1 && K <= 8 && fits) {
        if (K <= 4) {
            if (L == 3 && K == 4 && !f2) return launch_tc<4, false, 3, true>(h, qb, max_n, st);
            return f2 ? launch_tc<4, true, 0, true>(h, qb, max_n, st) : launch_tc<4, false, 0, true>(h, qb, max_n, st);
        }
        return f2 ? launch_tc<8, true, 0, true>(h, qb, max_n, st) : launch_tc<8, false, 0, true>(h, qb, max_n, st);
    }
    // The small three-layer four-lobe networks get an instance with the layer
    // and lobe loops unrolled (measured faster there; on the four-layer
    // paper-shaped networks unrolling was slower).
    if (K <= 4) {
        if (L == 3 && K == 4 && !f2) return launch_tc<4, false, 3>(h, qb, max_n, st);
        return f2 ? launch_tc<4, true, 0>(h, qb, max_n, st) : launch_tc<4, false, 0>(h, qb, max_n, st);
    }
    if (K <= 8) {
        // Hash-grid networks: three tile groups sharing the weights, where
        // they fit (more tiles in flight for the gathers).
        if (f2 && tc_groups_fit(h->tc, 3)) return launch_tc<8, true, 0, false, false, 3>(h, qb, max_n, st);
        return f2 ? launch_tc<8, true, 0>(h, qb, max_n, st) : launch_tc<8, false, 0>(h, qb, max_n, st);
    }
    return f2 ? launch_tc<16, true, 0>(h, qb, max_n, st) : launch_tc<16, false, 0>(h, qb, max_n, st);
}

npm_status tc_query(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux,
                    const float* uin, float ufrac, bool sample, float* dir_out, float* pdf_out,
                    float* mix_out, cudaStream_t st, bool log_pdf) {
    QueryBatch qb;
    memset(&qb, 0, sizeof(qb));
    qb.nseg = 1;
    qb.sample = sample ? 1 : 0;
    qb.log_pdf = (!sample && log_pdf) ? 1 : 0;
    QuerySeg& q = qb.seg[0];
    q.n = n;
    q.ld = ld;
    q.pos = pos;
    q.aux = aux;
    q.uin = uin;
    q.ufrac = sample ? ufrac : 0.0f;
    q.dir = sample ? dir_out : nullptr;
    q.pdf = pdf_out;
    q.mix = sample ? mix_out : nullptr;
    return tc_query_batch(h, qb, n, st) == cudaSuccess ? NPM_OK : NPM_ERR_CUDA;
}

}  // namespace npm
