// npm_fp32.cu -- FP32 CUDA-core path of the NPM hot path.
//
// Tile groups of 128 threads walk 64-query tiles. Per tile:
//   encode  : 2 threads per query gather the 8 corners of every level and
//             blend them (Sec. 5.1, Eq. 11); product mode appends the SH
//             encodings and the roughness (Sec. 4.3).
//   MLP     : each layer is a 64 x N x K tile GEMM from shared memory; thread
//             (qg, g) owns queries qg + 8j (j < 8) and outputs g*NI .. g*NI+NI-1
//             (Sec. 5.3, Eq. 12). Weights are staged once per CTA.
//   epilogue: 2 threads per query (lobes split in halves, combined with
//             warp shuffles) map the raw outputs (Table 1), then sample and/or
//             evaluate the mixture (Eq. 3-4).
// The forward kernel for 64-wide networks splits these roles: one group
// encodes for three groups that run the MLP and the epilogue
// (k_forward_fp32_ws); other networks run every step in each group
// (k_forward_fp32).
// The training kernel recomputes the forward pass, forms the gradient of the
// weighted log-likelihood in the log domain (Eq. 9), back-propagates through
// the layers and scatters grid gradients with vector atomics.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "npm_device.cuh"
#include "npm_kernels.h"

namespace npm {

constexpr int kTQ = 64;   // queries per tile
constexpr int kNT = 128;  // threads per CTA
constexpr unsigned kFull = 0xffffffffu;

// Activation row stride (floats) of the forward kernel instance whose
// widest layer is 16 * I: the padding of 4 keeps the 16 rows a warp reads
// in distinct banks.
__host__ __device__ constexpr int fwd_act_stride(int I) { return 16 * I + 4; }

// Tile groups per CTA of that instance: the register file holds 4 groups at
// 128 registers a thread, 6 at 80 (enough for the narrow instance only).
__host__ __device__ constexpr int fwd_max_groups(int I) { return I <= 2 ? 6 : 4; }

// ----------------------------------------------------------- tile GEMM

// Named barrier of tile group `group` (kNT threads; barrier 0 is the CTA's).
__device__ __forceinline__ void group_sync(int group) {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(kNT) : "memory");
}

template <int NI>
__device__ __forceinline__ void load_w(const float* p, float (&w)[NI]) {
    if constexpr (NI == 1) {
        w[0] = p[0];
    } else if constexpr (NI == 2) {
        float2 v = *reinterpret_cast<const float2*>(p);
        w[0] = v.x;
        w[1] = v.y;
    } else {
#pragma unroll
        for (int c = 0; c < NI; c += 4) {
            float4 v = *reinterpret_cast<const float4*>(p + c);
            w[c] = v.x;
            w[c + 1] = v.y;
            w[c + 2] = v.z;
            w[c + 3] = v.w;
        }
    }
}

// out[q][n] = f(sum_k in[q][k] * WT[k][n]) for q < 64, n < N. WT rows are
// padded to NP = 16 * NI columns (zeros beyond N). mode 0: identity,
// 1: ReLU, 2: keep where mask[q][n] > 0 (ReLU derivative), else 0.
// AST > 0: the activation row stride is the compile-time AST (so row and
// weight addresses are immediate offsets of two pointers); else AS_rt.
// OST > 0: the output rows have the compile-time stride OST (the input may
// then have another); else the input's.
// INPLACE: out may equal in; the tile group (named barrier group + 1)
// synchronises between the last read of in and the first store.
template <int NI, int AST, bool INPLACE, int OST = 0>
__device__ __forceinline__ void tile_gemm(int t, const float* in, int AS_rt, int K,
                                          const float* __restrict__ WT, float* out, int N, int mode,
                                          const float* __restrict__ mask, int group) {
    const int AS = AST > 0 ? AST : AS_rt;
    const int OS = OST > 0 ? OST : AS;
    constexpr int NP = 16 * NI;
    // Thread t owns output group g (16 groups) and query group qg (8): a
    // warp covers all 16 output groups and 2 query groups, lanes 2i and
    // 2i + 1 sharing output group i. Lanes that read the same shared-memory
    // vector are adjacent, which keeps a warp's 16-byte shared loads at two
    // wavefronts (sharing between strided lanes costs four).
    const int g = (t & 31) >> 1, qg = (t & 1) | ((t >> 5) << 1);
    // Accumulators paired along adjacent outputs: one packed two-lane FMA
    // (fma.rn on each lane, the same rounding as fmaf) per pair.
    constexpr int NP2 = NI >= 2 ? NI / 2 : 1;
    float2 acc[8][NP2];
    float acc1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc1[j] = 0.0f;
#pragma unroll
        for (int i = 0; i < NP2; ++i) acc[j][i] = make_float2(0.0f, 0.0f);
    }
    if constexpr (NI <= 2) {
        // Narrow layers: the K step's 4 x NI weights stay in registers and the
        // activation rows stream through one at a time (fewer live registers,
        // so more tile groups fit).
        for (int k = 0; k < K; k += 4) {
            float w[4][NI];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) load_w<NI>(WT + (k + kk) * NP + g * NI, w[kk]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 a = *reinterpret_cast<const float4*>(in + (qg + 8 * j) * AS + k);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float av = kk == 0 ? a.x : kk == 1 ? a.y : kk == 2 ? a.z : a.w;
                    if constexpr (NI == 1)
                        acc1[j] = fmaf(av, w[kk][0], acc1[j]);
                    else
                        acc[j][0] = __ffma2_rn(make_float2(av, av), make_float2(w[kk][0], w[kk][1]), acc[j][0]);
                }
            }
        }
    } else {
        for (int k = 0; k < K; k += 4) {
            float4 a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = *reinterpret_cast<const float4*>(in + (qg + 8 * j) * AS + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float w[NI];
                load_w<NI>(WT + (k + kk) * NP + g * NI, w);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float av = kk == 0 ? a[j].x : kk == 1 ? a[j].y : kk == 2 ? a[j].z : a[j].w;
                    const float2 aa = make_float2(av, av);
#pragma unroll
                    for (int i = 0; i < NP2; ++i)
                        acc[j][i] = __ffma2_rn(aa, make_float2(w[2 * i], w[2 * i + 1]), acc[j][i]);
                }
            }
        }
    }
    if constexpr (INPLACE) group_sync(group);
    const bool full = g * NI + NI <= N;  // all NI outputs of this thread exist
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int row = (qg + 8 * j) * OS;
        float v[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            v[i] = NI == 1 ? acc1[j] : ((i & 1) ? acc[j][i >> 1].y : acc[j][i >> 1].x);
            if (mode == 1) v[i] = fmaxf(v[i], 0.0f);
            if (mode == 2) v[i] = (g * NI + i < N && mask[row + g * NI + i] > 0.0f) ? v[i] : 0.0f;
        }
        if constexpr (NI % 4 == 0) {
            if (full) {
#pragma unroll
                for (int i = 0; i < NI; i += 4)
                    *reinterpret_cast<float4*>(out + row + g * NI + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                continue;
            }
        }
#pragma unroll
        for (int i = 0; i < NI; ++i)
            if (g * NI + i < N) out[row + g * NI + i] = v[i];
    }
}

// One layer for the tile; only the register tiles up to NIMAX outputs per
// thread are instantiated (NP = 16 NI <= 16 * NIMAX is guaranteed by the
// launcher). AST as in tile_gemm.
template <int NIMAX, int AST = 0, bool INPLACE = false, int OST = 0>
__device__ __forceinline__ void layer(int t, const float* in, int AS, int K, const float* WT, int NP,
                                      float* out, int N, int mode, const float* mask, int group = 0) {
    if (NP == 16) tile_gemm<1, AST, INPLACE, OST>(t, in, AS, K, WT, out, N, mode, mask, group);
    else if (NIMAX >= 2 && NP == 32)
        tile_gemm<(NIMAX >= 2 ? 2 : 1), AST, INPLACE, OST>(t, in, AS, K, WT, out, N, mode, mask, group);
    else if (NIMAX >= 4 && NP == 64)
        tile_gemm<(NIMAX >= 4 ? 4 : 1), AST, INPLACE, OST>(t, in, AS, K, WT, out, N, mode, mask, group);
    else if (NIMAX >= 8)
        tile_gemm<(NIMAX >= 8 ? 8 : 1), AST, INPLACE, OST>(t, in, AS, K, WT, out, N, mode, mask, group);
}

// ------------------------------------------------------------- encode

// Blend of level l at cell cl (F features) into s[0..F).
__device__ __forceinline__ void gather_level(const DevCfg& cfg, const float* __restrict__ grid, int l,
                                             const Cell& cl, float (&s)[8]) {
    const int F = cfg.feat;
    const float* gl = grid + (size_t)cfg.level_off[l] * F;
    uint32_t idx[8];
    corner_idx8(cfg, l, cl, idx);
    float w[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) s[f] = 0.0f;
    if (F == 2) {
        float2 v[8];
#pragma unroll
        for (int c = 0; c < 8; c += 2) gather_pair2(gl, cfg.level_off[l], idx[c], idx[c + 1], v[c], v[c + 1]);
        corner_w8(cl, w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            s[0] = fmaf(w[c], v[c].x, s[0]);
            s[1] = fmaf(w[c], v[c].y, s[1]);
        }
    } else if (F == 4) {
        float4 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = __ldg(reinterpret_cast<const float4*>(gl) + idx[c]);
        corner_w8(cl, w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            s[0] = fmaf(w[c], v[c].x, s[0]);
            s[1] = fmaf(w[c], v[c].y, s[1]);
            s[2] = fmaf(w[c], v[c].z, s[2]);
            s[3] = fmaf(w[c], v[c].w, s[3]);
        }
    } else {
        corner_w8(cl, w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float* e = gl + (size_t)idx[c] * F;
#pragma unroll
            for (int f = 0; f < 8; ++f)
                if (f < F) s[f] = fmaf(w[c], __ldg(e + f), s[f]);
        }
    }
}

// Fills act[q][0 .. widths[0]) for the tile's 64 queries; local thread t
// handles query t % 64 and every other level (two levels in flight).
// FOUR: 2-feature grids keep four levels' loads in flight (registers the
// wide instances have to spare).
template <bool FOUR>
__device__ __forceinline__ void encode_tile(int t, const DevCfg& cfg, const float* __restrict__ grid,
                                            int64_t base, int64_t n, int64_t ld,
                                            const float* __restrict__ pos,
                                            const float* __restrict__ aux, float* act, int AS) {
    const int q = t & (kTQ - 1), part = t >> 6;
    const int64_t j = base + q;
    const bool valid = j < n;
    float x = 0.0f, y = 0.0f, z = 0.0f;
    if (valid) {
        x = pos[j];
        y = pos[ld + j];
        z = pos[2 * ld + j];
    }
    float* row = act + q * AS;
    const int F = cfg.feat;
    int l = part;
    if (FOUR && F == 2) {
        // Four levels' corner loads in flight (levels l, l+2, l+4, l+6).
        for (; l + 6 < cfg.n_levels; l += 8) {
            Cell cs[4];
            uint32_t idx[4][8];
            float2 v[4][8];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cs[r] = make_cell(x, y, z, cfg.level_res[l + 2 * r]);
                corner_idx8(cfg, l + 2 * r, cs[r], idx[r]);
                const float* gr = grid + (size_t)cfg.level_off[l + 2 * r] * 2;
#pragma unroll
                for (int c = 0; c < 8; c += 2)
                    gather_pair2(gr, cfg.level_off[l + 2 * r], idx[r][c], idx[r][c + 1], v[r][c], v[r][c + 1]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float w[8];
                corner_w8(cs[r], w);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    a0 = fmaf(w[c], v[r][c].x, a0);
                    a1 = fmaf(w[c], v[r][c].y, a1);
                }
                row[(l + 2 * r) * 2] = a0;
                row[(l + 2 * r) * 2 + 1] = a1;
            }
        }
    }
    for (; l + 2 < cfg.n_levels; l += 4) {
        const Cell c0 = make_cell(x, y, z, cfg.level_res[l]);
        const Cell c1 = make_cell(x, y, z, cfg.level_res[l + 2]);
        float s0[8], s1[8];
        gather_level(cfg, grid, l, c0, s0);
        gather_level(cfg, grid, l + 2, c1, s1);
#pragma unroll
        for (int f = 0; f < 8; ++f)
            if (f < F) {
                row[l * F + f] = s0[f];
                row[(l + 2) * F + f] = s1[f];
            }
    }
    for (; l < cfg.n_levels; l += 2) {
        const Cell c0 = make_cell(x, y, z, cfg.level_res[l]);
        float s0[8];
        gather_level(cfg, grid, l, c0, s0);
#pragma unroll
        for (int f = 0; f < 8; ++f)
            if (f < F) row[l * F + f] = s0[f];
    }
    const int o = cfg.grid_feats;
    const int w0 = cfg.widths[0];
    if (cfg.mode == NPM_PRODUCT) {
        if (part == 0) {
            float wo[3] = {0.0f, 0.0f, 1.0f};
            if (valid) {
                wo[0] = aux[j];
                wo[1] = aux[ld + j];
                wo[2] = aux[2 * ld + j];
            }
            float sh[16];
            sh_band4(wo[0], wo[1], wo[2], sh);
#pragma unroll
            for (int i = 0; i < 16; ++i) row[o + i] = sh[i];
        } else {
            float nn[3] = {0.0f, 0.0f, 1.0f}, r = 0.0f;
            if (valid) {
                nn[0] = aux[3 * ld + j];
                nn[1] = aux[4 * ld + j];
                nn[2] = aux[5 * ld + j];
                r = aux[6 * ld + j];
            }
            float sh[4];
            sh_band2(nn[0], nn[1], nn[2], sh);
#pragma unroll
            for (int i = 0; i < 4; ++i) row[o + 16 + i] = sh[i];
            row[o + 20] = r;
            for (int i = o + 21; i < w0; ++i) row[i] = 0.0f;
        }
    } else if (part == 1) {
        for (int i = o; i < w0; ++i) row[i] = 0.0f;
    }
}

// -------------------------------------------------------- vMF epilogue

// Mapping of one half of the lobes of query q (Table 1). Returns the local
// lobe count; lam holds normalised weights.
template <int KH>
struct HalfMix {
    Lobe lob[KH];
    float cn[KH];
    float mx, ssum;  // largest weight logit and sum of e^{logit - mx}, both halves
    int l0, cnt;
};

template <int KH>
__device__ __forceinline__ void decode_half(const DevCfg& cfg, const float* raw, int half,
                                            HalfMix<KH>& hm, float* mix_out, int64_t ld, int64_t j,
                                            bool valid) {
    const int K = cfg.K, kh = (K + 1) >> 1;
    hm.l0 = half * kh;
    hm.cnt = min(K, hm.l0 + kh) - hm.l0;
    float mx = -INFINITY;
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) mx = fmaxf(mx, raw[4 * (hm.l0 + ii)]);
    mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 1));
    float ssum = 0.0f;
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) {
            hm.lob[ii].lam = __expf(raw[4 * (hm.l0 + ii)] - mx);
            ssum += hm.lob[ii].lam;
        }
    ssum += __shfl_xor_sync(kFull, ssum, 1);
    hm.mx = mx;
    hm.ssum = ssum;
    const float inv = __fdividef(1.0f, ssum);  // ssum in [1, K]
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) {
            const int i = hm.l0 + ii;
            hm.lob[ii].lam *= inv;
            float th, ph;
            decode_lobe_fast(cfg.kappa_act, raw[4 * i + 1], raw[4 * i + 2], raw[4 * i + 3], hm.lob[ii],
                        &th, &ph);
            hm.cn[ii] = vmf_scaled_norm_fast(hm.lob[ii].kap);
            if (mix_out && valid) {
                mix_out[(4 * i + 0) * ld + j] = hm.lob[ii].lam;
                mix_out[(4 * i + 1) * ld + j] = hm.lob[ii].kap;
                mix_out[(4 * i + 2) * ld + j] = th;
                mix_out[(4 * i + 3) * ld + j] = ph;
            }
        }
}

template <int KH>
__device__ __forceinline__ float half_pdf(const HalfMix<KH>& hm, const float w[3]) {
    float pv = 0.0f;
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) pv += hm.lob[ii].lam * vmf_eval_fast(hm.lob[ii], hm.cn[ii], w[0], w[1], w[2]);
    return pv + __shfl_xor_sync(kFull, pv, 1);
}

// log V at w (Eq. 4 in log-sum-exp form): the log of each lobe's term,
// log lambda_i + log c(kappa_i) + kappa_i (mu_i.w - 1), with log lambda_i
// taken from the logits so that it stays finite where lambda_i underflows.
template <int KH>
__device__ __forceinline__ float half_log_pdf(const HalfMix<KH>& hm, const float* raw, const float w[3]) {
    const float lnorm = hm.mx + __logf(hm.ssum);
    float a[KH];
    float m = -INFINITY;
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) {
            const Lobe& L = hm.lob[ii];
            const float d = L.mu[0] * w[0] + L.mu[1] * w[1] + L.mu[2] * w[2];
            a[ii] = (raw[4 * (hm.l0 + ii)] - lnorm) + __logf(hm.cn[ii]) + L.kap * (d - 1.0f);
            m = fmaxf(m, a[ii]);
        }
    m = fmaxf(m, __shfl_xor_sync(kFull, m, 1));
    float s = 0.0f;
#pragma unroll
    for (int ii = 0; ii < KH; ++ii)
        if (ii < hm.cnt) s += __expf(a[ii] - m);
    s += __shfl_xor_sync(kFull, s, 1);
    return m + __logf(s);
}

template <bool SAMPLE, int KH>
__device__ __forceinline__ void epilogue_tile(int t, const DevCfg& cfg, const float* act, int AS,
                                              int64_t base, int64_t n, int64_t ld,
                                              const float* __restrict__ uin, float ufrac,
                                              float* __restrict__ dir_out,
                                              float* __restrict__ pdf_out,
                                              float* __restrict__ mix_out, bool log_pdf = false) {
    const int q = t >> 1, half = t & 1;
    const int64_t j = base + q;
    const bool valid = j < n;
    const float* raw = act + q * AS;
    HalfMix<KH> hm;
    decode_half(cfg, raw, half, hm, mix_out, ld, j, valid);
    float w[3];
    bool uni = false;
    if (SAMPLE) {
        float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
        if (valid) {
            u0 = uin[j];
            u1 = uin[ld + j];
            u2 = uin[2 * ld + j];
            uni = ufrac > 0.0f && uin[3 * ld + j] < ufrac;
        }
        // Lobe choice: smallest i with u0 < lambda_0 + ... + lambda_i, the
        // cumulative sum taken in lobe order: half 0 sums its lobes from 0,
        // half 1 continues from half 0's total.
        float run = 0.0f;
        int sel = -1;
        if (half == 0) {
#pragma unroll
            for (int ii = 0; ii < KH; ++ii)
                if (ii < hm.cnt) {
                    run += hm.lob[ii].lam;
                    if (sel < 0 && u0 < run) sel = ii;
                }
        }
        const float tot0 = __shfl_xor_sync(kFull, run, 1);
        if (half == 1) {
            float cum = tot0;
#pragma unroll
            for (int ii = 0; ii < KH; ++ii)
                if (ii < hm.cnt) {
                    cum += hm.lob[ii].lam;
                    if (sel < 0 && u0 < cum) sel = ii;
                }
        }
        const int osel = __shfl_xor_sync(kFull, sel, 1);
        const int sel0 = half ? osel : sel, sel1 = half ? sel : osel;
        const int kh = (cfg.K + 1) >> 1;
        int owner, lidx;
        if (sel0 >= 0) {
            owner = 0;
            lidx = sel0;
        } else if (sel1 >= 0) {
            owner = 1;
            lidx = sel1;
        } else {
            const int last = cfg.K - 1;
            owner = last >= kh ? 1 : 0;
            lidx = last - owner * kh;
        }
        float d[3] = {0.0f, 0.0f, 1.0f};
        if (half == owner) {
            if (uni) {
                uniform_sphere(u1, u2, d);
            } else {
                Lobe sl = hm.lob[0];
#pragma unroll
                for (int ii = 1; ii < KH; ++ii)
                    if (ii == lidx) sl = hm.lob[ii];
                vmf_sample(sl, u1, u2, d);
            }
        }
        const int src = (threadIdx.x & 31 & ~1) | owner;
#pragma unroll
        for (int a = 0; a < 3; ++a) w[a] = __shfl_sync(kFull, d[a], src);
    } else {
        w[0] = w[1] = 0.0f;
        w[2] = 1.0f;
        if (valid) {
            w[0] = uin[j];
            w[1] = uin[ld + j];
            w[2] = uin[2 * ld + j];
        }
    }
    float pv;
    if (!SAMPLE && log_pdf) {
        pv = half_log_pdf(hm, raw, w);
    } else {
        pv = half_pdf(hm, w);
        if (SAMPLE && ufrac > 0.0f) pv = ufrac * kInv4Pi + (1.0f - ufrac) * pv;
    }
    if (valid) {
        if (half == 0) {
            if (SAMPLE) {
                dir_out[j] = w[0];
                dir_out[ld + j] = w[1];
                dir_out[2 * ld + j] = w[2];
            }
        } else {
            pdf_out[j] = pv;
        }
    }
}

// ------------------------------------------------------ forward kernel

// One CTA per SM holds G tile groups of 128 threads. The groups share one
// copy of the weights in shared memory and each walks its own 64-query tiles
// with its own activation buffers and named barrier.
template <bool SAMPLE, int NIMAX, int KH>
__global__ void __launch_bounds__(fwd_max_groups(NIMAX) * kNT, 1) k_forward_fp32(const __grid_constant__ DevCfg cfg,
                                                         const float* __restrict__ grid,
                                                         const float* __restrict__ wfwd,
                                                         const __grid_constant__ QueryBatch qb) {
    extern __shared__ float4 smem4[];
    float* sW = reinterpret_cast<float*>(smem4);
    constexpr int AS = fwd_act_stride(NIMAX);
    const int G = blockDim.x / kNT;
    const int group = threadIdx.x / kNT;
    const int t = threadIdx.x % kNT;
    float* act = sW + cfg.fwd_floats + group * kTQ * AS;  // one tile, layers in place
    for (int i = threadIdx.x; i < cfg.fwd_floats / 4; i += blockDim.x)
        smem4[i] = __ldg(reinterpret_cast<const float4*>(wfwd) + i);
    __syncthreads();
    int64_t total = qb.total_tiles, n0 = qb.seg[0].n;
    if (qb.n_dev) {
        n0 = *qb.n_dev;
        total = (n0 + kTQ - 1) / kTQ;
    }
    for (int64_t tile = (int64_t)blockIdx.x * G + group; tile < total; tile += (int64_t)gridDim.x * G) {
        int s = 0;
        while (s + 1 < qb.nseg && tile >= qb.seg[s + 1].tile0) ++s;
        const QuerySeg& S = qb.seg[s];
        const int64_t n = (s == 0 && qb.n_dev) ? n0 : S.n;
        const int64_t base = (tile - S.tile0) * kTQ;
        encode_tile<(NIMAX >= 4)>(t, cfg, grid, base, n, S.ld, S.pos, S.aux, act, AS);
        group_sync(group);
        // Bring the next tile's positions and this tile's uniforms into L2
        // while the MLP runs (one thread per 32 consecutive queries).
        if ((t & 31) == 0 && t < 2 * kTQ) {
            const int row = t >> 5;  // 0..3: u rows 0..2 of this tile, pos of the next
            if (row < 3) {
                const int64_t jj = base + (t & (kTQ - 1));
                if (jj < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(S.uin + row * S.ld + jj));
            } else {
                const int64_t nt = tile + (int64_t)gridDim.x * G;
                if (nt < total) {
                    int s2 = s;
                    while (s2 + 1 < qb.nseg && nt >= qb.seg[s2 + 1].tile0) ++s2;
                    const QuerySeg& S2 = qb.seg[s2];
                    const int64_t b2 = (nt - S2.tile0) * kTQ;
                    for (int r = 0; r < 3; ++r) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(S2.pos + r * S2.ld + b2));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(S2.pos + r * S2.ld + b2 + 32));
                    }
                }
            }
        }
        for (int l = 0; l < cfg.n_layers; ++l) {
            const bool last = l == cfg.n_layers - 1;
            layer<NIMAX, AS, true>(t, act, AS, cfg.widths[l], sW + cfg.off_fwd[l], cfg.np_fwd[l], act,
                                   cfg.widths[l + 1], last ? 0 : 1, nullptr, group);
            group_sync(group);
        }
        epilogue_tile<SAMPLE, KH>(t, cfg, act, AS, base, n, S.ld, S.uin, S.ufrac, S.dir, S.pdf, S.mix,
                                      qb.log_pdf != 0);
        group_sync(group);
    }
}

// ------------------------------------- warp-specialised forward kernel

// mbarrier primitives (CTA scope). Waits are bounded: false after `limit`
// SM clock cycles (2^31 by default, about a second), so a broken hand-off
// ends the kernel with an error status instead of hanging it. limit <= 0
// makes the wait one non-blocking test.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void fbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool fbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    if (limit <= 0) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    }
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        // sleeps in the barrier until the phase completes or ~20 us pass
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// AND of p over the 128 threads of tile group `group` (its named barrier);
// also orders their memory accesses like group_sync.
__device__ __forceinline__ bool group_all(int group, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, r;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred r, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, r;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(group + 1), "r"(kNT)
        : "memory");
    return r != 0;
}

// Row stride (floats) of an encoded tile: the network input width rounded
// up to 4, plus 4 (the float4 row reads of the first layer stay aligned).
__host__ __device__ constexpr int enc_stride(int w0) { return (w0 + 3) / 4 * 4 + 4; }

// Producer / consumer form of the fused forward pass. The CTA (one per SM)
// holds 1 + GC tile groups of 128 threads sharing the weights in shared
// memory. Group 0 only encodes: it walks the CTA's tiles in order, gathers
// and blends the grid corners of each (Sec. 5.1, Eq. 11; plus the
// product-mode encodings) and leaves the encoded tile in the mailbox of the
// consumer group that owns it. Consumer group g owns the CTA's tiles
// g, g + GC, g + 2 GC, ...: it runs the MLP (Eq. 12), the first layer
// straight from its mailbox (released as soon as that layer has read it),
// and the vMF epilogue (Table 1, Eq. 3-4, Sec. 5.3). The gathers' L2 latency
// is thus spent by the producer while the consumers keep the FMA pipes busy.
// Hand-offs use one 'full' and one 'empty' mbarrier per mailbox; one thread
// per group waits on it (bounded) and the group's named barrier passes the
// outcome on. A wait that gives up after wait_limit cycles sets
// kStatusTimeout in *status (if given) and every group leaves its loop; the
// kernel issues no asynchronous copies, so nothing is left in flight.
template <bool SAMPLE, int NIMAX, int KH, int GC, int DEPTH>
__global__ void __launch_bounds__((GC + 1) * kNT, 1) k_forward_fp32_ws(const __grid_constant__ DevCfg cfg,
                                                                      const float* __restrict__ grid,
                                                                      const float* __restrict__ wfwd,
                                                                      const __grid_constant__ QueryBatch qb,
                                                                      int* __restrict__ status,
                                                                      long long wait_limit) {
    extern __shared__ float4 smem4[];
    float* sW = reinterpret_cast<float*>(smem4);
    constexpr int AS = fwd_act_stride(NIMAX);
    const int ES = enc_stride(cfg.widths[0]);
    const int group = threadIdx.x / kNT;
    const int t = threadIdx.x % kNT;
    constexpr int NB = GC * DEPTH;          // mailboxes: DEPTH per consumer group
    float* act0 = sW + cfg.fwd_floats;      // GC activation tiles
    float* box0 = act0 + GC * kTQ * AS;     // NB mailboxes (encoded tiles)
    uint64_t* bars = reinterpret_cast<uint64_t*>(box0 + NB * kTQ * ES);  // full[NB], empty[NB]
    for (int i = threadIdx.x; i < cfg.fwd_floats / 4; i += blockDim.x)
        smem4[i] = __ldg(reinterpret_cast<const float4*>(wfwd) + i);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2 * NB; ++b) fbar_init(smem_addr(&bars[b]), 1);
    }
    __syncthreads();
    int64_t total = qb.total_tiles, n0 = qb.seg[0].n;
    if (qb.n_dev) {
        n0 = *qb.n_dev;
        total = (n0 + kTQ - 1) / kTQ;
    }
    bool ok = true;
    if (group == 0) {
        // Producer: tile k of this CTA goes to mailbox k % NB.
        for (int64_t k = 0; ok; ++k) {
            const int64_t tile = blockIdx.x + k * gridDim.x;
            if (tile >= total) break;
            const int b = (int)(k % NB);
            const uint32_t use = (uint32_t)(k / NB);
            // the mailbox's previous tile (if any) has been read
            bool w = true;
            if (t == 0) w = fbar_wait(smem_addr(&bars[NB + b]), (use & 1u) ^ 1u, wait_limit);
            ok = group_all(0, w);
            if (!ok) break;
            int sg = 0;
            while (sg + 1 < qb.nseg && tile >= qb.seg[sg + 1].tile0) ++sg;
            const QuerySeg& S = qb.seg[sg];
            const int64_t n = (sg == 0 && qb.n_dev) ? n0 : S.n;
            const int64_t base = (tile - S.tile0) * kTQ;
            // four levels' loads in flight where the registers allow (GC <= 3)
            encode_tile<(GC <= 3)>(t, cfg, grid, base, n, S.ld, S.pos, S.aux, box0 + b * kTQ * ES, ES);
            // positions of the CTA's next tile into L2
            if ((t & 31) == 0 && t < 2 * kTQ) {
                const int64_t nt = tile + gridDim.x;
                if (nt < total) {
                    int s2 = sg;
                    while (s2 + 1 < qb.nseg && nt >= qb.seg[s2 + 1].tile0) ++s2;
                    const QuerySeg& S2 = qb.seg[s2];
                    const int64_t b2 = (nt - S2.tile0) * kTQ + (t >> 5) * 16;
                    for (int r = 0; r < 3; ++r)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(S2.pos + r * S2.ld + b2));
                }
            }
            group_sync(0);
            if (t == 0) fbar_arrive(smem_addr(&bars[b]));
        }
    } else {
        const int g = group - 1;
        float* act = act0 + g * kTQ * AS;
        for (int64_t i = 0; ok; ++i) {
            const int64_t k = g + i * GC;
            const int64_t tile = blockIdx.x + k * gridDim.x;
            if (tile >= total) break;
            const int b = (int)(k % NB);
            const float* box = box0 + b * kTQ * ES;
            bool w = true;
            if (t == 0) w = fbar_wait(smem_addr(&bars[b]), (uint32_t)((k / NB) & 1), wait_limit);
            ok = group_all(group, w);
            if (!ok) break;
            int sg = 0;
            while (sg + 1 < qb.nseg && tile >= qb.seg[sg + 1].tile0) ++sg;
            const QuerySeg& S = qb.seg[sg];
            const int64_t n = (sg == 0 && qb.n_dev) ? n0 : S.n;
            const int64_t base = (tile - S.tile0) * kTQ;
            // this tile's uniforms (or directions) into L2 for the epilogue
            if ((t & 31) == 0 && t < 3 * 32) {
                const int64_t jj = base + (t & (kTQ - 1));
                if (jj < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(S.uin + (t >> 5) * S.ld + jj));
            }
            const bool one = cfg.n_layers == 1;
            layer<NIMAX, 0, false, AS>(t, box, ES, cfg.widths[0], sW + cfg.off_fwd[0], cfg.np_fwd[0], act,
                                   cfg.widths[1], one ? 0 : 1, nullptr, group);
            group_sync(group);
            if (t == 0) fbar_arrive(smem_addr(&bars[NB + b]));  // mailbox read
            for (int l = 1; l < cfg.n_layers; ++l) {
                const bool last = l == cfg.n_layers - 1;
                layer<NIMAX, AS, true>(t, act, AS, cfg.widths[l], sW + cfg.off_fwd[l], cfg.np_fwd[l], act,
                                       cfg.widths[l + 1], last ? 0 : 1, nullptr, group);
                group_sync(group);
            }
            epilogue_tile<SAMPLE, KH>(t, cfg, act, AS, base, n, S.ld, S.uin, S.ufrac, S.dir, S.pdf, S.mix,
                                      qb.log_pdf != 0);
            group_sync(group);
        }
    }
    if (!ok && t == 0 && status) atomicOr(status, kStatusTimeout);
}

// ------------------------------------------------------ training kernel

// Per query: raw outputs -> d(sum_j s_j log V_j)/d raw, written in place,
// and s_j log V_j accumulated into *loss. Log-domain mixture so that log V
// and the responsibilities r_i stay finite when V underflows FP32.
__device__ __forceinline__ void grad_epilogue(const DevCfg& cfg, float* act, int AS, int64_t base,
                                              int64_t n, int64_t ld,
                                              const float* __restrict__ dir,
                                              const float* __restrict__ rad,
                                              const float* __restrict__ spdf,
                                              const float* __restrict__ dlogv, float inv_n,
                                              float* __restrict__ loss) {
    const int t = threadIdx.x;
    const int q = t >> 1, half = t & 1;
    const int64_t j = base + q;
    const bool valid = j < n;
    float* raw = act + q * AS;
    const int K = cfg.K, KH = (K + 1) >> 1;
    const int l0 = half * KH, cnt = min(K, l0 + KH) - l0;
    float w[3] = {0.0f, 0.0f, 1.0f};
    float s = 0.0f;
    if (valid) {
        w[0] = dir[j];
        w[1] = dir[ld + j];
        w[2] = dir[2 * ld + j];
        s = dlogv ? dlogv[j] : -(rad[j] / spdf[j]) * inv_n;
    }
    constexpr int H = NPM_MAX_LOBES / 2;
    float lp[H], a[H], kap[H], md[H], wdt[H], wdp[H], sk[H], st[H], sp[H];
    float mx = -INFINITY;
#pragma unroll
    for (int ii = 0; ii < H; ++ii)
        if (ii < cnt) mx = fmaxf(mx, raw[4 * (l0 + ii)]);
    mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 1));
    float ssum = 0.0f;
#pragma unroll
    for (int ii = 0; ii < H; ++ii)
        if (ii < cnt) ssum += expf(raw[4 * (l0 + ii)] - mx);
    ssum += __shfl_xor_sync(kFull, ssum, 1);
    const float lse = mx + logf(ssum);
    float amax = -INFINITY;
#pragma unroll
    for (int ii = 0; ii < H; ++ii)
        if (ii < cnt) {
            const int i = l0 + ii;
            lp[ii] = raw[4 * i] - lse;  // log lambda_i
            const float rk = raw[4 * i + 1];
            if (cfg.kappa_act == NPM_EXP) {
                kap[ii] = expf(rk);
                sk[ii] = kap[ii];
            } else {
                kap[ii] = softplus(rk);
                sk[ii] = logistic(rk);
            }
            st[ii] = logistic(raw[4 * i + 2]);
            sp[ii] = logistic(raw[4 * i + 3]);
            float sth, cth, sph, cph;
            sincosf(kPi * st[ii], &sth, &cth);
            sincosf(2.0f * kPi * sp[ii], &sph, &cph);
            md[ii] = sth * cph * w[0] + sth * sph * w[1] + cth * w[2];
            wdt[ii] = cth * cph * w[0] + cth * sph * w[1] - sth * w[2];
            wdp[ii] = -sth * sph * w[0] + sth * cph * w[1];
            a[ii] = lp[ii] + logf(vmf_scaled_norm(kap[ii])) + kap[ii] * (md[ii] - 1.0f);
            amax = fmaxf(amax, a[ii]);
        }
    amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, 1));
    float es = 0.0f;
#pragma unroll
    for (int ii = 0; ii < H; ++ii)
        if (ii < cnt) es += expf(a[ii] - amax);
    es += __shfl_xor_sync(kFull, es, 1);
    const float logV = amax + logf(es);
#pragma unroll
    for (int ii = 0; ii < H; ++ii)
        if (ii < cnt) {
            const int i = l0 + ii;
            const float r = expf(a[ii] - logV);
            const float lam = expf(lp[ii]);
            const float sr = s * r;
            raw[4 * i + 0] = s * (r - lam);
            raw[4 * i + 1] = sr * (inv_minus_coth(kap[ii]) + md[ii]) * sk[ii];
            raw[4 * i + 2] = sr * kap[ii] * wdt[ii] * kPi * st[ii] * (1.0f - st[ii]);
            raw[4 * i + 3] = sr * kap[ii] * wdp[ii] * 2.0f * kPi * sp[ii] * (1.0f - sp[ii]);
        }
    // Zero the padding columns of the raw buffer (4K == widths[n_layers], so
    // nothing to do) and accumulate the loss once per query.
    float lv = (valid && half == 0) ? s * logV : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(kFull, lv, o);
    if ((threadIdx.x & 31) == 0 && lv != 0.0f) atomicAdd(loss, lv);
}

// dW[n][k] += sum_q dl[q][n] * h[q][k] (global atomics).
__device__ __forceinline__ void weight_grad(const float* dl, const float* h, int AS, int N, int K,
                                            float* __restrict__ gW) {
    const int t = threadIdx.x;
    const int a = t >> 4, b = t & 15;
    for (int n0 = a * 8; n0 < N; n0 += 64)
        for (int k0 = b * 4; k0 < K; k0 += 64) {
            float acc[8][4];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
            const bool two = n0 + 4 < N;
            for (int q = 0; q < kTQ; ++q) {
                const float4 hv = *reinterpret_cast<const float4*>(h + q * AS + k0);
                const float4 d0 = *reinterpret_cast<const float4*>(dl + q * AS + n0);
                float4 d1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (two) d1 = *reinterpret_cast<const float4*>(dl + q * AS + n0 + 4);
                const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
                const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(dv[r], hh[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (n0 + r < N) {
                    float* dst = gW + (size_t)(n0 + r) * K + k0;
                    atomicAdd(reinterpret_cast<float4*>(dst),
                              make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
                }
        }
}

// Grid gradient: dV_l[corner] += weight * dG_l (Eq. 11 transposed).
__device__ __forceinline__ void grid_scatter(const DevCfg& cfg, const float* denc, int AS,
                                             int64_t base, int64_t n, int64_t ld,
                                             const float* __restrict__ pos,
                                             float* __restrict__ ggrid) {
    const int t = threadIdx.x;
    const int q = t & (kTQ - 1), part = t >> 6;
    const int64_t j = base + q;
    if (j >= n) return;
    const float x = pos[j], y = pos[ld + j], z = pos[2 * ld + j];
    const float* row = denc + q * AS;
    const int F = cfg.feat;
    for (int l = part; l < cfg.n_levels; l += 2) {
        const Cell cl = make_cell(x, y, z, cfg.level_res[l]);
        float* gl = ggrid + (size_t)cfg.level_off[l] * F;
        const float* dg = row + l * F;
        uint32_t idx[8];
        float ws[8];
        corners8(cfg, l, cl, idx, ws);
        if (F == 2) {
#pragma unroll
            for (int c = 0; c < 8; c += 2)
                scatter_pair2(gl, cfg.level_off[l], idx[c], idx[c + 1], ws[c], ws[c + 1], dg[0], dg[1]);
            continue;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float w = ws[c];
            float* e = gl + (size_t)idx[c] * F;
            if (F == 4) {
                atomicAdd(reinterpret_cast<float4*>(e),
                          make_float4(w * dg[0], w * dg[1], w * dg[2], w * dg[3]));
            } else {
                for (int f = 0; f < F; ++f) atomicAdd(e + f, w * dg[f]);
            }
        }
    }
}

__global__ void __launch_bounds__(kNT) k_train_fp32(DevCfg cfg, const float* __restrict__ params,
                                                    int64_t mlp_off,
                                                    const float* __restrict__ wfwd,
                                                    const float* __restrict__ wbwd, int64_t n,
                                                    int64_t ld, const float* __restrict__ pos,
                                                    const float* __restrict__ aux,
                                                    const float* __restrict__ dir,
                                                    const float* __restrict__ rad,
                                                    const float* __restrict__ spdf,
                                                    const float* __restrict__ dlogv, float inv_n,
                                                    float* __restrict__ grad,
                                                    float* __restrict__ loss) {
    extern __shared__ float4 smem4[];
    float* sW = reinterpret_cast<float*>(smem4);
    const int AS = cfg.max_width + 4;
    const int L = cfg.n_layers;
    float* buf0 = sW + cfg.fwd_floats;  // L + 2 activation buffers
    auto buf = [&](int i) { return buf0 + i * kTQ * AS; };
    for (int i = threadIdx.x; i < cfg.fwd_floats / 4; i += kNT)
        smem4[i] = __ldg(reinterpret_cast<const float4*>(wfwd) + i);
    __syncthreads();
    const int64_t ntiles = (n + kTQ - 1) / kTQ;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kTQ;
        encode_tile<false>(threadIdx.x, cfg, params, base, n, ld, pos, aux, buf(0), AS);
        __syncthreads();
        for (int l = 0; l < L; ++l) {
            layer<8>(threadIdx.x, buf(l), AS, cfg.widths[l], sW + cfg.off_fwd[l], cfg.np_fwd[l],
                     buf(l + 1), cfg.widths[l + 1], l == L - 1 ? 0 : 1, nullptr);
            __syncthreads();
        }
        grad_epilogue(cfg, buf(L), AS, base, n, ld, dir, rad, spdf, dlogv, inv_n, loss);
        __syncthreads();
        // Backward: delta_L lives in buf(L); delta_{L-1} in buf(L+1);
        // delta_{i-1} (i < L) overwrites buf(i), whose activations are spent.
        float* dcur = buf(L);
        for (int i = L; i >= 1; --i) {
            const int N = cfg.widths[i], Kw = cfg.widths[i - 1];
            float* h = buf(i - 1);
            // Offset of W_i inside the packed MLP region.
            int64_t woff = 0;
            for (int m = 0; m < i - 1; ++m) woff += (int64_t)cfg.widths[m] * cfg.widths[m + 1];
            weight_grad(dcur, h, AS, N, Kw, grad + mlp_off + woff);
            float* dnext = (i == L) ? buf(L + 1) : buf(i);
            layer<8>(threadIdx.x, dcur, AS, N, wbwd + cfg.off_bwd[i - 1], cfg.np_bwd[i - 1], dnext,
                     Kw, i > 1 ? 2 : 0, h);
            __syncthreads();
            dcur = dnext;
        }
        grid_scatter(cfg, dcur, AS, base, n, ld, pos, grad);
        __syncthreads();
    }
}

// ------------------------------------------------------- utility kernels

// Arrange the MLP weights (row-major [out][in] per layer, packed) into the
// padded forward (W^T [in][np_fwd]) and backward (W [out][np_bwd]) blobs.
__global__ void k_arrange_weights(DevCfg cfg, const float* __restrict__ mlp,
                                  float* __restrict__ wfwd, float* __restrict__ wbwd) {
    int64_t woff = 0;
    for (int l = 0; l < cfg.n_layers; ++l) {
        const int K = cfg.widths[l], N = cfg.widths[l + 1];
        const int npf = cfg.np_fwd[l], npb = cfg.np_bwd[l];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * npf; i += gridDim.x * blockDim.x) {
            const int k = i / npf, nn = i % npf;
            wfwd[cfg.off_fwd[l] + i] = nn < N ? mlp[woff + (int64_t)nn * K + k] : 0.0f;
        }
        if (wbwd)  // backward copy (training only)
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * npb; i += gridDim.x * blockDim.x) {
                const int nn = i / npb, k = i % npb;
                wbwd[cfg.off_bwd[l] + i] = k < K ? mlp[woff + (int64_t)nn * K + k] : 0.0f;
            }
        woff += (int64_t)K * N;
    }
}

// Dense Adam with bias correction (Kingma and Ba) at step t = *steps + 1,
// c1 = 1 - b1^t, c2 = 1 - b2^t; the step count lives in device memory so that
// captured graphs replay correctly (k_step_done advances it afterwards).
// Skips the update when *loss is not finite and flags it. Clears the
// gradient. Optionally refreshes an FP16 copy of the first n_half parameters
// (the grid). With ema set, also the exponential moving average
// e <- d e + (1 - d) p of the updated parameters that inference evaluates
// (Sec. 5.3); the FP16 copy (inference only) is then taken from e.
__global__ void k_adam(int64_t n4, float4* __restrict__ p, float4* __restrict__ g,
                       float4* __restrict__ m, float4* __restrict__ v, float lr, float b1, float b2,
                       float eps, const int* __restrict__ steps, const float* __restrict__ loss,
                       int* __restrict__ status, __half2* __restrict__ half_copy, int64_t n_half,
                       float4* __restrict__ ema, float ema_decay) {
    const bool skip = loss != nullptr && !isfinite(*loss);
    if (skip && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusNumeric);
    const float t = (float)(*steps + 1);
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    // Two float4 groups per thread and iteration: more bytes in flight.
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n4; i0 += 2 * stride) {
        float4 gg[2], mm[2], vv[2], pp[2];
        bool in[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = i0 + u * stride;
            in[u] = i < n4;
            if (in[u]) {
                gg[u] = g[i];
                mm[u] = m[i];
                vv[u] = v[i];
                pp[u] = p[i];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = i0 + u * stride;
            if (!in[u]) continue;
            g[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (skip) continue;
            float* pm = &mm[u].x;
            float* pv = &vv[u].x;
            const float* pg = &gg[u].x;
            float* pq = &pp[u].x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                pm[c] = b1 * pm[c] + (1.0f - b1) * pg[c];
                pv[c] = b2 * pv[c] + (1.0f - b2) * pg[c] * pg[c];
                const float mh = pm[c] / c1, vh = pv[c] / c2;
                pq[c] -= lr * mh / (sqrtf(vh) + eps);
            }
            m[i] = mm[u];
            v[i] = vv[u];
            p[i] = pp[u];
            float4 inf = pp[u];
            if (ema) {
                float4 e = ema[i];
                const float d = ema_decay, d1 = 1.0f - ema_decay;
                e.x = d * e.x + d1 * pp[u].x;
                e.y = d * e.y + d1 * pp[u].y;
                e.z = d * e.z + d1 * pp[u].z;
                e.w = d * e.w + d1 * pp[u].w;
                ema[i] = e;
                inf = e;
            }
            if (half_copy && 4 * i < n_half) {
                if (4 * i + 4 <= n_half) {
                    half_copy[2 * i] = __floats2half2_rn(inf.x, inf.y);
                    half_copy[2 * i + 1] = __floats2half2_rn(inf.z, inf.w);
                } else {
                    // The copy's last entries (n_half not a multiple of 4).
                    __half* hc = reinterpret_cast<__half*>(half_copy) + 4 * i;
                    const float iv[4] = {inf.x, inf.y, inf.z, inf.w};
                    for (int c = 0; c < (int)(n_half - 4 * i); ++c) hc[c] = __float2half_rn(iv[c]);
                }
            }
        }
    }
}

__global__ void k_step_done(int* steps) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *steps += 1;
}

__global__ void k_grid_indices(DevCfg cfg, int64_t n, int64_t ld, const float* __restrict__ pos,
                               int32_t* __restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float x = pos[j], y = pos[ld + j], z = pos[2 * ld + j];
        for (int l = 0; l < cfg.n_levels; ++l) {
            const Cell cl = make_cell(x, y, z, cfg.level_res[l]);
            uint32_t idx[8];
            float w[8];
            corners8(cfg, l, cl, idx, w);  // the routine every encoder and scatter uses
#pragma unroll
            for (int c = 0; c < 8; ++c) out[((int64_t)l * 8 + c) * n + j] = (int32_t)idx[c];
        }
    }
}

__global__ void k_to_half(int64_t n, const float* __restrict__ src, __half* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

__global__ void k_copy_loss(const float* __restrict__ acc, float* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = *acc;
}

// ----------------------------------------------------------- launchers


size_t train_smem_bytes(const DevCfg& c) {
    return sizeof(float) *
           ((size_t)c.fwd_floats + (size_t)(c.n_layers + 2) * kTQ * (c.max_width + 4));
}

static int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    }
    return cached;
}

template <typename KernelT>
static int persistent_grid(KernelT kern, size_t smem, int64_t ntiles) {
    int per_sm = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)per_sm * sm_count();
    if (g > ntiles) g = ntiles;
    return (int)(g < 1 ? 1 : g);
}

// Shared-memory carveout (percent of the 228 KB maximum) that holds `bytes`.
int carveout_percent(size_t bytes) {
    const size_t max_smem = 228 * 1024;
    int pct = (int)((bytes * 100 + max_smem - 1) / max_smem);
    return pct < 1 ? 1 : pct > 100 ? 100 : pct;
}

// Template instance (register tile of the widest layer, lobes per half).
static int fp32_instance(const DevCfg& cfg) {
    int need = 1;
    for (int l = 0; l < cfg.n_layers; ++l) need = cfg.np_fwd[l] / 16 > need ? cfg.np_fwd[l] / 16 : need;
    // the activation rows (stride fwd_act_stride(I)) hold every width
    const int mw = (cfg.max_width + 15) / 16;
    need = mw > need ? mw : need;
    const int kh = (cfg.K + 1) / 2;
    need = kh > need ? kh : need;
    return need <= 2 ? 2 : need <= 4 ? 4 : 8;
}

// Shared memory of a one-group CTA: weights and one activation tile.
size_t fwd_smem_bytes(const DevCfg& c) {
    return sizeof(float) * ((size_t)c.fwd_floats + (size_t)kTQ * fwd_act_stride(fp32_instance(c)));
}

template <bool SAMPLE, int I>
static cudaError_t launch_fwd_inst(const DevCfg& cfg, const float* grid, const float* wfwd,
                                   const QueryBatch& qb, int64_t tiles_hint, cudaStream_t st) {
    auto kern = k_forward_fp32<SAMPLE, I, I>;
    const size_t wbytes = sizeof(float) * (size_t)cfg.fwd_floats;
    const size_t gbytes = sizeof(float) * (size_t)kTQ * fwd_act_stride(I);
    int G = (int)((227 * 1024 - wbytes) / gbytes);
    if (G > fwd_max_groups(I)) G = fwd_max_groups(I);
    // Tuning override (groups per CTA) for launch-configuration sweeps.
    static std::atomic<int> env_groups{INT32_MIN + 1};
    const int og = env_override("NPM_FP32_GROUPS", env_groups);
    if (og >= 1 && og < G) G = og;
    if (G < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = wbytes + G * gbytes;
    // Carve out only the shared memory this CTA needs; the rest of the
    // 256 KB stays L1 for the grid gathers.
    static std::atomic<uint64_t> attrs{~0ull};
    cudaError_t e = set_smem_attrs(kern, smem, carveout_percent(smem + 1024), attrs);
    if (e != cudaSuccess) return e;
    int64_t g = sm_count();
    const int64_t need = (tiles_hint + G - 1) / G;
    if (need < g) g = need < 1 ? 1 : need;
    kern<<<(int)g, G * kNT, smem, st>>>(cfg, grid, wfwd, qb);
    return cudaGetLastError();
}

// Mailboxes per consumer group of the warp-specialised kernel.
constexpr int kWsDepth = 2;

// Shared memory of the warp-specialised kernel with GC consumer groups:
// weights, GC activation tiles, GC * kWsDepth mailboxes and two mbarriers
// per mailbox.
static size_t ws_smem_bytes(const DevCfg& cfg, int I, int GC) {
    const size_t nb = (size_t)GC * kWsDepth;
    return sizeof(float) * ((size_t)cfg.fwd_floats + (size_t)GC * kTQ * fwd_act_stride(I) +
                            nb * kTQ * enc_stride(cfg.widths[0])) +
           2 * nb * sizeof(uint64_t);
}

template <bool SAMPLE, int GC>
static cudaError_t launch_fwd_ws(const DevCfg& cfg, const float* grid, const float* wfwd,
                                 const QueryBatch& qb, int64_t tiles_hint, int* status, long long wait_limit,
                                 cudaStream_t st) {
    auto kern = k_forward_fp32_ws<SAMPLE, 4, 4, GC, kWsDepth>;
    const size_t smem = ws_smem_bytes(cfg, 4, GC);
    static std::atomic<uint64_t> attrs{~0ull};
    cudaError_t e = set_smem_attrs(kern, smem, carveout_percent(smem + 1024), attrs);
    if (e != cudaSuccess) return e;
    int64_t g = sm_count();
    const int64_t need = (tiles_hint + GC - 1) / GC;
    if (need < g) g = need < 1 ? 1 : need;
    kern<<<(int)g, (GC + 1) * kNT, smem, st>>>(cfg, grid, wfwd, qb, status, wait_limit);
    return cudaGetLastError();
}

// Consumer groups of the warp-specialised kernel for this model, or 0 for
// the tile-group kernel. It serves the instance with 64-wide register tiles
// and at most 8 lobes whose buffers fit (the paper-shaped networks).
// NPM_FP32_WS (0, 3 or 4) overrides the choice for launch sweeps.
static int ws_groups(const DevCfg& cfg, int inst) {
    // three consumer groups at 128 registers beat four at 96 (measured)
    static std::atomic<int> env_ws{INT32_MIN + 1};
    const int ov = env_override("NPM_FP32_WS", env_ws);
    const int gc = ov == INT32_MIN ? 3 : ov;
    if (gc != 3 && gc != 4) return 0;
    if (inst != 4 || (cfg.K + 1) / 2 > 4) return 0;
    if (ws_smem_bytes(cfg, 4, gc) > 227 * 1024) return 0;
    return gc;
}

cudaError_t launch_forward_fp32_batch(const DevCfg& cfg, const float* grid, const float* wfwd,
                                      QueryBatch& qb, int64_t max_n, cudaStream_t st, int* status,
                                      long long wait_limit, bool wait_free) {
    int64_t t0 = 0;
    for (int s = 0; s < qb.nseg; ++s) {
        qb.seg[s].tile0 = t0;
        t0 += (qb.seg[s].n + kTQ - 1) / kTQ;
    }
    qb.total_tiles = t0;
    const int64_t hint = qb.n_dev ? (max_n + kTQ - 1) / kTQ : t0;
    const int inst = fp32_instance(cfg);
    const int gc = wait_free ? 0 : ws_groups(cfg, inst);
    if (gc == 4)
        return qb.sample ? launch_fwd_ws<true, 4>(cfg, grid, wfwd, qb, hint, status, wait_limit, st)
                         : launch_fwd_ws<false, 4>(cfg, grid, wfwd, qb, hint, status, wait_limit, st);
    if (gc == 3)
        return qb.sample ? launch_fwd_ws<true, 3>(cfg, grid, wfwd, qb, hint, status, wait_limit, st)
                         : launch_fwd_ws<false, 3>(cfg, grid, wfwd, qb, hint, status, wait_limit, st);
    if (qb.sample) {
        if (inst == 2) return launch_fwd_inst<true, 2>(cfg, grid, wfwd, qb, hint, st);
        if (inst == 4) return launch_fwd_inst<true, 4>(cfg, grid, wfwd, qb, hint, st);
        return launch_fwd_inst<true, 8>(cfg, grid, wfwd, qb, hint, st);
    }
    if (inst == 2) return launch_fwd_inst<false, 2>(cfg, grid, wfwd, qb, hint, st);
    if (inst == 4) return launch_fwd_inst<false, 4>(cfg, grid, wfwd, qb, hint, st);
    return launch_fwd_inst<false, 8>(cfg, grid, wfwd, qb, hint, st);
}

cudaError_t launch_forward_fp32(const DevCfg& cfg, const float* grid, const float* wfwd, int64_t n,
                                int64_t ld, const float* pos, const float* aux, const float* uin,
                                float ufrac, bool sample, float* dir_out, float* pdf_out,
                                float* mix_out, cudaStream_t st, int* status, long long wait_limit,
                                bool wait_free, bool log_pdf) {
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
    return launch_forward_fp32_batch(cfg, grid, wfwd, qb, n, st, status, wait_limit, wait_free);
}

cudaError_t launch_train_fp32(const DevCfg& cfg, const float* params, int64_t mlp_off,
                              const float* wfwd, const float* wbwd, int64_t n, int64_t ld,
                              const float* pos, const float* aux, const float* dir,
                              const float* rad, const float* spdf, const float* dlogv,
                              float* grad, float* loss, cudaStream_t st) {
    const size_t smem = train_smem_bytes(cfg);
    const int64_t ntiles = (n + kTQ - 1) / kTQ;
    const int g = persistent_grid(k_train_fp32, smem, ntiles);
    k_train_fp32<<<g, kNT, smem, st>>>(cfg, params, mlp_off, wfwd, wbwd, n, ld, pos, aux, dir, rad,
                                       spdf, dlogv, 1.0f / (float)n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_arrange_weights(const DevCfg& cfg, const float* mlp, float* wfwd, float* wbwd,
                                   cudaStream_t st) {
    k_arrange_weights<<<32, 256, 0, st>>>(cfg, mlp, wfwd, wbwd);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float* p, float* g, float* m, float* v, float lr, float b1,
                        float b2, float eps, int* steps, const float* loss, int* status,
                        __half* half_copy, int64_t n_half, float* ema, float ema_decay,
                        cudaStream_t st) {
    const int64_t n4 = n / 4;
    int grid = (int)((n4 + 255) / 256);
    const int cap = sm_count() * 16;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_adam<<<grid, 256, 0, st>>>(n4, reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(g),
                                 reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), lr, b1,
                                 b2, eps, steps, loss, status,
                                 reinterpret_cast<__half2*>(half_copy), n_half,
                                 reinterpret_cast<float4*>(ema), ema_decay);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_step_done<<<1, 32, 0, st>>>(steps);
    return cudaGetLastError();
}

cudaError_t launch_grid_indices(const DevCfg& cfg, int64_t n, int64_t ld, const float* pos,
                                int32_t* out, cudaStream_t st) {
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_grid_indices<<<grid, 256, 0, st>>>(cfg, n, ld, pos, out);
    return cudaGetLastError();
}

cudaError_t launch_to_half(int64_t n, const float* src, __half* dst, cudaStream_t st) {
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_to_half<<<grid, 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_copy_loss(const float* acc, float* out, cudaStream_t st) {
    k_copy_loss<<<1, 32, 0, st>>>(acc, out);
    return cudaGetLastError();
}

}  // namespace npm
