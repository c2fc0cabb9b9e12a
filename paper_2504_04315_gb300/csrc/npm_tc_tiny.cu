// npm_tc_tiny.cu -- fused tensor-core forward for the small serving networks:
// one dense grid level of 4 FP16 features, three bias-free layers of at most
// 32 outputs (tcgen05.mma on BF16, split BF16 or FP16 operands, FP32
// accumulation in tensor memory) and K = 4 vMF lobes (the reduced-precision
// serving workload).
//
// The general kernel (npm_tc.cu) serves every shape; this one trims the
// per-query instruction count of the shape the serving loop runs, where the
// kernel is bound by instruction issue rather than memory or tensor work:
//   - encode: the level's 8 corners as 8-byte FP16 loads at 32-bit indices,
//     the blend as packed FP32 (two features per instruction);
//   - hidden activations: ReLU and BF16 rounding in one conversion per pair
//     of values (round-to-zero high part, residual rounded to nearest);
//   - decode (Table 1), normaliser, sampling weights and mixture density
//     (Eq. 3-4) on lobe pairs in packed FP32, with the hardware exponential,
//     logarithm, reciprocal, sine and cosine on arguments kept in their
//     accurate ranges; the sampler itself (Sec. 5.3, Jakob's inversion) is
//     the general kernel's vmf_sample_rp.
// Tiles, weights, shared-memory layout and the bounded waits are those of
// the general kernel: thread t owns query t of a 128-query tile and lane t
// of tensor memory; one elected thread issues the MMAs.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <atomic>

#include "npm_handle.h"
#include "npm_kernels.h"
#include "npm_tc.cuh"

namespace npm {
namespace tc {

namespace {

constexpr float kL2E = 1.4426950408889634f;  // log2(e)
constexpr float kLn2 = 0.69314718055994531f;

// Hardware approximations (PTX ex2/lg2/rcp/sin/cos .approx): e^x is
// evaluated as 2^(x log2 e) with the scaling folded into the caller's FMA.
__device__ __forceinline__ float hw_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 ex2x2(float2 x) { return make_float2(hw_ex2(x.x), hw_ex2(x.y)); }
__device__ __forceinline__ float2 rcpx2(float2 x) { return make_float2(hw_rcp(x.x), hw_rcp(x.y)); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ReLU and BF16 rounding of a pair (v0, v1): round-to-zero high parts
// packed (v0 in the low half) and, in split mode, the residuals
// v - hi (exact in FP32, never negative) rounded to nearest. A negative
// value gives zero in both.
__device__ __forceinline__ uint32_t cvt_rz_relu(float v0, float v1) {
    uint32_t d;
    asm("cvt.rz.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}
__device__ __forceinline__ uint32_t cvt_rn_relu(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}
__device__ __forceinline__ uint32_t cvt_rn(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}
// The two BF16 halves of a packed pair as FP32 (low half first).
__device__ __forceinline__ float2 bf16x2_to_f2(uint32_t h) {
    return make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xffff0000u));
}

// Operand formats of the tiny kernel: BF16, BF16 split into high part and
// residual, FP16 (weights FP16 plus an FP16 residual).
enum : int { kOpsBf16 = 0, kOpsBf16x3 = 1, kOpsFp16 = 2 };

__device__ __forceinline__ uint32_t cvt_f16_relu(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.satfinite.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}

template <int OPS>
__device__ __forceinline__ void relu_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    if (OPS == kOpsFp16) {
        hi = cvt_f16_relu(v0, v1);
    } else if (OPS == kOpsBf16x3) {
        hi = cvt_rz_relu(v0, v1);
        const float2 r = fma2(bf16x2_to_f2(hi), f2(-1.0f), make_float2(v0, v1));
        lo = cvt_rn_relu(r.x, r.y);
    } else {
        hi = cvt_rn_relu(v0, v1);
    }
}

// Encoding features (any sign): high parts rounded to nearest, residuals
// v - hi rounded to nearest.
template <int OPS>
__device__ __forceinline__ void feat_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    if (OPS == kOpsFp16) {
        hi = pack_f16_sat(v0, v1);
        return;
    }
    hi = cvt_rn(v0, v1);
    if (OPS == kOpsBf16x3) {
        const float2 r = fma2(bf16x2_to_f2(hi), f2(-1.0f), make_float2(v0, v1));
        lo = cvt_rn(r.x, r.y);
    }
}

// One lobe pair's decoded state: weights, kappa, the mean's components
// with the signs of the decode (mu = (-nx, -ny, -sa)), the weight times the
// normaliser, and -kappa log2(e).
struct LobePair {
    float2 lam, kap, nx, ny, sa, lc, nkl;
};

// Normaliser c(kappa) = kappa / (2 pi (1 - e^{-2 kappa})) of a pair: the
// three-term series of 1 - e^{-x} below x = 2 kappa = 1/16 (truncation
// < 1e-5 relative), the hardware exponential above (< 2e-6 relative there);
// kappa floored at 1e-30 so that kappa -> 0 gives 1 / (4 pi).
__device__ __forceinline__ float2 norm_pair(float2 kap) {
    const float2 k = make_float2(fmaxf(kap.x, 1e-30f), fmaxf(kap.y, 1e-30f));
    const float2 x = add2(k, k);
    const float2 ee = ex2x2(mul2(x, f2(-kL2E)));
    const float2 em_exp = fma2(ee, f2(-1.0f), f2(1.0f));
    const float2 c = fma2(x, f2(-1.0f / 6.0f), f2(0.5f));
    const float2 em_ser = mul2(x, fma2(mul2(x, f2(-1.0f)), c, f2(1.0f)));
    const float2 em = make_float2(x.x < 0.0625f ? em_ser.x : em_exp.x, x.y < 0.0625f ? em_ser.y : em_exp.y);
    return mul2(k, rcpx2(mul2(em, f2(2.0f * kPi))));
}

// Table 1 for lobes (i, i + 1) from their raw outputs; lam / inv applied by
// the caller. theta = pi s(t'), phi = 2 pi s(p') with
// sin(theta) = cos(a), cos(theta) = -sin(a), a = theta - pi/2 in [-pi/2, pi/2],
// sin(phi) = -sin(b), cos(phi) = -cos(b), b = phi - pi in [-pi, pi].
// mix (or NULL): rows (lambda, kappa, theta, phi) of lobes i, i + 1 of
// query j are written.
__device__ __forceinline__ void decode_pair(float2 lam, float2 rk, float2 rt, float2 rp, LobePair& L,
                                            float* __restrict__ mix, int i, int64_t ld, int64_t j) {
    L.lam = lam;
    // kappa = softplus(k') = max(k', 0) + ln(1 + e^{-|k'|})
    const float2 q = ex2x2(mul2(make_float2(fabsf(rk.x), fabsf(rk.y)), f2(-kL2E)));
    const float2 l = make_float2(hw_lg2(1.0f + q.x), hw_lg2(1.0f + q.y));
    L.kap = fma2(l, f2(kLn2), make_float2(fmaxf(rk.x, 0.0f), fmaxf(rk.y, 0.0f)));
    // logistic s(t) = 1 / (1 + e^{-t})
    const float2 st = rcpx2(add2(ex2x2(mul2(rt, f2(-kL2E))), f2(1.0f)));
    const float2 sp = rcpx2(add2(ex2x2(mul2(rp, f2(-kL2E))), f2(1.0f)));
    const float2 a = fma2(st, f2(kPi), f2(-0.5f * kPi));
    const float2 b = fma2(sp, f2(2.0f * kPi), f2(-kPi));
    float sa0, ca0, sa1, ca1, sb0, cb0, sb1, cb1;
    __sincosf(a.x, &sa0, &ca0);
    __sincosf(a.y, &sa1, &ca1);
    __sincosf(b.x, &sb0, &cb0);
    __sincosf(b.y, &sb1, &cb1);
    // sin(theta) = ca; mu_x = ca cos(phi) = -(ca cb), mu_y = -(ca sb), mu_z = -sa
    const float2 sth = make_float2(ca0, ca1);
    L.nx = mul2(sth, make_float2(cb0, cb1));
    L.ny = mul2(sth, make_float2(sb0, sb1));
    L.sa = make_float2(sa0, sa1);
    L.lc = mul2(lam, norm_pair(L.kap));
    L.nkl = mul2(L.kap, f2(-kL2E));
    if (mix) {
        mix[(4 * i + 0) * ld + j] = lam.x;
        mix[(4 * i + 1) * ld + j] = L.kap.x;
        mix[(4 * i + 2) * ld + j] = a.x + 0.5f * kPi;
        mix[(4 * i + 3) * ld + j] = b.x + kPi;
        mix[(4 * i + 4) * ld + j] = lam.y;
        mix[(4 * i + 5) * ld + j] = L.kap.y;
        mix[(4 * i + 6) * ld + j] = a.y + 0.5f * kPi;
        mix[(4 * i + 7) * ld + j] = b.y + kPi;
    }
}

// Sum over the pair of lam_i c_i e^{kappa_i (mu_i . w - 1)}.
__device__ __forceinline__ float pair_pdf(const LobePair& L, const float w[3]) {
    // -mu.w = nx wx + ny wy + sa wz
    const float2 dn = fma2(L.sa, f2(w[2]), fma2(L.ny, f2(w[1]), mul2(L.nx, f2(w[0]))));
    // kappa (mu.w - 1) log2(e) = -kappa log2(e) (dn + 1)
    const float2 v = ex2x2(mul2(L.nkl, add2(dn, f2(1.0f))));
    const float2 p = mul2(L.lc, v);
    return p.x + p.y;
}

// log of each lobe's term, log lambda_i + log c(kappa_i) + kappa_i (mu_i.w - 1),
// for the pair (log-sum-exp evaluation); log lambda_i = logit - lnorm stays
// finite where lambda_i underflows.
__device__ __forceinline__ float2 pair_log_terms(const LobePair& L, float2 logit, float lnorm, const float w[3]) {
    const float2 dn = fma2(L.sa, f2(w[2]), fma2(L.ny, f2(w[1]), mul2(L.nx, f2(w[0]))));
    const float2 e = mul2(L.kap, add2(dn, f2(1.0f)));  // -kappa (mu.w - 1)
    const float2 cn = norm_pair(L.kap);
    return make_float2(logit.x - lnorm + kLn2 * hw_lg2(cn.x) - e.x, logit.y - lnorm + kLn2 * hw_lg2(cn.y) - e.y);
}

// Tile groups per CTA: one CTA per SM, each group of 128 threads walks its
// own tiles with its own activation tile, tensor-memory columns, MMA
// barrier and named CTA barrier, sharing one copy of the weights and of the
// grid table in shared memory.
constexpr int kGroups = 8;

// Named barrier of group g (id 0 is the CTA-wide __syncthreads).
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kThreads) : "memory");
}
// Barrier of group g that also ORs a predicate over its threads.
__device__ __forceinline__ bool group_sync_or(int g, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %3, 0;\n\t"
        "bar.red.or.pred o, %1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}\n"
        : "=r"(r)
        : "r"(1 + g), "r"(kThreads), "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

// Shared-memory layout of the CTA (byte offsets).
struct TinyLayout {
    uint32_t grid, a, a_stride, bars, bytes;
};

__host__ __device__ inline TinyLayout tiny_layout(const TcCfg& c, uint32_t grid_bytes) {
    TinyLayout L;
    const uint32_t nw = (c.split || c.f16) ? 2u : 1u;       // weight blobs
    const uint32_t na = c.split ? 2u : 1u;                  // activation tiles
    L.grid = nw * c.w_bytes;                                // weights first (hi, then lo)
    L.a = (L.grid + grid_bytes + 1023u) & ~1023u;           // per-group activation tiles
    L.a_stride = na * c.a_bytes;                            // hi tile, then its residual
    L.bars = L.a + (uint32_t)kGroups * L.a_stride;          // [0] weights + grid, [1 + g] MMA
    L.bytes = L.bars + 8u * (1u + kGroups) + 16u;           // + tensor-memory slot
    return L;
}

template <int OPS>
__global__ void __launch_bounds__(kThreads * kGroups, 1) k_forward_tiny(const __grid_constant__ TcCfg tc,
                                                                        const uint2* __restrict__ grid4,
                                                                        uint32_t grid_bytes,
                                                                        const uint8_t* __restrict__ wblob,
                                                                        const __grid_constant__ QueryBatch qb,
                                                                        int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr bool SPLIT = OPS == kOpsBf16x3;
    constexpr int nw = OPS == kOpsBf16 ? 1 : 2;  // weight blobs (hi, residual)
    const TinyLayout lay = tiny_layout(tc, grid_bytes);
    const int g = threadIdx.x >> 7;      // tile group
    const int t = threadIdx.x & 127;     // row of the group's tile
    const int warp = t >> 5;             // warp within the group (its TMEM lane quarter)
    uint8_t* sW = smem;
    const uint2* sG = reinterpret_cast<const uint2*>(smem + lay.grid);
    uint8_t* sA = smem + lay.a + (uint32_t)g * lay.a_stride;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 1 + kGroups);
    const uint32_t bar_w = smem_u32(&bars[0]);
    const uint32_t bar_mma = smem_u32(&bars[1 + g]);

    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(32u * kGroups)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i <= kGroups; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // This group's 32 tensor-memory columns.
    const uint32_t tmem = *tslot + 32u * (uint32_t)g;
    if (threadIdx.x == 0) {
        // Weights and grid table: two bulk copies on one barrier.
        const uint32_t wb = (uint32_t)nw * tc.w_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w), "r"(wb + grid_bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sW)),
            "l"(wblob), "r"(wb), "r"(bar_w)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(smem + lay.grid)),
            "l"(grid4), "r"(grid_bytes), "r"(bar_w)
            : "memory");
    }
    // Launched as a programmatic dependent (the wavefront frames), the steps
    // above overlap the previous kernel; the queries and their count are
    // read only after it has completed. The weights and grid copied above
    // are not written by that kernel.
    grid_dep_wait();
    grid_dep_launch();
    bool ok = !__syncthreads_or(threadIdx.x < 32 && !mbar_wait_bounded(bar_w, 0));
    uint32_t phase = 0;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // This thread's row in the K-major activation tile: 16-column layout
    // (layer 0) and 32-column layout (layers 1 and 2); chunk c of 8 columns
    // is 128 bytes further.
    const uint32_t row16 = (uint32_t)((t >> 3) * 256 + (t & 7) * 16);
    const uint32_t row32 = (uint32_t)((t >> 3) * 512 + (t & 7) * 16);
    const uint32_t lo_off = SPLIT ? tc.a_bytes : 0u;
    const int D = tc.base.level_res[0];
    const uint32_t uD = (uint32_t)D, uD2 = uD * uD;
    const int np0 = tc.layer[0].Np, np1 = tc.layer[1].Np;

    int64_t ntiles = qb.total_tiles, n0 = qb.seg[0].n;
    if (qb.n_dev) {
        n0 = *qb.n_dev;
        ntiles = (n0 + kTile - 1) / kTile;
    }
    const int64_t stride = (int64_t)gridDim.x * kGroups;
    for (int64_t tile = (int64_t)blockIdx.x * kGroups + g; ok && tile < ntiles; tile += stride) {
        int sg = 0;
        while (sg + 1 < qb.nseg && tile >= qb.seg[sg + 1].tile0) ++sg;
        const QuerySeg& S = qb.seg[sg];
        const int64_t n = (sg == 0 && qb.n_dev) ? n0 : S.n;
        const int64_t ld = S.ld;
        const int64_t j = (tile - S.tile0) * kTile + t;
        const bool valid = j < n;
        if (warp == 3) {
            // Into L2 while this tile is encoded and run through the MLP: its
            // uniforms (or directions) and the group's next tile's positions.
            const int lane = t & 31, r = lane >> 2;
            const int64_t b0 = (tile - S.tile0) * kTile + 32 * (lane & 3);
            if (r < 4) {
                if ((r < 3 || S.ufrac > 0.0f) && b0 < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(S.uin + r * ld + b0));
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
        // ---- encode (Sec. 5.1, Eq. 11): the 8 corners of the cell from the
        // shared-memory table, blended in FP32, written as this row's first
        // 8-column chunk (4 features, 4 zeros); the second chunk of the
        // 16-column input is zero.
        {
            float x = 0.0f, y = 0.0f, z = 0.0f;
            if (valid) {
                x = S.pos[j];
                y = S.pos[ld + j];
                z = S.pos[2 * ld + j];
            }
            const Cell cl = make_cell(x, y, z, D);
            // Corners (x, x + 1) are adjacent entries: four row addresses,
            // the x-neighbour one entry on.
            // (the last corner, b + D^2 + D + 1, is below D^3 by the cell clamp)
            const uint2* r00 = sG + bounded_index(cl.c[0] + uD * (cl.c[1] + uD * cl.c[2]), uD2 * uD - uD2 - uD - 1u);
            const uint2* rows[4] = {r00, r00 + uD, r00 + uD2, r00 + uD2 + uD};
            uint2 raw[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) raw[c] = rows[c >> 1][c & 1];
            float w8[8];
            corner_w8(cl, w8);
            float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float2 v01 = __half22float2(*reinterpret_cast<const __half2*>(&raw[c].x));
                const float2 v23 = __half22float2(*reinterpret_cast<const __half2*>(&raw[c].y));
                a01 = fma2(f2(w8[c]), v01, a01);
                a23 = fma2(f2(w8[c]), v23, a23);
            }
            uint32_t h01, h23, l01 = 0u, l23 = 0u;
            feat_pair<OPS>(a01.x, a01.y, h01, l01);
            feat_pair<OPS>(a23.x, a23.y, h23, l23);
            *reinterpret_cast<uint4*>(sA + row16) = make_uint4(h01, h23, 0u, 0u);
            *reinterpret_cast<uint4*>(sA + row16 + 128) = make_uint4(0u, 0u, 0u, 0u);
            if (SPLIT) {
                *reinterpret_cast<uint4*>(sA + lo_off + row16) = make_uint4(l01, l23, 0u, 0u);
                *reinterpret_cast<uint4*>(sA + lo_off + row16 + 128) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        fence_async_smem();
        tc_fence_before();
        group_sync(g);
        uint32_t rawu[16];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const TcLayer& ly = tc.layer[l];
            if (t == 0) {
                tc_fence_after();
                // Descriptors of K step s are those of step 0 with the start
                // address 256 bytes (16 units) further.
                const uint64_t ad = umma_desc(smem_u32(sA), 128u, (uint32_t)(ly.Kp >> 3) * 128u);
                const uint64_t bd = umma_desc(smem_u32(sW) + ly.w_off, 128u, (uint32_t)(ly.Kp >> 3) * 128u);
                const uint64_t bl = bd + (uint64_t)(tc.w_bytes >> 4), al = ad + (uint64_t)(lo_off >> 4);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    if (s < (ly.Kp >> 4)) {
                        const uint64_t o = (uint64_t)(16 * s);
                        mma_bf16(tmem, ad + o, bd + o, ly.idesc, s > 0 ? 1u : 0u);
                        if (OPS != kOpsBf16) mma_bf16(tmem, ad + o, bl + o, ly.idesc, 1u);
                        if (SPLIT) mma_bf16(tmem, al + o, bd + o, ly.idesc, 1u);
                    }
                }
                mma_commit(bar_mma);
            }
            // Warp 0 of the group waits on the MMA barrier; the group's other
            // warps wait in its named barrier, which also passes the outcome.
            const bool done = warp != 0 || mbar_wait_bounded(bar_mma, phase);
            phase ^= 1u;
            ok = !group_sync_or(g, !done);
            if (!ok) break;
            tc_fence_after();
            if (l < 2) {
                // ReLU, BF16 high part and residual of this row's outputs,
                // as the next layer's input (32-column layout).
                const int np = l == 0 ? np0 : np1;
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    if (c0 < np) {
                        uint32_t r[16];
                        tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
                        tmem_wait16(r);
                        uint32_t hi[8], lo[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            relu_pair<OPS>(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]), hi[i], lo[i]);
                        const uint32_t o = row32 + (uint32_t)(c0 >> 3) * 128u;
                        *reinterpret_cast<uint4*>(sA + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<uint4*>(sA + o + 128) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                        if (SPLIT) {
                            *reinterpret_cast<uint4*>(sA + lo_off + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                            *reinterpret_cast<uint4*>(sA + lo_off + o + 128) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                        }
                    }
                }
                fence_async_smem();
                tc_fence_before();
                group_sync(g);
            } else {
                tmem_ld16(tmem + lane_base, rawu);
                tmem_wait16(rawu);
                tc_fence_before();
            }
        }
        if (!ok) break;
        // ---- decode (Table 1), sample (Sec. 5.3) and density (Eq. 4).
        float r[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(rawu[i]);
        const float mx = fmaxf(fmaxf(r[0], r[4]), fmaxf(r[8], r[12]));
        const float2 mxl = f2(-mx * kL2E);
        const float2 e01 = ex2x2(fma2(make_float2(r[0], r[4]), f2(kL2E), mxl));
        const float2 e23 = ex2x2(fma2(make_float2(r[8], r[12]), f2(kL2E), mxl));
        const float ssum = (e01.x + e01.y) + (e23.x + e23.y);  // in [1, 4]
        const float inv = hw_rcp(ssum);
        LobePair P0, P1;
        float* mix = valid ? S.mix : nullptr;
        decode_pair(mul2(e01, f2(inv)), make_float2(r[1], r[5]), make_float2(r[2], r[6]), make_float2(r[3], r[7]),
                    P0, mix, 0, ld, j);
        decode_pair(mul2(e23, f2(inv)), make_float2(r[9], r[13]), make_float2(r[10], r[14]),
                    make_float2(r[11], r[15]), P1, mix, 2, ld, j);
        float w[3] = {0.0f, 0.0f, 1.0f};
        const bool sample = qb.sample != 0;
        if (sample) {
            float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
            bool uni = false;
            if (valid) {
                u0 = S.uin[j];
                u1 = S.uin[ld + j];
                u2 = S.uin[2 * ld + j];
                uni = S.ufrac > 0.0f && S.uin[3 * ld + j] < S.ufrac;
            }
            if (uni) {
                uniform_sphere(u1, u2, w);
            } else {
                // Smallest lobe i with u0 below the running sum of the
                // weights (the last lobe if rounding leaves u0 above all).
                const float c0 = P0.lam.x, c1 = c0 + P0.lam.y, c2 = c1 + P1.lam.x;
                // The sums are non-decreasing, so the lobe index is
                // g0 + g1 + g2: the second pair when g1, the odd lobe of the
                // pair when exactly one or all three hold.
                const bool g0 = u0 >= c0, g1 = u0 >= c1, g2 = u0 >= c2;
                Lobe sl;
                const float2 kk = g1 ? P1.kap : P0.kap, xx = g1 ? P1.nx : P0.nx, yy = g1 ? P1.ny : P0.ny,
                             zz = g1 ? P1.sa : P0.sa;
                const bool odd = g2 || (g0 && !g1);
                sl.kap = odd ? kk.y : kk.x;
                sl.mu[0] = -(odd ? xx.y : xx.x);
                sl.mu[1] = -(odd ? yy.y : yy.x);
                sl.mu[2] = -(odd ? zz.y : zz.x);
                sl.lam = 0.0f;
                vmf_sample_rp(sl, u1, u2, w);
            }
            float pv = pair_pdf(P0, w) + pair_pdf(P1, w);
            if (S.ufrac > 0.0f) pv = S.ufrac * kInv4Pi + (1.0f - S.ufrac) * pv;
            if (valid) {
                S.dir[j] = w[0];
                S.dir[ld + j] = w[1];
                S.dir[2 * ld + j] = w[2];
                S.pdf[j] = pv;
            }
        } else {
            if (valid) {
                w[0] = S.uin[j];
                w[1] = S.uin[ld + j];
                w[2] = S.uin[2 * ld + j];
            }
            float pv;
            if (qb.log_pdf) {
                const float lnorm = mx + kLn2 * hw_lg2(ssum);
                const float2 a0 = pair_log_terms(P0, make_float2(r[0], r[4]), lnorm, w);
                const float2 a1 = pair_log_terms(P1, make_float2(r[8], r[12]), lnorm, w);
                const float m = fmaxf(fmaxf(a0.x, a0.y), fmaxf(a1.x, a1.y));
                const float s = __expf(a0.x - m) + __expf(a0.y - m) + __expf(a1.x - m) + __expf(a1.y - m);
                pv = m + __logf(s);
            } else {
                pv = pair_pdf(P0, w) + pair_pdf(P1, w);
            }
            if (valid) S.pdf[j] = pv;
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(status, kStatusTimeout);
        // Drain this group's own asynchronous work (bounded) before the
        // tensor memory is released: the MMA batch whose wait gave up (and,
        // for group 0, the weights' and grid's bulk copies).
        if (warp == 0) {
            if (g == 0) (void)mbar_wait_bounded(bar_w, 0);
            (void)mbar_wait_bounded(bar_mma, phase ^ 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(32u * kGroups)
                     : "memory");
    }
}

}  // namespace

bool tiny_qualifies(const TcCfg& c) {
    const DevCfg& d = c.base;
    const uint32_t grid_bytes = (uint32_t)d.level_res[0] * d.level_res[0] * d.level_res[0] * 8u;
    return !c.fp32 && d.mode == NPM_RADIANCE && d.n_levels == 1 && d.feat == 4 && (d.dense_mask & 1u) && d.n_layers == 3 &&
           d.K == 4 && d.kappa_act == NPM_SOFTPLUS && c.layer[0].Kp == 16 && c.layer[0].Np <= 32 &&
           c.layer[1].Kp == 32 && c.layer[1].Np <= 32 && c.layer[2].Kp == 32 && c.layer[2].Np == 16 &&
           c.a0_bytes == 0 && c.a_bytes == (uint32_t)(kTile * 32 * 2) && grid_bytes % 16u == 0 &&
           tiny_layout(c, grid_bytes).bytes <= 227u * 1024u;
}

cudaError_t launch_tiny(const TcCfg& c, size_t, const __half* grid_h, const uint8_t* wblob, QueryBatch& qb,
                        int64_t max_n, int* status, cudaStream_t st, bool pdl) {
    auto kern = c.split ? k_forward_tiny<kOpsBf16x3> : c.f16 ? k_forward_tiny<kOpsFp16> : k_forward_tiny<kOpsBf16>;
    const uint32_t grid_bytes = (uint32_t)c.base.level_res[0] * c.base.level_res[0] * c.base.level_res[0] * 8u;
    const size_t smem = tiny_layout(c, grid_bytes).bytes;
    // One CTA per SM (kGroups x 128 threads at 64 registers); carve out just
    // its shared memory so the rest stays L1.
    static std::atomic<uint64_t> attrs_s{~0ull}, attrs_h{~0ull}, attrs_p{~0ull};
    cudaError_t e = set_smem_attrs(kern, smem, carveout_percent(smem + 1024),
                                   c.split ? attrs_s : c.f16 ? attrs_h : attrs_p);
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
    const int64_t hint = qb.n_dev ? (max_n + kTile - 1) / kTile : t0;
    int64_t g = (hint + kGroups - 1) / kGroups;
    if (g > sms) g = sms;
    if (g < 1) g = 1;
    return launch_maybe_pdl(kern, dim3((unsigned)g), dim3(kThreads * kGroups), smem, st, pdl, c,
                            reinterpret_cast<const uint2*>(grid_h), grid_bytes, wblob, qb, status);
}

}  // namespace tc
}  // namespace npm
