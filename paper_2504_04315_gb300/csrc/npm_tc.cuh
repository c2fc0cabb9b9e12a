// npm_tc.cuh -- shared pieces of the tensor-core (tcgen05) kernels on
// sm_103a: the model's layer layout for the MMAs and the inline-PTX helpers
// (tensor memory, MMA issue, mbarriers, shared-memory matrix descriptors and
// the BF16 operand stores). Internal to the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "npm_device.cuh"

namespace npm {
namespace tc {

constexpr int kTile = 128;
constexpr int kThreads = 128;

struct TcLayer {
    int K, N;        // logical widths
    int Kp, Np;      // padded to multiples of 16
    uint32_t w_off;  // byte offset of this layer's weights in the blob
    uint32_t idesc;  // instruction descriptor
};

struct TcCfg {
    DevCfg base;
    TcLayer layer[NPM_MAX_LAYERS];
    uint32_t w_bytes;  // bytes of one weight blob (multiple of 128); the
                       // residual (lo) blob follows when split
    uint32_t a_bytes;  // bytes of one activation tile; the lo tile follows
    uint32_t a0_bytes; // bytes of the layer-0 input tile when it has its own
                       // buffer (the encoding leaves all-zero 8-column chunks);
                       // 0 when layer 0 shares the buffer of layers >= 1
    int split;         // 1: BF16 residual operands (three MMAs per K step)
    int f16;           // 1: FP16 operands: activations rounded to FP16, weights
                       // FP16 plus an FP16 residual (two MMAs per K step);
                       // with split, activations FP16 plus an FP16 residual too
    int fp32;          // 1: the FP32-accuracy mode (split FP16 operands, FP32
                       // grid table, the FP32 path's sampler)
    uint32_t tmem_cols;
    int enc_width;     // meaningful network inputs
};

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle (core matrices of 8 rows x
// 16 bytes): lbo = byte step between core matrices along K, sbo = byte step
// between 8-row groups along M/N; bit 46 is the tcgen05 descriptor version.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One potentially blocking test of phase `parity`: the thread sleeps in the
// barrier until the phase completes or about 20 microseconds pass (the
// suspend-time hint), so a waiting warp issues almost nothing.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; false after ~2^32 cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 32)) return false;
    return true;
}

// 16 consecutive FP32 columns of this thread's TMEM lane. The values are
// valid only after tmem_wait16 on the same registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// tcgen05.wait::ld with the loaded registers as in/out operands, so that no
// use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// (a, b) rounded to nearest FP16 and packed (a in the low half); values
// beyond the FP16 range saturate to +-65504 rather than becoming infinite.
__device__ __forceinline__ uint32_t pack_f16_sat(float a, float b) {
    uint32_t d;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// Named barrier of 128-thread tile group g of a CTA (id 1 + g; id 0 is the
// CTA-wide __syncthreads), and its form that also ORs a predicate over the
// group's threads.
__device__ __forceinline__ void tc_group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(128) : "memory");
}
__device__ __forceinline__ bool tc_group_sync_or(int g, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %3, 0;\n\t"
        "bar.red.or.pred o, %1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}\n"
        : "=r"(r)
        : "r"(1 + g), "r"(128), "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

// FP16 residuals (a - hi_a, b - hi_b) of a packed FP16 pair hp = (hi_a,
// hi_b), rounded to nearest and packed the same way.
__device__ __forceinline__ uint32_t f16_residual(uint32_t hp, float a, float b) {
    const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hp));
    return pack_f16_sat(a - hf.x, b - hf.y);
}

// A pair of MMA operands in the model's operand format.
__device__ __forceinline__ uint32_t pack_op(float a, float b, bool f16) {
    return f16 ? pack_f16_sat(a, b) : pack_bf16(a, b);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile whose rows
// hold kp elements: 8x8 core matrices (128 bytes), K-adjacent core matrices
// 128 bytes apart, 8-row groups kp/8 * 128 bytes apart.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int kp) {
    return (uint32_t)((row >> 3) * (kp >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Rounds v to BF16 (hi) and, when lo_off != 0, also stores the BF16
// residual v - hi at the same position of the residual tile lo_off bytes on.
__device__ __forceinline__ void store16(uint8_t* sA, uint32_t off0, uint32_t off1, const float (&v)[16],
                                        uint32_t lo_off) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        h[i] = *reinterpret_cast<uint32_t*>(&hb);
        const float2 hf = __bfloat1622float2(hb);
        l[i] = pack_bf16(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    }
    *reinterpret_cast<uint4*>(sA + off0) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(sA + off1) = make_uint4(h[4], h[5], h[6], h[7]);
    if (lo_off) {
        *reinterpret_cast<uint4*>(sA + lo_off + off0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(sA + lo_off + off1) = make_uint4(l[4], l[5], l[6], l[7]);
    }
}

// Forward-pass form of store16. With a residual tile, hi is v truncated to
// BF16 (its upper 16 bits: one byte permute per pair) and the residual
// v - hi, exact in FP32 and of the same sign as v, is rounded to BF16 (one
// packed subtraction and one conversion per pair); the product error that
// split BF16 drops stays below 2^-15 relative. Without a residual tile, v is
// rounded to nearest (to FP16 with saturation when f16).
__device__ __forceinline__ void store16_fwd(uint8_t* sA, uint32_t off0, uint32_t off1, const float (&v)[16],
                                            uint32_t lo_off, bool f16 = false) {
    uint32_t h[8];
    if (f16) {
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = pack_f16_sat(v[2 * i], v[2 * i + 1]);
        if (lo_off) {
            // FP16 residuals v - hi, rounded to nearest.
            uint32_t l[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) l[i] = f16_residual(h[i], v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4*>(sA + lo_off + off0) = make_uint4(l[0], l[1], l[2], l[3]);
            *reinterpret_cast<uint4*>(sA + lo_off + off1) = make_uint4(l[4], l[5], l[6], l[7]);
        }
    } else if (lo_off) {
        uint32_t l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t a = __float_as_uint(v[2 * i]), b = __float_as_uint(v[2 * i + 1]);
            h[i] = __byte_perm(a, b, 0x7632);
            const float2 nh = make_float2(__uint_as_float((a & 0xffff0000u) ^ 0x80000000u),
                                          __uint_as_float((b & 0xffff0000u) ^ 0x80000000u));
            const float2 r = __fadd2_rn(make_float2(v[2 * i], v[2 * i + 1]), nh);
            l[i] = pack_bf16(r.x, r.y);
        }
        *reinterpret_cast<uint4*>(sA + lo_off + off0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(sA + lo_off + off1) = make_uint4(l[4], l[5], l[6], l[7]);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
    }
    *reinterpret_cast<uint4*>(sA + off0) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(sA + off1) = make_uint4(h[4], h[5], h[6], h[7]);
}

// One or two BF16 values (and their residuals when lo_off != 0), or FP16
// values when f16.
__device__ __forceinline__ void store_pair(uint8_t* sA, uint32_t off, float a, float b, uint32_t lo_off,
                                           bool f16 = false) {
    if (f16) {
        const uint32_t hp = pack_f16_sat(a, b);
        *reinterpret_cast<uint32_t*>(sA + off) = hp;
        if (lo_off) *reinterpret_cast<uint32_t*>(sA + lo_off + off) = f16_residual(hp, a, b);
        return;
    }
    __nv_bfloat162 hb = __floats2bfloat162_rn(a, b);
    *reinterpret_cast<__nv_bfloat162*>(sA + off) = hb;
    if (lo_off) {
        const float2 hf = __bfloat1622float2(hb);
        *reinterpret_cast<uint32_t*>(sA + lo_off + off) = pack_bf16(a - hf.x, b - hf.y);
    }
}

__device__ __forceinline__ void store_one(uint8_t* sA, uint32_t off, float a, uint32_t lo_off, bool f16 = false) {
    if (f16) {
        const uint32_t hp = pack_f16_sat(a, 0.0f);
        *reinterpret_cast<uint16_t*>(sA + off) = (uint16_t)(hp & 0xffffu);
        if (lo_off) *reinterpret_cast<uint16_t*>(sA + lo_off + off) = (uint16_t)(f16_residual(hp, a, 0.0f) & 0xffffu);
        return;
    }
    const __nv_bfloat16 hb = __float2bfloat16_rn(a);
    *reinterpret_cast<__nv_bfloat16*>(sA + off) = hb;
    if (lo_off)
        *reinterpret_cast<__nv_bfloat16*>(sA + lo_off + off) = __float2bfloat16_rn(a - __bfloat162float(hb));
}

// Sampler of the reduced-precision path (Sec. 5.3, Jakob's inversion as in
// vmf_sample) on the hardware approximations: 1 - e^{-2k} and log(1 + y) by
// their series where the direct forms lose relative accuracy (2k < 0.1,
// four terms, truncation < 1e-6 relative; |y| < 1/16, seven terms,
// truncation < 1e-9 relative), the fast exponential, logarithm and divide
// elsewhere, and sqrt as x rsqrt(x). The fast logarithm's absolute error
// (about 2^-21.4 near 1) is at most 6e-6 of log(1 + y) for |y| >= 1/16. The
// density is always evaluated at the direction returned, so its accuracy
// bar does not depend on these approximations.
__device__ __forceinline__ void vmf_sample_rp(const Lobe& L, float u1, float u2, float out[3]) {
    const float k = L.kap;
    const float x = 2.0f * k;
    const float em1 = x < 0.1f ? -x * (1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f))))
                               : __expf(-x) - 1.0f;  // e^{-2k} - 1
    const float y = u1 * em1;                        // in (-1, 0]
    const float ser =
        y * (1.0f + y * (-0.5f + y * (1.0f / 3.0f + y * (-0.25f + y * (0.2f + y * (-1.0f / 6.0f + y * (1.0f / 7.0f)))))));
    const float l1p = fabsf(y) < 0.0625f ? ser : __logf(1.0f + y);
    float t1 = k > 1e-20f ? __fdividef(-l1p, k) : 2.0f * u1;
    t1 = fminf(fmaxf(t1, 0.0f), 2.0f);
    const float W = 1.0f - t1;
    const float q = t1 * (2.0f - t1);
    const float sn = q > 0.0f ? q * rsqrtf(q) : 0.0f;
    float sp, cp;
    __sincosf(2.0f * kPi * (u2 - 0.5f), &sp, &cp);
    const float lx = -sn * cp, ly = -sn * sp;
    float tt[3], bb[3];
    frame(L.mu, tt, bb);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = lx * tt[a] + ly * bb[a] + W * L.mu[a];
}

// Fused forward of the small serving networks (npm_tc_tiny.cu): radiance
// mode, one dense level of 4 features, three layers of at most 32 outputs
// (padded input 16), K = 4, softplus kappa, layer 0 sharing the activation
// buffer. launch_tiny takes the general kernel's configuration, shared
// memory size, FP16 grid and weight blob. With pdl the kernel is launched as
// a programmatic dependent of the stream's previous kernel: its prologue
// (tensor-memory allocation, copies of the weights and grid) overlaps that
// kernel, which therefore must not write the weights or the grid.
bool tiny_qualifies(const TcCfg& c);
cudaError_t launch_tiny(const TcCfg& c, size_t smem, const __half* grid_h, const uint8_t* wblob, QueryBatch& qb,
                        int64_t max_n, int* status, cudaStream_t st, bool pdl = false);

}  // namespace tc
}  // namespace npm
