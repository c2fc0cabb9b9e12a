// npm_frame.cu -- a synthetic wavefront path tracer driving the NPM hot path
// (the per-bounce batched inference and per-frame training of Sec. 5.2),
// standing in for the paper's OptiX renderer and scenes.
//
// Per frame: every path starts at a seeded position in [0,1)^3. Each bounce
// draws four uniforms per live path, queries the guide on the compacted
// queue (one-sample mixture with a uniform-sphere BSDF stand-in), evaluates
// the analytic radiance at the sampled direction times Exponential(1) noise,
// records training samples, and keeps each path with probability `survival`
// (Bernoulli), moving it along the sampled direction (wrapping into the unit
// box). The first `train_batch` paths' first-bounce samples form the frame's
// training batch; one npm_train_step follows the last bounce.
//
// The queue size lives in device memory, so a whole frame is captured once
// into a CUDA graph and replayed; a device frame counter keys the random
// numbers, and %globaltimer stamps at bounce boundaries give per-bounce
// latencies.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "npm_handle.h"
#include "npm_kernels.h"

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Key of the random stream (frame, bounce, purpose).
__device__ __forceinline__ uint64_t key(uint64_t seed, uint64_t frame, uint64_t bounce, uint64_t what) {
    return mix64(mix64(seed ^ (frame * 0x632BE59BD9B4E019ull)) ^ (bounce * 64 + what));
}

// 32-bit finaliser (two xor-multiply rounds; Wellons' "lowbias32" constants).
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Uniform in [0, 1) with 24 random bits: element i of the stream keyed by
// s0. Two 32-bit hash rounds cost a fraction of a 64-bit mix per draw, and
// the driver draws eight per path and bounce. The high word of i (zero below
// 2^32, i.e. below 2^30 paths) joins the key, so larger indices do not wrap
// onto smaller ones.
__device__ __forceinline__ float uni(uint64_t s0, uint64_t i) {
    const uint32_t hi = (uint32_t)(s0 >> 32) ^ ((uint32_t)(i >> 32) * 0x9E3779B9u);
    const uint32_t h = hash32(hash32((uint32_t)i + (uint32_t)s0) ^ hi);
    return (float)(h >> 8) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct WfState {
    int64_t P, T;
    int bounces;
    float survival;
    uint64_t seed;
    float* pos[2];        // [3][P] each
    int32_t* pid[2];      // [P]
    int64_t* count;       // [2]
    float* u;             // [4][P]
    float* dir;           // [3][P]
    float* pdf;           // [P]
    float* tpos;          // [3][T]
    float* tdir;          // [3][T]
    float* trad;          // [T]
    float* tpdf;          // [T]
    uint64_t* frame;      // device frame counter
    // [max_frames][2 bounces + 2]: 0 after the frame start; 1 + 2b when
    // bounce b's query kernel has finished (taken as the bounce's advance
    // kernel starts); 2 + 2b after that advance; 2 bounces + 1 after the
    // training step.
    uint64_t* stamps;
    int64_t* live;        // [max_frames][bounces]: paths queried per bounce
    unsigned long long* queries;  // total queries served
    int max_frames;
};

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

__device__ __forceinline__ void stamp(const WfState& s, int slot) {
    const uint64_t f = *s.frame;
    if ((int64_t)f < s.max_frames) s.stamps[f * (2 * s.bounces + 2) + slot] = globaltimer();
}

// Sampling uniforms of path p at bounce b, written at queue slot i.
__device__ __forceinline__ void write_uniforms(const WfState& s, uint64_t ku, int64_t i, uint64_t p) {
    for (int r = 0; r < 4; ++r) s.u[r * s.P + i] = uni(ku, r * (uint64_t)s.P + p);
}

// Camera rays of the frame: positions, path ids and bounce 0's uniforms.
__global__ void k_wf_start(WfState s) {
    const uint64_t f = *s.frame;
    const uint64_t kp = key(s.seed, f, 0, 1), ku = key(s.seed, f, 0, 2);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < s.P;
         p += (int64_t)gridDim.x * blockDim.x) {
        for (int r = 0; r < 3; ++r) s.pos[0][r * s.P + p] = uni(kp, (uint64_t)(r * s.P + p));
        s.pid[0][p] = (int32_t)p;
        write_uniforms(s, ku, p, (uint64_t)p);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.count[0] = s.P;
        s.count[1] = 0;
    }
}

// Timestamp slot of the current frame, taken after every earlier kernel of
// the stream has completed; clear >= 0 also zeroes that queue counter (the
// next bounce's destination, which no later kernel reads before the next
// advance appends to it).
__global__ void k_wf_stamp(WfState s, int slot, int clear) {
    npm::grid_dep_wait();
    npm::grid_dep_launch();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        stamp(s, slot);
        if (clear >= 0) s.count[clear] = 0;
    }
}

// Threads per block of k_wf_advance. Its compaction takes a full-warp
// ballot and keeps one count per warp in a 32-entry shared table, so the
// block must be whole warps and at most 32 of them.
constexpr int kAdvanceThreads = 256;
static_assert(kAdvanceThreads % 32 == 0 && kAdvanceThreads <= 1024,
              "k_wf_advance needs whole warps, at most 32 of them");

// Radiance estimate, training record, survival and compaction of one
// bounce; each survivor also gets the next bounce's uniforms at its new
// queue slot (this bounce's query kernel has consumed the old ones).
__global__ void __launch_bounds__(kAdvanceThreads) k_wf_advance(WfState s, int b, int src) {
    // Launched as a programmatic dependent of the query kernel: its blocks
    // may be scheduled early, and read nothing until that kernel completes.
    npm::grid_dep_wait();
    npm::grid_dep_launch();
    const uint64_t f = *s.frame;
    const int64_t n = s.count[src];
    const int dst = src ^ 1;
    const uint64_t kn = key(s.seed, f, b, 3), ks = key(s.seed, f, b, 4), kj = key(s.seed, f, b, 5);
    const uint64_t ku = key(s.seed, f, b + 1, 2);
    const bool next = b + 1 < s.bounces;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // The query kernel of this bounce has completed (stream order).
        stamp(s, 1 + 2 * b);
        if ((int64_t)f < s.max_frames) s.live[f * s.bounces + b] = n;
    }
    const unsigned lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = kAdvanceThreads / 32;
    __shared__ int s_off[kAdvanceThreads / 32];  // survivors per warp, then their offsets
    __shared__ long long s_base;   // the block's first slot in the next queue
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const bool valid = i < n;
        bool keep = false;
        float x[3] = {0.0f, 0.0f, 0.0f};
        int32_t p = 0;
        if (valid) {
            p = s.pid[src][i];
            const float w[3] = {s.dir[i], s.dir[s.P + i], s.dir[2 * s.P + i]};
            for (int r = 0; r < 3; ++r) x[r] = s.pos[src][r * s.P + i];
            if (b == 0 && p < s.T) {
                const float L = field(x, w) * -log1pf(-uni(kn, (uint64_t)p));
                for (int r = 0; r < 3; ++r) {
                    s.tpos[r * s.T + p] = x[r];
                    s.tdir[r * s.T + p] = w[r];
                }
                s.trad[p] = L;
                s.tpdf[p] = s.pdf[i];
            }
            keep = uni(ks, (uint64_t)p) < s.survival;
            if (keep)
                for (int r = 0; r < 3; ++r) {
                    float y = x[r] + 0.25f * w[r] + 0.1f * (uni(kj, r * (uint64_t)s.P + p) - 0.5f);
                    x[r] = y - floorf(y);
                }
        }
        // Block-aggregated compaction into the next queue: one atomic per
        // block and pass, since atomics on one address serialise.
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_off[warp] = __popc(mask);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < nwarps; ++w) {
                const int c = s_off[w];
                s_off[w] = (int)tot;
                tot += (unsigned long long)c;
            }
            s_base = tot ? (long long)atomicAdd((unsigned long long*)&s.count[dst], tot) : 0ll;
        }
        __syncthreads();
        if (keep) {
            const int64_t j = npm::bounded_slot((int64_t)s_base + s_off[warp] + __popc(mask & ((1u << lane) - 1u)), s.P);
            for (int r = 0; r < 3; ++r) s.pos[dst][r * s.P + j] = x[r];
            s.pid[dst][j] = p;
            if (next) write_uniforms(s, ku, j, (uint64_t)p);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(s.queries, (unsigned long long)n);
}

__global__ void k_wf_end(WfState s) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        stamp(s, 2 * s.bounces + 1);
        *s.frame += 1;
    }
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : g < 1 ? 1 : g);
}

}  // namespace

struct npm_wavefront {
    npm_handle* h = nullptr;
    npm_frame_config cfg;
    WfState st;
    void* mem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    float* loss = nullptr;
};

namespace {

npm_status enqueue_frame(npm_wavefront* w, cudaStream_t st) {
    WfState& s = w->st;
    npm_handle* h = w->h;
    const int g = grid_for(s.P);
    // Within a frame the stamp, query and advance kernels of the bounces are
    // programmatic dependents of their predecessors (each waits for it
    // before reading its results; the query kernel's prologue and every
    // launch overlap the previous kernel's tail). None of them writes the
    // model, which only the training step at the end of the frame updates.
    k_wf_start<<<g, 256, 0, st>>>(s);  // also zeroes count[1]
    cudaError_t le = npm::launch_maybe_pdl(k_wf_stamp, dim3(1), dim3(32), 0, st, true, s, 0, -1);
    if (le != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(le));
    for (int b = 0; b < s.bounces; ++b) {
        const int src = b & 1;
        npm::QueryBatch qb;
        memset(&qb, 0, sizeof(qb));
        qb.nseg = 1;
        qb.sample = 1;
        qb.n_dev = &s.count[src];
        npm::QuerySeg& q = qb.seg[0];
        q.n = s.P;
        q.ld = s.P;
        q.pos = s.pos[src];
        q.uin = s.u;
        q.dir = s.dir;
        q.pdf = s.pdf;
        q.ufrac = w->cfg.uniform_frac;
        cudaError_t e = h->tc ? npm::tc_query_batch(h, qb, s.P, st, true)
                              : npm::launch_forward_fp32_batch(h->dc, inf_params(h), inf_wfwd(h), qb, s.P, st, status_word(h), h->wait_limit);
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
        e = npm::launch_maybe_pdl(k_wf_advance, dim3(g), dim3(kAdvanceThreads), 0, st, true, s, b, src);
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
        // count[src] was this bounce's queue: the next advance appends to it
        e = npm::launch_maybe_pdl(k_wf_stamp, dim3(1), dim3(32), 0, st, true, s, 2 + 2 * b, src);
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
    }
    npm_status rs = npm_train_step(h, s.T, s.tpos, nullptr, s.tdir, s.trad, s.tpdf, s.T, w->loss, st);
    if (rs != NPM_OK) return rs;
    k_wf_end<<<1, 32, 0, st>>>(s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NPM_OK : npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

npm_status npm_wavefront_create(npm_handle* h, const npm_frame_config* cfg, npm_wavefront** out) {
    npm::CallRange range("npm_wavefront_create");
    if (!h || !cfg || !out) return npm::set_error(NPM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (h->cfg.mode != NPM_RADIANCE)
        return npm::set_error(NPM_ERR_UNSUPPORTED, "the wavefront driver runs radiance-mode models");
    if (cfg->paths < 1 || cfg->paths > h->cfg.max_batch || cfg->bounces < 1 || cfg->bounces > 64 ||
        cfg->train_batch < 1 || cfg->train_batch > cfg->paths || cfg->train_batch > h->cfg.max_batch ||
        !(cfg->survival >= 0.0f && cfg->survival <= 1.0f) ||
        !(cfg->uniform_frac > 0.0f && cfg->uniform_frac <= 1.0f) || cfg->max_frames < 1)
        return npm::set_error(NPM_ERR_INVALID_ARG, "bad wavefront configuration");
    npm_wavefront* w = new npm_wavefront();
    w->h = h;
    w->cfg = *cfg;
    WfState& s = w->st;
    s.P = cfg->paths;
    s.T = cfg->train_batch;
    s.bounces = cfg->bounces;
    s.survival = cfg->survival;
    s.seed = cfg->seed;
    s.max_frames = cfg->max_frames;
    const size_t P = (size_t)s.P, T = (size_t)s.T;
    const size_t floats = 2 * 3 * P + 4 * P + 3 * P + P + 3 * T + 3 * T + T + T + 1;
    const size_t nstamp = (size_t)cfg->max_frames * (2 * cfg->bounces + 2);
    const size_t nlive = (size_t)cfg->max_frames * cfg->bounces;
    const size_t bytes = floats * 4 + 2 * P * 4 + 64 + (nstamp + nlive) * 8 + 256 * 20;
    if (cudaMalloc(&w->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return npm::set_error(NPM_ERR_OOM, "cannot allocate wavefront buffers");
    }
    cudaMemset(w->mem, 0, bytes);
    char* p = static_cast<char*>(w->mem);
    auto take = [&](size_t b) {
        char* r = p;
        p += (b + 255) / 256 * 256;
        return r;
    };
    s.pos[0] = (float*)take(3 * P * 4);
    s.pos[1] = (float*)take(3 * P * 4);
    s.u = (float*)take(4 * P * 4);
    s.dir = (float*)take(3 * P * 4);
    s.pdf = (float*)take(P * 4);
    s.tpos = (float*)take(3 * T * 4);
    s.tdir = (float*)take(3 * T * 4);
    s.trad = (float*)take(T * 4);
    s.tpdf = (float*)take(T * 4);
    s.pid[0] = (int32_t*)take(P * 4);
    s.pid[1] = (int32_t*)take(P * 4);
    s.count = (int64_t*)take(16);
    s.frame = (uint64_t*)take(8);
    s.queries = (unsigned long long*)take(8);
    w->loss = (float*)take(4);
    s.stamps = (uint64_t*)take(nstamp * 8);
    s.live = (int64_t*)take(nlive * 8);
    if ((size_t)(p - static_cast<char*>(w->mem)) > bytes) {
        cudaFree(w->mem);
        delete w;
        return npm::set_error(NPM_ERR_INVALID_ARG, "internal layout error");
    }
    *out = w;
    return NPM_OK;
}

npm_status npm_wavefront_run(npm_wavefront* w, int frames, void* stream, npm_frame_stats* out) {
    npm::CallRange range("npm_wavefront_run");
    if (!w || frames < 0 || !out) return npm::set_error(NPM_ERR_INVALID_ARG, "bad argument");
    WfState& s = w->st;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t f0 = 0;
    unsigned long long q0 = 0;
    if (cudaMemcpy(&f0, s.frame, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&q0, s.queries, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return npm::set_error(NPM_ERR_CUDA, "read wavefront counters");
    if ((int64_t)(f0 + frames) > s.max_frames)
        return npm::set_error(NPM_ERR_CAPACITY, "more frames than max_frames");
    npm_status rs;
    if (w->cfg.use_graph && !w->exec) {
        if (!w->cap && cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking) != cudaSuccess)
            return npm::set_error(NPM_ERR_CUDA, "cannot create the capture stream");
        if (cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return npm::set_error(NPM_ERR_CUDA, "cannot begin capture");
        rs = enqueue_frame(w, w->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(w->cap, &g);
        if (rs != NPM_OK) {
            if (g) cudaGraphDestroy(g);
            return rs;
        }
        if (e != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, cudaGetErrorString(e));
        w->graph = g;
        if (cudaGraphInstantiate(&w->exec, g, 0) != cudaSuccess)
            return npm::set_error(NPM_ERR_CUDA, "cannot instantiate the frame graph");
    }
    // Timing events, released on every return path.
    struct Events {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    if (cudaEventCreate(&ev.e0) != cudaSuccess || cudaEventCreate(&ev.e1) != cudaSuccess)
        return npm::set_error(NPM_ERR_CUDA, "cannot create timing events");
    const cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    cudaEventRecord(e0, st);
    for (int f = 0; f < frames; ++f) {
        if (w->exec) {
            if (cudaGraphLaunch(w->exec, st) != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, "graph launch");
        } else if ((rs = enqueue_frame(w, st)) != NPM_OK) {
            return rs;
        }
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return npm::set_error(NPM_ERR_CUDA, "frames failed");
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long q1 = 0;
    cudaMemcpy(&q1, s.queries, 8, cudaMemcpyDeviceToHost);
    const int stride = 2 * s.bounces + 2;
    std::vector<uint64_t> t((size_t)frames * stride);
    std::vector<int64_t> live((size_t)frames * s.bounces);
    cudaMemcpy(t.data(), s.stamps + f0 * stride, t.size() * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(live.data(), s.live + f0 * s.bounces, live.size() * 8, cudaMemcpyDeviceToHost);
    std::vector<double> lat;
    double train_ms = 0.0, query_ms = 0.0, adv_ms = 0.0;
    memset(out, 0, sizeof(*out));
    for (int f = 0; f < frames; ++f) {
        const uint64_t* r = &t[(size_t)f * stride];
        for (int b = 0; b < s.bounces; ++b) {
            lat.push_back((double)(r[2 * b + 2] - r[2 * b]) * 1e-6);
            const double q = (double)(r[2 * b + 1] - r[2 * b]) * 1e-6;
            query_ms += q;
            adv_ms += (double)(r[2 * b + 2] - r[2 * b + 1]) * 1e-6;
            if (b < NPM_FRAME_BOUNCE_STATS) {
                out->bounce_queries[b] += (double)live[(size_t)f * s.bounces + b] / frames;
                out->bounce_query_ms[b] += q / frames;
            }
        }
        train_ms += (double)(r[2 * s.bounces + 1] - r[2 * s.bounces]) * 1e-6;
    }
    std::sort(lat.begin(), lat.end());
    out->frames = frames;
    out->queries = (int64_t)(q1 - q0);
    out->seconds = ms * 1e-3;
    out->queries_per_s = ms > 0 ? (double)(q1 - q0) / (ms * 1e-3) : 0.0;
    if (!lat.empty()) {
        out->bounce_p50_ms = lat[lat.size() / 2];
        out->bounce_p99_ms = lat[std::min(lat.size() - 1, (size_t)(0.99 * (double)lat.size()))];
    }
    out->train_ms_mean = frames ? train_ms / frames : 0.0;
    out->query_ms_mean = frames ? query_ms / frames : 0.0;
    out->advance_ms_mean = frames ? adv_ms / frames : 0.0;
    out->frame_ms_mean = frames ? ms / frames : 0.0;
    cudaMemcpy(&out->last_loss, w->loss, 4, cudaMemcpyDeviceToHost);
    return NPM_OK;
}

npm_status npm_wavefront_destroy(npm_wavefront* w) {
    if (!w) return NPM_OK;
    cudaDeviceSynchronize();
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    if (w->cap) cudaStreamDestroy(w->cap);
    cudaFree(w->mem);
    delete w;
    return NPM_OK;
}

}  // extern "C"
