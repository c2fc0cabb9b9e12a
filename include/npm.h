/*
 * npm.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of
 * Neural Parametric Mixtures (NPM) for path guiding (Dong, Wang, Li,
 * SIGGRAPH 2023).
 *
 * What the library computes, per path vertex (a "query"):
 *   1. G(x): a multi-resolution grid embedding of the position x in [0,1]^3,
 *      trilinear blending of the 8 corner features on each level, levels
 *      concatenated (Sec. 5.1, Eq. 11). Levels with D^3 > T are hashed.
 *   2. In product mode (Sec. 4.3, Eq. 13-14) the network input also holds the
 *      spherical-harmonics encoding of the outgoing direction (4 bands, 16
 *      values) and of the normal (2 bands, 4 values) and the roughness.
 *   3. A bias-free MLP with ReLU hidden layers (Sec. 5.3, Eq. 12) decodes the
 *      input into 4K raw outputs, mapped per lobe by Table 1 into a K-lobe
 *      von Mises-Fisher mixture (Eq. 3-4).
 *   4. The mixture is sampled (Sec. 5.3: numerically stable vMF sampling) and
 *      its density evaluated (Eq. 4); training minimises the KL divergence to
 *      the target through its Monte Carlo gradient (Sec. 4.2, Eq. 7-10) with
 *      Adam (Sec. 5.3).
 *
 * Conventions (every entry point):
 *   - Per-query arrays are structure-of-arrays FP32 with a leading dimension
 *     ld >= n: component c of query j is at p[c * ld + j]. (Sec. 5.2 keeps
 *     the wavefront queues in SoA layout.)
 *   - Array arguments of the hot calls are DEVICE pointers owned by the
 *     caller unless the name ends in _host. The library never keeps them.
 *   - The library owns the parameters, the gradient, the Adam moments and a
 *     workspace sized at npm_create from max_batch; the hot calls allocate
 *     nothing.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream). Argument errors are detected on the host and returned
 *     before anything is launched. A failed launch returns NPM_ERR_CUDA. An
 *     asynchronous device fault surfaces as NPM_ERR_CUDA on a later call.
 *   - n == 0 is valid and launches nothing. n > max_batch returns
 *     NPM_ERR_CAPACITY.
 *   - Positions outside [0,1]^3 are clamped to the box; direction arguments
 *     are unit vectors.
 *   - npm_last_error() returns a thread-local description of the last error.
 *   - Each entry point opens an NVTX range named after itself, so profiler
 *     timelines group the kernels of each call.
 *   - Test-only fault injection (host side; off unless set in the
 *     environment): NPM_TEST_FAIL_ALLOC=N fails the N-th device allocation
 *     of each npm_create with NPM_ERR_OOM (everything allocated before is
 *     freed); NPM_TEST_FAIL_LAUNCH=N makes the N-th hot call of the process
 *     (query, evaluation, training or backward) return NPM_ERR_CUDA as if
 *     its launch had failed, launching nothing.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef NPM_H
#define NPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NPM_OK = 0,
    NPM_ERR_INVALID_ARG = 1, /* bad pointer, size, stride or configuration */
    NPM_ERR_OOM = 2,         /* device allocation failed (npm_create only) */
    NPM_ERR_CUDA = 3,        /* a CUDA call or kernel launch failed */
    NPM_ERR_CAPACITY = 4,    /* n > max_batch */
    NPM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    NPM_ERR_NUMERIC = 6,     /* non-finite loss: the Adam step was skipped */
    NPM_ERR_UNSUPPORTED = 7, /* valid but not built (e.g. shape limits) */
    NPM_ERR_IO = 8           /* npm_save / npm_load file error */
} npm_status;

enum { NPM_RADIANCE = 0, NPM_PRODUCT = 1 };  /* Sec. 4.1 / Sec. 4.3 */
enum { NPM_SOFTPLUS = 0, NPM_EXP = 1 };      /* kappa mapping; Table 1 uses exp */
enum { NPM_FP32 = 0, NPM_BF16 = 1, NPM_BF16X3 = 2, NPM_FP16 = 3, NPM_FP32_TC = 4 };  /* MLP / grid arithmetic */

#define NPM_MAX_LEVELS 32
#define NPM_MAX_LAYERS 8
#define NPM_MAX_WIDTH 128
#define NPM_MAX_LOBES 16

/*
 * Model configuration (all fields explicit, no hidden defaults).
 *   level_res[l]   D_l, lattice points per axis on level l (D_l >= 2).
 *   log2_table     T = 2^log2_table entries per hashed level; a level with
 *                  D_l^3 <= T is stored densely (index i + D (j + D k)),
 *                  otherwise hashed: (i ^ j*2654435761 ^ k*805459861) mod T.
 *   widths[0..n_layers]  MLP widths; widths[0] is the network input (grid
 *                  features, plus 21 SH/roughness values in product mode,
 *                  zero-padded), widths[n_layers] must equal 4K. Every width
 *                  is a multiple of 4 and at most NPM_MAX_WIDTH.
 *   precision      NPM_FP32: FP32 grid and CUDA-core FP32 MLP.
 *                  NPM_BF16: FP16 grid copy, BF16 tensor-core MLP (tcgen05)
 *                  with FP32 accumulation; all vMF math stays FP32. Single-
 *                  pass BF16 inference does NOT meet the reduced-precision
 *                  accuracy bar (density within 2e-2 at the 99.9th
 *                  percentile) on mixtures with sharp lobes: at kappa up to
 *                  ~35 its 8-bit significands put the density 1.5e-2 to
 *                  6e-2 off. Use it only where that error is acceptable.
 *                  NPM_BF16X3: as NPM_BF16, but every activation and weight
 *                  is split into a BF16 high part and a BF16 residual, and
 *                  each product is hi*hi + hi*lo + lo*hi (three MMAs per
 *                  K step), which recovers about 16 significant bits; meets
 *                  the bar.
 *                  NPM_FP16: FP16 grid copy, tensor-core MLP on FP16
 *                  operands with FP32 accumulation: activations rounded to
 *                  nearest FP16 (11-bit significands, saturating at the FP16
 *                  range), weights as an FP16 high part plus an FP16
 *                  residual (two MMAs per K step); vMF math in FP32. Meets
 *                  the bar (the FP16 rounding of the activations puts the
 *                  density within about 5e-3 at the 99.9th percentile).
 *                  NPM_FP32_TC: the FP32 path's accuracy on tensor cores:
 *                  the FP32 grid table, and every activation and weight
 *                  split into an FP16 high part and an FP16 residual (about
 *                  22 significant bits), each product hi*hi + hi*lo + lo*hi
 *                  (three MMAs per K step) with FP32 accumulation; vMF math
 *                  and sampling as in NPM_FP32. Held to the FP32 bars
 *                  (density and direction within 1e-4). Values beyond the
 *                  FP16 range (|v| > 65504) saturate; below |v| = 0.125 the
 *                  residual is an FP16 subnormal, so such values are held
 *                  to an absolute error of 2^-25 rather than 22 bits.
 *                  Training in this mode runs the FP32 kernels.
 *                  Training (npm_train_step, npm_backward) multiplies split
 *                  BF16 operands in the reduced-precision modes. Master
 *                  parameters and Adam state are FP32 in all modes.
 *   lr, beta1, beta2, eps   Adam (Sec. 5.3 uses lr 0.005).
 *   max_batch      largest n of any call; sizes the workspace.
 *   seed           seeds npm_create's parameter initialisation
 *                  (grid U[-1e-4, 1e-4], MLP Glorot-uniform).
 */
typedef struct npm_config {
    int mode;
    int n_levels;
    int feat_per_level;
    int log2_table;
    int level_res[NPM_MAX_LEVELS];
    int n_layers;
    int widths[NPM_MAX_LAYERS + 1];
    int K;
    int kappa_act;
    int precision;
    float lr, beta1, beta2, eps;
    int64_t max_batch;
    uint64_t seed;
} npm_config;

typedef struct npm_handle npm_handle;

/* Create a model on the current CUDA device. Parameters start from the
 * seeded initialisation; replace them with npm_set_params. Errors:
 * NPM_ERR_INVALID_ARG for an inconsistent config, NPM_ERR_OOM. */
npm_status npm_create(const npm_config* cfg, npm_handle** out);

/* Free every device buffer of the handle (synchronises the device first).
 * NULL is a no-op. */
npm_status npm_destroy(npm_handle* h);

/*
 * Guided sampling: encode + decode + sample + pdf (Sec. 5.2 steps 1-5).
 *   pos   [3][ld]  positions x.
 *   aux   [7][ld]  product mode: wo (3), normal (3), roughness; NULL in
 *                  radiance mode.
 *   u     [3][ld]  uniforms in [0,1): u0 picks the lobe against the
 *                  cumulative weights, u1 the cosine to the lobe mean
 *                  (inverse CDF), u2 the azimuth. When uniform_frac > 0, u is
 *                  [4][ld] and u3 < uniform_frac draws the direction
 *                  uniformly on the sphere from (u1, u2) instead (a
 *                  one-sample mixture with a BSDF stand-in, Sec. 6.1).
 *   dir_out  [3][ld]  sampled unit directions.
 *   pdf_out  [n]      density of the whole strategy at dir_out:
 *                  uniform_frac/(4 pi) + (1 - uniform_frac) V(dir_out).
 *   mix_out  [4K][ld] or NULL: decoded mixture, rows (lambda, kappa,
 *                  theta, phi) per lobe (Table 1).
 */
npm_status npm_query_sample(npm_handle* h, int64_t n, const float* pos, const float* aux,
                            const float* u, int64_t ld, float uniform_frac, float* dir_out,
                            float* pdf_out, float* mix_out, void* stream);

/* npm_query_sample with every array in HOST memory (pinned memory lets the
 * copies overlap): the library copies the inputs into its own device staging
 * buffers (sized by max_batch at npm_create), runs the same kernel in chunks
 * on two internal streams so that copies and compute overlap, copies dir_out
 * and pdf_out back, and returns after `stream` has completed the work. The
 * host arrays use the same [c][ld] layout. */
npm_status npm_query_sample_host(npm_handle* h, int64_t n, const float* pos, const float* aux,
                                 const float* u, int64_t ld, float uniform_frac, float* dir_out,
                                 float* pdf_out, void* stream);

/* Mixture density V(dir | Theta(x)) (Eq. 4) at given unit directions
 * dir [3][ld]; pdf_out [n]. */
npm_status npm_eval_pdf(npm_handle* h, int64_t n, const float* pos, const float* aux,
                        const float* dir, int64_t ld, float* pdf_out, void* stream);

/* log V(dir | Theta(x)) at given unit directions dir [3][ld]; logpdf_out
 * [n]. Evaluated by the same kernels as npm_eval_pdf in log-sum-exp form:
 * each lobe's term log lambda_i + log c(kappa_i) + kappa_i (mu_i.dir - 1),
 * with log lambda_i taken from the logits, so the result stays finite where
 * V itself underflows FP32 (directions far from every sharp lobe). This is
 * the quantity the training loss (Sec. 4.2, Eq. 8-9) differentiates. */
npm_status npm_eval_log_pdf(npm_handle* h, int64_t n, const float* pos, const float* aux,
                            const float* dir, int64_t ld, float* logpdf_out, void* stream);

/*
 * One training step (Sec. 4.2 and 5.3): the loss
 *   l = -(1/n) sum_j (radiance_j / sample_pdf_j) log V(dir_j | Theta(x_j)),
 * whose gradient is the Monte Carlo KL gradient of Eq. 9 up to the constant
 * normalisation of the target; back-propagation through the mapping, the
 * MLP and the grid (activations recomputed); then one dense Adam step over
 * all parameters.
 *   radiance [n]  noisy estimates L_j >= 0; sample_pdf [n] > 0 the density
 *                 dir_j was drawn from (a constant of the step).
 *   loss_out      device float or NULL; receives l (written, not added).
 * The call does not synchronise. If the loss is not finite the Adam kernel
 * skips the update on the device (parameters and moments unchanged, the step
 * counter still advances) and records NPM_ERR_NUMERIC in the device status
 * word, which npm_check_device_status reports.
 * Training keeps a tile's activations of every layer on chip; networks whose
 * tiles do not fit (for example 128-wide hidden layers with a 128-wide
 * input) return NPM_ERR_UNSUPPORTED here and in npm_backward before anything
 * is launched; inference supports every valid configuration.
 */
npm_status npm_train_step(npm_handle* h, int64_t n, const float* pos, const float* aux,
                          const float* dir, const float* radiance, const float* sample_pdf,
                          int64_t ld, float* loss_out, void* stream);

/* Gradient only: zero the gradient buffer, then accumulate
 * d/dparams of sum_j dlogv_j log V(dir_j | Theta(x_j)) into it.
 * dlogv [n] are the per-query upstream weights (npm_train_step uses
 * -radiance/(n sample_pdf)). */
npm_status npm_backward(npm_handle* h, int64_t n, const float* pos, const float* aux,
                        const float* dir, const float* dlogv, int64_t ld, void* stream);

/* One dense Adam step (with bias correction) from the gradient buffer;
 * clears the gradient. */
npm_status npm_adam_step(npm_handle* h, void* stream);

/* ------------------------------------------------------------- serving */

/*
 * Continuous-batching request loop over one handle (the batched per-bounce
 * queries and the interleaved training batches of Sec. 5.2).
 *
 * Requests carry HOST arrays in the [c][ld] layout (pinned memory lets the
 * copies overlap); they stay owned by the caller until npm_server_wait
 * returns for the request's ticket. A worker thread admits requests in
 * arrival order as soon as a device staging pool of pool_queries queries has
 * room for them (admission by memory): every admitted query request of a
 * round is served by ONE launch of the fused kernel over all of them, on one
 * of two streams, so that requests arriving while others run join the next
 * batch. A training request runs after every earlier query request and
 * before every later one. Results equal those of npm_query_sample for the
 * same inputs and parameters. While a server is attached, the handle must
 * not be used directly. Errors: NPM_ERR_CAPACITY for n > pool_queries or
 * n > the handle's max_batch, NPM_ERR_INVALID_ARG for bad arguments.
 */
typedef struct npm_server npm_server;

typedef struct npm_server_stats {
    int64_t batches;                /* kernel launches (query) and training steps */
    int64_t requests_done;
    int64_t queries_done;
    int64_t train_done;
    int64_t max_requests_per_batch; /* most requests served by one launch */
    int64_t pool_queries;
    int64_t pool_peak_used;
    double latency_p50_ms;          /* submit -> results on the host */
    double latency_p99_ms;
} npm_server_stats;

npm_status npm_server_create(npm_handle* h, int64_t pool_queries, npm_server** out);
npm_status npm_server_submit_query(npm_server* s, int64_t n, const float* pos, const float* aux,
                                   const float* u, int64_t ld, float uniform_frac, float* dir_out,
                                   float* pdf_out, uint64_t* ticket);
npm_status npm_server_submit_train(npm_server* s, int64_t n, const float* pos, const float* aux,
                                   const float* dir, const float* radiance,
                                   const float* sample_pdf, int64_t ld, uint64_t* ticket);
/* hold != 0 pauses admission (submitted requests queue up); hold == 0
 * resumes it, and everything queued is admitted together as memory allows.
 * npm_server_destroy releases a hold. */
npm_status npm_server_hold(npm_server* s, int hold);
/* Blocks until the request is complete; latency_ms (optional) receives
 * submit-to-completion time. Each ticket can be waited for once. */
npm_status npm_server_wait(npm_server* s, uint64_t ticket, double* latency_ms);
npm_status npm_server_get_stats(npm_server* s, npm_server_stats* out);
/* Completes every submitted request, then frees the server. */
npm_status npm_server_destroy(npm_server* s);

/* ------------------------------------------------- wavefront frame driver */

/*
 * A synthetic wavefront path tracer around a radiance-mode handle, standing
 * in for the paper's renderer (Sec. 5.2): per frame, `paths` paths start at
 * seeded positions; each of `bounces` bounces queries the guide on the
 * compacted queue of live paths (npm_query_sample with uniform_frac),
 * evaluates the analytic radiance of the stand-in scene times Exponential(1)
 * noise at the sampled direction, and keeps each path with probability
 * `survival`, moving it along the sampled direction; the first-bounce
 * samples of the first `train_batch` paths feed one npm_train_step per frame.
 * Queue sizes live in device memory: with use_graph the whole frame is
 * captured once into a CUDA graph and replayed. Buffers are allocated at
 * create; run allocates nothing. The handle must not be used by others while
 * frames run.
 */
typedef struct npm_wavefront npm_wavefront;

typedef struct npm_frame_config {
    int64_t paths;        /* paths per frame (<= the handle's max_batch) */
    int bounces;          /* bounces per frame */
    float survival;       /* Bernoulli survival probability per bounce */
    int64_t train_batch;  /* training samples per frame (<= paths) */
    float uniform_frac;   /* probability of the uniform-sphere BSDF stand-in */
    uint64_t seed;
    int use_graph;        /* capture one frame as a CUDA graph and replay it */
    int max_frames;       /* frames over the driver's lifetime (timestamp space) */
} npm_frame_config;

#define NPM_FRAME_BOUNCE_STATS 16  /* bounces with per-bounce figures */

typedef struct npm_frame_stats {
    int64_t frames;
    int64_t queries;        /* guided queries served (sum of live paths) */
    double seconds;         /* device time of the frames */
    double queries_per_s;   /* queries / seconds, training included */
    double bounce_p50_ms;   /* per-bounce batch latency on the device */
    double bounce_p99_ms;   /* (query kernel + scene evaluation and compaction) */
    double frame_ms_mean;
    double train_ms_mean;   /* the per-frame training step */
    float last_loss;
    /* Breakdown of a frame's device time (means over the run's frames):
     * the guide's query kernels of all bounces, and the stand-in scene's
     * evaluation and compaction kernels of all bounces. */
    double query_ms_mean;
    double advance_ms_mean;
    /* Per bounce b < NPM_FRAME_BOUNCE_STATS, means over the run's frames:
     * live paths queried and the query kernel's time. */
    double bounce_queries[NPM_FRAME_BOUNCE_STATS];
    double bounce_query_ms[NPM_FRAME_BOUNCE_STATS];
} npm_frame_stats;

npm_status npm_wavefront_create(npm_handle* h, const npm_frame_config* cfg, npm_wavefront** out);
/* Runs `frames` frames on `stream`, waits for them and fills *out. */
npm_status npm_wavefront_run(npm_wavefront* w, int frames, void* stream, npm_frame_stats* out);
npm_status npm_wavefront_destroy(npm_wavefront* w);

/* ------------------------------------------------- synthetic stand-in scene */

/*
 * Seeded inputs and an analytic target on the device, standing in for the
 * paper's renderer and scenes (which are not part of the method). Random
 * numbers: SplitMix64 at counter i of (seed, stream), uniform = (bits >> 40)
 * * 2^-24; element (r, j) of an [rows][n] block uses counter r*n + j.
 *
 * npm_scene_generate: positions pos [3][ld] uniform in [0,1)^3; in product
 * mode aux [7][ld] = (wo on the normal's hemisphere, normal uniform on the
 * sphere, roughness U[0.05, 1]); sampling uniforms u [urows][ld].
 *
 * npm_scene_radiance: the analytic target at (pos, dir): a sum of three vMF
 * lobes (amplitudes 0.5/0.3/0.2, means and sharpness 1..50 varying smoothly
 * with position; it integrates to 1 over the sphere), times in product mode
 * max(0, n.w)(0.3 + 0.7 D(n.h)/D(1)) with a GGX D of alpha = roughness^2.
 * clean_out [n] (optional) receives the target, noisy_out [n] (optional) the
 * target times Exponential(1) noise drawn from (noise_seed).
 * All pointers are device pointers; both calls are asynchronous.
 */
npm_status npm_scene_generate(uint64_t seed, int64_t n, int product, float* pos, float* aux,
                              float* u, int urows, int64_t ld, void* stream);
npm_status npm_scene_radiance(int product, uint64_t noise_seed, int64_t n, const float* pos,
                              const float* aux, const float* dir, int64_t ld, float* clean_out,
                              float* noisy_out, void* stream);

/* ---------------------------------------------------- allocation-free */

/* Largest padded forward-weight copy npm_eval_pdf_noalloc accepts, in
 * floats (128 KiB of static device memory): the sum over layers of
 * widths[l] * round_up(widths[l+1]) with round_up to 16, 32, 64 or 128. */
#define NPM_NOALLOC_MAX_WEIGHT_FLOATS 32768

/*
 * npm_eval_pdf_noalloc -- mixture density V(dir | Theta(x)) of the FP32 path
 * for callers that cannot allocate device memory. The paper has no
 * counterpart; this is a deployment interface. Examples of such callers: a
 * renderer whose device memory is owned by its own allocator or reserved up
 * front, a plug-in that runs under a host framework that forbids
 * cudaMalloc/cudaFree during a frame, or code that runs between other work on
 * a stream and must not trigger the synchronisation an allocation implies.
 *
 * No handle is needed and nothing is allocated: the caller passes the
 * configuration, the parameters and every input and output; the one piece of
 * scratch the kernel needs (the padded, transposed copy of the MLP weights)
 * lives in a file-scope device array of NPM_NOALLOC_MAX_WEIGHT_FLOATS floats
 * that is loaded with the library on every GPU that uses it and stays
 * resident until the process exits.
 *   cfg      model configuration (precision is ignored: FP32 arithmetic).
 *   params   DEVICE pointer, 16-byte aligned, npm_num_params FP32 values in
 *            the public layout (grid, then each weight matrix row-major).
 *   pos, aux, dir, ld, pdf_out   as for npm_eval_pdf (device pointers);
 *            n is not limited by cfg->max_batch.
 * Errors: NPM_ERR_INVALID_ARG (configuration or arguments),
 * NPM_ERR_CAPACITY when the padded weights exceed
 * NPM_NOALLOC_MAX_WEIGHT_FLOATS, NPM_ERR_CUDA on a failed launch.
 * Kernel: the FP32 tile-group forward kernel, which has no kernel-internal
 * waits (no mailbox hand-offs between thread groups), so no launch can give
 * up part-way: when the call returns NPM_OK, every pdf_out value is written
 * by the work it queued. (npm_eval_pdf on a handle may run the
 * warp-specialised kernel instead, whose bounded waits report through the
 * handle's status word; this entry point has no such word.)
 * Set-up: every call looks up the device address of the scratch array on
 * the current device (cudaGetSymbolAddress: no allocation; the first call
 * on a device also loads the library's device code there, so make the first
 * call on each device before any stream capture). A device reset therefore
 * needs no special handling.
 * Sharing: every call on a device uses the same scratch array, which keeps
 * the contents of the last call. Each call rewrites every value it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (different
 * streams without ordering between them) race on the array and may read
 * each other's weights: order them on one stream or with events.
 */
npm_status npm_eval_pdf_noalloc(const npm_config* cfg, const float* params, int64_t n,
                                const float* pos, const float* aux, const float* dir, int64_t ld,
                                float* pdf_out, void* stream);

/* ------------------------------------------------------------ support */

/* Number of FP32 parameters: grid (level, entry, feature), then each weight
 * matrix row-major [out][in]. */
int64_t npm_num_params(const npm_handle* h);

/* Copy parameters from / to a HOST FP32 buffer of npm_num_params values.
 * set also refreshes the reduced-precision copies and resets nothing else.
 * Both synchronise the device. */
npm_status npm_set_params(npm_handle* h, const float* host, int64_t count);
npm_status npm_get_params(npm_handle* h, float* host, int64_t count);
/* Copy the gradient buffer to a HOST buffer (it holds the result of the last
 * npm_backward; npm_adam_step and npm_train_step leave it zeroed). */
npm_status npm_get_grads(npm_handle* h, float* host, int64_t count);

/* Device-memory forms of npm_set_params / npm_get_grads, ordered on
 * `stream` and not synchronising (for differentiable wrappers that keep the
 * parameters in a framework's device tensor). dev: npm_num_params FP32
 * values in the same public layout, DEVICE memory, owned by the caller.
 * set also refreshes the reduced-precision and padded copies (and restarts
 * the weight average, as npm_set_params does). Errors: NPM_ERR_INVALID_ARG
 * (NULL or a count other than npm_num_params), NPM_ERR_CUDA. */
npm_status npm_set_params_device(npm_handle* h, const float* dev, int64_t count, void* stream);
npm_status npm_get_grads_device(npm_handle* h, float* dev, int64_t count, void* stream);

/* Device pointers to the FP32 master parameters and gradient (owned by the
 * handle, valid until npm_destroy). */
float* npm_params_device(npm_handle* h);
float* npm_grads_device(npm_handle* h);

/*
 * Moving average of the weights for inference (Sec. 5.3: inference applies
 * an exponential moving average of the weights of the previous training
 * steps, which damps the noise of the Monte Carlo gradients).
 *   decay in (0, 1): from now on every Adam step also updates
 *            e <- decay * e + (1 - decay) * p over all parameters (grid and
 *            MLP, fused into the Adam kernel), and every inference call
 *            (npm_query_sample, npm_query_sample_host, npm_eval_pdf, the
 *            server) evaluates the network with e; training keeps using p.
 *            The first enable starts e at the current parameters; calling
 *            again with another decay keeps e. npm_set_params restarts e at
 *            the new parameters.
 *   decay 0: off; inference evaluates p again (e is released).
 * Allocates the average and its padded weight copies on the first enable
 * (not a hot call) and synchronises `stream`. A wavefront driver captures
 * its frame graph on its first run: enable or disable the average before
 * that. Checkpoints (npm_save) do not hold e.
 * Errors: NPM_ERR_INVALID_ARG (decay outside [0, 1)), NPM_ERR_OOM.
 */
npm_status npm_set_ema(npm_handle* h, float decay, void* stream);

/* The moving average in the public parameter layout (host buffer of
 * npm_num_params floats); NPM_ERR_INVALID_ARG when it is off. */
npm_status npm_get_ema_params(npm_handle* h, float* host, int64_t count);

/* Adam state: step counter and moments (host buffers of npm_num_params). */
npm_status npm_get_adam(npm_handle* h, int* step, float* m_host, float* v_host);
npm_status npm_set_adam(npm_handle* h, int step, const float* m_host, const float* v_host);

/* Grid indices for the bit-exact check: out [L][8][n] int32 (level,
 * corner with bit0=+x bit1=+y bit2=+z, query), device pointer. */
npm_status npm_grid_indices(npm_handle* h, int64_t n, const float* pos, int64_t ld,
                            int32_t* out, void* stream);

/* Checkpoint: configuration, parameters, Adam moments and step counter in a
 * binary file. npm_load requires a handle created with the same
 * configuration. */
npm_status npm_save(npm_handle* h, const char* path);
npm_status npm_load(npm_handle* h, const char* path);

/* Reads and clears the device-side status word (non-finite loss, bounded
 * wait timeouts). Synchronises the stream. */
npm_status npm_check_device_status(npm_handle* h, void* stream);

/* Validation (not a hot call): for each of n_pos positions x_p (pos
 * [3][ld], aux [7][ld] in product mode, device memory), the integral over
 * the sphere of the mixture density, I_p = sum_k weights[k] V(dirs_k | x_p),
 * by the caller's quadrature (dirs [3][n_dir] unit vectors and weights
 * [n_dir] doubles, device memory, e.g. Gauss-Legendre in cos(theta) times
 * uniform in phi). V is a density on the sphere (Eq. 3-4), so I_p = 1 up to
 * the quadrature and the density's own rounding. The densities come from
 * npm_eval_pdf (the same kernels as every query); the weighted sums are
 * reduced on the GPU in FP64. out [n_pos] doubles, device memory. Works in
 * chunks through the handle's staging buffers (no allocation), so it must
 * not overlap npm_query_sample_host on the same handle. Asynchronous.
 * Errors: NPM_ERR_INVALID_ARG, NPM_ERR_CAPACITY (n_dir > max_batch). */
npm_status npm_pdf_integral(npm_handle* h, int64_t n_pos, const float* pos, const float* aux, int64_t ld,
                            int64_t n_dir, const float* dirs, const double* weights, double* out,
                            void* stream);

/* Bound of the device-side waits inside the FP32 forward kernel of this
 * handle (its encoder and MLP thread groups hand tiles over through
 * shared-memory mailboxes; failure handling, not part of the method).
 *   cycles > 0: a wait gives up after about `cycles` SM clock cycles
 *               (default 2^31, about a second at 2 GHz);
 *   cycles <= 0: every wait is one non-blocking test, so a hand-off that is
 *               not already complete gives up at once (this lets a test
 *               exercise the timeout path without waiting).
 * A wait that gives up ends the kernel early: the outputs of that call are
 * incomplete and npm_check_device_status then returns NPM_ERR_TIMEOUT. The
 * kernel issues no asynchronous copies, so nothing is left in flight and the
 * context stays usable. Applies to launches made after the call; the
 * tensor-core kernels keep their fixed bound. Errors: NPM_ERR_INVALID_ARG
 * (NULL handle). */
npm_status npm_set_wait_limit(npm_handle* h, int64_t cycles);

/* Debug builds (compiled with NPM_DEBUG_BOUNDS; not a hot call): every
 * kernel checks each grid-entry index and queue slot it computes against
 * its buffer before the access; an index out of range is counted and
 * replaced by 0 (the kernel carries on; no trap). Returns the count since
 * the library was loaded on the current device, -1 in a normal build
 * (checks compiled out), -2 if the count cannot be read. Synchronises
 * with the device. The paper has no counterpart. */
int64_t npm_debug_bounds_violations(void);

/* Thread-local text of the last error returned on this thread. */
const char* npm_last_error(void);

/* ------------------------------------------------------- unit peaks */

/*
 * npm_measure_unit_peaks -- measured throughput of the units the hot path's
 * roofline bounds are built from, on the current device (the paper has no
 * counterpart; these are the denominators of the L2 and ALU/MUFU bounds,
 * next to the HBM copy and tensor GEMM peaks measured elsewhere):
 *   fp32_fma_tflops     packed two-lane FP32 FMA, 2 FLOP per lane-FMA
 *   fp32_fma_scalar_tflops  the same with scalar FMA
 *   mufu_gops           MUFU 2^x results per second
 *   l2_sector_read_gbs  random 32-byte sector reads that bypass L1, from a
 *                       64 MiB buffer resident in L2, bytes of sectors/s
 *   l2_atomic_gops      random FP32 atomic adds (no return) into that buffer
 *   l2_atomic_v2_gops   the same with two-wide FP32 vector atomic adds
 *   l2_atomic_v4_gops   the same with four-wide FP32 vector atomic adds
 *   sm_count, max_sm_clock_mhz  the device's SM count and rated clock
 * Allocates and frees 64 MiB of device memory; runs a few milliseconds of
 * kernels on `stream` and synchronises it. Not for use inside a capture.
 * Errors: NPM_ERR_INVALID_ARG (out NULL), NPM_ERR_OOM, NPM_ERR_CUDA.
 */
typedef struct npm_unit_peaks {
    double fp32_fma_tflops, fp32_fma_scalar_tflops, mufu_gops, l2_sector_read_gbs, l2_atomic_gops,
        l2_atomic_v2_gops, l2_atomic_v4_gops;
    int sm_count;
    double max_sm_clock_mhz;
} npm_unit_peaks;

npm_status npm_measure_unit_peaks(npm_unit_peaks* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NPM_H */
