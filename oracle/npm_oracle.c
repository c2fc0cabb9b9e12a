/*
 * npm_oracle.c -- plain FP64 CPU reference of the Neural Parametric Mixtures
 * (NPM) hot path (Dong, Wang, Li, SIGGRAPH 2023).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers. It shares no code, header, table or
 * constant with the CUDA library and includes nothing from it.
 *
 * Every function below is a direct, slow restatement of one step of the
 * method, in the paper's order and notation, computed in double precision.
 * The only single-precision step is the lattice coordinate p = x * (D - 1)
 * (one float multiply) and its floor, which decide integer grid indices and
 * therefore must be taken in the precision of the fast path (the indices are
 * then compared bit for bit). Everything after the index is FP64.
 *
 * Readings of points the paper leaves open:
 *  - Eq. 11 says "bilinear" but interpolates the eight corners of a 3D cell:
 *    trilinear blending.
 *  - D_l lattice points per axis; p = x (D - 1); cell c = min(floor p, D - 2);
 *    x is clamped to [0, 1].
 *  - A level whose D^3 exceeds the table size T is hashed with the spatial
 *    hash of Instant-NGP (primes 1, 2654435761, 805459861, xor, mod T);
 *    otherwise it is indexed densely as i + D (j + D k).
 *  - Raw outputs per lobe i are interleaved (lambda', kappa', theta', phi').
 *    Table 1: lambda = softmax(lambda'); kappa = exp(kappa') (paper) or
 *    softplus(kappa'); theta = pi * logistic(theta'); phi = 2 pi *
 *    logistic(phi'); mu = (sin t cos p, sin t sin p, cos t).
 *  - The MLP has no biases; hidden layers use ReLU; the last layer is linear.
 *  - Training minimises the weighted negative log-likelihood
 *    -(1/N) sum_j (L_j / p_j) log V(w_j), whose gradient is Eq. 9 with the
 *    unnormalised target L in place of D (a constant factor).
 *  - Sampling: the smallest lobe i with u0 < cumulative weight; the last lobe
 *    if rounding leaves u0 above the total. The lobe's cos-angle is drawn by
 *    the inversion of Jakob 2012; azimuth 2 pi u2; frame of Duff et al. 2017.
 *    The returned density is the mixture density at the sample.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int mode;            /* 0: radiance NPM, 1: product NPM (Sec. 4.3) */
    int n_levels;        /* L (Sec. 5.1) */
    int feat;            /* F features per lattice point */
    int log2_table;      /* T = 2^log2_table entries per hashed level */
    int level_res[32];   /* D_l, lattice points per axis */
    int n_layers;        /* number of weight matrices */
    int widths[17];      /* widths[0] = MLP input, widths[n_layers] = 4K */
    int K;               /* number of vMF lobes */
    int kappa_act;       /* 0: softplus, 1: exp (Table 1) */
} orc_cfg;

/* ---------------------------------------------------------------- sizes */

static int64_t level_entries(const orc_cfg* c, int l) {
    int64_t d = c->level_res[l];
    int64_t t = (int64_t)1 << c->log2_table;
    int64_t d3 = d * d * d;
    return d3 <= t ? d3 : t;
}

/* Entry offset of each level (levels stored back to back); returns total. */
int64_t orc_grid_offsets(const orc_cfg* c, int64_t* offsets) {
    int64_t off = 0;
    for (int l = 0; l < c->n_levels; ++l) {
        if (offsets) offsets[l] = off;
        off += level_entries(c, l);
    }
    return off;
}

int64_t orc_n_params(const orc_cfg* c) {
    int64_t n = orc_grid_offsets(c, NULL) * c->feat;
    for (int i = 0; i < c->n_layers; ++i) n += (int64_t)c->widths[i] * c->widths[i + 1];
    return n;
}

/* ------------------------------------------- Sec. 5.1: lattice and index */

/* Lattice index of integer point (i, j, k) on level l. */
uint32_t orc_lattice_index(const orc_cfg* c, int l, uint32_t i, uint32_t j, uint32_t k) {
    uint32_t d = (uint32_t)c->level_res[l];
    uint64_t t = (uint64_t)1 << c->log2_table;
    if ((uint64_t)d * d * d <= t) return i + d * (j + d * k);
    uint32_t h = (i * 1u) ^ (j * 2654435761u) ^ (k * 805459861u);
    return (uint32_t)(h % (uint32_t)t);
}

/* Eight corner indices and trilinear weights of x on level l (Eq. 11).
 * Corner order: bit 0 = +x, bit 1 = +y, bit 2 = +z. */
void orc_grid_corners(const orc_cfg* c, int l, const float x[3], uint32_t idx[8], double w[8]) {
    int d = c->level_res[l];
    uint32_t cell[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        float xa = x[a];
        if (!(xa >= 0.0f)) xa = 0.0f;          /* also maps NaN to 0 */
        if (xa > 1.0f) xa = 1.0f;
        volatile float p = xa * (float)(d - 1); /* one float multiply */
        float fl = floorf(p);
        int ci = (int)fl;
        if (ci > d - 2) ci = d - 2;
        cell[a] = (uint32_t)ci;
        f[a] = (double)p - (double)ci;
    }
    for (int corner = 0; corner < 8; ++corner) {
        uint32_t o[3];
        double wt = 1.0;
        for (int a = 0; a < 3; ++a) {
            int bit = (corner >> a) & 1;
            o[a] = cell[a] + (uint32_t)bit;
            wt *= bit ? f[a] : 1.0 - f[a];
        }
        idx[corner] = orc_lattice_index(c, l, o[0], o[1], o[2]);
        w[corner] = wt;
    }
}

/* G(x) of Eq. 11: per level, the trilinear blend of the corner features,
 * levels concatenated. out has n_levels * feat entries. */
void orc_grid_encode(const orc_cfg* c, const double* params, const float x[3], double* out) {
    int64_t off[32];
    orc_grid_offsets(c, off);
    for (int l = 0; l < c->n_levels; ++l) {
        uint32_t idx[8];
        double w[8];
        orc_grid_corners(c, l, x, idx, w);
        for (int q = 0; q < c->feat; ++q) {
            double s = 0.0;
            for (int corner = 0; corner < 8; ++corner)
                s += w[corner] * params[(off[l] + idx[corner]) * c->feat + q];
            out[l * c->feat + q] = s;
        }
    }
}

/* ------------------------------- Sec. 4.3: spherical-harmonics encoding */

/* Real orthonormal spherical harmonics of a unit vector, bands 0..bands-1
 * (bands <= 4), written out from their closed forms
 * Y_l^m = N_l^m P_l^|m|(z) * {cos, sin}(|m| phi) in Cartesian coordinates. */
void orc_sh(int bands, const double d[3], double* out) {
    double x = d[0], y = d[1], z = d[2];
    int n = 0;
    if (bands >= 1) out[n++] = 0.5 * sqrt(1.0 / ORC_PI);
    if (bands >= 2) {
        double c1 = sqrt(3.0 / (4.0 * ORC_PI));
        out[n++] = c1 * y;
        out[n++] = c1 * z;
        out[n++] = c1 * x;
    }
    if (bands >= 3) {
        double c2 = 0.5 * sqrt(15.0 / ORC_PI);
        out[n++] = c2 * x * y;
        out[n++] = c2 * y * z;
        out[n++] = 0.25 * sqrt(5.0 / ORC_PI) * (3.0 * z * z - 1.0);
        out[n++] = c2 * x * z;
        out[n++] = 0.25 * sqrt(15.0 / ORC_PI) * (x * x - y * y);
    }
    if (bands >= 4) {
        double a = 0.25 * sqrt(35.0 / (2.0 * ORC_PI));
        double b = 0.5 * sqrt(105.0 / ORC_PI);
        double e = 0.25 * sqrt(21.0 / (2.0 * ORC_PI));
        out[n++] = a * y * (3.0 * x * x - y * y);
        out[n++] = b * x * y * z;
        out[n++] = e * y * (5.0 * z * z - 1.0);
        out[n++] = 0.25 * sqrt(7.0 / ORC_PI) * z * (5.0 * z * z - 3.0);
        out[n++] = e * x * (5.0 * z * z - 1.0);
        out[n++] = 0.25 * sqrt(105.0 / ORC_PI) * z * (x * x - y * y);
        out[n++] = a * x * (x * x - 3.0 * y * y);
    }
}

/* Network input: G(x), then in product mode SH of wo (4 bands), SH of the
 * normal (2 bands) and the roughness; zero padding up to widths[0]. */
void orc_encode(const orc_cfg* c, const double* params, const float x[3], const float* aux7,
                double* enc) {
    int w0 = c->widths[0];
    for (int i = 0; i < w0; ++i) enc[i] = 0.0;
    orc_grid_encode(c, params, x, enc);
    if (c->mode == 1) {
        int o = c->n_levels * c->feat;
        double wo[3] = {aux7[0], aux7[1], aux7[2]};
        double nn[3] = {aux7[3], aux7[4], aux7[5]};
        orc_sh(4, wo, enc + o);
        orc_sh(2, nn, enc + o + 16);
        enc[o + 20] = aux7[6];
    }
}

/* ------------------------------------------------ Sec. 5.3: decoder MLP */

static const double* mlp_weights(const orc_cfg* c, const double* params, int layer) {
    int64_t o = orc_grid_offsets(c, NULL) * c->feat;
    for (int i = 0; i < layer; ++i) o += (int64_t)c->widths[i] * c->widths[i + 1];
    return params + o;
}

/* Forward pass. acts (optional) receives every layer's pre-activation z_i
 * (i = 1..n_layers) back to back; raw receives the last layer's output. */
void orc_mlp(const orc_cfg* c, const double* params, const double* in, double* raw, double* acts) {
    double h[2][256];
    int wi = c->widths[0];
    for (int k = 0; k < wi; ++k) h[0][k] = in[k];
    int cur = 0;
    int64_t ao = 0;
    for (int layer = 0; layer < c->n_layers; ++layer) {
        const double* W = mlp_weights(c, params, layer);
        int wo = c->widths[layer + 1];
        int last = layer == c->n_layers - 1;
        for (int j = 0; j < wo; ++j) {
            double z = 0.0;
            for (int k = 0; k < wi; ++k) z += W[(int64_t)j * wi + k] * h[cur][k];
            if (acts) acts[ao + j] = z;
            h[1 - cur][j] = last ? z : (z > 0.0 ? z : 0.0);
        }
        ao += wo;
        cur = 1 - cur;
        wi = wo;
    }
    for (int j = 0; j < wi; ++j) raw[j] = h[cur][j];
}

/* --------------------------------------------- Table 1: output mapping */

typedef struct {
    double lam, kap, th, ph, mu[3];
} orc_lobe;

static double logistic(double t) { return 1.0 / (1.0 + exp(-t)); }

static double softplus(double t) { return t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t)); }

void orc_decode(const orc_cfg* c, const double* raw, orc_lobe* lobes) {
    int K = c->K;
    double mx = -INFINITY;
    for (int i = 0; i < K; ++i) mx = raw[4 * i] > mx ? raw[4 * i] : mx;
    double s = 0.0;
    for (int i = 0; i < K; ++i) s += exp(raw[4 * i] - mx);
    for (int i = 0; i < K; ++i) {
        orc_lobe* L = &lobes[i];
        L->lam = exp(raw[4 * i] - mx) / s;
        L->kap = c->kappa_act == 1 ? exp(raw[4 * i + 1]) : softplus(raw[4 * i + 1]);
        L->th = ORC_PI * logistic(raw[4 * i + 2]);
        L->ph = 2.0 * ORC_PI * logistic(raw[4 * i + 3]);
        L->mu[0] = sin(L->th) * cos(L->ph);
        L->mu[1] = sin(L->th) * sin(L->ph);
        L->mu[2] = cos(L->th);
    }
}

/* --------------------------------------------------- Eq. 3-4: densities */

/* vMF normaliser, kappa / (4 pi sinh kappa) times e^kappa so that it pairs
 * with exp(kappa (mu.w - 1)); the kappa -> 0 limit is 1 / (4 pi). */
double orc_vmf_scaled_norm(double k) {
    if (k < 1e-8) return (1.0 + k) / (4.0 * ORC_PI);
    return k / (2.0 * ORC_PI * (-expm1(-2.0 * k)));
}

double orc_vmf_pdf(const double mu[3], double k, const double w[3]) {
    double d = mu[0] * w[0] + mu[1] * w[1] + mu[2] * w[2];
    return orc_vmf_scaled_norm(k) * exp(k * (d - 1.0));
}

double orc_mixture_pdf(int K, const orc_lobe* lobes, const double w[3]) {
    double v = 0.0;
    for (int i = 0; i < K; ++i) v += lobes[i].lam * orc_vmf_pdf(lobes[i].mu, lobes[i].kap, w);
    return v;
}

/* ----------------------------------------------------- Sec. 5.3: sampling */

/* Orthonormal basis (t, b) completing the unit vector n, following
 * Duff et al. 2017, "Building an Orthonormal Basis, Revisited". */
void orc_frame(const double n[3], double t[3], double b[3]) {
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double bb = n[0] * n[1] * a;
    t[0] = 1.0 + sg * n[0] * n[0] * a;
    t[1] = sg * bb;
    t[2] = -sg * n[0];
    b[0] = bb;
    b[1] = sg + n[1] * n[1] * a;
    b[2] = -n[1];
}

/* Cosine of the angle to the mean for one lobe: inverse of the CDF
 * P(W <= w) = (e^{k w} - e^{-k}) / (2 sinh k), in the log1p/expm1 form of
 * Jakob 2012 (numerically stable for large k). */
double orc_vmf_sample_w(double k, double u1) {
    if (k <= 0.0) return 1.0 - 2.0 * u1;
    double w = 1.0 + log1p(u1 * expm1(-2.0 * k)) / k;
    if (w > 1.0) w = 1.0;
    if (w < -1.0) w = -1.0;
    return w;
}

void orc_vmf_sample(const double mu[3], double k, double u1, double u2, double out[3]) {
    double W = orc_vmf_sample_w(k, u1);
    double s = sqrt(fmax(0.0, (1.0 - W) * (1.0 + W)));
    double p = 2.0 * ORC_PI * u2;
    double lx = s * cos(p), ly = s * sin(p);
    double t[3], b[3];
    orc_frame(mu, t, b);
    for (int a = 0; a < 3; ++a) out[a] = lx * t[a] + ly * b[a] + W * mu[a];
}

/* Lobe picked by u0: smallest i with u0 < lambda_0 + ... + lambda_i. Also
 * returns the distance of u0 to the nearest inner boundary of the CDF. */
int orc_pick_lobe(int K, const orc_lobe* lobes, double u0, double* margin) {
    double cum = 0.0, m = INFINITY;
    int sel = -1;
    for (int i = 0; i < K; ++i) {
        cum += lobes[i].lam;
        if (i < K - 1 && fabs(u0 - cum) < m) m = fabs(u0 - cum);
        if (sel < 0 && u0 < cum) sel = i;
    }
    if (sel < 0) sel = K - 1;
    if (margin) *margin = m;
    return sel;
}

/* ------------------------------------------------------ batch drivers */

/* One query: x (and aux) -> decoded lobes. */
static void decode_query(const orc_cfg* c, const double* params, const float x[3],
                         const float* aux7, orc_lobe* lobes, double* raw) {
    double enc[256];
    orc_encode(c, params, x, aux7, enc);
    orc_mlp(c, params, enc, raw, NULL);
    orc_decode(c, raw, lobes);
}

static void gather3(const float* base, int64_t ld, int64_t j, float out[3]) {
    out[0] = base[j];
    out[1] = base[ld + j];
    out[2] = base[2 * ld + j];
}

/* Decoded mixture per query: out [4K][ld] rows (lambda, kappa, theta, phi)
 * per lobe. */
void orc_decode_batch(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                      const float* aux, int64_t ld, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        float x[3], a7[7];
        gather3(pos, ld, j, x);
        if (c->mode == 1)
            for (int r = 0; r < 7; ++r) a7[r] = aux[r * ld + j];
        orc_lobe lobes[64];
        double raw[256];
        decode_query(c, params, x, a7, lobes, raw);
        for (int i = 0; i < c->K; ++i) {
            out[(4 * i + 0) * ld + j] = lobes[i].lam;
            out[(4 * i + 1) * ld + j] = lobes[i].kap;
            out[(4 * i + 2) * ld + j] = lobes[i].th;
            out[(4 * i + 3) * ld + j] = lobes[i].ph;
        }
    }
}

/* Guided sampling (Sec. 5.2-5.3). u is [3][ld], or [4][ld] when alpha > 0:
 * with probability alpha (u3 < alpha) the direction is drawn uniformly on
 * the sphere from (u1, u2) instead -- the one-sample mixture with a 50 %
 * BSDF-selection probability of Sec. 6.1, a uniform sphere standing in for
 * the BSDF. pdf_out is the density of the whole strategy at the returned
 * direction: alpha / (4 pi) + (1 - alpha) V(w). forced (optional, [n]) forces
 * the lobe when >= 0. lobe_out / margin_out are optional diagnostics. */
void orc_query_sample(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                      const float* aux, const float* u, int64_t ld, double alpha,
                      const int* forced, double* dir_out, double* pdf_out, int* lobe_out,
                      double* margin_out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        float x[3], a7[7];
        gather3(pos, ld, j, x);
        if (c->mode == 1)
            for (int r = 0; r < 7; ++r) a7[r] = aux[r * ld + j];
        orc_lobe lobes[64];
        double raw[256];
        decode_query(c, params, x, a7, lobes, raw);
        double u0 = u[j], u1 = u[ld + j], u2 = u[2 * ld + j];
        double w[3], margin = INFINITY;
        int sel = -1;
        if (alpha > 0.0 && (double)u[3 * ld + j] < alpha) {
            double z = 1.0 - 2.0 * u1;
            double r = sqrt(fmax(0.0, 1.0 - z * z));
            double p = 2.0 * ORC_PI * u2;
            w[0] = r * cos(p);
            w[1] = r * sin(p);
            w[2] = z;
        } else {
            sel = orc_pick_lobe(c->K, lobes, u0, &margin);
            if (forced && forced[j] >= 0) sel = forced[j];
            orc_vmf_sample(lobes[sel].mu, lobes[sel].kap, u1, u2, w);
        }
        double v = orc_mixture_pdf(c->K, lobes, w);
        for (int a = 0; a < 3; ++a) dir_out[a * ld + j] = w[a];
        pdf_out[j] = alpha > 0.0 ? alpha / (4.0 * ORC_PI) + (1.0 - alpha) * v : v;
        if (lobe_out) lobe_out[j] = sel;
        if (margin_out) margin_out[j] = margin;
    }
}

/* Mixture density V(w | Theta(x)) at given directions (Eq. 4). */
void orc_eval_pdf(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                  const float* aux, const float* dir, int64_t ld, double* pdf_out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        float x[3], a7[7], wf[3];
        gather3(pos, ld, j, x);
        gather3(dir, ld, j, wf);
        if (c->mode == 1)
            for (int r = 0; r < 7; ++r) a7[r] = aux[r * ld + j];
        orc_lobe lobes[64];
        double raw[256];
        decode_query(c, params, x, a7, lobes, raw);
        double w[3] = {wf[0], wf[1], wf[2]};
        pdf_out[j] = orc_mixture_pdf(c->K, lobes, w);
    }
}

/* Same as orc_eval_pdf with FP64 directions (used for quadrature). */
void orc_eval_pdf64(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                    const float* aux, const double* dir, int64_t ld, double* pdf_out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        float x[3], a7[7];
        gather3(pos, ld, j, x);
        if (c->mode == 1)
            for (int r = 0; r < 7; ++r) a7[r] = aux[r * ld + j];
        orc_lobe lobes[64];
        double raw[256];
        decode_query(c, params, x, a7, lobes, raw);
        double w[3] = {dir[j], dir[ld + j], dir[2 * ld + j]};
        pdf_out[j] = orc_mixture_pdf(c->K, lobes, w);
    }
}

/* Grid indices for the bit-exact check: out [L][8][n] (level, corner,
 * query). */
void orc_grid_indices(const orc_cfg* c, int64_t n, const float* pos, int64_t ld, int32_t* out) {
    for (int64_t j = 0; j < n; ++j) {
        float x[3];
        gather3(pos, ld, j, x);
        for (int l = 0; l < c->n_levels; ++l) {
            uint32_t idx[8];
            double w[8];
            orc_grid_corners(c, l, x, idx, w);
            for (int corner = 0; corner < 8; ++corner)
                out[((int64_t)l * 8 + corner) * n + j] = (int32_t)idx[corner];
        }
    }
}

/* ------------------------------------------ Sec. 4.2: loss and gradient */

/* 1/k - coth k, the derivative of log(k / sinh k). */
static double inv_minus_coth(double k) {
    if (k < 1e-4) return -k / 3.0 + k * k * k / 45.0;
    return 1.0 / k - 1.0 / tanh(k);
}

/* Gradient of the training loss l = -(1/N) sum_j w_j log V(w_j | Theta(x_j)),
 * w_j = L_j / p_j (Eq. 8-9 with the unnormalised target), with respect to
 * every parameter (grid, then weight matrices). Single-threaded, fixed order.
 * grad (n_params doubles) is overwritten. Returns the loss. */
double orc_train_grad(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                      const float* aux, const float* dir, const float* L, const float* pt,
                      int64_t ld, double* grad) {
    int64_t np = orc_n_params(c);
    for (int64_t i = 0; i < np; ++i) grad[i] = 0.0;
    int64_t goff[32];
    int64_t ng = orc_grid_offsets(c, goff) * c->feat;
    int nl = c->n_layers, K = c->K;
    int64_t woff[17];
    woff[0] = ng;
    int tot_act = 0;
    for (int i = 0; i < nl; ++i) {
        woff[i + 1] = woff[i] + (int64_t)c->widths[i] * c->widths[i + 1];
        tot_act += c->widths[i + 1];
    }
    double* z = (double*)malloc(sizeof(double) * (size_t)tot_act);
    double loss = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        float x[3], a7[7], wf[3];
        gather3(pos, ld, j, x);
        gather3(dir, ld, j, wf);
        if (c->mode == 1)
            for (int r = 0; r < 7; ++r) a7[r] = aux[r * ld + j];
        double w[3] = {wf[0], wf[1], wf[2]};
        double enc[256], raw[256];
        orc_encode(c, params, x, a7, enc);
        orc_mlp(c, params, enc, raw, z);
        orc_lobe lobes[64];
        orc_decode(c, raw, lobes);
        double v[64], V = 0.0;
        for (int i = 0; i < K; ++i) {
            v[i] = orc_vmf_pdf(lobes[i].mu, lobes[i].kap, w);
            V += lobes[i].lam * v[i];
        }
        double wt = (double)L[j] / (double)pt[j];
        double s = -wt / (double)n; /* d loss / d log V */
        loss += s * log(V);
        /* d log V / d raw, Table 1 chain rule. */
        double delta[256];
        for (int i = 0; i < K; ++i) {
            const orc_lobe* lb = &lobes[i];
            double r = lb->lam * v[i] / V;
            double md = lb->mu[0] * w[0] + lb->mu[1] * w[1] + lb->mu[2] * w[2];
            double dk = c->kappa_act == 1 ? lb->kap : logistic(raw[4 * i + 1]);
            double st = logistic(raw[4 * i + 2]), sp = logistic(raw[4 * i + 3]);
            double dmu_dth[3] = {cos(lb->th) * cos(lb->ph), cos(lb->th) * sin(lb->ph), -sin(lb->th)};
            double dmu_dph[3] = {-sin(lb->th) * sin(lb->ph), sin(lb->th) * cos(lb->ph), 0.0};
            double wdth = dmu_dth[0] * w[0] + dmu_dth[1] * w[1] + dmu_dth[2] * w[2];
            double wdph = dmu_dph[0] * w[0] + dmu_dph[1] * w[1] + dmu_dph[2] * w[2];
            delta[4 * i + 0] = s * (r - lb->lam);
            delta[4 * i + 1] = s * r * (inv_minus_coth(lb->kap) + md) * dk;
            delta[4 * i + 2] = s * r * lb->kap * wdth * ORC_PI * st * (1.0 - st);
            delta[4 * i + 3] = s * r * lb->kap * wdph * 2.0 * ORC_PI * sp * (1.0 - sp);
        }
        /* Back-propagate through the MLP, layer by layer. */
        int zo = tot_act;
        for (int layer = nl - 1; layer >= 0; --layer) {
            int wi = c->widths[layer], wo = c->widths[layer + 1];
            zo -= wo;
            const double* W = params + woff[layer];
            double hin[256];
            if (layer == 0) {
                for (int k = 0; k < wi; ++k) hin[k] = enc[k];
            } else {
                int zp = zo - wi;
                for (int k = 0; k < wi; ++k) hin[k] = z[zp + k] > 0.0 ? z[zp + k] : 0.0;
            }
            double* gW = grad + woff[layer];
            for (int o = 0; o < wo; ++o)
                for (int k = 0; k < wi; ++k) gW[(int64_t)o * wi + k] += delta[o] * hin[k];
            double back[256];
            for (int k = 0; k < wi; ++k) {
                double sacc = 0.0;
                for (int o = 0; o < wo; ++o) sacc += W[(int64_t)o * wi + k] * delta[o];
                back[k] = sacc;
            }
            if (layer > 0) {
                int zp = zo - wi;
                for (int k = 0; k < wi; ++k) delta[k] = z[zp + k] > 0.0 ? back[k] : 0.0;
            } else {
                for (int k = 0; k < wi; ++k) delta[k] = back[k];
            }
        }
        /* delta now holds d loss / d encoding; scatter the grid part. */
        for (int l = 0; l < c->n_levels; ++l) {
            uint32_t idx[8];
            double cw[8];
            orc_grid_corners(c, l, x, idx, cw);
            for (int corner = 0; corner < 8; ++corner)
                for (int q = 0; q < c->feat; ++q)
                    grad[(goff[l] + idx[corner]) * c->feat + q] += cw[corner] * delta[l * c->feat + q];
        }
    }
    free(z);
    return loss;
}

/* Loss only (same definition as orc_train_grad, no gradient). */
double orc_train_loss(const orc_cfg* c, const double* params, int64_t n, const float* pos,
                      const float* aux, const float* dir, const float* L, const float* pt,
                      int64_t ld) {
    double* pdf = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_eval_pdf(c, params, n, pos, aux, dir, ld, pdf);
    double loss = 0.0;
    for (int64_t j = 0; j < n; ++j) loss -= ((double)L[j] / (double)pt[j]) * log(pdf[j]) / (double)n;
    free(pdf);
    return loss;
}

/* --------------------------------------------------- Sec. 5.3: Adam */

/* One Adam step (Kingma and Ba) with bias correction at step t (1-based). */
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v, int t, double lr,
              double b1, double b2, double eps) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Sec. 5.3, inference weights: the exponential moving average of the
 * parameters after each training step, e <- d e + (1 - d) p. */
void orc_ema(int64_t n, double* e, const double* p, double d) {
    for (int64_t i = 0; i < n; ++i) e[i] = d * e[i] + (1.0 - d) * p[i];
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
