/*
 * qt_oracle.c -- plain FP64 CPU oracle for the forward step of the Quantization
 * Tree algorithm (Pages & Wilbertz, "GPGPUs in computational finance: Massive
 * parallel computing for American style options", arXiv:1101.3228).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file;
 * it exists so that the tests, the smoke check and the CPU-baseline leg of the
 * benchmark can check the CUDA library.  It shares no source with the CUDA
 * library: every function here is written from the paper (and, for the
 * sampler, from the published definitions it names) and nothing more.
 *
 * What it computes, in the paper's order:
 *   Sec. 3, Prop. 1   -- X_{k+1} = A_k X_k + T_k eps_k (AR(1) form of the chain),
 *                        with the pair (X_k, eps_k) drawn directly (Sec. 4,
 *                        the remark that precedes Algorithm III);
 *   Sec. 2            -- nearest-neighbour (Voronoi) projection onto Gamma_k;
 *   Algorithm III     -- for every layer k and sample m: i = NN(X_k, Gamma_k),
 *                        j = NN(A_k X_k + T_k eps_k, Gamma_{k+1}), count p^k_ij;
 *   Algorithm I/III   -- pi^k_ij = p^k_ij / p^k_i;
 *   Sec. 2 (BDP on the tree) -- V_n = phi_n, V_k = max(phi_k, sum_j pi^k_ij V_{k+1}(j)).
 *   Algorithm II      -- the path-wise estimator (each path through every layer,
 *                        one search per layer), also for an Euler-scheme chain;
 *   eq. (stochCtrl)   -- the swing option's bang-bang BDP over consumption states.
 *
 * Readings where the paper is silent (each is restated in the design notes):
 *   - distance and ties: the cell of z is argmin_i D64(z, x_i) with
 *     D64 = sum_l (z_l - x_il)^2 summed left to right in IEEE binary64,
 *     round to nearest, no fused multiply-add; ties go to the lowest index
 *     (Sec. 2 only says C_i is a subset of the closed Voronoi cell);
 *   - pi^k maps Gamma_k to Gamma_{k+1} (Algorithm III's convention);
 *   - a row with p^k_i = 0 has no continuation value: V_k(i) = phi_k(i);
 *   - samples are produced in single precision (the paper's Sec. 3 data
 *     table states single precision) or in double precision, by the sampler
 *     defined below; both sides compute that sampler exactly.
 *
 * Sampler (the paper leaves the generator open; Sec. 3.1 discusses
 * counter/skip-ahead streams, of which a counter-based generator is the
 * limiting case):
 *   - Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3" (SC'11): key (seed_lo, seed_hi),
 *     counter (m_lo, m_hi, k, r) for sample m, layer k, call r;
 *   - uniforms: FP32 u = (2*(w>>9)+1) * 2^-24;
 *               FP64 u = (2*((w_a>>6)*2^26 + (w_b>>6))+1) * 2^-53;
 *   - normals: Box & Muller (1958), z0 = sqrt(-2 ln u0) cos(2 pi u1),
 *     z1 = sqrt(-2 ln u0) sin(2 pi u1), where ln is 2 atanh((f-1)/(f+1))
 *     after splitting off the binary exponent, and sin/cos are Taylor
 *     polynomials after an exact quarter-turn reduction of u1.  Every step is
 *     a correctly rounded +, -, *, / or sqrt in a fixed order, so any IEEE
 *     machine computes the same bits.
 *   - normal stream: FP32 calls give 4 normals each, FP64 calls give 2;
 *     z = normals [0, d), eps = normals [d, 2d).
 *   - X_k = m_k + L_k z, Y = A_k X_k + b_k + T_k eps, evaluated in the
 *     sample precision, products and sums rounded one at a time in the order
 *     written; L and T are read as lower triangular.
 *
 * Build: cc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__FP_FAST_FMA) && !defined(QTO_ALLOW_FMA_MACRO)
/* Not an error by itself: contraction is controlled by -ffp-contract=off. */
#endif

#define QTO_OK 0
#define QTO_EINVAL 1
#define QTO_ENOMEM 2

#define QTO_PREC_F64 0
#define QTO_PREC_F32 1

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                                      */
/* ------------------------------------------------------------------------ */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u; /* Weyl increments, golden ratio and sqrt(3)-1 */
        k[1] += 0xBB67AE85u;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Vectorised entry for the tests: count blocks, ctr/out are [count][4]. */
void qto_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count)
{
    for (int64_t t = 0; t < count; ++t) philox4x32_10(ctr + 4 * t, key, out + 4 * t);
}

static void sample_counter(uint64_t seed, int32_t k, int64_t m, uint32_t r,
                           uint32_t ctr[4], uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    ctr[0] = (uint32_t)(uint64_t)m;
    ctr[1] = (uint32_t)((uint64_t)m >> 32);
    ctr[2] = (uint32_t)k;
    ctr[3] = r;
}

/* ------------------------------------------------------------------------ */
/* Uniforms                                                                   */
/* ------------------------------------------------------------------------ */

static float uniform_f32(uint32_t w)
{
    /* odd multiple of 2^-24 in (0,1): exact in binary32 */
    const uint32_t j = w >> 9;
    return (float)(2u * j + 1u) * 0x1p-24f;
}

static double uniform_f64(uint32_t wa, uint32_t wb)
{
    const uint64_t j = ((uint64_t)(wa >> 6) << 26) | (uint64_t)(wb >> 6);
    return (double)(2u * j + 1u) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm from 2 atanh(s), s = (f-1)/(f+1)                         */
/* ------------------------------------------------------------------------ */

float qto_ln_f32(float u)
{
    uint32_t bits;
    memcpy(&bits, &u, 4);
    int32_t e = (int32_t)((bits >> 23) & 0xFFu) - 127;
    uint32_t fb = (bits & 0x007FFFFFu) | 0x3F800000u;
    float f;
    memcpy(&f, &fb, 4);
    if (f > 1.41421354f) { /* fold the mantissa into (sqrt(1/2), sqrt(2)] */
        f = f * 0.5f;
        e = e + 1;
    }
    const float s = (f - 1.0f) / (f + 1.0f);
    const float z = s * s;
    float p = (1.0f / 11.0f);
    p = p * z + (1.0f / 9.0f);
    p = p * z + (1.0f / 7.0f);
    p = p * z + (1.0f / 5.0f);
    p = p * z + (1.0f / 3.0f);
    const float t = (s * z) * p;
    const float at = s + t;          /* atanh(s) */
    const float lnf = at + at;       /* ln f = 2 atanh(s) */
    return (float)e * 0.693147182f + lnf;
}

double qto_ln_f64(double u)
{
    uint64_t bits;
    memcpy(&bits, &u, 8);
    int64_t e = (int64_t)((bits >> 52) & 0x7FFu) - 1023;
    uint64_t fb = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double f;
    memcpy(&f, &fb, 8);
    if (f > 1.4142135623730951) {
        f = f * 0.5;
        e = e + 1;
    }
    const double s = (f - 1.0) / (f + 1.0);
    const double z = s * s;
    double p = (1.0 / 21.0);
    p = p * z + (1.0 / 19.0);
    p = p * z + (1.0 / 17.0);
    p = p * z + (1.0 / 15.0);
    p = p * z + (1.0 / 13.0);
    p = p * z + (1.0 / 11.0);
    p = p * z + (1.0 / 9.0);
    p = p * z + (1.0 / 7.0);
    p = p * z + (1.0 / 5.0);
    p = p * z + (1.0 / 3.0);
    const double t = (s * z) * p;
    const double at = s + t;
    const double lnf = at + at;
    return (double)e * 0.6931471805599453 + lnf;
}

/* ------------------------------------------------------------------------ */
/* sin and cos of 2*pi*u for u in (0,1), u a dyadic rational                  */
/* ------------------------------------------------------------------------ */

static void sincos_quarter_f32(float t, float* s, float* c)
{
    /* t in [0, pi/4]: Taylor polynomials in t^2 */
    const float t2 = t * t;
    float ps = (1.0f / 362880.0f);
    ps = ps * t2 + (-1.0f / 5040.0f);
    ps = ps * t2 + (1.0f / 120.0f);
    ps = ps * t2 + (-1.0f / 6.0f);
    *s = t + (t * t2) * ps;
    float pc = (-1.0f / 3628800.0f);
    pc = pc * t2 + (1.0f / 40320.0f);
    pc = pc * t2 + (-1.0f / 720.0f);
    pc = pc * t2 + (1.0f / 24.0f);
    pc = pc * t2 + (-1.0f / 2.0f);
    *c = 1.0f + t2 * pc;
}

void qto_sincos2pi_f32(float u, float* sn, float* cs)
{
    const float v = u * 4.0f;            /* exact */
    const int q = (int)v;                /* quadrant, v >= 0 */
    const float f = v - (float)q;        /* exact, in [0,1) */
    float st, ct, s0, c0;
    if (f > 0.5f) {
        const float g = 1.0f - f;        /* exact */
        sincos_quarter_f32(g * 1.57079637f, &st, &ct);
        s0 = ct;
        c0 = st;
    } else {
        sincos_quarter_f32(f * 1.57079637f, &st, &ct);
        s0 = st;
        c0 = ct;
    }
    switch (q & 3) {
    case 0: *sn = s0; *cs = c0; break;
    case 1: *sn = c0; *cs = -s0; break;
    case 2: *sn = -s0; *cs = -c0; break;
    default: *sn = -c0; *cs = s0; break;
    }
}

static void sincos_quarter_f64(double t, double* s, double* c)
{
    const double t2 = t * t;
    double ps = (1.0 / 355687428096000.0);
    ps = ps * t2 + (-1.0 / 1307674368000.0);
    ps = ps * t2 + (1.0 / 6227020800.0);
    ps = ps * t2 + (-1.0 / 39916800.0);
    ps = ps * t2 + (1.0 / 362880.0);
    ps = ps * t2 + (-1.0 / 5040.0);
    ps = ps * t2 + (1.0 / 120.0);
    ps = ps * t2 + (-1.0 / 6.0);
    *s = t + (t * t2) * ps;
    double pc = (-1.0 / 6402373705728000.0);
    pc = pc * t2 + (1.0 / 20922789888000.0);
    pc = pc * t2 + (-1.0 / 87178291200.0);
    pc = pc * t2 + (1.0 / 479001600.0);
    pc = pc * t2 + (-1.0 / 3628800.0);
    pc = pc * t2 + (1.0 / 40320.0);
    pc = pc * t2 + (-1.0 / 720.0);
    pc = pc * t2 + (1.0 / 24.0);
    pc = pc * t2 + (-1.0 / 2.0);
    *c = 1.0 + t2 * pc;
}

void qto_sincos2pi_f64(double u, double* sn, double* cs)
{
    const double v = u * 4.0;
    const int q = (int)v;
    const double f = v - (double)q;
    double st, ct, s0, c0;
    if (f > 0.5) {
        const double g = 1.0 - f;
        sincos_quarter_f64(g * 1.5707963267948966, &st, &ct);
        s0 = ct;
        c0 = st;
    } else {
        sincos_quarter_f64(f * 1.5707963267948966, &st, &ct);
        s0 = st;
        c0 = ct;
    }
    switch (q & 3) {
    case 0: *sn = s0; *cs = c0; break;
    case 1: *sn = c0; *cs = -s0; break;
    case 2: *sn = -s0; *cs = -c0; break;
    default: *sn = -c0; *cs = s0; break;
    }
}

/* ------------------------------------------------------------------------ */
/* Normal stream of one (layer, sample): g[0 .. count)                       */
/* ------------------------------------------------------------------------ */

static void normals_f32(uint64_t seed, int32_t k, int64_t m, int count, float* g)
{
    uint32_t ctr[4], key[2], w[4];
    int have = 0;
    for (uint32_t r = 0; have < count; ++r) {
        sample_counter(seed, k, m, r, ctr, key);
        philox4x32_10(ctr, key, w);
        for (int pair = 0; pair < 2; ++pair) {
            const float u0 = uniform_f32(w[2 * pair]);
            const float u1 = uniform_f32(w[2 * pair + 1]);
            const float rad = sqrtf(-2.0f * qto_ln_f32(u0));
            float sn, cs;
            qto_sincos2pi_f32(u1, &sn, &cs);
            if (have < count) g[have++] = rad * cs;
            if (have < count) g[have++] = rad * sn;
        }
    }
}

static void normals_f64(uint64_t seed, int32_t k, int64_t m, int count, double* g)
{
    uint32_t ctr[4], key[2], w[4];
    int have = 0;
    for (uint32_t r = 0; have < count; ++r) {
        sample_counter(seed, k, m, r, ctr, key);
        philox4x32_10(ctr, key, w);
        const double u0 = uniform_f64(w[0], w[1]);
        const double u1 = uniform_f64(w[2], w[3]);
        const double rad = sqrt(-2.0 * qto_ln_f64(u0));
        double sn, cs;
        qto_sincos2pi_f64(u1, &sn, &cs);
        if (have < count) g[have++] = rad * cs;
        if (have < count) g[have++] = rad * sn;
    }
}

/* First `count` normals of samples m0 .. m0+M-1 of layer k, widened to FP64. */
int qto_normals(int32_t prec, uint64_t seed, int32_t k, int64_t m0, int64_t M, int32_t count, double* g)
{
    if (count <= 0 || count > 64 || M < 0) return QTO_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) {
        if (prec == QTO_PREC_F32) {
            float tmp[64];
            normals_f32(seed, k, m0 + t, count, tmp);
            for (int q = 0; q < count; ++q) g[t * count + q] = (double)tmp[q];
        } else {
            normals_f64(seed, k, m0 + t, count, g + t * count);
        }
    }
    return QTO_OK;
}

/* Uniform stream for the Monte Carlo pi experiment (Sec. 3.1, Table 2):
 * u[t] = the q-th uniform of Philox call (m0+t, k, r); FP32 layout. */
int qto_uniforms_f32(uint64_t seed, int32_t k, uint32_t r, int64_t m0, int64_t M, float* u4)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) {
        uint32_t ctr[4], key[2], w[4];
        sample_counter(seed, k, m0 + t, r, ctr, key);
        philox4x32_10(ctr, key, w);
        for (int q = 0; q < 4; ++q) u4[4 * t + q] = uniform_f32(w[q]);
    }
    return QTO_OK;
}

/* ------------------------------------------------------------------------ */
/* Pair sampling (Prop. 1 and the pair form used by Algorithm III)            */
/* ------------------------------------------------------------------------ */

#define QTO_DMAX 16

typedef struct {
    int d;
    int prec;
    /* parameters of one layer k, in the sample precision */
    float mf[QTO_DMAX], Lf[QTO_DMAX * QTO_DMAX], Af[QTO_DMAX * QTO_DMAX], bf[QTO_DMAX], Tf[QTO_DMAX * QTO_DMAX];
    double md[QTO_DMAX], Ld[QTO_DMAX * QTO_DMAX], Ad[QTO_DMAX * QTO_DMAX], bd[QTO_DMAX], Td[QTO_DMAX * QTO_DMAX];
} layer_params;

static void load_layer(layer_params* P, int d, int prec, const double* mk, const double* Lk,
                       const double* Ak, const double* bk, const double* Tk)
{
    P->d = d;
    P->prec = prec;
    for (int l = 0; l < d; ++l) {
        P->md[l] = mk[l];
        P->bd[l] = bk[l];
        P->mf[l] = (float)mk[l];
        P->bf[l] = (float)bk[l];
        for (int q = 0; q < d; ++q) {
            P->Ld[l * d + q] = Lk[l * d + q];
            P->Ad[l * d + q] = Ak[l * d + q];
            P->Td[l * d + q] = Tk[l * d + q];
            P->Lf[l * d + q] = (float)Lk[l * d + q];
            P->Af[l * d + q] = (float)Ak[l * d + q];
            P->Tf[l * d + q] = (float)Tk[l * d + q];
        }
    }
}

/* X_k = m_k + L_k z ; Y = A_k X_k + b_k + T_k eps   (one sample) */
static void sample_pair(const layer_params* P, uint64_t seed, int32_t k, int64_t m, double* X, double* Y)
{
    const int d = P->d;
    if (P->prec == QTO_PREC_F32) {
        float g[2 * QTO_DMAX], x[QTO_DMAX];
        normals_f32(seed, k, m, 2 * d, g);
        for (int l = 0; l < d; ++l) {
            float acc = P->mf[l];
            for (int q = 0; q <= l; ++q) acc = acc + P->Lf[l * d + q] * g[q];
            x[l] = acc;
        }
        for (int l = 0; l < d; ++l) {
            float acc = P->bf[l];
            for (int q = 0; q < d; ++q) acc = acc + P->Af[l * d + q] * x[q];
            for (int q = 0; q <= l; ++q) acc = acc + P->Tf[l * d + q] * g[d + q];
            X[l] = (double)x[l];
            Y[l] = (double)acc;
        }
    } else {
        double g[2 * QTO_DMAX], x[QTO_DMAX];
        normals_f64(seed, k, m, 2 * d, g);
        for (int l = 0; l < d; ++l) {
            double acc = P->md[l];
            for (int q = 0; q <= l; ++q) acc = acc + P->Ld[l * d + q] * g[q];
            x[l] = acc;
        }
        for (int l = 0; l < d; ++l) {
            double acc = P->bd[l];
            for (int q = 0; q < d; ++q) acc = acc + P->Ad[l * d + q] * x[q];
            for (int q = 0; q <= l; ++q) acc = acc + P->Td[l * d + q] * g[d + q];
            X[l] = x[l];
            Y[l] = acc;
        }
    }
}

/* Samples m0 .. m0+M-1 of layer k: X, Y are [M][d] FP64 (FP32 values widened). */
int qto_sample_pairs(int32_t d, int32_t prec, uint64_t seed, int32_t k, int64_t m0, int64_t M,
                     const double* mk, const double* Lk, const double* Ak, const double* bk,
                     const double* Tk, double* X, double* Y)
{
    if (d < 1 || d > QTO_DMAX || M < 0) return QTO_EINVAL;
    layer_params P;
    load_layer(&P, d, prec, mk, Lk, Ak, bk, Tk);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) sample_pair(&P, seed, k, m0 + t, X + t * d, Y + t * d);
    return QTO_OK;
}

/* ------------------------------------------------------------------------ */
/* Nearest-neighbour projection (Sec. 2): brute force, FP64, lowest index     */
/* ------------------------------------------------------------------------ */

static double dist64(int d, const double* z, const double* x)
{
    double acc = 0.0;
    for (int l = 0; l < d; ++l) {
        const double t = z[l] - x[l];
        acc = acc + t * t;
    }
    return acc;
}

static int32_t nearest_one(int d, const double* grid, int64_t N, const double* z)
{
    int32_t best = 0;
    double bd = dist64(d, z, grid);
    for (int64_t i = 1; i < N; ++i) {
        const double di = dist64(d, z, grid + i * d);
        if (di < bd) { /* strict: equal distances keep the lower index */
            bd = di;
            best = (int32_t)i;
        }
    }
    return best;
}

int qto_nearest(int32_t d, const double* grid, int64_t N, const double* Z, int64_t M, int32_t* idx)
{
    if (d < 1 || N < 1 || M < 0 || N > 0x7FFFFFFF) return QTO_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) idx[t] = nearest_one(d, grid, N, Z + t * d);
    return QTO_OK;
}

/* Squared distance to the nearest point (quantization error of Sec. 2). */
int qto_nearest_dist(int32_t d, const double* grid, int64_t N, const double* Z, int64_t M, double* dist)
{
    if (d < 1 || N < 1 || M < 0) return QTO_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) {
        const int32_t i = nearest_one(d, grid, N, Z + t * d);
        dist[t] = dist64(d, Z + t * d, grid + (int64_t)i * d);
    }
    return QTO_OK;
}

/* ------------------------------------------------------------------------ */
/* Transition counts p^k_ij (Algorithm III counting step)                     */
/* ------------------------------------------------------------------------ */

/* counts[NA][NB] += #{t : NN(X_t, gA) = i, NN(Y_t, gB) = j}.  Counts are
 * accumulated, not cleared, so several sample ranges can be added up. */
int qto_counts_from_samples(int32_t d, const double* gA, int64_t NA, const double* gB, int64_t NB,
                            const double* X, const double* Y, int64_t M, int64_t* counts)
{
    if (d < 1 || NA < 1 || NB < 1 || M < 0) return QTO_EINVAL;
    int32_t* ii = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    int32_t* jj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    if (!ii || !jj) {
        free(ii);
        free(jj);
        return QTO_ENOMEM;
    }
    qto_nearest(d, gA, NA, X, M, ii);
    qto_nearest(d, gB, NB, Y, M, jj);
    for (int64_t t = 0; t < M; ++t) counts[(int64_t)ii[t] * NB + jj[t]] += 1;
    free(ii);
    free(jj);
    return QTO_OK;
}

/* Whole forward step: every layer k = 0..n-1 draws samples m0..m0+M-1.
 * grids: concatenated [sum_k N_k][d]; counts: concatenated [N_k][N_{k+1}],
 * accumulated (the caller zeroes them).  If ii/jj are non-NULL they receive
 * the cells of every sample, [n][M] each. */
int qto_transitions(int32_t d, int32_t n, const int64_t* N, const double* A, const double* b,
                    const double* T, const double* m, const double* L, const double* grids,
                    int64_t m0, int64_t M, uint64_t seed, int32_t prec, int64_t* counts,
                    int32_t* ii_out, int32_t* jj_out)
{
    if (d < 1 || d > QTO_DMAX || n < 1 || M < 0) return QTO_EINVAL;
    int64_t goff = 0, coff = 0;
    double* X = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1) * (size_t)d);
    double* Y = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1) * (size_t)d);
    int32_t* ii = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    int32_t* jj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    if (!X || !Y || !ii || !jj) {
        free(X); free(Y); free(ii); free(jj);
        return QTO_ENOMEM;
    }
    for (int32_t k = 0; k < n; ++k) {
        const int64_t Nk = N[k], Nk1 = N[k + 1];
        const double* gA = grids + goff * d;
        const double* gB = grids + (goff + Nk) * d;
        qto_sample_pairs(d, prec, seed, k, m0, M, m + (int64_t)k * d, L + (int64_t)k * d * d,
                         A + (int64_t)k * d * d, b + (int64_t)k * d, T + (int64_t)k * d * d, X, Y);
        qto_nearest(d, gA, Nk, X, M, ii);
        qto_nearest(d, gB, Nk1, Y, M, jj);
        int64_t* ck = counts + coff;
        for (int64_t t = 0; t < M; ++t) ck[(int64_t)ii[t] * Nk1 + jj[t]] += 1;
        if (ii_out) memcpy(ii_out + (int64_t)k * M, ii, sizeof(int32_t) * (size_t)M);
        if (jj_out) memcpy(jj_out + (int64_t)k * M, jj, sizeof(int32_t) * (size_t)M);
        goff += Nk;
        coff += Nk * Nk1;
    }
    free(X); free(Y); free(ii); free(jj);
    return QTO_OK;
}

/* ------------------------------------------------------------------------ */
/* Backward dynamic programming on the tree (Sec. 2)                         */
/* ------------------------------------------------------------------------ */

/* phi, V: concatenated [sum_k N_k].  pi^k_ij = p^k_ij / p^k_i (Algorithm III),
 * E(V_{k+1} | X^_k = x_i) = sum_j pi^k_ij V_{k+1}(j) (Sec. 2),
 * V_k(i) = max(phi_k(i), that), V_n = phi_n.  Empty rows: V_k(i) = phi_k(i). */
int qto_backward(int32_t n, const int64_t* N, const int64_t* counts, const double* phi, double* V)
{
    if (n < 1) return QTO_EINVAL;
    int64_t* goff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 2));
    int64_t* coff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!goff || !coff) {
        free(goff); free(coff);
        return QTO_ENOMEM;
    }
    goff[0] = 0;
    coff[0] = 0;
    for (int32_t k = 0; k <= n; ++k) goff[k + 1] = goff[k] + N[k];
    for (int32_t k = 0; k < n; ++k) coff[k + 1] = coff[k] + N[k] * N[k + 1];
    for (int64_t i = 0; i < N[n]; ++i) V[goff[n] + i] = phi[goff[n] + i];
    for (int32_t k = n - 1; k >= 0; --k) {
        const int64_t Nk = N[k], Nk1 = N[k + 1];
        const int64_t* ck = counts + coff[k];
        const double* Vn = V + goff[k + 1];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < Nk; ++i) {
            int64_t ci = 0;
            for (int64_t j = 0; j < Nk1; ++j) ci += ck[i * Nk1 + j];
            const double ph = phi[goff[k] + i];
            if (ci == 0) {
                V[goff[k] + i] = ph;
                continue;
            }
            double cont = 0.0;
            for (int64_t j = 0; j < Nk1; ++j) {
                const double pij = (double)ck[i * Nk1 + j] / (double)ci;
                cont = cont + pij * Vn[j];
            }
            V[goff[k] + i] = ph > cont ? ph : cont;
        }
    }
    free(goff);
    free(coff);
    return QTO_OK;
}

/* Price from V_0: a single root (N_0 = 1) gives V_0(0); otherwise the
 * estimated law of X^_0, p^0_i / M, weights V_0(i). */
double qto_price_from_V(const int64_t* N, const int64_t* counts, const double* V)
{
    const int64_t N0 = N[0], N1 = N[1];
    if (N0 == 1) return V[0];
    int64_t total = 0;
    for (int64_t i = 0; i < N0 * N1; ++i) total += counts[i];
    double price = 0.0;
    for (int64_t i = 0; i < N0; ++i) {
        int64_t ci = 0;
        for (int64_t j = 0; j < N1; ++j) ci += counts[i * N1 + j];
        price = price + ((double)ci / (double)total) * V[i];
    }
    return price;
}

/* ------------------------------------------------------------------------ */
/* Algorithm II: the path-wise estimator (Sec. 3, Algorithms I and II)       */
/* ------------------------------------------------------------------------ */
/*
 * Every path m is simulated layer after layer, as in Algorithms I and II:
 *   X_0 = m_0 + L_0 z,  z = normals [0, d) of stream (m, layer 0);
 *   for k = 0 .. n-1:
 *     eps_k = normals [d, 2d) of stream (m, k);
 *     X_{k+1} = b_k + A_k X_k + S_k(X_k) T_k eps_k;
 *     j = NN(X_{k+1}, Gamma_{k+1});  p^k_ij += 1;  i <- j      (i_0 = NN(X_0, Gamma_0)).
 * S_k = I is the AR(1) chain of Prop. 1.  The Euler-scheme chain (a chain that
 * is not AR(1): its layers cannot be drawn independently, which is what
 * Algorithm III needs) scales row l of the innovation by
 *   s_{k,l}(x) = sqrt(max(alpha_{k,l} + beta_{k,l} x_l, 0)),
 * the Euler step of a square-root diffusion dX = (drift) dt + sqrt(alpha + beta X) dW.
 * In the sample precision, rounded one operation at a time in this order:
 *   s_l = sqrt(max(alpha_l + beta_l * x_l, 0));  t_lq = s_l * T_lq;
 *   acc = b_l; acc += A_lq * x_q (q = 0..d-1); acc += t_lq * eps_q (q = 0..l).
 * (With the AR(1) chain t_lq = T_lq, which is also what s_l = 1 gives.)  The
 * step of layer 0 is therefore the pair Algorithm III draws for layer 0.
 */
typedef struct {
    float af[QTO_DMAX], bf[QTO_DMAX];
    double ad[QTO_DMAX], bd[QTO_DMAX];
    int on;
} euler_params;

static void load_euler(euler_params* E, int d, const double* alpha, const double* beta)
{
    E->on = alpha != NULL && beta != NULL;
    for (int l = 0; l < d; ++l) {
        E->ad[l] = E->on ? alpha[l] : 1.0;
        E->bd[l] = E->on ? beta[l] : 0.0;
        E->af[l] = (float)E->ad[l];
        E->bf[l] = (float)E->bd[l];
    }
}

/* One step of path m from state x (sample precision, widened) at layer k. */
static void path_step(const layer_params* P, const euler_params* E, uint64_t seed, int32_t k, int64_t m,
                      const double* x, double* xn)
{
    const int d = P->d;
    if (P->prec == QTO_PREC_F32) {
        float g[2 * QTO_DMAX], xf[QTO_DMAX], sc[QTO_DMAX];
        normals_f32(seed, k, m, 2 * d, g);
        for (int l = 0; l < d; ++l) xf[l] = (float)x[l];
        for (int l = 0; l < d; ++l) {
            float u = E->af[l] + E->bf[l] * xf[l];
            sc[l] = sqrtf(u > 0.0f ? u : 0.0f);
        }
        for (int l = 0; l < d; ++l) {
            float acc = P->bf[l];
            for (int q = 0; q < d; ++q) acc = acc + P->Af[l * d + q] * xf[q];
            for (int q = 0; q <= l; ++q) {
                const float t = E->on ? sc[l] * P->Tf[l * d + q] : P->Tf[l * d + q];
                acc = acc + t * g[d + q];
            }
            xn[l] = (double)acc;
        }
    } else {
        double g[2 * QTO_DMAX], sc[QTO_DMAX];
        normals_f64(seed, k, m, 2 * d, g);
        for (int l = 0; l < d; ++l) {
            double u = E->ad[l] + E->bd[l] * x[l];
            sc[l] = sqrt(u > 0.0 ? u : 0.0);
        }
        for (int l = 0; l < d; ++l) {
            double acc = P->bd[l];
            for (int q = 0; q < d; ++q) acc = acc + P->Ad[l * d + q] * x[q];
            for (int q = 0; q <= l; ++q) {
                const double t = E->on ? sc[l] * P->Td[l * d + q] : P->Td[l * d + q];
                acc = acc + t * g[d + q];
            }
            xn[l] = acc;
        }
    }
}

/* X_0 = m_0 + L_0 z of path m (z = normals [0, d) of stream (m, 0)). */
static void path_start(const layer_params* P0, uint64_t seed, int64_t m, double* x)
{
    const int d = P0->d;
    if (P0->prec == QTO_PREC_F32) {
        float g[2 * QTO_DMAX];
        normals_f32(seed, 0, m, d, g);
        for (int l = 0; l < d; ++l) {
            float acc = P0->mf[l];
            for (int q = 0; q <= l; ++q) acc = acc + P0->Lf[l * d + q] * g[q];
            x[l] = (double)acc;
        }
    } else {
        double g[2 * QTO_DMAX];
        normals_f64(seed, 0, m, d, g);
        for (int l = 0; l < d; ++l) {
            double acc = P0->md[l];
            for (int q = 0; q <= l; ++q) acc = acc + P0->Ld[l * d + q] * g[q];
            x[l] = acc;
        }
    }
}

/* Paths m0 .. m0+M-1 through layers 0..n.  counts: concatenated [N_k][N_{k+1}],
 * accumulated (the caller zeroes them).  alpha/beta: [n][d] (both NULL: the
 * AR(1) chain).  paths_out (optional): [n+1][M][d] FP64 states; cells_out
 * (optional): [n+1][M] cells. */
int qto_pathwise(int32_t d, int32_t n, const int64_t* N, const double* A, const double* b, const double* T,
                 const double* m, const double* L, const double* alpha, const double* beta, const double* grids,
                 int64_t m0, int64_t M, uint64_t seed, int32_t prec, int64_t* counts, double* paths_out,
                 int32_t* cells_out)
{
    if (d < 1 || d > QTO_DMAX || n < 1 || M < 0) return QTO_EINVAL;
    if ((alpha == NULL) != (beta == NULL)) return QTO_EINVAL;
    int64_t* goff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 2));
    int64_t* coff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    layer_params* LP = (layer_params*)malloc(sizeof(layer_params) * (size_t)(n + 1));
    euler_params* EP = (euler_params*)malloc(sizeof(euler_params) * (size_t)(n + 1));
    if (!goff || !coff || !LP || !EP) {
        free(goff); free(coff); free(LP); free(EP);
        return QTO_ENOMEM;
    }
    goff[0] = 0;
    coff[0] = 0;
    for (int32_t k = 0; k <= n; ++k) goff[k + 1] = goff[k] + N[k];
    for (int32_t k = 0; k < n; ++k) coff[k + 1] = coff[k] + N[k] * N[k + 1];
    /* layer k's step uses A_k, b_k, T_k; layer 0 also m_0, L_0 */
    for (int32_t k = 0; k < n; ++k) {
        load_layer(&LP[k], d, prec, m + (int64_t)k * d, L + (int64_t)k * d * d, A + (int64_t)k * d * d,
                   b + (int64_t)k * d, T + (int64_t)k * d * d);
        load_euler(&EP[k], d, alpha ? alpha + (int64_t)k * d : NULL, beta ? beta + (int64_t)k * d : NULL);
    }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) {
        double x[QTO_DMAX], xn[QTO_DMAX];
        const int64_t mm = m0 + t;
        path_start(&LP[0], seed, mm, x);
        int32_t i = nearest_one(d, grids, N[0], x);
        if (paths_out) for (int l = 0; l < d; ++l) paths_out[t * d + l] = x[l];
        if (cells_out) cells_out[t] = i;
        for (int32_t k = 0; k < n; ++k) {
            path_step(&LP[k], &EP[k], seed, k, mm, x, xn);
            for (int l = 0; l < d; ++l) x[l] = xn[l];
            const int32_t j = nearest_one(d, grids + goff[k + 1] * d, N[k + 1], x);
            int64_t* cell = counts + coff[k] + (int64_t)i * N[k + 1] + j;
#pragma omp atomic
            *cell += 1;
            if (paths_out) for (int l = 0; l < d; ++l) paths_out[((int64_t)(k + 1) * M + t) * d + l] = x[l];
            if (cells_out) cells_out[(int64_t)(k + 1) * M + t] = j;
            i = j;
        }
    }
    free(goff); free(coff); free(LP); free(EP);
    return QTO_OK;
}

/* ------------------------------------------------------------------------ */
/* Swing option on the tree (Sec. 2, eq. (stochCtrl) and its bang-bang BDP)  */
/* ------------------------------------------------------------------------ */
/*
 * Controls q_k in {0, 1} at dates k = 0 .. n-1 (a bang-bang control exists, so
 * the BDP runs over these two values), payoff q_k v_k(X_k), and the global
 * constraint sum_k q_k in [Qmin, Qmax].  The state carries the consumption Q
 * before date k.  Reading of the paper's I_Q and chi: chi(Q, x) = Q + x, and x
 * is admissible at (k, Q) when the consumption can still end inside
 * [Qmin, Qmax]:  F(k+1, Q + x)  with  F(k, Q) = (Q <= Qmax and Q + (n - k) >= Qmin).
 *   P_n(., Q) = 0 where F(n, Q), -inf elsewhere;
 *   P_k(i, Q) = max over admissible x of  x v_k(x_i) + sum_j pi^k_ij P_{k+1}(j, Q + x),
 *               -inf where no x is admissible;  an empty row (p^k_i = 0) has
 *               continuation 0.
 * P: concatenated Q-major blocks, layer k = [Qmax + 1][N_k] at offset
 * (Qmax + 1) * sum_{q<k} N_q.  v: concatenated [sum_k N_k] (layer n unused).
 */
static int swing_feasible(int32_t n, int32_t k, int64_t Q, int32_t Qmin, int32_t Qmax)
{
    return Q <= Qmax && Q + (n - k) >= Qmin;
}

int qto_swing(int32_t n, const int64_t* N, const int64_t* counts, const double* v, int32_t Qmin, int32_t Qmax,
              double* P)
{
    if (n < 1 || Qmin < 0 || Qmax < Qmin) return QTO_EINVAL;
    const int64_t nq = (int64_t)Qmax + 1;
    int64_t* goff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 2));
    int64_t* coff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!goff || !coff) {
        free(goff); free(coff);
        return QTO_ENOMEM;
    }
    goff[0] = 0;
    coff[0] = 0;
    for (int32_t k = 0; k <= n; ++k) goff[k + 1] = goff[k] + N[k];
    for (int32_t k = 0; k < n; ++k) coff[k + 1] = coff[k] + N[k] * N[k + 1];
    double* Pn = P + nq * goff[n];
    for (int64_t Q = 0; Q < nq; ++Q)
        for (int64_t j = 0; j < N[n]; ++j)
            Pn[Q * N[n] + j] = swing_feasible(n, n, Q, Qmin, Qmax) ? 0.0 : -INFINITY;
    for (int32_t k = n - 1; k >= 0; --k) {
        const int64_t Nk = N[k], Nk1 = N[k + 1];
        const int64_t* ck = counts + coff[k];
        const double* Pk1 = P + nq * goff[k + 1];
        double* Pk = P + nq * goff[k];
        const double* vk = v + goff[k];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < Nk; ++i) {
            int64_t ci = 0;
            for (int64_t j = 0; j < Nk1; ++j) ci += ck[i * Nk1 + j];
            for (int64_t Q = 0; Q < nq; ++Q) {
                double best = -INFINITY;
                for (int x = 0; x <= 1; ++x) {
                    const int64_t Q1 = Q + x;
                    if (!swing_feasible(n, k + 1, Q1, Qmin, Qmax)) continue;
                    double cont = 0.0;
                    if (ci > 0) {
                        for (int64_t j = 0; j < Nk1; ++j) {
                            const double pij = (double)ck[i * Nk1 + j] / (double)ci;
                            cont = cont + pij * Pk1[Q1 * Nk1 + j];
                        }
                    }
                    const double val = x ? vk[i] + cont : cont;
                    if (val > best) best = val;
                }
                Pk[Q * Nk + i] = best;
            }
        }
    }
    free(goff);
    free(coff);
    return QTO_OK;
}

int qto_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
