/*
 * Plain CPU oracle for the batched BP decoders of Zhao & Lau,
 * "Implementation of Decoders for LDPC Block Codes and LDPC Convolutional
 * Codes Based on GPUs" (arXiv 1204.0334).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Everything here is slow on purpose: one frame at a time, plain loops over
 * the edge lists of a general sparse H, double precision, in the order the
 * paper states the steps.  OpenMP only distributes independent frames
 * (the paper's own multi-thread CPU decoder is an OpenMP loop, Sec. IV-C).
 *
 * Contents
 *   or_philox4x32_10   counter-based generator (Salmon et al., SC'11)
 *   or_ln_f32,         the channel generator's binary32 ln and sin/cos of 2 pi u
 *   or_sincos2pi_f32   (range reduction + minimax polynomials, defined op by op)
 *   or_channel_awgn    BPSK over AWGN, channel LLR (Sec. II-B: x = 1 - 2c,
 *   or_channel_awgn_cw y = x + g, mu = 2y/sigma^2), all-zero or given codeword,
 *                      in binary32 as the generator defines it
 *   or_sp_decode       sum-product BP, Algorithm 1 (eqs. bphs, bpvs, bpd,
 *                      hrddcs), phi-form or literal tanh-form check update
 *   or_ms_decode       integer min-sum (fixed-point variant of the CN rule)
 *   or_noms_forward /  normalized/offset min-sum with per-iteration,
 *   or_noms_backward   per-circulant parameters, and its reverse-mode
 *                      gradient (hand-derived)
 *   or_ldpccc_decode   pipelined BP of the LDPC convolutional code derived
 *                      from a QC base matrix, Algorithm 2 and Sec. IV-B-2
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the two-multiplier S-box with a   */
/* Weyl-sequence key schedule.                                               */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ c[1] ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c[3] ^ k1;
        uint32_t n3 = lo_a;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ------------------------------------------------------------------------ */
/* The channel generator in binary32.  The LLRs the decoders receive are      */
/* binary32, and this generator is defined operation by operation so that any */
/* implementation of the same definition produces the same bits.  Every       */
/* arithmetic step below is one IEEE-754 binary32 operation rounded to        */
/* nearest-even: + - * / sqrtf, and fmaf where written (this file is compiled */
/* with -ffp-contract=off, so nothing else is fused).                         */
/*                                                                            */
/* Uniforms: a Philox word w gives u = (2 floor(w / 2^9) + 1) 2^-24, an odd   */
/* multiple of 2^-24 in (0, 1), exact in binary32.                            */
/*                                                                            */
/* ln u: u = m 2^e with m in [sqrt(1/2), sqrt(2)) (from the bit pattern; the  */
/* threshold is the binary32 value 0x3fb504f3), f = m - 1 (exact),            */
/* ln(1 + f) = f + f^2 (-1/2 + f R(f)), R a degree-7 minimax polynomial, and  */
/* ln u = e LN2_HI + (e LN2_LO + ln(1 + f)) with the Cody-Waite split of ln 2 */
/* (LN2_HI has 15 significant bits, so e LN2_HI is exact).                    */
/*                                                                            */
/* sin and cos of 2 pi u: with v = 2 floor(w / 2^9) + 1 (u = v 2^-24), the    */
/* nearest quarter turn j = floor((v + 2^21) / 2^22) and r = (v - j 2^22)     */
/* 2^-24 in [-1/8, 1/8] are exact integer steps; sin(2 pi r) = r S(r^2) and   */
/* cos(2 pi r) = 1 + r^2 C(r^2) with degree-4 minimax polynomials S and C;    */
/* the quadrant j mod 4 swaps and negates them.                               */
/*                                                                            */
/* The coefficients are binary32 minimax fits (Lawson's algorithm) made once  */
/* for this generator; the fitting procedure is documented with the input     */
/* generators.                                                                */
/* ------------------------------------------------------------------------ */
static const float OR_LN_R[8] = { /* degree 7 down to 0 */
    -0x1.38c9dep-4f, 0x1.055ec6p-3f, -0x1.0d8242p-3f, 0x1.22d92ep-3f,
    -0x1.54728ap-3f, 0x1.99a01cp-3f, -0x1.000226p-2f, 0x1.555554p-2f};
static const float OR_SIN_S[5] = { /* degree 4 down to 0 */
    0x1.a0b0c6p+8f, -0x1.61b22ap+6f, 0x1.46e1p+6f, -0x1.4abc8ap+5f, 0x1.921fb6p+2f};
static const float OR_COS_C[5] = { /* degree 4 down to 0 */
    0x1.c33bfap+6f, 0x1.b78f76p+5f, -0x1.558c8p+6f, 0x1.03c192p+6f, -0x1.3bd3ccp+4f};
static const float OR_LN2_HI = 0x1.62e4p-1f, OR_LN2_LO = 0x1.7f7d1cp-20f;

/* ln u for a positive normal binary32 u */
float or_ln_f32(float u)
{
    uint32_t b;
    memcpy(&b, &u, 4);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u; /* m in [1, 2) */
    if (mb > 0x3fb504f3u) {                       /* m > sqrt(2): use m / 2 */
        mb -= 0x00800000u;
        e += 1;
    }
    float m;
    memcpy(&m, &mb, 4);
    float f = m - 1.0f;
    float R = OR_LN_R[0];
    for (int i = 1; i < 8; ++i) R = fmaf(R, f, OR_LN_R[i]);
    float t = fmaf(f, R, -0.5f);
    float f2 = f * f;
    float lnm = fmaf(f2, t, f);
    float ef = (float)e;
    return fmaf(ef, OR_LN2_HI, fmaf(ef, OR_LN2_LO, lnm));
}

/* sin and cos of 2 pi v 2^-24 for an odd v in (0, 2^24) */
void or_sincos2pi_f32(uint32_t v, float *s_out, float *c_out)
{
    int32_t j = (int32_t)((v + (1u << 21)) >> 22);
    int32_t ri = (int32_t)v - j * (1 << 22);
    float r = (float)ri * 0x1p-24f;
    float z = r * r;
    float S = OR_SIN_S[0], C = OR_COS_C[0];
    for (int i = 1; i < 5; ++i) {
        S = fmaf(S, z, OR_SIN_S[i]);
        C = fmaf(C, z, OR_COS_C[i]);
    }
    float sn = r * S;
    float cs = fmaf(z, C, 1.0f);
    switch (j & 3) {
        case 0: *s_out = sn; *c_out = cs; break;
        case 1: *s_out = cs; *c_out = -sn; break;
        case 2: *s_out = -sn; *c_out = -cs; break;
        default: *s_out = -cs; *c_out = sn; break;
    }
}

/* arrays of the two functions (for the accuracy tests) */
void or_ln_f32_array(const float *u, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_ln_f32(u[i]);
}
void or_sincos2pi_f32_array(const uint32_t *v, float *s, float *c, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) or_sincos2pi_f32(v[i], s + i, c + i);
}

/*
 * Channel of Sec. II-B: BPSK x_n = 1 - 2 c_n, y_n = x_n + sigma*g_n with g_n
 * standard normal, mu_n = 2 y_n / sigma^2.  cw (row-major [nfr][N], 0/1) is
 * the transmitted codeword; NULL sends the all-zero codeword (x_n = +1).
 * Bit n of frame F uses counter (n/4, F_lo, F_hi, tag) under key
 * (seed_lo, seed_hi); words (w0, w1) and (w2, w3) are two Box-Muller pairs
 * giving the normals of bits 4q, 4q+1 and 4q+2, 4q+3:
 *   rho = sqrtf(-2 ln u(w0)),  g0 = rho cos(2 pi u(w1)),  g1 = rho sin(2 pi u(w1)).
 * In binary32: sf = sigma and s2 = 2 / sigma^2 rounded from double, and
 *   mu = s2 * fmaf(sf, g, x).
 * g_out (if non-NULL) receives g (binary32 values).
 */
void or_channel_awgn_cw(uint64_t seed, uint64_t first_frame, int nfr, int N, double sigma,
                        uint32_t tag, const uint8_t *cw, float *mu_out, double *g_out)
{
    const float sf = (float)sigma, s2 = (float)(2.0 / (sigma * sigma));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int f = 0; f < nfr; ++f) {
        uint64_t F = first_frame + (uint64_t)f;
        for (int q = 0; 4 * q < N; ++q) {
            uint32_t ctr[4] = {(uint32_t)q, (uint32_t)F, (uint32_t)(F >> 32), tag};
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            float g[4];
            for (int pair = 0; pair < 2; ++pair) {
                uint32_t v0 = 2u * (w[2 * pair] >> 9) + 1u;
                uint32_t v1 = 2u * (w[2 * pair + 1] >> 9) + 1u;
                float u0 = (float)v0 * 0x1p-24f;
                float rho = sqrtf(-2.0f * or_ln_f32(u0));
                float sn, cs;
                or_sincos2pi_f32(v1, &sn, &cs);
                g[2 * pair] = rho * cs;
                g[2 * pair + 1] = rho * sn;
            }
            for (int e = 0; e < 4; ++e) {
                int n = 4 * q + e;
                if (n >= N) break;
                float x = (cw && cw[(size_t)f * N + n]) ? -1.0f : 1.0f;
                mu_out[(size_t)f * N + n] = s2 * fmaf(sf, g[e], x);
                if (g_out) g_out[(size_t)f * N + n] = (double)g[e];
            }
        }
    }
}

void or_channel_awgn(uint64_t seed, uint64_t first_frame, int nfr, int N, double sigma,
                     uint32_t tag, float *mu_out, double *g_out)
{
    or_channel_awgn_cw(seed, first_frame, nfr, N, sigma, tag, NULL, mu_out, g_out);
}

/* ------------------------------------------------------------------------ */
/* Graph helpers.  H is given as CSR rows in the paper's edge order: row by   */
/* row, left to right (Sec. IV-A, data structure H).  Edge e of row m is      */
/* col[e] for e in [row_ptr[m], row_ptr[m+1]).  The column view (LUT_v)       */
/* lists, for every variable, its edges in increasing edge index.             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int M, N, E;
    const int *row_ptr, *col;
    int *vptr, *vedge; /* column view */
} or_graph;

static int or_graph_init(or_graph *g, int M, int N, const int *row_ptr, const int *col)
{
    g->M = M; g->N = N; g->row_ptr = row_ptr; g->col = col;
    g->E = row_ptr[M];
    g->vptr = (int *)calloc((size_t)N + 1, sizeof(int));
    g->vedge = (int *)malloc(sizeof(int) * (size_t)(g->E > 0 ? g->E : 1));
    if (!g->vptr || !g->vedge) return -1;
    for (int e = 0; e < g->E; ++e) g->vptr[col[e] + 1]++;
    for (int n = 0; n < N; ++n) g->vptr[n + 1] += g->vptr[n];
    int *fill = (int *)calloc((size_t)N, sizeof(int));
    if (!fill) return -1;
    for (int e = 0; e < g->E; ++e) {
        int n = col[e];
        g->vedge[g->vptr[n] + fill[n]++] = e;
    }
    free(fill);
    return 0;
}

static void or_graph_free(or_graph *g)
{
    free(g->vptr);
    free(g->vedge);
}

/* LUT_v of the paper: for each variable, the indices of its edges.  Exposed  */
/* so the worked example of Sec. IV-A can be checked.                         */
int or_variable_edges(int M, int N, const int *row_ptr, const int *col, int *vptr_out, int *vedge_out)
{
    or_graph g;
    if (or_graph_init(&g, M, N, row_ptr, col)) return -1;
    memcpy(vptr_out, g.vptr, sizeof(int) * (size_t)(N + 1));
    memcpy(vedge_out, g.vedge, sizeof(int) * (size_t)g.E);
    or_graph_free(&g);
    return 0;
}

static double or_clip(double x, double c)
{
    if (x > c) return c;
    if (x < -c) return -c;
    return x;
}

/* ------------------------------------------------------------------------ */
/* Real type of the sum-product and LDPCCC decoders.  The oracle is double    */
/* precision; the same source compiled with -DOR_REAL_FLOAT is a binary32     */
/* build of the same steps in the same order (a diagnostic that shows how far */
/* any FP32 implementation of Algorithm 1 moves from the FP64 result; it is   */
/* not a reference).                                                          */
/* ------------------------------------------------------------------------ */
#ifdef OR_REAL_FLOAT
typedef float or_real;
#define OR_R(fn) fn##f
#else
typedef double or_real;
#define OR_R(fn) fn
#endif

static or_real or_clip_r(or_real x, or_real c)
{
    if (x > c) return c;
    if (x < -c) return -c;
    return x;
}

/* phi(x) = -ln tanh(x/2) = ln((e^x + 1)/(e^x - 1)) for x >= 0; phi(0) = +inf. */
/* phi is its own inverse on [0, inf], and tanh(x/2) = exp(-phi(|x|)), so the   */
/* product of tanh in eq. (bphs) becomes a sum of phi values.                   */
static or_real or_phi(or_real x)
{
    if (x <= (or_real)0) return INFINITY;
    return OR_R(log1p)((or_real)2 / OR_R(expm1)(x));
}

/*
 * Horizontal step of Algorithm 1 for one check node, eq. (bphs).
 * form 0: phi-form  alpha = prod(sign) * phi( sum_{n' != n} phi(|beta_n'|) )
 * form 1: literal   alpha = 2 atanh( prod_{n' != n} tanh(beta_n'/2) )
 * The extrinsic set excludes the edge itself; an empty product is 1.
 * Every output is clipped to +-clip.
 */
static void or_check_update(const or_real *beta, or_real *alpha, int d, or_real clip, int form)
{
    for (int a = 0; a < d; ++a) {
        if (form == 1) {
            or_real prod = 1;
            for (int b = 0; b < d; ++b)
                if (b != a) prod *= OR_R(tanh)(beta[b] / 2);
            or_real v;
            if (prod >= 1) v = INFINITY;
            else if (prod <= -1) v = -INFINITY;
            else v = 2 * OR_R(atanh)(prod);
            alpha[a] = or_clip_r(v, clip);
        } else {
            or_real s = 0;
            int neg = 0;
            for (int b = 0; b < d; ++b) {
                if (b == a) continue;
                s += or_phi(OR_R(fabs)(beta[b]));
                if (beta[b] < 0) neg ^= 1;
            }
            or_real mag = or_phi(s); /* phi(0) = inf for an empty set */
            if (mag > clip) mag = clip;
            alpha[a] = neg ? -mag : mag;
        }
    }
}

/* One frame of Algorithm 1 with the syndrome stopping rule.                 */
static void or_sp_frame(const or_graph *g, const float *mu_f, int max_iter, int early_stop, double clip_d,
                        int form, double *post, uint8_t *hard, int *iters, int *ok)
{
    int E = g->E, M = g->M, N = g->N;
    const or_real clip = (or_real)clip_d;
    or_real *beta = (or_real *)malloc(sizeof(or_real) * (size_t)(E ? E : 1));
    or_real *alpha = (or_real *)malloc(sizeof(or_real) * (size_t)(E ? E : 1));
    or_real *mu = (or_real *)malloc(sizeof(or_real) * (size_t)(N ? N : 1));
    or_real *in = (or_real *)malloc(sizeof(or_real) * (size_t)(N + 1));
    or_real *outv = (or_real *)malloc(sizeof(or_real) * (size_t)(N + 1));
    for (int n = 0; n < N; ++n) mu[n] = or_clip_r((or_real)mu_f[n], clip);

    /* [Initialization] beta_mn = mu_n on every edge. */
    for (int e = 0; e < E; ++e) beta[e] = mu[g->col[e]];

    int it_done = max_iter, satisfied = 0;
    for (int it = 1; it <= max_iter; ++it) {
        /* [Horizontal step] every check node, eq. (bphs). */
        for (int m = 0; m < M; ++m) {
            int e0 = g->row_ptr[m], d = g->row_ptr[m + 1] - e0;
            for (int k = 0; k < d; ++k) in[k] = beta[e0 + k];
            or_check_update(in, outv, d, clip, form);
            for (int k = 0; k < d; ++k) alpha[e0 + k] = outv[k];
        }
        /* [Vertical step] eqs. (bpvs) and (bpd). */
        for (int n = 0; n < N; ++n) {
            int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
            or_real total = mu[n];
            for (int k = 0; k < dv; ++k) total += alpha[g->vedge[v0 + k]];
            for (int k = 0; k < dv; ++k) {
                or_real s = mu[n];
                for (int k2 = 0; k2 < dv; ++k2)
                    if (k2 != k) s += alpha[g->vedge[v0 + k2]];
                beta[g->vedge[v0 + k]] = or_clip_r(s, clip);
            }
            post[n] = (double)or_clip_r(total, clip);
            /* eq. (hrddcs): 0 if beta_n >= 0, else 1 */
            hard[n] = post[n] < 0.0 ? 1 : 0;
        }
        /* Syndrome of the current hard decisions. */
        satisfied = 1;
        for (int m = 0; m < M && satisfied; ++m) {
            int par = 0;
            for (int e = g->row_ptr[m]; e < g->row_ptr[m + 1]; ++e) par ^= hard[g->col[e]];
            if (par) satisfied = 0;
        }
        if (early_stop && satisfied) {
            it_done = it;
            break;
        }
    }
    *iters = it_done;
    *ok = satisfied;
    free(beta); free(alpha); free(mu); free(in); free(outv);
}

int or_sp_decode(int M, int N, const int *row_ptr, const int *col, int nfr, const float *mu, int max_iter,
                 int early_stop, double clip, int form, double *post, uint8_t *hard, int *iters, int *ok,
                 int nthreads)
{
    or_graph g;
    if (max_iter < 1) return -1;
    if (or_graph_init(&g, M, N, row_ptr, col)) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int f = 0; f < nfr; ++f)
        or_sp_frame(&g, mu + (size_t)f * N, max_iter, early_stop, clip, form, post + (size_t)f * N,
                    hard + (size_t)f * N, iters + f, ok + f);
    or_graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Integer min-sum.  The paper cites 8-bit min-sum GPU decoders as prior art  */
/* (Sec. I) but gives no definition; this follows the usual definition:       */
/* quantize mu to q = clamp(rint(mu * 2^F), -127, 127) (round half to even),  */
/* check update alpha = prod(sign) * min_{n' != n} |beta_n'|  (sign(0) = +),  */
/* variable update beta = clamp(q + sum_{m' != m} alpha, -127, 127),          */
/* posterior = q + sum alpha (int32, unclamped), hard = posterior < 0.        */
/* ------------------------------------------------------------------------ */
static int or_sat(int x, int lim)
{
    return x > lim ? lim : (x < -lim ? -lim : x);
}

int or_quantize(const float *mu, int count, int frac_bits, int8_t *q)
{
    double scale = ldexp(1.0, frac_bits);
    for (int i = 0; i < count; ++i) {
        double v = nearbyint((double)mu[i] * scale); /* default mode: half to even */
        if (v > 127.0) v = 127.0;
        if (v < -127.0) v = -127.0;
        q[i] = (int8_t)v;
    }
    return 0;
}

static void or_ms_frame(const or_graph *g, const float *mu_f, int frac_bits, int max_iter, int early_stop,
                        int32_t *post, uint8_t *hard, int *iters, int *ok)
{
    int E = g->E, M = g->M, N = g->N;
    int *beta = (int *)malloc(sizeof(int) * (size_t)(E ? E : 1));
    int *alpha = (int *)malloc(sizeof(int) * (size_t)(E ? E : 1));
    int8_t *q8 = (int8_t *)malloc((size_t)(N ? N : 1));
    or_quantize(mu_f, N, frac_bits, q8);
    for (int e = 0; e < E; ++e) beta[e] = q8[g->col[e]];
    int it_done = max_iter, satisfied = 0;
    for (int it = 1; it <= max_iter; ++it) {
        for (int m = 0; m < M; ++m) {
            int e0 = g->row_ptr[m], e1 = g->row_ptr[m + 1];
            for (int e = e0; e < e1; ++e) {
                int mag = 127, neg = 0; /* empty set: saturated + */
                for (int e2 = e0; e2 < e1; ++e2) {
                    if (e2 == e) continue;
                    int a = beta[e2] < 0 ? -beta[e2] : beta[e2];
                    if (a < mag) mag = a;
                    if (beta[e2] < 0) neg ^= 1;
                }
                alpha[e] = neg ? -mag : mag;
            }
        }
        for (int n = 0; n < N; ++n) {
            int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
            int total = q8[n];
            for (int k = 0; k < dv; ++k) total += alpha[g->vedge[v0 + k]];
            for (int k = 0; k < dv; ++k) {
                int s = q8[n];
                for (int k2 = 0; k2 < dv; ++k2)
                    if (k2 != k) s += alpha[g->vedge[v0 + k2]];
                beta[g->vedge[v0 + k]] = or_sat(s, 127);
            }
            post[n] = total;
            hard[n] = total < 0 ? 1 : 0;
        }
        satisfied = 1;
        for (int m = 0; m < M && satisfied; ++m) {
            int par = 0;
            for (int e = g->row_ptr[m]; e < g->row_ptr[m + 1]; ++e) par ^= hard[g->col[e]];
            if (par) satisfied = 0;
        }
        if (early_stop && satisfied) {
            it_done = it;
            break;
        }
    }
    *iters = it_done;
    *ok = satisfied;
    free(beta); free(alpha); free(q8);
}

int or_ms_decode(int M, int N, const int *row_ptr, const int *col, int nfr, const float *mu, int frac_bits,
                 int max_iter, int early_stop, int32_t *post, uint8_t *hard, int *iters, int *ok, int nthreads)
{
    or_graph g;
    if (max_iter < 1) return -1;
    if (or_graph_init(&g, M, N, row_ptr, col)) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int f = 0; f < nfr; ++f)
        or_ms_frame(&g, mu + (size_t)f * N, frac_bits, max_iter, early_stop, post + (size_t)f * N,
                    hard + (size_t)f * N, iters + f, ok + f);
    or_graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pipelined BP of an LDPC convolutional code, Algorithm 2.                   */
/*                                                                            */
/* H is the unwrapped parity-check matrix H_[0,T) truncated to T check layers */
/* and T variable frames, given as CSR rows in the paper's edge order.  Check */
/* layer R holds rows [R*cb, (R+1)*cb), frame F holds columns [F*c, (F+1)*c); */
/* cb = c - b.  A layer only touches frames R - ms .. R.                      */
/*                                                                            */
/* Slot t (0-based) of Algorithm 2:                                           */
/*   [Initialization] frame t enters processor 1: beta = mu on its edges;     */
/*   shifting frames between processors moves no data (Sec. IV-B-2).          */
/*   Processor i = 1..I: horizontal step on layer t-(i-1)(ms+1), eq. (bph);   */
/*   then, for all i, vertical step on frame t-(i-1)(ms+1)-ms, eq. (bpvs).    */
/*   The frame leaving processor I, t-(I-1)(ms+1)-ms, gets its a-posteriori   */
/*   LLR and hard decision.  Indices outside [0,T) are skipped: the first     */
/*   ms frames see only the layers that exist (start-up, Sec. IV-B-2 step 3). */
/*                                                                            */
/* Outputs post/hard are [T][c]; decided[F] = 1 for the frames decided within */
/* the T slots (F <= T - I(ms+1)).  If log is non-NULL it receives one        */
/* (slot, kind, index, processor) record per event, kind 0 = frame enters,    */
/* 1 = check layer update, 2 = frame update, 3 = decision; at most log_cap.   */
/* Returns the number of decided frames, or -1.                               */
/* ------------------------------------------------------------------------ */
static int or_ldpccc_stream(const or_graph *g, int T, int c, int cb, int ms, int I, const float *mu_f,
                            double clip_d, double *post, uint8_t *hard, uint8_t *decided, int *log,
                            int log_cap, int *log_n)
{
    int E = g->E;
    const or_real clip = (or_real)clip_d;
    or_real *beta = (or_real *)calloc((size_t)(E ? E : 1), sizeof(or_real));
    or_real *alpha = (or_real *)calloc((size_t)(E ? E : 1), sizeof(or_real));
    or_real *in = (or_real *)malloc(sizeof(or_real) * (size_t)(g->N + 1));
    or_real *outv = (or_real *)malloc(sizeof(or_real) * (size_t)(g->N + 1));
    int ndec = 0, nl = 0;
#define OR_LOG(t_, k_, x_, i_)                                                                     \
    do {                                                                                           \
        if (log && nl < log_cap) {                                                                 \
            log[4 * nl] = (t_); log[4 * nl + 1] = (k_); log[4 * nl + 2] = (x_); log[4 * nl + 3] = (i_); \
        }                                                                                          \
        ++nl;                                                                                      \
    } while (0)
    for (int F = 0; F < T; ++F) decided[F] = 0;
    for (int t = 0; t < T; ++t) {
        /* [Initialization] frame t and its channel messages enter processor 1. */
        for (int v = t * c; v < (t + 1) * c; ++v) {
            or_real m = or_clip_r((or_real)mu_f[v], clip);
            for (int k = g->vptr[v]; k < g->vptr[v + 1]; ++k) beta[g->vedge[k]] = m;
        }
        OR_LOG(t, 0, t, 1);
        /* [Horizontal step] processor i updates check layer t-(i-1)(ms+1). */
        for (int i = 1; i <= I; ++i) {
            int R = t - (i - 1) * (ms + 1);
            if (R < 0 || R >= T) continue;
            OR_LOG(t, 1, R, i);
            for (int m = R * cb; m < (R + 1) * cb; ++m) {
                int e0 = g->row_ptr[m], d = g->row_ptr[m + 1] - e0;
                for (int k = 0; k < d; ++k) in[k] = beta[e0 + k];
                or_check_update(in, outv, d, clip, 0);
                for (int k = 0; k < d; ++k) alpha[e0 + k] = outv[k];
            }
        }
        /* [Vertical step] processor i updates frame t-(i-1)(ms+1)-ms. */
        for (int i = 1; i <= I; ++i) {
            int F = t - (i - 1) * (ms + 1) - ms;
            if (F < 0 || F >= T) continue;
            OR_LOG(t, 2, F, i);
            for (int n = F * c; n < (F + 1) * c; ++n) {
                int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
                or_real m0 = or_clip_r((or_real)mu_f[n], clip);
                for (int k = 0; k < dv; ++k) {
                    or_real s = m0;
                    for (int k2 = 0; k2 < dv; ++k2)
                        if (k2 != k) s += alpha[g->vedge[v0 + k2]];
                    beta[g->vedge[v0 + k]] = or_clip_r(s, clip);
                }
            }
        }
        /* [Making hard decision] for the frame leaving processor I. */
        {
            int F = t - (I - 1) * (ms + 1) - ms;
            if (F >= 0 && F < T) {
                OR_LOG(t, 3, F, I);
                for (int n = F * c; n < (F + 1) * c; ++n) {
                    int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
                    or_real total = or_clip_r((or_real)mu_f[n], clip);
                    for (int k = 0; k < dv; ++k) total += alpha[g->vedge[v0 + k]];
                    total = or_clip_r(total, clip);
                    post[n] = (double)total;
                    hard[n] = total < 0 ? 1 : 0;
                }
                decided[F] = 1;
                ++ndec;
            }
        }
    }
#undef OR_LOG
    if (log_n) *log_n = nl;
    free(beta); free(alpha); free(in); free(outv);
    return ndec;
}

int or_ldpccc_decode(int M, int N, const int *row_ptr, const int *col, int T, int c, int cb, int ms, int I,
                     int nstreams, const float *mu, double clip, double *post, uint8_t *hard, uint8_t *decided,
                     int *log, int log_cap, int *log_n, int nthreads)
{
    if (I < 1 || ms < 0 || c <= 0 || cb <= 0 || M != T * cb || N != T * c) return -1;
    or_graph g;
    if (or_graph_init(&g, M, N, row_ptr, col)) return -1;
    int ndec = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(max : ndec)
    for (int s = 0; s < nstreams; ++s) {
        int r = or_ldpccc_stream(&g, T, c, cb, ms, I, mu + (size_t)s * N, clip, post + (size_t)s * N,
                                 hard + (size_t)s * N, decided + (size_t)s * T, s == 0 ? log : NULL,
                                 log_cap, s == 0 ? log_n : NULL);
        if (r > ndec) ndec = r;
    }
    or_graph_free(&g);
    return ndec;
}

/* ------------------------------------------------------------------------ */
/* Neural normalized/offset min-sum (NOMS).  The paper only cites reduced-    */
/* complexity BP (Sec. II-B); this is the usual parameterized min-sum with a   */
/* weight w and an offset o per iteration and per circulant block:            */
/*   beta^(0)_e = clip(mu_v)                                                   */
/*   alpha^(l)_e = s_e * min(max(w_{l,c(e)} * m_e - o_{l,c(e)}, 0), clip)     */
/*        (every message clipped at +-clip, like the other decoders; an empty */
/*        set of other edges gives m_e = inf, i.e. alpha = s_e * clip),       */
/*        m_e = min_{e' != e in the row} |beta^(l-1)_e'|,                      */
/*        s_e = prod_{e' != e} sign(beta^(l-1)_e')   (sign(0) = +)             */
/*   beta^(l)_e = clip(mu_v + sum_{e' != e in the column} alpha^(l)_e'),       */
/*   post^(l)_v = mu_v + sum_e alpha^(l)_e                                    */
/*   loss = 1/(T N nfr) sum_l sum_v softplus(-post^(l)_v)                     */
/* (multi-loss over iterations, target = the all-zero codeword).  cblk[e] is  */
/* the circulant index of edge e; params is [T][ncirc][2] = (w, o).           */
/* The gradient is reverse mode written out by hand: through the arg-min edge */
/* of each m_e (the lowest index among ties), through max(., 0) where it is   */
/* positive and below clip, and through the clip where |beta| < clip; signs  */
/* carry none.                                                                */
/* ------------------------------------------------------------------------ */
static double or_softplus(double x)
{
    return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

static double or_sigmoid(double x)
{
    return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}

/* CN of one iteration; also returns, per edge, the arg-min edge, m_e, s_e and the active flag */
static void or_noms_cn(const or_graph *g, const double *beta, const int *cblk, const double *par_l, double clip,
                       double *alpha, int *amin, double *mval, double *sval, int *act)
{
    for (int m = 0; m < g->M; ++m) {
        int e0 = g->row_ptr[m], e1 = g->row_ptr[m + 1];
        for (int e = e0; e < e1; ++e) {
            double best = INFINITY;
            int arg = -1, neg = 0;
            for (int e2 = e0; e2 < e1; ++e2) {
                if (e2 == e) continue;
                double a = fabs(beta[e2]);
                if (a < best) { best = a; arg = e2; }
                if (beta[e2] < 0.0) neg ^= 1;
            }
            double s = neg ? -1.0 : 1.0;
            double w = par_l[2 * cblk[e]], o = par_l[2 * cblk[e] + 1];
            double z = (arg < 0) ? INFINITY : w * best - o;
            int on = z > 0.0;
            alpha[e] = on ? s * (z < clip ? z : clip) : 0.0;
            /* the gradient passes where alpha = s (w m - o): positive, below the clip */
            amin[e] = arg; mval[e] = best; sval[e] = s; act[e] = on && arg >= 0 && z < clip;
        }
    }
}

/* x rounded to the nearest binary16 value (ties to even; beyond 65504 -> inf): the storage
   of the FP16-message variant.  Binary16 keeps 11 significant bits down to 2^-14 and a
   fixed quantum of 2^-24 below (subnormals). */
double or_round_half(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e); /* ax = m 2^e, m in [0.5, 1) */
    int q = e - 11;
    if (q < -24) q = -24;
    double r = ldexp(nearbyint(ldexp(ax, -q)), q);
    if (r > 65504.0) r = INFINITY;
    return copysign(r, x);
}

void or_round_half_array(const double *x, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_round_half(x[i]);
}

static void or_noms_vn(const or_graph *g, const double *mu, const double *alpha, double clip, double *beta,
                       double *post)
{
    for (int n = 0; n < g->N; ++n) {
        int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
        double tot = mu[n];
        for (int k = 0; k < dv; ++k) tot += alpha[g->vedge[v0 + k]];
        post[n] = tot;
        for (int k = 0; k < dv; ++k) {
            double s = mu[n];
            for (int k2 = 0; k2 < dv; ++k2)
                if (k2 != k) s += alpha[g->vedge[v0 + k2]];
            beta[g->vedge[v0 + k]] = or_clip(s, clip);
        }
    }
}

/* The FP16-message variant's forward (store16).  Rounding a message to binary16 and picking
   the arg-min of the rounded messages are decisions taken on a floating-point value, so this
   forward takes them on the value the device computes: binary32 arithmetic, w * m - o as one
   fused multiply-add, the sums of the variable rule in the column's edge order (increasing
   check index).  Every input of these steps (binary16 messages, binary32 channel LLRs and
   parameters) is exact in binary32; results are stored as doubles.  Both message kinds are
   kept as binary16 (alpha after the check step, beta after the variable step), as the FP16
   decoder stores them; the gradient treats that rounding as the identity, as it treats the
   clip where inactive. */
static void or_noms_cn_f32(const or_graph *g, const double *beta, const int *cblk, const double *par_l, double clip,
                           double *alpha, int *amin, double *mval, double *sval, int *act)
{
    const float cf = (float)clip;
    for (int m = 0; m < g->M; ++m) {
        int e0 = g->row_ptr[m], e1 = g->row_ptr[m + 1];
        for (int e = e0; e < e1; ++e) {
            float best = INFINITY;
            int arg = -1, neg = 0;
            for (int e2 = e0; e2 < e1; ++e2) {
                if (e2 == e) continue;
                float a = fabsf((float)beta[e2]);
                if (a < best) { best = a; arg = e2; }
                if (beta[e2] < 0.0) neg ^= 1;
            }
            float sg = neg ? -1.0f : 1.0f;
            float w = (float)par_l[2 * cblk[e]], o = (float)par_l[2 * cblk[e] + 1];
            float z = (arg < 0) ? INFINITY : fmaf(w, best, -o);
            int on = z > 0.0f;
            /* stored as binary16, like beta */
            alpha[e] = on ? or_round_half((double)(sg * (z < cf ? z : cf))) : 0.0;
            amin[e] = arg; mval[e] = best; sval[e] = sg; act[e] = on && arg >= 0 && z < cf;
        }
    }
}

static void or_noms_vn_f32(const or_graph *g, const double *mu, const double *alpha, double clip, double *beta,
                           double *post)
{
    for (int n = 0; n < g->N; ++n) {
        int v0 = g->vptr[n], dv = g->vptr[n + 1] - v0;
        float tot = (float)mu[n];
        for (int k = 0; k < dv; ++k) tot += (float)alpha[g->vedge[v0 + k]];
        post[n] = tot;
        for (int k = 0; k < dv; ++k) {
            float sm = (float)mu[n];
            for (int k2 = 0; k2 < dv; ++k2)
                if (k2 != k) sm += (float)alpha[g->vedge[v0 + k2]];
            beta[g->vedge[v0 + k]] = or_round_half(or_clip(sm, clip));
        }
    }
}

/*
 * or_noms: forward (and, if grad != NULL, backward) over nfr frames.
 * post_out (nullable) receives post^(T) [nfr][N]; returns the loss.  grad is [T][ncirc][2],
 * accumulated (the caller zeroes it).  store16: the FP16-message variant (alpha^(l) and beta^(l),
 * l >= 1, rounded to binary16 when stored; its forward in binary32, see or_noms_cn_f32).
 */
double or_noms(int M, int N, const int *row_ptr, const int *col, const int *cblk, int nfr, const float *mu_f,
               int T, const double *params, int ncirc, double clip, double *post_out, double *grad, int nthreads,
               int store16)
{
    or_graph g;
    if (T < 1 || or_graph_init(&g, M, N, row_ptr, col)) return NAN;
    int E = g.E;
    double Z = (double)T * N * nfr;
    double loss = 0.0;
    (void)ncirc;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : loss)
    for (int f = 0; f < nfr; ++f) {
        double *mu = malloc(sizeof(double) * N);
        double *beta = malloc(sizeof(double) * (size_t)E * (T + 1)); /* beta^(0..T) */
        double *alpha = malloc(sizeof(double) * (size_t)E * T);
        double *post = malloc(sizeof(double) * (size_t)N * T);
        double *mval = malloc(sizeof(double) * (size_t)E * T), *sval = malloc(sizeof(double) * (size_t)E * T);
        int *amin = malloc(sizeof(int) * (size_t)E * T), *act = malloc(sizeof(int) * (size_t)E * T);
        double *gb = calloc((size_t)E, sizeof(double)), *ga = malloc(sizeof(double) * E);
        double *gb_prev = malloc(sizeof(double) * E);
        double lf = 0.0;
        for (int n = 0; n < N; ++n) mu[n] = or_clip((double)mu_f[(size_t)f * N + n], clip);
        for (int e = 0; e < E; ++e) beta[e] = mu[col[e]];
        for (int l = 0; l < T; ++l) {
            if (store16) {
                or_noms_cn_f32(&g, beta + (size_t)l * E, cblk, params + (size_t)l * 2 * ncirc, clip,
                               alpha + (size_t)l * E, amin + (size_t)l * E, mval + (size_t)l * E,
                               sval + (size_t)l * E, act + (size_t)l * E);
                or_noms_vn_f32(&g, mu, alpha + (size_t)l * E, clip, beta + (size_t)(l + 1) * E,
                               post + (size_t)l * N);
            } else {
                or_noms_cn(&g, beta + (size_t)l * E, cblk, params + (size_t)l * 2 * ncirc, clip,
                           alpha + (size_t)l * E, amin + (size_t)l * E, mval + (size_t)l * E,
                           sval + (size_t)l * E, act + (size_t)l * E);
                or_noms_vn(&g, mu, alpha + (size_t)l * E, clip, beta + (size_t)(l + 1) * E,
                           post + (size_t)l * N);
            }
            for (int n = 0; n < N; ++n) lf += or_softplus(-post[(size_t)l * N + n]);
        }
        if (post_out)
            for (int n = 0; n < N; ++n) post_out[(size_t)f * N + n] = post[(size_t)(T - 1) * N + n];
        loss += lf / Z;
        if (grad) {
            /* gb = adjoint of beta^(l) (zero for l = T) */
            for (int l = T - 1; l >= 0; --l) {
                const double *bl = beta + (size_t)l * E;                 /* input of CN l */
                /* VN l output as stored: the clip was inactive where |beta| < clip (with binary16
                   storage, where the stored value is below the clip) */
                const double *bn = beta + (size_t)(l + 1) * E;
                const double *pl = post + (size_t)l * N;
                /* adjoint of alpha^(l) */
                for (int n = 0; n < N; ++n) {
                    int v0 = g.vptr[n], dv = g.vptr[n + 1] - v0;
                    double dpost = -or_sigmoid(-pl[n]) / Z;
                    for (int k = 0; k < dv; ++k) {
                        double s = dpost;
                        for (int k2 = 0; k2 < dv; ++k2) {
                            if (k2 == k) continue;
                            int e2 = g.vedge[v0 + k2];
                            if (fabs(bn[e2]) < clip) s += gb[e2];
                        }
                        ga[g.vedge[v0 + k]] = s;
                    }
                }
                /* parameters and the adjoint of beta^(l) */
                double *pg = grad ? grad + (size_t)l * 2 * ncirc : NULL;
                for (int e = 0; e < E; ++e) gb_prev[e] = 0.0;
                for (int e = 0; e < E; ++e) {
                    if (!act[(size_t)l * E + e]) continue;
                    double s = sval[(size_t)l * E + e], mv = mval[(size_t)l * E + e];
                    int c = cblk[e];
                    double w = params[(size_t)l * 2 * ncirc + 2 * c];
#pragma omp atomic
                    pg[2 * c] += ga[e] * s * mv;
#pragma omp atomic
                    pg[2 * c + 1] += -ga[e] * s;
                    int a = amin[(size_t)l * E + e];
                    double sb = bl[a] > 0 ? 1.0 : (bl[a] < 0 ? -1.0 : 0.0);
                    gb_prev[a] += ga[e] * s * w * sb;
                }
                for (int e = 0; e < E; ++e) gb[e] = gb_prev[e];
            }
        }
        free(mu); free(beta); free(alpha); free(post); free(mval); free(sval); free(amin); free(act);
        free(gb); free(ga); free(gb_prev);
    }
    or_graph_free(&g);
    return loss;
}
