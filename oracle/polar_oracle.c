/*
 * polar_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU implementation of what the GPU library
 * computes: polar encoding, CRC, Gaussian-approximation code construction and
 * successive-cancellation list (SCL) decoding with CRC aid, tree pruning
 * (R0/R1/REP/SPC), fixed-point arithmetic and the adaptive list schedules,
 * after Leonardon et al., "Fast and Flexible Software Polar List Decoders".
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this file.  It shares no code, header or table with the CUDA library.
 * Every decoder path copies whole per-path arrays and recurses exactly as the
 * SCL pseudo-code (Algorithm 1) does; nothing here is blocked, fused or
 * reordered for speed.
 *
 * Readings of the paper taken where it is silent (all listed in the design
 * notes of the repository):
 *   - |A| = K includes the c CRC bits; info bits then CRC bits fill A in
 *     increasing index order.
 *   - CRC: MSB-first polynomial division, initial value 0, no reflection,
 *     no final XOR; the remainder is appended MSB first.
 *   - Path metric: the min-sum (LLR-based) metric, PM += |lambda| when the
 *     decided bit differs from the hard decision of lambda (Sec. II-B cites
 *     Balatsoukas-Stimming et al. without printing it); an exact mode uses
 *     PM += ln(1 + exp(-(1 - 2u) lambda)) with the exact f.
 *   - Hard decision: HD(lambda) = 1 iff lambda < 0 (so +0 and -0 give 0).
 *   - Candidates: path p (slot order) yields M candidates j; candidate id
 *     c = p*M + j; the min(L, n) smallest (PM, c) survive; survivors take new
 *     slots in increasing c.
 *   - Node handlers (Sec. II-B, IV-C): R0 one candidate; REP two (all-0,
 *     all-1); R1 flips of the t least reliable positions (Chase-t, "two
 *     maximum" read as the two least reliable); SPC the even-parity subset of
 *     those flips.  Sums over node positions use a balanced pairwise tree over
 *     index order; flip penalties are a left fold in ascending flip rank.
 *   - Fixed point (Sec. III-B-3): q = clamp(rint_half_even(lambda * 2^f), -Q, Q);
 *     every add saturates to [-Q, Q]; the PM shares the type and is
 *     normalised (minimum subtracted) after every node/leaf step.
 *
 * Pins (tests/test_oracle_*.py) tie every function to something outside
 * itself (closed forms, catalogue values, brute-force ML, exact MAP metrics,
 * an independent SC decoder, brute-force enumeration of the Chase-t and SPC
 * candidate lists at flip depths below the node size with L > 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "polar_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Encoding matrix F^{(x)n} (Sec. II-A footnote): F^{(x)1} = [[1,0],[1,1]] and
 * F^{(x)n} = [[F', 0], [F', F']] with F' = F^{(x)(n-1)}, row vector times
 * matrix.  For v = (a, b) (halves) that block form gives
 * v F = ((a xor b) F', b F'), applied here recursively in place.            */
void orc_polar_transform(int N, uint8_t *v)
{
    if (N <= 1) return;
    int h = N / 2;
    for (int i = 0; i < h; i++) v[i] ^= v[i + h];
    orc_polar_transform(h, v);
    orc_polar_transform(h, v + h);
}

/* CRC (Sec. II-A, Sec. IV-B): remainder of M(x) x^c divided by the generator
 * x^c + poly, bits taken MSB first (bits[0] is the highest power).          */
uint32_t orc_crc(const uint8_t *bits, int nbits, int c, uint32_t poly)
{
    if (c <= 0) return 0;
    uint32_t mask = (c == 32) ? 0xFFFFFFFFu : ((1u << c) - 1u);
    uint32_t reg = 0;
    for (int i = 0; i < nbits; i++) {
        uint32_t top = (reg >> (c - 1)) & 1u;
        uint32_t fb = top ^ (uint32_t)(bits[i] & 1u);
        reg = (reg << 1) & mask;
        if (fb) reg ^= (poly & mask);
    }
    return reg;
}

static int code_info_positions(const orc_code *cd, int *A)
{
    int k = 0;
    for (int i = 0; i < cd->N; i++)
        if (!cd->frozen[i]) A[k++] = i;
    return k;
}

/* Build u_A = (info || crc) (Sec. II-A): info bits then the c CRC bits, the
 * CRC remainder written MSB first.                                          */
static void build_uA(const orc_code *cd, const uint8_t *info, uint8_t *uA)
{
    int kinfo = cd->K - cd->crc_len;
    memcpy(uA, info, (size_t)kinfo);
    uint32_t r = orc_crc(info, kinfo, cd->crc_len, cd->crc_poly);
    for (int k = 0; k < cd->crc_len; k++)
        uA[kinfo + k] = (uint8_t)((r >> (cd->crc_len - 1 - k)) & 1u);
}

/* Encoder (Sec. II-A).  Systematic: u' = u F, zero u'_{A^c}, x = u' F, and
 * then x_A = u_A.  Non-systematic: x = u F.  Returns 0, or -1 if the
 * systematic property fails (it cannot for a polar frozen set that is closed
 * under the domination order, which GA sets are).                          */
int orc_encode(const orc_code *cd, const uint8_t *info, uint8_t *x)
{
    int N = cd->N;
    int *A = (int *)malloc(sizeof(int) * (size_t)N);
    uint8_t *uA = (uint8_t *)malloc((size_t)N);
    int nA = code_info_positions(cd, A);
    if (nA != cd->K) { free(A); free(uA); return -2; }
    build_uA(cd, info, uA);
    memset(x, 0, (size_t)N);
    for (int k = 0; k < nA; k++) x[A[k]] = uA[k];
    orc_polar_transform(N, x);
    int rc = 0;
    if (cd->systematic) {
        for (int i = 0; i < N; i++)
            if (cd->frozen[i]) x[i] = 0;
        orc_polar_transform(N, x);
        for (int k = 0; k < nA; k++)
            if (x[A[k]] != uA[k]) rc = -1;
    }
    free(A);
    free(uA);
    return rc;
}

void orc_encode_batch(const orc_code *cd, int n_frames, const uint8_t *info, uint8_t *x, int *rc)
{
    int kinfo = cd->K - cd->crc_len;
    *rc = 0;
    for (int f = 0; f < n_frames; f++) {
        int r = orc_encode(cd, info + (size_t)f * (size_t)kinfo, x + (size_t)f * (size_t)cd->N);
        if (r) *rc = r;
    }
}

/* ------------------------------------------------------------------------ */
/* Gaussian approximation construction (cited in Sec. II-A; formulas from
 * Trifonov 2012 with Chung, Richardson and Urbanke's phi approximation).
 * z holds the mean of each bit-channel's LLR; a check-node combination gives
 * phi^-1(1 - (1 - phi(za))(1 - phi(zb))), a variable-node combination za + zb.
 * The f (check) branch feeds the left child, the g (variable) branch the
 * right child, matching the decoding tree.                                  */
static double ga_phi(double x)
{
    if (x <= 0.0) return 1.0;
    if (x < 10.0) {
        double v = exp(-0.4527 * pow(x, 0.86) + 0.0218);
        return v > 1.0 ? 1.0 : v;
    }
    return sqrt(M_PI / x) * exp(-x / 4.0) * (1.0 - 10.0 / (7.0 * x));
}

static double ga_check(double za, double zb)
{
    double pa = ga_phi(za), pb = ga_phi(zb);
    /* 1 - (1 - pa)(1 - pb), written without cancellation */
    double y = pa + pb - pa * pb;
    double hi = za < zb ? za : zb;
    if (y <= 0.0) return hi;
    if (y >= 1.0) return 0.0;
    double lo = 0.0;
    /* phi is decreasing: bisection for phi(x) = y on [0, min(za, zb)] */
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (ga_phi(mid) > y) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static void ga_rec(int S, const double *z, double *out_leaves, double *tmp)
{
    if (S == 1) { out_leaves[0] = z[0]; return; }
    int h = S / 2;
    double *child = tmp;
    for (int i = 0; i < h; i++) child[i] = ga_check(z[i], z[i + h]);
    ga_rec(h, child, out_leaves, tmp + h);
    for (int i = 0; i < h; i++) child[i] = z[i] + z[i + h];
    ga_rec(h, child, out_leaves + h, tmp + h);
}

void orc_ga_reliability(int N, const uint8_t *punct, double sigma2, double *z_leaves)
{
    double *z0 = (double *)malloc(sizeof(double) * (size_t)N);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(2 * N + 2));
    for (int i = 0; i < N; i++) z0[i] = (punct && punct[i]) ? 0.0 : 2.0 / sigma2;
    ga_rec(N, z0, z_leaves, tmp);
    free(z0);
    free(tmp);
}

/* Frozen set: the |A| = K most reliable channels are information; ties go to
 * the larger index.  sigma^2 = 1 / (2 R 10^(EbN0/10)), R = K_info / (N - P). */
void orc_ga_frozen(int N, int K, int K_info, const uint8_t *punct, double design_ebn0_db,
                   uint8_t *frozen, double *z_out)
{
    int P = 0;
    if (punct)
        for (int i = 0; i < N; i++) P += punct[i] ? 1 : 0;
    double R = (double)K_info / (double)(N - P);
    double sigma2 = 1.0 / (2.0 * R * pow(10.0, design_ebn0_db / 10.0));
    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    orc_ga_reliability(N, punct, sigma2, z);
    if (z_out) memcpy(z_out, z, sizeof(double) * (size_t)N);
    for (int i = 0; i < N; i++) frozen[i] = 1;
    for (int k = 0; k < K; k++) {
        int best = -1;
        for (int i = 0; i < N; i++) {
            if (!frozen[i]) continue;
            if (best < 0 || z[i] > z[best] || (z[i] == z[best] && i > best)) best = i;
        }
        frozen[best] = 0;
    }
    free(z);
}

/* ------------------------------------------------------------------------ */
/* Density-evolution construction (Sec. II-A cites Tal and Vardy, "How to
 * construct polar codes").  A binary memoryless symmetric channel is held as
 * a mixture of binary symmetric channels: component j is used with
 * probability q_j and flips the bit with probability p_j <= 1/2.  The two
 * polarising transforms act on pairs of components:
 *   check (left child):  p = p_a (1 - p_b) + p_b (1 - p_a),  weight q_a q_b;
 *   variable (right child): the two observations agree with probability
 *     s = p_a p_b + (1 - p_a)(1 - p_b), leaving a BSC of crossover
 *     p_a p_b / s, or disagree, leaving min(p_a (1-p_b), p_b (1-p_a)) / (1-s).
 * After each transform the mixture is brought back to at most mu components
 * by merging all components whose capacity 1 - h2(p) falls in the same of mu
 * equal bins: a merged component has the weighted mean crossover, which
 * forgets which BSC was used, so the result is a degraded version of the true
 * bit channel and its error probability sum_j q_j p_j is an upper bound.   */
typedef struct {
    double q, p;
} de_comp;

static double de_cap(double p)
{
    if (p <= 0.0) return 1.0;
    if (p >= 0.5) return 0.0;
    return 1.0 + p * log2(p) + (1.0 - p) * log2(1.0 - p);
}

/* merge m components into at most mu (binned by capacity); returns the count */
static int de_merge(const de_comp *in, int m, int mu, de_comp *out, double *Q, double *E)
{
    for (int b = 0; b < mu; b++) Q[b] = E[b] = 0.0;
    for (int j = 0; j < m; j++) {
        if (in[j].q <= 0.0) continue;
        int b = (int)(de_cap(in[j].p) * mu);
        if (b >= mu) b = mu - 1;
        if (b < 0) b = 0;
        Q[b] += in[j].q;
        E[b] += in[j].q * in[j].p;
    }
    int k = 0;
    for (int b = 0; b < mu; b++)
        if (Q[b] > 0.0) {
            out[k].q = Q[b];
            out[k].p = E[b] / Q[b];
            k++;
        }
    return k;
}

typedef struct {
    int mu;
    de_comp *work;  /* 2 mu^2 components */
    double *Q, *E;  /* mu bins */
} de_ctx;

static int de_check(const de_ctx *D, const de_comp *a, int na, const de_comp *b, int nb, de_comp *out)
{
    int m = 0;
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            D->work[m].q = a[i].q * b[j].q;
            D->work[m].p = a[i].p * (1.0 - b[j].p) + b[j].p * (1.0 - a[i].p);
            m++;
        }
    return de_merge(D->work, m, D->mu, out, D->Q, D->E);
}

static int de_var(const de_comp *D_a, int na, const de_comp *b, int nb, const de_ctx *D, de_comp *out)
{
    int m = 0;
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            double pa = D_a[i].p, pb = b[j].p, w = D_a[i].q * b[j].q;
            double s = pa * pb + (1.0 - pa) * (1.0 - pb);
            if (s > 0.0) {
                D->work[m].q = w * s;
                D->work[m].p = pa * pb / s;
                m++;
            }
            if (s < 1.0) {
                double x = pa * (1.0 - pb), y = pb * (1.0 - pa);
                D->work[m].q = w * (1.0 - s);
                D->work[m].p = (x < y ? x : y) / (1.0 - s);
                m++;
            }
        }
    return de_merge(D->work, m, D->mu, out, D->Q, D->E);
}

/* chans: S channels of at most mu components each (counts in cnt); writes
 * the error-probability bound of each leaf channel in tree order */
static void de_rec(const de_ctx *D, int S, const de_comp *chans, const int *cnt, double *pe, de_comp *tmp,
                   int *tcnt)
{
    int mu = D->mu;
    if (S == 1) {
        double e = 0.0;
        for (int j = 0; j < cnt[0]; j++) e += chans[j].q * chans[j].p;
        pe[0] = e;
        return;
    }
    int h = S / 2;
    de_comp *child = tmp;
    int *ccnt = tcnt;
    for (int i = 0; i < h; i++)
        ccnt[i] = de_check(D, chans + (size_t)i * mu, cnt[i], chans + (size_t)(i + h) * mu, cnt[i + h],
                           child + (size_t)i * mu);
    de_rec(D, h, child, ccnt, pe, tmp + (size_t)h * mu, tcnt + h);
    for (int i = 0; i < h; i++)
        ccnt[i] = de_var(chans + (size_t)i * mu, cnt[i], chans + (size_t)(i + h) * mu, cnt[i + h], D,
                         child + (size_t)i * mu);
    de_rec(D, h, child, ccnt, pe + h, tmp + (size_t)h * mu, tcnt + h);
}

/* Error-probability bounds of the N bit channels when every channel use is
 * the BMS mixture (q[0..m), p[0..m)) and punctured positions carry nothing
 * (a BSC with crossover 1/2).  m <= mu.                                      */
void orc_de_bms(int N, const uint8_t *punct, int m, const double *q, const double *p, int mu, double *pe)
{
    de_ctx D;
    D.mu = mu;
    D.work = (de_comp *)malloc(sizeof(de_comp) * (size_t)(2 * mu * mu));
    D.Q = (double *)malloc(sizeof(double) * (size_t)mu);
    D.E = (double *)malloc(sizeof(double) * (size_t)mu);
    de_comp *ch = (de_comp *)calloc((size_t)N * (size_t)mu, sizeof(de_comp));
    de_comp *tmp = (de_comp *)calloc((size_t)(2 * N + 2) * (size_t)mu, sizeof(de_comp));
    int *cnt = (int *)calloc((size_t)N, sizeof(int));
    int *tcnt = (int *)calloc((size_t)(2 * N + 2), sizeof(int));
    for (int i = 0; i < N; i++) {
        if (punct && punct[i]) {
            ch[(size_t)i * mu].q = 1.0;
            ch[(size_t)i * mu].p = 0.5;
            cnt[i] = 1;
        } else {
            for (int j = 0; j < m; j++) {
                ch[(size_t)i * mu + j].q = q[j];
                ch[(size_t)i * mu + j].p = p[j];
            }
            cnt[i] = m;
        }
    }
    de_rec(&D, N, ch, cnt, pe, tmp, tcnt);
    free(D.work); free(D.Q); free(D.E); free(ch); free(tmp); free(cnt); free(tcnt);
}

/* standard normal tail beyond x */
static double q_tail(double x) { return 0.5 * erfc(x / sqrt(2.0)); }

/* BPSK over AWGN of variance sigma2 as a mixture of mu BSCs: the reliability
 * |LLR| = a of a channel output is a BSC with crossover 1 / (1 + e^a); the
 * axis of a is cut where that BSC's capacity crosses b / mu, b = 1..mu-1, and
 * the BSCs of each interval are merged (their mean crossover is the error
 * mass of the interval over its probability).  With x = 0 sent, y ~ N(1,
 * sigma2), LLR = 2 y / sigma2, |LLR| in [A, B) for y in +-[A, B) sigma2 / 2. */
int orc_de_awgn_channel(double sigma2, int mu, double *q, double *p)
{
    double sigma = sqrt(sigma2);
    double prev_a = 0.0;
    int k = 0;
    for (int b = 1; b <= mu; b++) {
        double a;
        if (b == mu) {
            a = INFINITY;
        } else {
            /* capacity of the BSC at reliability a rises from 0 to 1: bisection */
            double lo = 0.0, hi = 200.0, target = (double)b / mu;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi);
                if (de_cap(1.0 / (1.0 + exp(mid))) < target) lo = mid; else hi = mid;
            }
            a = 0.5 * (lo + hi);
        }
        double u = prev_a * sigma2 / 2.0, v = isinf(a) ? INFINITY : a * sigma2 / 2.0;
        /* P(y in [u, v)) and P(y in (-v, -u]) for y ~ N(1, sigma2) */
        double good = q_tail((u - 1.0) / sigma) - (isinf(v) ? 0.0 : q_tail((v - 1.0) / sigma));
        double bad = q_tail((u + 1.0) / sigma) - (isinf(v) ? 0.0 : q_tail((v + 1.0) / sigma));
        if (good + bad > 0.0) {
            q[k] = good + bad;
            p[k] = bad / (good + bad);
            k++;
        }
        prev_a = a;
    }
    return k;
}

void orc_de_reliability(int N, const uint8_t *punct, double sigma2, int mu, double *pe)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)mu);
    double *p = (double *)malloc(sizeof(double) * (size_t)mu);
    int m = orc_de_awgn_channel(sigma2, mu, q, p);
    orc_de_bms(N, punct, m, q, p, mu, pe);
    free(q);
    free(p);
}

/* Frozen set from the bounds: the |A| = K channels with the smallest error
 * probability carry information; ties go to the larger index.              */
void orc_de_frozen(int N, int K, int K_info, const uint8_t *punct, double design_ebn0_db, int mu,
                   uint8_t *frozen, double *pe_out)
{
    int P = 0;
    if (punct)
        for (int i = 0; i < N; i++) P += punct[i] ? 1 : 0;
    double R = (double)K_info / (double)(N - P);
    double sigma2 = 1.0 / (2.0 * R * pow(10.0, design_ebn0_db / 10.0));
    double *pe = (double *)malloc(sizeof(double) * (size_t)N);
    orc_de_reliability(N, punct, sigma2, mu, pe);
    if (pe_out) memcpy(pe_out, pe, sizeof(double) * (size_t)N);
    for (int i = 0; i < N; i++) frozen[i] = 1;
    for (int k = 0; k < K; k++) {
        int best = -1;
        for (int i = 0; i < N; i++) {
            if (!frozen[i]) continue;
            if (best < 0 || pe[i] < pe[best] || (pe[i] == pe[best] && i > best)) best = i;
        }
        frozen[best] = 0;
    }
    free(pe);
}

/* Quasi-uniform puncturing (cited in Sec. III-A, Niu et al.): the first P
 * positions in bit-reversed order are not transmitted.                      */
void orc_qup_pattern(int N, int P, uint8_t *punct)
{
    int n = 0;
    while ((1 << n) < N) n++;
    memset(punct, 0, (size_t)N);
    for (int i = 0; i < P; i++) {
        int r = 0;
        for (int b = 0; b < n; b++)
            if (i & (1 << b)) r |= 1 << (n - 1 - b);
        punct[r] = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Arithmetic of the decoder (Sec. II-B f, g, h; Sec. III-B-3 fixed point).
 * Every value is kept in a double; in the float mode each operation is done
 * in float and the float result stored (exact, a float is a double), in the
 * fixed-point modes values are integers and every add saturates to [-Q, Q]. */
typedef struct {
    int mode;     /* ORC_MODE_F32, ORC_MODE_FIXED, ORC_MODE_EXACT */
    int frac;     /* fixed point: fractional bits */
    double Q;     /* fixed point: saturation bound */
} arith_t;

static double sat(const arith_t *A, double v)
{
    if (v > A->Q) return A->Q;
    if (v < -A->Q) return -A->Q;
    return v;
}

static int hd(double v) { return v < 0.0; }

/* log(1 + exp(x)) without overflow */
static double softplus(double x)
{
    if (x > 0.0) return x + log1p(exp(-x));
    return log1p(exp(x));
}

/* f (Sec. II-B): sign(a b) min(|a|, |b|).  The sign is taken from the sign
 * bits (so f(-0, 3) = -0, which decides 0 like +0).  Exact mode: the exact
 * check-node rule 2 atanh(tanh(a/2) tanh(b/2)) in its numerically stable form
 * sign(a)sign(b)min(|a|,|b|) + ln(1+e^-|a+b|) - ln(1+e^-|a-b|).             */
static double a_f(const arith_t *A, double a, double b)
{
    if (A->mode == ORC_MODE_EXACT) {
        double s = ((a < 0) != (b < 0)) ? -1.0 : 1.0;
        double m = fmin(fabs(a), fabs(b));
        return s * m + log1p(exp(-fabs(a + b))) - log1p(exp(-fabs(a - b)));
    }
    if (A->mode == ORC_MODE_F32) {
        float fa = (float)a, fb = (float)b;
        float m = fminf(fabsf(fa), fabsf(fb));
        int neg = (signbit(fa) != 0) != (signbit(fb) != 0);
        return (double)(neg ? -m : m);
    }
    double m = fmin(fabs(a), fabs(b));
    int neg = (a < 0) != (b < 0);
    return neg ? -m : m;
}

/* g (Sec. II-B): (1 - 2 s) a + b, computed as (s ? -a : a) + b.              */
static double a_g(const arith_t *A, double a, double b, int s)
{
    if (A->mode == ORC_MODE_F32) {
        float fa = (float)a, fb = (float)b;
        float t = s ? -fa : fa;
        volatile float r = t + fb; /* one float rounding, never fused */
        return (double)r;
    }
    if (A->mode == ORC_MODE_EXACT) return (s ? -a : a) + b;
    return sat(A, (s ? -a : a) + b);
}

/* addition of non-negative metric terms (path metric, penalties) */
static double a_add(const arith_t *A, double x, double y)
{
    if (A->mode == ORC_MODE_F32) {
        volatile float r = (float)x + (float)y;
        return (double)r;
    }
    if (A->mode == ORC_MODE_EXACT) return x + y;
    return sat(A, x + y);
}

static double a_abs(const arith_t *A, double v)
{
    (void)A;
    return fabs(v);
}

/* Channel LLR into the decoder's number format (Sec. III-B-3).              */
static double a_quant(const arith_t *A, double lam)
{
    if (A->mode == ORC_MODE_F32) return (double)(float)lam;
    if (A->mode == ORC_MODE_EXACT) return lam;
    double x = ldexp(lam, A->frac);
    if (x > A->Q) x = A->Q;
    if (x < -A->Q) x = -A->Q;
    return nearbyint(x); /* default rounding mode: half to even */
}

/* Balanced pairwise sum over index order: s(lo,hi) = s(lo,mid) + s(mid,hi). */
static double tree_sum(const arith_t *A, const double *v, int lo, int hi)
{
    if (hi - lo == 1) return v[lo];
    int mid = lo + (hi - lo) / 2;
    return a_add(A, tree_sum(A, v, lo, mid), tree_sum(A, v, mid, hi));
}

/* ------------------------------------------------------------------------ */
/* Node classification for tree pruning (Sec. II-B, Sec. III-B-2): the
 * top-most node whose leaves match a type that is enabled and within its size
 * limit replaces its subtree.  Precedence R0 > R1 > REP > SPC.  A size-1 node
 * is a frozen leaf (R0) or an information leaf (R1 of size 1).  Nodes below
 * node_min leaves are internal: their subtrees are decoded leaf by leaf.   */
static int classify(const orc_code *cd, const orc_pruning *pr, int o, int S)
{
    int nf = 0;
    for (int i = o; i < o + S; i++) nf += cd->frozen[i] ? 1 : 0;
    if (S == 1) return nf ? ORC_NODE_R0 : ORC_NODE_R1;
    if (!pr || S < pr->node_min) return ORC_NODE_INTERNAL;
    if (nf == S && (pr->mask & ORC_PRUNE_R0)) return ORC_NODE_R0;
    if (nf == 0 && (pr->mask & ORC_PRUNE_R1) && (pr->r1_max == 0 || S <= pr->r1_max))
        return ORC_NODE_R1;
    if (nf == S - 1 && !cd->frozen[o + S - 1] && (pr->mask & ORC_PRUNE_REP) &&
        (pr->rep_max == 0 || S <= pr->rep_max))
        return ORC_NODE_REP;
    if (nf == 1 && cd->frozen[o] && S >= 4 && (pr->mask & ORC_PRUNE_SPC) &&
        (pr->spc_max == 0 || S <= pr->spc_max))
        return ORC_NODE_SPC;
    return ORC_NODE_INTERNAL;
}

typedef struct {
    double pm;
    int c;
    int p;
    int j;
} cand_t;

static int cmp_pm_c(const void *x, const void *y)
{
    const cand_t *a = (const cand_t *)x, *b = (const cand_t *)y;
    if (a->pm < b->pm) return -1;
    if (a->pm > b->pm) return 1;
    return (a->c > b->c) - (a->c < b->c);
}

static int cmp_c(const void *x, const void *y)
{
    const cand_t *a = (const cand_t *)x, *b = (const cand_t *)y;
    return (a->c > b->c) - (a->c < b->c);
}

/* Sort positions of a node by (|alpha|, index) ascending (least reliable
 * first); used by R1 and SPC.                                               */
static void reliability_order(const double *alpha, int S, int *order)
{
    for (int i = 0; i < S; i++) order[i] = i;
    /* insertion sort: plain and stable by index */
    for (int i = 1; i < S; i++) {
        int k = order[i];
        int m = i - 1;
        while (m >= 0) {
            double am = fabs(alpha[order[m]]), ak = fabs(alpha[k]);
            if (am > ak) { order[m + 1] = order[m]; m--; }
            else break;
        }
        order[m + 1] = k;
    }
}

static int popcount_u(unsigned v)
{
    int c = 0;
    while (v) { c += (int)(v & 1u); v >>= 1; }
    return c;
}


/* ------------------------------------------------------------------------ */
/* Node handlers (Sec. II-B "Simplified SC and SCL", Sec. IV-C sorting).
 * For one path at one node: M candidates, candidate j has a penalty and a
 * node codeword beta (the node's partial sums, S bits).                     */
typedef struct {
    int type, S, t;
    const double *alpha; /* node LLRs of the path, S values */
    int *order;          /* positions by (|alpha|, index) ascending */
    uint8_t *h;          /* hard decisions */
    int parity;          /* XOR of h */
    double *buf;         /* scratch, S values */
} node_ctx;

static int node_M(const node_ctx *nc)
{
    switch (nc->type) {
    case ORC_NODE_R0: return 1;
    case ORC_NODE_REP: return 2;
    case ORC_NODE_R1: return 1 << nc->t;
    case ORC_NODE_SPC: return 1 << (nc->t - 1);
    }
    return 0;
}

/* Flip pattern of SPC candidate m: the m-th j (increasing) among 0..2^t-1
 * whose flips of the t least reliable bits make the parity even.            */
static int spc_j(const node_ctx *nc, int m)
{
    int seen = 0;
    for (int j = 0; j < (1 << nc->t); j++) {
        if ((popcount_u((unsigned)j) & 1) == nc->parity) {
            if (seen == m) return j;
            seen++;
        }
    }
    return -1;
}

static double node_pen(const arith_t *A, const node_ctx *nc, int cand)
{
    int S = nc->S;
    if (A->mode == ORC_MODE_EXACT) {
        /* exact metric, leaves only: ln(1 + exp(-(1 - 2u) lambda)) */
        double lam = nc->alpha[0];
        int u = (nc->type == ORC_NODE_R0) ? 0 : (hd(lam) ^ cand);
        return softplus(-(1.0 - 2.0 * u) * lam);
    }
    if (nc->type == ORC_NODE_R0 || nc->type == ORC_NODE_REP) {
        /* R0 and REP j=0: all-zero word, REP j=1: all-one word; the penalty
         * sums |alpha_i| over positions that disagree with the word.        */
        int ones = (nc->type == ORC_NODE_REP) && cand == 1;
        for (int i = 0; i < S; i++) {
            double a = nc->alpha[i];
            int disagree = ones ? (a > 0) : hd(a);
            nc->buf[i] = disagree ? a_abs(A, a) : 0.0;
        }
        return tree_sum(A, nc->buf, 0, S);
    }
    /* R1 / SPC: left fold of |alpha| over flipped ranks, ascending rank */
    int j = (nc->type == ORC_NODE_SPC) ? spc_j(nc, cand) : cand;
    double pen = 0.0;
    for (int k = 0; k < nc->t; k++)
        if (j & (1 << k)) pen = a_add(A, pen, a_abs(A, nc->alpha[nc->order[k]]));
    return pen;
}

static void node_beta(const node_ctx *nc, int cand, uint8_t *beta)
{
    int S = nc->S;
    if (nc->type == ORC_NODE_R0) { memset(beta, 0, (size_t)S); return; }
    if (nc->type == ORC_NODE_REP) { memset(beta, cand ? 1 : 0, (size_t)S); return; }
    int j = (nc->type == ORC_NODE_SPC) ? spc_j(nc, cand) : cand;
    memcpy(beta, nc->h, (size_t)S);
    for (int k = 0; k < nc->t; k++)
        if (j & (1 << k)) beta[nc->order[k]] ^= 1;
}

/* ------------------------------------------------------------------------ */
/* SCL decoder (Algorithm 1).  Per path: lambda[2N] and s[N].  The root LLRs
 * sit at lambda[0..N); a node of size Nv at offset o_l has its children's
 * LLRs at o_l + Nv.  Partial sums of a node covering leaves [o_s, o_s + Nv)
 * sit at s[o_s .. o_s + Nv).                                                 */
typedef struct {
    double *lam;
    uint8_t *s;
    double pm;
} path_t;

typedef struct {
    const orc_code *cd;
    const orc_pruning *pr;
    arith_t A;
    int L;
    int n_active;
    path_t *paths; /* L live paths (slots 0..n_active-1) */
    path_t *next;  /* L paths being built by update_paths */
    int *order;
    uint8_t *h;
    double *buf;
    uint8_t *beta;
    cand_t *cands;
    node_ctx *ctx; /* one per active path */
    orc_stats *st;
    int err;
} dec_t;

static void normalise(dec_t *D)
{
    if (D->A.mode != ORC_MODE_FIXED) return;
    double mn = D->paths[0].pm;
    for (int p = 1; p < D->n_active; p++)
        if (D->paths[p].pm < mn) mn = D->paths[p].pm;
    for (int p = 0; p < D->n_active; p++) D->paths[p].pm -= mn;
}

static void prepare_node(dec_t *D, node_ctx *nc, int p, int type, int S, int o_l)
{
    nc->type = type;
    nc->S = S;
    nc->alpha = D->paths[p].lam + o_l;
    nc->order = D->order + (size_t)p * (size_t)D->cd->N;
    nc->h = D->h + (size_t)p * (size_t)D->cd->N;
    nc->buf = D->buf;
    nc->t = 0;
    if (type == ORC_NODE_R1) {
        int t = D->pr && D->pr->r1_t > 0 ? D->pr->r1_t : S;
        nc->t = t < S ? t : S;
        if (D->A.mode == ORC_MODE_EXACT) nc->t = 1;
    } else if (type == ORC_NODE_SPC) {
        int t = D->pr && D->pr->spc_t > 0 ? D->pr->spc_t : S;
        nc->t = t < S ? t : S;
    }
    int par = 0;
    for (int i = 0; i < S; i++) {
        nc->h[i] = (uint8_t)hd(nc->alpha[i]);
        par ^= nc->h[i];
    }
    nc->parity = par;
    if (type == ORC_NODE_R1 || type == ORC_NODE_SPC) reliability_order(nc->alpha, S, nc->order);
}

/* update_paths() generalised to a node (Algorithm 1 leaf step; Sec. II-B):
 * every active path p offers M candidates, c = p*M + j; the min(L, n)
 * smallest (PM, c) survive and take new slots in increasing c.             */
static void update_paths(dec_t *D, int type, int S, int o_l, int o_s)
{
    int na = D->n_active;
    if (type != ORC_NODE_R0 && type != ORC_NODE_R1 && type != ORC_NODE_REP && type != ORC_NODE_SPC) {
        D->err = 1;
        return;
    }
    for (int p = 0; p < na; p++) prepare_node(D, &D->ctx[p], p, type, S, o_l);
    int M = node_M(&D->ctx[0]);
    if (M > 4096 || M < 1) { D->err = 2; return; }
    int n = 0;
    for (int p = 0; p < na; p++) {
        for (int j = 0; j < M; j++) {
            cand_t *c = &D->cands[n++];
            c->pm = a_add(&D->A, D->paths[p].pm, node_pen(&D->A, &D->ctx[p], j));
            c->c = p * M + j;
            c->p = p;
            c->j = j;
        }
    }
    int keep = n < D->L ? n : D->L;
    if (D->st) {
        D->st->node_steps++;
        if (n > D->L) D->st->sorts++;
        D->st->cand_total += n;
    }
    qsort(D->cands, (size_t)n, sizeof(cand_t), cmp_pm_c);
    qsort(D->cands, (size_t)keep, sizeof(cand_t), cmp_c);
    int N = D->cd->N;
    for (int q = 0; q < keep; q++) {
        const cand_t *c = &D->cands[q];
        path_t *src = &D->paths[c->p];
        path_t *dst = &D->next[q];
        memcpy(dst->lam, src->lam, sizeof(double) * (size_t)(2 * N));
        memcpy(dst->s, src->s, (size_t)N);
        dst->pm = c->pm;
        node_beta(&D->ctx[c->p], c->j, dst->s + o_s);
    }
    path_t *tmp = D->paths;
    D->paths = D->next;
    D->next = tmp;
    D->n_active = keep;
    normalise(D);
}

static void scl_rec(dec_t *D, int Nv, int o_l, int o_s)
{
    if (D->err) return;
    int type = classify(D->cd, D->pr, o_s, Nv);
    if (type != ORC_NODE_INTERNAL) {
        update_paths(D, type, Nv, o_l, o_s);
        return;
    }
    int h = Nv / 2;
    for (int p = 0; p < D->n_active; p++) {
        double *lam = D->paths[p].lam;
        for (int i = 0; i < h; i++) lam[o_l + Nv + i] = a_f(&D->A, lam[o_l + i], lam[o_l + h + i]);
    }
    if (D->st) D->st->fg_elems += (long long)h * D->n_active;
    scl_rec(D, h, o_l + Nv, o_s);
    for (int p = 0; p < D->n_active; p++) {
        double *lam = D->paths[p].lam;
        const uint8_t *s = D->paths[p].s;
        for (int i = 0; i < h; i++)
            lam[o_l + Nv + i] = a_g(&D->A, lam[o_l + i], lam[o_l + h + i], s[o_s + i]);
    }
    if (D->st) D->st->fg_elems += (long long)h * D->n_active;
    scl_rec(D, h, o_l + Nv, o_s + h);
    for (int p = 0; p < D->n_active; p++) {
        uint8_t *s = D->paths[p].s;
        for (int i = 0; i < h; i++) s[o_s + i] ^= s[o_s + h + i];
    }
}

/* extract u_A from a decoded codeword x (systematic: x_A; otherwise the
 * transform is an involution, so u = x F) and check the CRC (Sec. IV-B).   */
static int extract_check(const orc_code *cd, const uint8_t *x, uint8_t *uA, uint8_t *work)
{
    int N = cd->N;
    memcpy(work, x, (size_t)N);
    if (!cd->systematic) orc_polar_transform(N, work);
    int k = 0;
    for (int i = 0; i < N; i++)
        if (!cd->frozen[i]) uA[k++] = work[i];
    int kinfo = cd->K - cd->crc_len;
    if (cd->crc_len == 0) return 1;
    uint32_t r = orc_crc(uA, kinfo, cd->crc_len, cd->crc_poly);
    for (int b = 0; b < cd->crc_len; b++)
        if (uA[kinfo + b] != (uint8_t)((r >> (cd->crc_len - 1 - b)) & 1u)) return 0;
    return 1;
}

typedef struct {
    int crc_ok;
    int slot;
    int L;
} stage_result;

/* One CA-SCL decode at list size L from the channel LLRs (Algorithm 1 and
 * select_best_path with sorted CRC checks, Sec. IV-B).                      */
static int scl_stage(const orc_code *cd, const double *llr_full, int L, const orc_pruning *pr,
                     const arith_t *A, orc_stats *st, uint8_t *info_out, double *pm_out,
                     uint8_t *paths_out, stage_result *res)
{
    int N = cd->N;
    dec_t D;
    memset(&D, 0, sizeof(D));
    D.cd = cd;
    D.pr = pr;
    D.A = *A;
    D.L = L;
    D.st = st;
    int cap = L;
    D.paths = (path_t *)calloc((size_t)cap, sizeof(path_t));
    D.next = (path_t *)calloc((size_t)cap, sizeof(path_t));
    for (int p = 0; p < cap; p++) {
        D.paths[p].lam = (double *)calloc((size_t)(2 * N), sizeof(double));
        D.paths[p].s = (uint8_t *)calloc((size_t)N, 1);
        D.next[p].lam = (double *)calloc((size_t)(2 * N), sizeof(double));
        D.next[p].s = (uint8_t *)calloc((size_t)N, 1);
    }
    D.order = (int *)calloc((size_t)cap * (size_t)N, sizeof(int));
    D.h = (uint8_t *)calloc((size_t)cap * (size_t)N, 1);
    D.buf = (double *)calloc((size_t)N, sizeof(double));
    D.ctx = (node_ctx *)calloc((size_t)cap, sizeof(node_ctx));
    /* the largest candidate set: R1 with t up to 12 or SPC; bounded here */
    size_t max_c = (size_t)cap * 4096u;
    D.cands = (cand_t *)calloc(max_c, sizeof(cand_t));
    for (int i = 0; i < N; i++) D.paths[0].lam[i] = llr_full[i];
    D.paths[0].pm = 0.0;
    D.n_active = 1;

    scl_rec(&D, N, 0, 0);

    int rc = D.err ? -3 : 0;
    if (!rc) {
        /* select_best_path: order by (PM, slot), first valid CRC wins */
        int na = D.n_active;
        int *ord = (int *)malloc(sizeof(int) * (size_t)na);
        for (int p = 0; p < na; p++) ord[p] = p;
        for (int a = 1; a < na; a++) {
            int k = ord[a], m = a - 1;
            while (m >= 0 && D.paths[ord[m]].pm > D.paths[k].pm) { ord[m + 1] = ord[m]; m--; }
            ord[m + 1] = k;
        }
        uint8_t *uA = (uint8_t *)malloc((size_t)N);
        uint8_t *work = (uint8_t *)malloc((size_t)N);
        int chosen = ord[0], ok = 0;
        for (int r = 0; r < na; r++) {
            if (extract_check(cd, D.paths[ord[r]].s, uA, work)) { chosen = ord[r]; ok = 1; break; }
        }
        extract_check(cd, D.paths[chosen].s, uA, work);
        int kinfo = cd->K - cd->crc_len;
        if (info_out) memcpy(info_out, uA, (size_t)kinfo);
        if (pm_out)
            for (int p = 0; p < L; p++) pm_out[p] = p < na ? D.paths[p].pm : INFINITY;
        if (paths_out)
            for (int p = 0; p < L; p++) {
                if (p < na) memcpy(paths_out + (size_t)p * (size_t)N, D.paths[p].s, (size_t)N);
                else memset(paths_out + (size_t)p * (size_t)N, 0, (size_t)N);
            }
        res->crc_ok = ok;
        res->slot = chosen;
        res->L = L;
        free(ord);
        free(uA);
        free(work);
    }
    for (int p = 0; p < cap; p++) {
        free(D.paths[p].lam); free(D.paths[p].s);
        free(D.next[p].lam); free(D.next[p].s);
    }
    free(D.paths); free(D.next); free(D.order); free(D.h); free(D.buf); free(D.ctx); free(D.cands);
    return rc;
}

static int set_arith(int mode, int frac, double Q, arith_t *A)
{
    A->frac = 0;
    A->Q = 0;
    switch (mode) {
    case ORC_F32: A->mode = ORC_MODE_F32; return 0;
    case ORC_I16: A->mode = ORC_MODE_FIXED; A->frac = 5; A->Q = 32767.0; return 0;
    case ORC_I8: A->mode = ORC_MODE_FIXED; A->frac = 2; A->Q = 127.0; return 0;
    case ORC_IWIDE: A->mode = ORC_MODE_FIXED; A->frac = frac; A->Q = Q; return 0;
    case ORC_EXACT: A->mode = ORC_MODE_EXACT; return 0;
    }
    return -1;
}

/* Channel LLRs (non-punctured positions, in increasing position order) to the
 * N root LLRs: a punctured position was never sent, so its LLR is 0.       */
static void scatter_llr(const orc_code *cd, const double *llr, const arith_t *A, double *full)
{
    int k = 0;
    for (int i = 0; i < cd->N; i++) {
        if (cd->punct && cd->punct[i]) full[i] = 0.0;
        else full[i] = a_quant(A, llr[k++]);
    }
}

/* The decoders of Sec. II-B: SC (L = 1), CA-SCL(L), and the adaptive
 * schedules FA (L = 1, 2, 4, ..., Lmax, stop at the first CRC pass) and PA
 * (L = 1 then Lmax), each stage a fresh decode from the channel LLRs.
 * status: bit 0 CRC passed (always 1 with no CRC), bits 8..15 the list size
 * of the stage that produced the output, bits 16..23 its slot.             */
int orc_decode(const orc_code *cd, const double *llr, int L, int algo, const orc_pruning *pr,
               int mode, int wide_frac, double wide_q, uint8_t *info_out, int32_t *status,
               double *pm_out, uint8_t *paths_out, orc_stats *st)
{
    arith_t A;
    if (set_arith(mode, wide_frac, wide_q, &A)) return -1;
    if (A.mode == ORC_MODE_EXACT && pr && pr->mask) return -1;
    int N = cd->N;
    if (N < 2 || (N & (N - 1))) return -1;
    int nA = 0;
    for (int i = 0; i < N; i++) nA += cd->frozen[i] ? 0 : 1;
    if (nA != cd->K || cd->crc_len > cd->K) return -1;
    if (L < 1) return -1;
    double *full = (double *)malloc(sizeof(double) * (size_t)N);
    scatter_llr(cd, llr, &A, full);
    int stages[16], ns = 0;
    if (algo == ORC_ALGO_SC) stages[ns++] = 1;
    else if (algo == ORC_ALGO_CASCL) stages[ns++] = L;
    else if (algo == ORC_ALGO_FA) {
        for (int l = 1; l < L; l *= 2) stages[ns++] = l;
        stages[ns++] = L;
    } else if (algo == ORC_ALGO_PA) {
        stages[ns++] = 1;
        if (L > 1) stages[ns++] = L;
    } else { free(full); return -1; }
    stage_result res = {0, 0, 0};
    int rc = 0;
    for (int s = 0; s < ns; s++) {
        if (pm_out) for (int p = 0; p < L; p++) pm_out[p] = INFINITY;
        rc = scl_stage(cd, full, stages[s], pr, &A, st, info_out, pm_out, paths_out, &res);
        if (rc) break;
        if (st) st->stages++;
        if (res.crc_ok) break;
    }
    free(full);
    if (rc) return rc;
    if (status) *status = (res.crc_ok ? 1 : 0) | (res.L << 8) | (res.slot << 16);
    return 0;
}

/* Plain SC and SSC decoding (Sec. II-B), written without any list
 * machinery: hard decisions at information leaves, zero at frozen leaves,
 * and the classic single-path node rules (R0 zero word, R1 hard decision,
 * REP the all-one word only when its penalty is strictly smaller, SPC hard
 * decision with the least reliable bit flipped when the parity is odd).
 * Writes the decoded codeword x (N bits).                                    */
static void sc_rec(const orc_code *cd, const orc_pruning *pr, const arith_t *A, double *lam,
                   uint8_t *s, int Nv, int o_l, int o_s, double *buf, int *order)
{
    int type = classify(cd, pr, o_s, Nv);
    const double *al = lam + o_l;
    if (type == ORC_NODE_R0) { memset(s + o_s, 0, (size_t)Nv); return; }
    if (type == ORC_NODE_R1) {
        for (int i = 0; i < Nv; i++) s[o_s + i] = (uint8_t)hd(al[i]);
        return;
    }
    if (type == ORC_NODE_REP) {
        for (int i = 0; i < Nv; i++) buf[i] = hd(al[i]) ? fabs(al[i]) : 0.0;
        double p0 = tree_sum(A, buf, 0, Nv);
        for (int i = 0; i < Nv; i++) buf[i] = (al[i] > 0) ? fabs(al[i]) : 0.0;
        double p1 = tree_sum(A, buf, 0, Nv);
        memset(s + o_s, p1 < p0 ? 1 : 0, (size_t)Nv);
        return;
    }
    if (type == ORC_NODE_SPC) {
        int par = 0;
        for (int i = 0; i < Nv; i++) { s[o_s + i] = (uint8_t)hd(al[i]); par ^= s[o_s + i]; }
        if (par) {
            reliability_order(al, Nv, order);
            s[o_s + order[0]] ^= 1;
        }
        return;
    }
    int h = Nv / 2;
    for (int i = 0; i < h; i++) lam[o_l + Nv + i] = a_f(A, lam[o_l + i], lam[o_l + h + i]);
    sc_rec(cd, pr, A, lam, s, h, o_l + Nv, o_s, buf, order);
    for (int i = 0; i < h; i++) lam[o_l + Nv + i] = a_g(A, lam[o_l + i], lam[o_l + h + i], s[o_s + i]);
    sc_rec(cd, pr, A, lam, s, h, o_l + Nv, o_s + h, buf, order);
    for (int i = 0; i < h; i++) s[o_s + i] ^= s[o_s + h + i];
}

int orc_sc_plain(const orc_code *cd, const double *llr, const orc_pruning *pr, int mode, int wide_frac,
                 double wide_q, uint8_t *x_out)
{
    arith_t A;
    if (set_arith(mode, wide_frac, wide_q, &A) || A.mode == ORC_MODE_EXACT) return -1;
    int N = cd->N;
    double *lam = (double *)calloc((size_t)(2 * N), sizeof(double));
    double *buf = (double *)calloc((size_t)N, sizeof(double));
    int *order = (int *)calloc((size_t)N, sizeof(int));
    scatter_llr(cd, llr, &A, lam);
    sc_rec(cd, pr, &A, lam, x_out, N, 0, 0, buf, order);
    free(lam);
    free(buf);
    free(order);
    return 0;
}

/* Node type of each node of the pruned tree, for tests: writes, in pre-order,
 * (depth, offset, type) triples of the nodes that are not internal.        */
static void types_rec(const orc_code *cd, const orc_pruning *pr, int Nv, int o, int d, int32_t *out,
                      int *n)
{
    int type = classify(cd, pr, o, Nv);
    if (type != ORC_NODE_INTERNAL) {
        out[3 * *n] = d;
        out[3 * *n + 1] = o;
        out[3 * *n + 2] = type;
        (*n)++;
        return;
    }
    types_rec(cd, pr, Nv / 2, o, d + 1, out, n);
    types_rec(cd, pr, Nv / 2, o + Nv / 2, d + 1, out, n);
}

int orc_node_list(const orc_code *cd, const orc_pruning *pr, int32_t *out)
{
    int n = 0;
    types_rec(cd, pr, cd->N, 0, 0, out, &n);
    return n;
}

/* Batch helper for the tests and the CPU baseline: frames are independent. */
int orc_decode_batch(const orc_code *cd, const double *llr, int n_frames, int L, int algo,
                     const orc_pruning *pr, int mode, int wide_frac, double wide_q, uint8_t *info_out,
                     int32_t *status, double *pm_out, orc_stats *st)
{
    int P = 0;
    if (cd->punct)
        for (int i = 0; i < cd->N; i++) P += cd->punct[i] ? 1 : 0;
    int stride = cd->N - P;
    int kinfo = cd->K - cd->crc_len;
    for (int f = 0; f < n_frames; f++) {
        int rc = orc_decode(cd, llr + (size_t)f * (size_t)stride, L, algo, pr, mode, wide_frac, wide_q,
                            info_out ? info_out + (size_t)f * (size_t)kinfo : NULL,
                            status ? status + f : NULL, pm_out ? pm_out + (size_t)f * (size_t)L : NULL,
                            NULL, st);
        if (rc) return rc;
    }
    return 0;
}
