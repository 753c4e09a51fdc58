/*
 * mrg_oracle.c -- plain, slow CPU oracle for combined multiple-recursive
 * generators (MRG32k3a; MRG31k3p for reproducing the paper's printed output).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is computed from the definitions, in the most direct way:
 *   - a component step is the order-3 linear recurrence of Sec. 2 evaluated
 *     with 128-bit signed integers and one `%` (no folding tricks);
 *   - a stream start is "jump ahead by Z steps" from the previous start
 *     (Sec. 2.1), evaluated as the companion-matrix power A^Z by
 *     square-and-multiply with 128-bit products;
 *   - uniforms are z * norm with norm = 1/(m1+1) in IEEE double (the kernel
 *     multiplies the integer output by a constant factor, Sec. 2.2 Listing 1);
 *   - normals follow the Box-Muller transform (Sec. 3.1, Algorithm 1),
 *     exponentials the inverse transform -log(u)/rate (Sec. 3.2), both in
 *     double with libm, using exact integer argument reductions so that the
 *     reference keeps full relative accuracy near zeros.
 *
 * State convention (Sec. 2.1 printout, current.g1.1 .. g2.3): per stream six
 * words, newest first:  x1[n-1], x1[n-2], x1[n-3], x2[n-1], x2[n-2], x2[n-3].
 *
 * Generator parameters are passed in as p[8] = {m1, m2, a1_1, a1_2, a1_3,
 * a2_1, a2_2, a2_3}, where a_c_j is the (signed) coefficient of x_c[n-j].
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * (-ffp-contract=off keeps every product and sum a separately rounded IEEE
 * operation on every host, including aarch64 where gcc would otherwise fuse.)
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

typedef struct {
    uint64_t m[2];
    int64_t a[2][3];
} gen_t;

static gen_t unpack(const int64_t *p)
{
    gen_t g;
    g.m[0] = (uint64_t)p[0];
    g.m[1] = (uint64_t)p[1];
    for (int j = 0; j < 3; ++j) {
        g.a[0][j] = p[2 + j];
        g.a[1][j] = p[5 + j];
    }
    return g;
}

/* v mod m in [0, m) for any signed 128-bit v. */
static uint64_t mod_signed(i128 v, uint64_t m)
{
    i128 r = v % (i128)m;
    if (r < 0)
        r += (i128)m;
    return (uint64_t)r;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)m);
}

/* ---------------------------------------------------------------------- */
/* The recurrence (Sec. 2; MRG32k3a constants from L'Ecuyer 1999, the      */
/* generator of RngStreams cited in Sec. 1).                                */
/* ---------------------------------------------------------------------- */

/* One step of component c on x = (x[n-1], x[n-2], x[n-3]); returns x[n]. */
static uint64_t comp_step(const gen_t *g, int c, uint64_t x[3])
{
    i128 acc = 0;
    for (int j = 0; j < 3; ++j)
        acc += (i128)g->a[c][j] * (i128)x[j];
    uint64_t xn = mod_signed(acc, g->m[c]);
    x[2] = x[1];
    x[1] = x[0];
    x[0] = xn;
    return xn;
}

/* One step of the combined generator: the output integer z in [1, m1]
 * (difference of the components mod m1, with 0 mapped to m1). */
static uint64_t gen_step(const gen_t *g, uint64_t s[6])
{
    uint64_t p1 = comp_step(g, 0, s);
    uint64_t p2 = comp_step(g, 1, s + 3);
    uint64_t z = mod_signed((i128)p1 - (i128)p2, g->m[0]);
    return z == 0 ? g->m[0] : z;
}

static void load_state(const uint32_t *st, uint64_t s[6])
{
    for (int k = 0; k < 6; ++k)
        s[k] = st[k];
}

static void store_state(const uint64_t s[6], uint32_t *st)
{
    for (int k = 0; k < 6; ++k)
        st[k] = (uint32_t)s[k];
}

/* ---------------------------------------------------------------------- */
/* Jump-ahead (Sec. 2.1): the companion matrix maps (x[n-1],x[n-2],x[n-3]) */
/* to (x[n],x[n-1],x[n-2]); k steps are its k-th power.                     */
/* ---------------------------------------------------------------------- */

static void companion(const gen_t *g, int c, uint64_t A[9])
{
    for (int j = 0; j < 3; ++j)
        A[j] = mod_signed((i128)g->a[c][j], g->m[c]);
    A[3] = 1; A[4] = 0; A[5] = 0;
    A[6] = 0; A[7] = 1; A[8] = 0;
}

static void matmul(const uint64_t X[9], const uint64_t Y[9], uint64_t m, uint64_t out[9])
{
    uint64_t t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            uint64_t acc = 0;
            for (int k = 0; k < 3; ++k)
                acc = (acc + mulmod(X[3 * r + k], Y[3 * k + c], m)) % m;
            t[3 * r + c] = acc;
        }
    memcpy(out, t, sizeof t);
}

static void matpow(const gen_t *g, int c, u128 e, uint64_t out[9])
{
    uint64_t base[9], res[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    companion(g, c, base);
    while (e) {
        if (e & 1)
            matmul(res, base, g->m[c], res);
        matmul(base, base, g->m[c], base);
        e >>= 1;
    }
    memcpy(out, res, sizeof res);
}

static void matvec(const uint64_t A[9], uint64_t x[3], uint64_t m)
{
    uint64_t y[3];
    for (int r = 0; r < 3; ++r) {
        uint64_t acc = 0;
        for (int k = 0; k < 3; ++k)
            acc = (acc + mulmod(A[3 * r + k], x[k], m)) % m;
        y[r] = acc;
    }
    memcpy(x, y, sizeof y);
}

/* A_c^(2^k): k successive squarings of the companion matrix (the stream
 * spacing 2^134 of MRG31k3p does not fit a 128-bit exponent). */
static void matpow2k(const gen_t *g, int c, unsigned k, uint64_t out[9])
{
    companion(g, c, out);
    for (unsigned i = 0; i < k; ++i)
        matmul(out, out, g->m[c], out);
}

void orc_matpow2k(const int64_t *p, int c, unsigned k, uint64_t out[9])
{
    gen_t g = unpack(p);
    matpow2k(&g, c, k, out);
}

/* out = A_c^e mod m_c, e = e_hi * 2^64 + e_lo. */
void orc_matpow(const int64_t *p, int c, uint64_t e_lo, uint64_t e_hi, uint64_t out[9])
{
    gen_t g = unpack(p);
    matpow(&g, c, ((u128)e_hi << 64) | e_lo, out);
}

/* st <- A^e st on both components: the state e steps later. */
void orc_jump(const int64_t *p, uint32_t st[6], uint64_t e_lo, uint64_t e_hi)
{
    gen_t g = unpack(p);
    u128 e = ((u128)e_hi << 64) | e_lo;
    uint64_t s[6], A[9];
    load_state(st, s);
    for (int c = 0; c < 2; ++c) {
        matpow(&g, c, e, A);
        matvec(A, s + 3 * c, g.m[c]);
    }
    store_state(s, st);
}

/* Streams are created one after another; each new stream starts Z = 2^zlog2
 * steps after the previous one (Sec. 2.1).  states: n x 6 (row = stream).
 * next_seed receives the creator state after the n-th stream. */
void orc_create_streams(const int64_t *p, const uint32_t seed[6], uint64_t n,
                        unsigned zlog2, uint32_t *states, uint32_t next_seed[6])
{
    gen_t g = unpack(p);
    uint64_t J[2][9], s[6];
    for (int c = 0; c < 2; ++c)
        matpow2k(&g, c, zlog2, J[c]);
    load_state(seed, s);
    for (uint64_t i = 0; i < n; ++i) {
        store_state(s, states + 6 * i);
        for (int c = 0; c < 2; ++c)
            matvec(J[c], s + 3 * c, g.m[c]);
    }
    store_state(s, next_seed);
}

/* ---------------------------------------------------------------------- */
/* Output transforms                                                       */
/* ---------------------------------------------------------------------- */

/* ln(z / M), M = m1 + 1, for z in [1, m1].  Above 1/2 the exact integer
 * complement M - z feeds log1p so that values near u = 1 keep their
 * relative accuracy. */
static double log_uniform(uint64_t z, uint64_t m1)
{
    uint64_t M = m1 + 1;
    if (2 * z > M)
        return log1p(-((double)(M - z) / (double)M));
    return log((double)z / (double)M);
}

/* sin and cos of 2*pi*z/M computed after an exact integer reduction:
 * 4z = q*M + r, angle = (pi/2) q + phi, phi = (pi/2) r / M in [0, pi/2);
 * phi above pi/4 is reflected (sin phi = cos(pi/2 - phi)). */
static void sincos_turn(uint64_t z, uint64_t m1, double *s, double *c)
{
    uint64_t M = m1 + 1;
    uint64_t q = (4 * z) / M, r = (4 * z) % M;
    double sp, cp;
    if (2 * r <= M) {
        double phi = (M_PI / 2) * ((double)r / (double)M);
        sp = sin(phi);
        cp = cos(phi);
    } else {
        double psi = (M_PI / 2) * ((double)(M - r) / (double)M);
        sp = cos(psi);
        cp = sin(psi);
    }
    switch (q & 3) {
    case 0: *s = sp;  *c = cp;  break;
    case 1: *s = cp;  *c = -sp; break;
    case 2: *s = -sp; *c = -cp; break;
    default: *s = -cp; *c = sp; break;
    }
}

/* Box-Muller (Sec. 3.1, Algorithm 1) on the pair (u1, u2) = (z1/M, z2/M):
 * R = sqrt(-2 ln u1), Theta = 2 pi u2, X = R cos Theta, Y = R sin Theta. */
static void box_muller(uint64_t z1, uint64_t z2, uint64_t m1, double *x, double *y)
{
    double R = sqrt(-2.0 * log_uniform(z1, m1));
    double s, c;
    sincos_turn(z2, m1, &s, &c);
    *x = R * c;
    *y = R * s;
}

/* The transforms applied to given output integers (pairs for Box-Muller). */
void orc_box_muller_pairs(const int64_t *p, const uint32_t *z, uint64_t npairs, double *out)
{
    for (uint64_t k = 0; k < npairs; ++k)
        box_muller(z[2 * k], z[2 * k + 1], (uint64_t)p[0], &out[2 * k], &out[2 * k + 1]);
}

void orc_exp_of(const int64_t *p, const uint32_t *z, uint64_t n, double rate, double *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = -log_uniform(z[i], (uint64_t)p[0]) / rate;
}

/* ---------------------------------------------------------------------- */
/* Single-stream generation.  st (6 words) is advanced in place.            */
/* ---------------------------------------------------------------------- */

void orc_raw(const int64_t *p, uint32_t st[6], uint64_t n, uint32_t *out)
{
    gen_t g = unpack(p);
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (uint32_t)gen_step(&g, s);
    store_state(s, st);
}

double orc_norm(const int64_t *p)
{
    return 1.0 / (double)((uint64_t)p[0] + 1);
}

void orc_uniform64(const int64_t *p, uint32_t st[6], uint64_t n, double *out)
{
    gen_t g = unpack(p);
    double norm = orc_norm(p);
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (double)gen_step(&g, s) * norm;
    store_state(s, st);
}

/* fp32 uniform = the fp64 uniform rounded to float (Listing 1 computes the
 * product in double and stores it into a float array). */
void orc_uniform32(const int64_t *p, uint32_t st[6], uint64_t n, float *out)
{
    gen_t g = unpack(p);
    double norm = orc_norm(p);
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (float)((double)gen_step(&g, s) * norm);
    store_state(s, st);
}

/* n standard normals from consecutive pairs of one stream: draws (2k, 2k+1)
 * give out[2k] = X, out[2k+1] = Y.  An odd n discards the last Y, so the
 * stream advances by n + (n mod 2) draws. */
void orc_normal(const int64_t *p, uint32_t st[6], uint64_t n, double *out)
{
    gen_t g = unpack(p);
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t i = 0; i < n; i += 2) {
        uint64_t z1 = gen_step(&g, s);
        uint64_t z2 = gen_step(&g, s);
        double x, y;
        box_muller(z1, z2, g.m[0], &x, &y);
        out[i] = x;
        if (i + 1 < n)
            out[i + 1] = y;
    }
    store_state(s, st);
}

/* Exponential(rate) by inversion (Sec. 3.2): E = -ln(u) / rate. */
void orc_exponential(const int64_t *p, uint32_t st[6], uint64_t n, double rate, double *out)
{
    gen_t g = unpack(p);
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t i = 0; i < n; ++i)
        out[i] = -log_uniform(gen_step(&g, s), g.m[0]) / rate;
    store_state(s, st);
}

/* ---------------------------------------------------------------------- */
/* Many streams: row i of `states` (6 words) is stream i; row i of out     */
/* starts at element i*ld.  dist: 0 raw (u32 out), 1 uniform, 2 normal,     */
/* 3 exponential; f32 selects float output for the uniform, otherwise       */
/* uniforms are double and normals/exponentials are the double reference.  */
/* ---------------------------------------------------------------------- */

void orc_generate_streams(const int64_t *p, uint32_t *states, uint64_t nstreams,
                          uint64_t n, int dist, int f32, double rate,
                          void *out, uint64_t ld, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
    for (uint64_t i = 0; i < nstreams; ++i) {
        uint32_t *st = states + 6 * i;
        switch (dist) {
        case 0:
            orc_raw(p, st, n, (uint32_t *)out + i * ld);
            break;
        case 1:
            if (f32)
                orc_uniform32(p, st, n, (float *)out + i * ld);
            else
                orc_uniform64(p, st, n, (double *)out + i * ld);
            break;
        case 2:
            orc_normal(p, st, n, (double *)out + i * ld);
            break;
        default:
            orc_exponential(p, st, n, rate, (double *)out + i * ld);
            break;
        }
    }
}

/* Fused consumer: per stream, `draws` draws as draws/2 pairs (za, zb).
 * count[i] = number of pairs with (za/M)^2 + (zb/M)^2 < 1, decided exactly
 * in integers as za^2 + zb^2 < M^2; sum[i] = sum over pairs of X + Y, the
 * Box-Muller normals of the same pair, accumulated left to right in double.
 * An odd `draws` is rounded up to whole pairs. */
void orc_fused(const int64_t *p, uint32_t *states, uint64_t nstreams, uint64_t draws,
               int64_t *count, double *sum, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    uint64_t M = (uint64_t)p[0] + 1;
    u128 M2 = (u128)M * M;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
    for (uint64_t i = 0; i < nstreams; ++i) {
        gen_t g = unpack(p);
        uint64_t s[6];
        load_state(states + 6 * i, s);
        int64_t cnt = 0;
        double acc = 0.0;
        for (uint64_t k = 0; k < draws; k += 2) {
            uint64_t za = gen_step(&g, s);
            uint64_t zb = gen_step(&g, s);
            if ((u128)za * za + (u128)zb * zb < M2)
                ++cnt;
            double x, y;
            box_muller(za, zb, g.m[0], &x, &y);
            acc += x;
            acc += y;
        }
        count[i] = cnt;
        sum[i] = acc;
        store_state(s, states + 6 * i);
    }
}

/* ---------------------------------------------------------------------- */
/* Fisher's exact test by Monte Carlo (Sec. 4): statistic, random tables   */
/* with the observed margins, and the count of simulated statistics at or  */
/* below the observed one.                                                  */
/* ---------------------------------------------------------------------- */

/* lf[k] = log(k!) for k = 0..n, from lgamma. */
void orc_logfact_table(uint64_t n, double *lf)
{
    for (uint64_t k = 0; k <= n; ++k)
        lf[k] = lgamma((double)k + 1.0);
}

/* The test statistic of a table (Sec. 4: "minus log-factorial of table"),
 * -sum_{i,j} log(n_ij!), summed row by row, left to right. */
double orc_logfact_sum(const int32_t *table, uint32_t I, uint32_t J, const double *lf)
{
    double t = 0.0;
    for (uint32_t i = 0; i < I; ++i)
        for (uint32_t j = 0; j < J; ++j)
            t -= lf[table[(size_t)i * J + j]];
    return t;
}

/* Probability that a draw of R items without replacement from a population
 * of S items, K of which are marked, holds exactly x marked items. */
static double hyper_pmf(int64_t S, int64_t K, int64_t R, int64_t x, const double *lf)
{
    double l = lf[K] - lf[x] - lf[K - x] + lf[S - K] - lf[R - x] - lf[S - K - R + x]
               - (lf[S] - lf[R] - lf[S - R]);
    return exp(l);
}

/* Standard inversion of that distribution's CDF with one uniform u: the
 * smallest x of the support with u <= F(x), F accumulated from the bottom
 * of the support (the largest x if rounding leaves F below u). */
int64_t orc_hyper_inv(int64_t S, int64_t K, int64_t R, double u, const double *lf)
{
    int64_t lo = R - (S - K) > 0 ? R - (S - K) : 0;
    int64_t hi = R < K ? R : K;
    double F = 0.0;
    for (int64_t x = lo; x < hi; ++x) {
        F += hyper_pmf(S, K, R, x, lf);
        if (u <= F)
            return x;
    }
    return hi;
}

/* One random table with row sums r[I] and column sums c[J] (Sec. 4 step 2,
 * Patefield's method as the paper describes it): entries sampled row by row,
 * left to right, each from its distribution conditional on the entries
 * already sampled -- the cell (i, j) holds x of the R units still to place
 * in row i among the S units left in columns j..J-1 of rows i..I-1, of which
 * C_j are in column j -- by inversion with one uniform; the last entry of a
 * row and the whole last row follow from the margins.  (I-1)(J-1) uniforms
 * per table.  Returns the table's statistic; `st` advances by those draws. */
static double fisher_table(const gen_t *g, uint64_t s[6], const int32_t *r, const int32_t *c,
                           uint32_t I, uint32_t J, const double *lf, int32_t *cell)
{
    double norm = 1.0 / (double)(g->m[0] + 1);
    int64_t C[64];
    int64_t rest = 0;
    for (uint32_t j = 0; j < J; ++j) {
        C[j] = c[j];
        rest += c[j];
    }
    for (uint32_t i = 0; i + 1 < I; ++i) {
        int64_t R = r[i];
        int64_t S = rest;
        for (uint32_t j = 0; j + 1 < J; ++j) {
            double u = (double)gen_step(g, s) * norm;
            int64_t x = orc_hyper_inv(S, C[j], R, u, lf);
            cell[(size_t)i * J + j] = (int32_t)x;
            S -= C[j];
            C[j] -= x;
            R -= x;
        }
        cell[(size_t)i * J + J - 1] = (int32_t)R;
        C[J - 1] -= R;
        rest -= r[i];
    }
    for (uint32_t j = 0; j < J; ++j)
        cell[(size_t)(I - 1) * J + j] = (int32_t)C[j];
    return orc_logfact_sum(cell, I, J, lf);
}

/* B replicates on nstreams streams: replicate b uses stream b mod nstreams,
 * taking that stream's next (I-1)(J-1) uniforms (replicates of one stream in
 * increasing b).  stats[b] (may be NULL) receives each statistic; the return
 * value is the number of replicates with statistic <= threshold (Sec. 4
 * step 3).  states advance in place.  2 <= I, J <= 64. */
uint64_t orc_fisher(const int64_t *p, uint32_t *states, uint64_t nstreams, const int32_t *table,
                    uint32_t I, uint32_t J, uint64_t B, double threshold, const double *lf,
                    double *stats, int nthreads)
{
    int32_t r[64], c[64];
    for (uint32_t i = 0; i < I; ++i) {
        r[i] = 0;
        for (uint32_t j = 0; j < J; ++j)
            r[i] += table[(size_t)i * J + j];
    }
    for (uint32_t j = 0; j < J; ++j) {
        c[j] = 0;
        for (uint32_t i = 0; i < I; ++i)
            c[j] += table[(size_t)i * J + j];
    }
    if (nthreads < 1)
        nthreads = 1;
    uint64_t count = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16) reduction(+ : count)
    for (uint64_t sidx = 0; sidx < nstreams; ++sidx) {
        gen_t g = unpack(p);
        uint64_t s[6];
        int32_t cell[64 * 64];
        load_state(states + 6 * sidx, s);
        for (uint64_t b = sidx; b < B; b += nstreams) {
            double t = fisher_table(&g, s, r, c, I, J, lf, cell);
            if (stats)
                stats[b] = t;
            if (t <= threshold)
                ++count;
        }
        store_state(s, states + 6 * sidx);
    }
    return count;
}

/* B random tables from one stream (state advanced in place): tables
 * [B][I][J] receives the cells, the return value is unused (0). */
int orc_fisher_tables(const int64_t *p, uint32_t st[6], const int32_t *table, uint32_t I,
                      uint32_t J, uint64_t B, const double *lf, int32_t *tables)
{
    gen_t g = unpack(p);
    int32_t r[64], c[64];
    for (uint32_t i = 0; i < I; ++i) {
        r[i] = 0;
        for (uint32_t j = 0; j < J; ++j)
            r[i] += table[(size_t)i * J + j];
    }
    for (uint32_t j = 0; j < J; ++j) {
        c[j] = 0;
        for (uint32_t i = 0; i < I; ++i)
            c[j] += table[(size_t)i * J + j];
    }
    uint64_t s[6];
    load_state(st, s);
    for (uint64_t b = 0; b < B; ++b)
        fisher_table(&g, s, r, c, I, J, lf, tables + b * (size_t)I * J);
    store_state(s, st);
    return 0;
}
