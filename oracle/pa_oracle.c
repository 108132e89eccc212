/*
 * pa_oracle.c -- plain, slow, single-thread CPU population annealing (PA).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this code; the library's product path
 * never does.  It shares no source, header, table or helper with the CUDA
 * path: every definition below is written out again from the method.
 *
 * One int8 per spin (sigma = +-1), one site at a time, the paper's step order
 * (Sec. 2, steps 1-5):
 *   step 1  R iid uniform configurations at beta_0 = 0 (exact sampling),
 *   step 2  resample from beta_{i-1} to beta_i with tau_j = exp(-dbeta E_j)/Q_i
 *           and Q_i of Eq. (Q); copies by one of five count rules (Sec. 3),
 *   step 3  theta_i checkerboard Metropolis sweeps at beta_i,
 *   step 4  population averages,
 *   step 5  loop.
 * The free energy follows Eq. (free-energy-estimator):
 *   -beta_i F_i = ln Z_0 + sum_k ln Q_k,   ln Z_0 = N ln 2.
 *
 * Discretisation (the paper leaves these open; both this oracle and the CUDA
 * path implement the same reading so that all integer state matches bit for
 * bit):
 *   - RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = 64-bit
 *     seed, counter = (c0, c1, c2, c3) with the domain in the top bits of c1.
 *   - Metropolis accepts a move with dE > 0 iff u < thr[dE/4], u a uint32
 *     uniform and thr[k] = floor(2^32 exp(-4 k beta)) (clamped to 2^32-1);
 *     the bits of u are bit planes shared by 32 consecutive replica slots.
 *   - The Boltzmann factors are evaluated per energy level,
 *     w_k = q^k with q = exp(-4 dbeta) by binary powering, summed in a fixed
 *     pairwise tree, and turned into 2^-40 fixed-point expected copy numbers
 *     f_k = floor(2^40 R w_k / S) (Eq. taus: tau-hat = (R/R_{i-1}) tau).
 *   - Copy counts are exact integer functions of f and the RNG draws.
 *
 * Every floating-point operation here is a single IEEE-754 double operation;
 * build with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of the 4x32 Philox S-box,  */
/* multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /   */
/* 0xBB67AE85 applied between rounds.                                       */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0, p1;
        uint32_t y0, y1, y2, y3;
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        y1 = (uint32_t)p1;
        y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                  uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = c0; ctr[1] = c1; ctr[2] = c2; ctr[3] = c3;
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox(ctr, key, out);
}

/* counter domains (top nibble of c1) */
#define DOM_SWEEP    0x00000000u
#define DOM_INIT     0x10000000u
#define DOM_RESAMPLE 0x20000000u
#define DOM_DISORDER 0x30000000u

#define SUB_NEAREST     0u
#define SUB_SYSTEMATIC  1u
#define SUB_MULTINOMIAL 2u
#define SUB_RESIDUAL    3u
#define SUB_POISSON     4u

/* resampler ids */
#define OR_MULTINOMIAL 0
#define OR_SYSTEMATIC  1
#define OR_RESIDUAL    2
#define OR_POISSON     3
#define OR_NEAREST     4

/* status */
#define OR_OK          0
#define OR_ERR_ARG     1
#define OR_ERR_CAP     4
#define OR_ERR_KMAX    5

#define FRAC_BITS 40
#define POISSON_KMAX 256

/* ------------------------------------------------------------------------ */
/* exp from its Taylor series after Cody-Waite reduction by ln 2:            */
/*   x = n ln2 + r, |r| <= ln2/2, exp(x) = 2^n sum_{k<=13} r^k/k!            */
/* (truncation error r^14/14! < 5e-18 relative).  Used only by the Poisson  */
/* count rule, on x in [-16, 0].                                            */
/* ------------------------------------------------------------------------ */
static const double INV_LN2 = 0x1.71547652b82fep+0;
static const double LN2_HI  = 0x1.62e42fefa3800p-1;  /* ln 2 to 42 bits     */
static const double LN2_LO  = 0x1.ef35793c76730p-45; /* ln 2 - LN2_HI       */
static const double INV_FACT[14] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1,
    0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
    0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
    0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};

double or_exp(double x)
{
    double z = x * INV_LN2;
    double nd = floor(z + 0.5);
    double r = (x - nd * LN2_HI) - nd * LN2_LO;
    double p = INV_FACT[13];
    int k;
    for (k = 12; k >= 0; --k)
        p = p * r + INV_FACT[k];
    return ldexp(p, (int)nd);
}

/* ------------------------------------------------------------------------ */
/* Lattice: periodic L^d, site s = x + L y (+ L^2 z), bonds (s, s + e_a).   */
/* ------------------------------------------------------------------------ */
static int nb_site(int d, int L, int s, int a, int dir)
{
    int stride = 1, c, i;
    for (i = 0; i < a; ++i) stride *= L;
    c = (s / stride) % L;
    if (dir > 0)
        return (c == L - 1) ? s - (L - 1) * stride : s + stride;
    return (c == 0) ? s + (L - 1) * stride : s - stride;
    (void)d;
}

static int site_colour(int d, int L, int s)
{
    int sum = 0, a;
    for (a = 0; a < d; ++a) {
        sum += s % L;
        s /= L;
    }
    return sum & 1;
}

static int npow(int L, int d)
{
    int n = 1, i;
    for (i = 0; i < d; ++i) n *= L;
    return n;
}

/* Hamiltonian H = -sum_<ij> J_ij s_i s_j (Eq. Hamiltonian), J[a*N + s] for
 * the bond between s and s + e_a. */
int32_t or_energy(int d, int L, const int8_t *J, const int8_t *sig)
{
    int N = npow(L, d), s, a;
    int32_t E = 0;
    for (s = 0; s < N; ++s)
        for (a = 0; a < d; ++a)
            E -= (int32_t)J[a * N + s] * sig[s] * sig[nb_site(d, L, s, a, +1)];
    return E;
}

int32_t or_magnetisation(int N, const int8_t *sig)
{
    int32_t m = 0;
    int s;
    for (s = 0; s < N; ++s) m += sig[s];
    return m;
}

/* EA +-J couplings, p = 1/2: bond b = a*N + s takes bit (b & 31) of lane
 * (b >> 5) & 3 of the DISORDER draw with c0 = b >> 7; bit 1 means J = -1. */
void or_disorder(int d, int L, uint64_t disorder_seed, uint32_t realization, int8_t *J)
{
    int N = npow(L, d), b;
    uint32_t x[4];
    for (b = 0; b < d * N; ++b) {
        draw4(disorder_seed, (uint32_t)(b >> 7), DOM_DISORDER, 0u, realization, x);
        J[b] = ((x[(b >> 5) & 3] >> (b & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

/* Step 1: exact sampling at beta_0 = 0.  Site s of replica j takes bit
 * (s & 31) of word s >> 5, word w being lane (w & 3) of the INIT draw with
 * c0 = w >> 2, c3 = j.  Bit 1 means sigma = -1. */
void or_init_replica(int d, int L, uint64_t seed, uint32_t j, int8_t *sig)
{
    int N = npow(L, d), s;
    uint32_t x[4];
    for (s = 0; s < N; ++s) {
        int w = s >> 5;
        draw4(seed, (uint32_t)(w >> 2), DOM_INIT, 0u, j, x);
        sig[s] = ((x[w & 3] >> (s & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

/* Metropolis thresholds thr[k] = floor(2^32 exp(-4 k beta)), k = 1..3,
 * clamped to 2^32 - 1; thr[0] is unused (moves with dE <= 0 always pass). */
void or_thresholds(double beta, uint32_t thr[4])
{
    int k;
    thr[0] = 0xFFFFFFFFu;
    for (k = 1; k < 4; ++k) {
        double x = beta * (double)(4 * k);
        double t = ldexp(exp(-x), 32);
        thr[k] = (t >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)floor(t);
    }
}

/* The uint32 uniform u of the Metropolis test of the replica in slot `slot`
 * at site s (round t, colour c, temperature step `step`) is made of 32 bit
 * planes: its bit 31 - p is bit (slot & 31) of plane word p, and plane word
 * p is lane p & 3 of the SWEEP draw with counter
 *   c0 = slot >> 5, c1 = (t << 4) | (c << 3) | (p >> 2), c2 = step, c3 = s.
 * u < thr is decided by comparing u and thr four bits (one draw) at a time
 * from the most significant end, which is the ordinary comparison of two
 * numbers digit by digit in base 16; equal numbers are not "less". */
int or_u_less(uint64_t seed, uint32_t slot, uint32_t step, uint32_t t, int c, int s,
              uint32_t thr)
{
    uint32_t g, x[4], r = slot & 31u;
    for (g = 0; g < 8; ++g) {
        uint32_t du, dt;
        draw4(seed, slot >> 5, DOM_SWEEP | (t << 4) | ((uint32_t)c << 3) | g, step, (uint32_t)s, x);
        du = (((x[0] >> r) & 1u) << 3) | (((x[1] >> r) & 1u) << 2) |
             (((x[2] >> r) & 1u) << 1) | ((x[3] >> r) & 1u);
        dt = (thr >> (28 - 4 * g)) & 15u;
        if (du != dt) return du < dt;
    }
    return 0;
}

/* Step 3: theta rounds of single-replica updates of the replica in slot
 * `slot` at temperature step `step`.  One round = all colour-0 sites in
 * ascending order, then all colour-1 sites.  A site flips if dE <= 0, else
 * iff u < thr[dE/4] with u the uniform above.
 * Returns the number of accepted flips; updates *E by the energy changes. */
uint64_t or_sweeps(int d, int L, const int8_t *J, int8_t *sig, int32_t *E,
                   uint64_t seed, uint32_t step, uint32_t slot, uint32_t theta,
                   const uint32_t thr[4])
{
    int N = npow(L, d);
    uint64_t acc = 0;
    uint32_t t;
    int c, s, a;
    for (t = 0; t < theta; ++t) {
        for (c = 0; c < 2; ++c) {
            for (s = 0; s < N; ++s) {
                int h = 0, dE, flip;
                if (site_colour(d, L, s) != c) continue;
                for (a = 0; a < d; ++a) {
                    h += J[a * N + s] * sig[nb_site(d, L, s, a, +1)];
                    h += J[a * N + nb_site(d, L, s, a, -1)] * sig[nb_site(d, L, s, a, -1)];
                }
                dE = 2 * sig[s] * h;
                if (dE <= 0) flip = 1;
                else flip = or_u_less(seed, slot, step, t, c, s, thr[dE / 4]);
                if (flip) {
                    sig[s] = (int8_t)-sig[s];
                    *E += dE;
                    ++acc;
                }
            }
        }
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Step 2: weights, Q (Eq. Q) and the copy counts.                          */
/* ------------------------------------------------------------------------ */

/* q^k by binary powering: multiply in q^(2^m) for every set bit m of k,
 * least significant first. */
static double pow_bin(double q, uint32_t k)
{
    double r = 1.0, b = q;
    while (k) {
        if (k & 1u) r = r * b;
        b = b * b;
        k >>= 1;
    }
    return r;
}

/* 128-bit helpers (gcc __int128) */
typedef unsigned __int128 u128;

/* N(x) of systematic resampling: number of labels (k + u/2^32) T / R, k in
 * [0, R), that lie below x. */
static uint64_t sys_below(uint64_t x, uint64_t R, uint64_t T, uint32_t u)
{
    u128 P = (u128)x * R;
    uint64_t a = (uint64_t)(P / T);
    uint64_t b = (uint64_t)(P % T);
    uint64_t n = a + (((u128)b << 32) > (u128)u * T ? 1u : 0u);
    return n < R ? n : R;
}

/* index j with C[j-1] <= p < C[j] (C inclusive prefix sums, C[-1] = 0) */
static uint32_t find_box(const uint64_t *C, uint32_t n, uint64_t p)
{
    uint32_t j;
    for (j = 0; j < n; ++j)
        if (p < C[j]) return j;
    return n; /* not reached for p < C[n-1] */
}

/*
 * Copy counts of the parents j < Rprev from their fixed-point expected copy
 * numbers f_rep (tau-hat in 2^-40 units), by the chosen rule (Sec. 3).
 * run_id enters the resampling draws' counter.  Returns a status code.
 */
static int counts_from_f(const uint64_t *f_rep, uint32_t Rprev, uint32_t R, int method,
                         uint64_t seed, uint32_t step, uint32_t run_id, uint32_t *counts,
                         uint64_t *Rnew)
{
    const uint32_t dom = DOM_RESAMPLE | (run_id << 8);
    uint32_t j;
    uint64_t *C = (uint64_t *)calloc(Rprev, sizeof(uint64_t)), T = 0, total = 0;
    uint32_t x[4];
    int status = OR_OK;
    for (j = 0; j < Rprev; ++j) {
        T += f_rep[j];
        C[j] = T;
        counts[j] = 0;
    }

    if (method == OR_NEAREST) {
        /* floor(tau) copies plus one more with probability tau - floor(tau) */
        for (j = 0; j < Rprev; ++j) {
            uint64_t u40, frac;
            draw4(seed, j, dom | SUB_NEAREST, step, 0u, x);
            u40 = (((uint64_t)x[1] << 32) | x[0]) >> 24;
            frac = f_rep[j] & ((1ull << FRAC_BITS) - 1);
            counts[j] = (uint32_t)(f_rep[j] >> FRAC_BITS) + (u40 < frac ? 1u : 0u);
        }
    } else if (method == OR_SYSTEMATIC) {
        /* one uniform U in [0,1); labels at (k + U) T/R on the cumulative
         * weight axis; replica j takes the labels in [C_{j-1}, C_j). */
        uint64_t prev = 0, below_prev = 0;
        draw4(seed, 0u, dom | SUB_SYSTEMATIC, step, 0u, x);
        for (j = 0; j < Rprev; ++j) {
            uint64_t below = sys_below(C[j], R, T, x[0]);
            counts[j] = (uint32_t)(below - below_prev);
            below_prev = below;
            prev = C[j];
        }
        (void)prev;
    } else if (method == OR_MULTINOMIAL) {
        /* R labels iid uniform on [0, T); replica j takes those in its box */
        uint32_t kk;
        for (kk = 0; kk < R; ++kk) {
            uint64_t u64, p;
            draw4(seed, kk >> 1, dom | SUB_MULTINOMIAL, step, 0u, x);
            u64 = (kk & 1u) ? (((uint64_t)x[3] << 32) | x[2]) : (((uint64_t)x[1] << 32) | x[0]);
            p = (uint64_t)(((u128)u64 * T) >> 64);
            counts[find_box(C, Rprev, p)] += 1;
        }
    } else if (method == OR_RESIDUAL) {
        /* floor(tau) deterministic copies, the R_res remaining ones drawn
         * multinomially with probabilities proportional to the remainders. */
        uint64_t A = 0, Tres = 0, Rres;
        uint64_t *G = (uint64_t *)calloc(Rprev, sizeof(uint64_t));
        const uint64_t *box;
        uint64_t boxT;
        uint32_t kk;
        for (j = 0; j < Rprev; ++j) {
            counts[j] = (uint32_t)(f_rep[j] >> FRAC_BITS);
            A += counts[j];
            Tres += f_rep[j] & ((1ull << FRAC_BITS) - 1);
            G[j] = Tres;
        }
        Rres = (uint64_t)R - A;
        box = (Tres > 0) ? G : C;
        boxT = (Tres > 0) ? Tres : T;
        for (kk = 0; kk < (uint32_t)Rres; ++kk) {
            uint64_t u64, p;
            draw4(seed, kk >> 1, dom | SUB_RESIDUAL, step, 0u, x);
            u64 = (kk & 1u) ? (((uint64_t)x[3] << 32) | x[2]) : (((uint64_t)x[1] << 32) | x[0]);
            p = (uint64_t)(((u128)u64 * boxT) >> 64);
            counts[find_box(box, Rprev, p)] += 1;
        }
        free(G);
    } else if (method == OR_POISSON) {
        /* r_j ~ Poisson(tau-hat_j), as the sum of M_j = floor(f_j/2^44) + 1
         * Poisson draws of mean tau-hat_j / M_j (each <= 16), each by
         * sequential inversion of the Poisson CDF. */
        for (j = 0; j < Rprev; ++j) {
            double lam = ldexp((double)f_rep[j], -FRAC_BITS);
            uint32_t M = (uint32_t)(f_rep[j] >> 44) + 1u, m;
            double lc = lam / (double)M;
            uint32_t total_k = 0;
            for (m = 0; m < M; ++m) {
                double u, p, Pc;
                uint32_t kp = 0;
                draw4(seed, j, dom | SUB_POISSON, step, m, x);
                u = ldexp((double)((((uint64_t)x[1] << 32) | x[0]) >> 11), -53);
                p = or_exp(-lc);
                Pc = p;
                while (u >= Pc) {
                    kp += 1;
                    if (kp > POISSON_KMAX) { status = OR_ERR_KMAX; break; }
                    p = (p * lc) / (double)kp;
                    Pc = Pc + p;
                }
                total_k += kp;
            }
            counts[j] = total_k;
        }
    } else {
        status = OR_ERR_ARG;
    }
    for (j = 0; j < Rprev; ++j) total += counts[j];
    *Rnew = total;
    free(C);
    return status;
}

/*
 * Resampling from beta_{i-1} to beta_i = beta_{i-1} + dbeta.  run_id enters
 * the resampling draws' counter (c1 = 2 << 28 | run_id << 8 | rule), so that
 * runs advanced together draw independent numbers; a lone run has run_id 0.
 * Inputs: E[0..Rprev) (energies at beta_{i-1}), nominal size R, method.
 * Outputs: counts[0..Rprev), f_rep[0..Rprev) (2^-40 fixed-point tau-hat),
 * *lnQ, *Rnew.  Returns a status code.
 */
int or_resample(const int32_t *E, uint32_t Rprev, uint32_t R, double dbeta,
                int method, uint64_t seed, uint32_t step, uint32_t run_id,
                uint32_t *counts, uint64_t *f_rep, double *lnQ, uint64_t *Rnew)
{
    int32_t Emin = E[0], Emax = E[0];
    uint32_t j, K, P, k, h;
    uint64_t *nlev, *flev;
    double *t, S, q;
    int status;

    for (j = 1; j < Rprev; ++j) {
        if (E[j] < Emin) Emin = E[j];
        if (E[j] > Emax) Emax = E[j];
    }
    K = (uint32_t)((Emax - Emin) / 4) + 1;
    P = 1;
    while (P < K) P <<= 1;
    nlev = (uint64_t *)calloc(K, sizeof(uint64_t));
    flev = (uint64_t *)calloc(K, sizeof(uint64_t));
    t = (double *)calloc(P, sizeof(double));
    for (j = 0; j < Rprev; ++j) nlev[(E[j] - Emin) / 4] += 1;

    /* Boltzmann factor relative to the lowest energy: exp(-dbeta (E - Emin))
     * = q^k for E = Emin + 4k. */
    q = exp(-(4.0 * dbeta));
    for (k = 0; k < K; ++k) t[k] = (double)nlev[k] * pow_bin(q, k);
    /* S = sum_k n_k w_k in a fixed pairwise tree: t[k] += t[k + h] for
     * h = P/2, P/4, ..., 1. */
    for (h = P >> 1; h >= 1; h >>= 1)
        for (k = 0; k < h; ++k) t[k] = t[k] + t[k + h];
    S = t[0];
    /* ln Q = ln( (1/R_{i-1}) sum_j exp(-dbeta E_j) ) */
    *lnQ = (log(S) - log((double)Rprev)) - dbeta * (double)Emin;
    /* tau-hat_k = R w_k / S in 2^-40 fixed point */
    for (k = 0; k < K; ++k) {
        double a = (double)R * pow_bin(q, k);
        a = a / S;
        a = ldexp(a, FRAC_BITS);
        flev[k] = (uint64_t)floor(a);
    }
    for (j = 0; j < Rprev; ++j) f_rep[j] = flev[(E[j] - Emin) / 4];
    status = counts_from_f(f_rep, Rprev, R, method, seed, step, run_id, counts, Rnew);
    free(nlev); free(flev); free(t);
    return status;
}

/* ------------------------------------------------------------------------ */
/* A whole run                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t R_i;
    double lnQ, sum_lnQ;
    int64_t sumE, sumE2, sumAbsM, sumM2, sumC2;
    double entropy, sv;
    uint64_t accepts;
    /* partial resampling: effective size of the reweighted population, whether
     * the step resampled, and the weighted sums sum_j w_j O_j */
    double ess;
    int32_t resampled;
    double wsum, wE, wE2, wAM, wM2;
} or_obs;

typedef struct {
    int d, L, N;
    int8_t *J;
    uint32_t R, Rcap;
    int n_steps;
    double *beta;
    uint32_t *theta;
    int method;
    uint64_t seed;
    uint32_t slot_base;   /* 32 x the replica groups of the runs before this one */
    uint32_t run_id;
    int step;
    uint32_t Rcur, Rprev;
    int8_t *sig, *sig2;
    int32_t *E, *E2;
    uint32_t *fam, *fam2;
    uint32_t *counts;  /* of the last resampling, over the R_prev parents */
    uint64_t *f_rep;
    uint32_t *anc;
    double sum_lnQ;
    or_obs obs;
    int status;
    /* partial resampling (alpha >= 0): per-replica weights w (double-buffered
     * with the population); alpha < 0 resamples at every step */
    double alpha;
    double *w, *w2, *wn;
    double ess;
    int32_t resampled;
} or_run;

/* Sum of v[0..n) as the balanced binary tree over P = 2^ceil(log2 n) slots
 * (slots past n hold 0): adjacent pairs are added, then adjacent pairs of
 * those sums, and so on. */
static double tree_sum(const double *v, uint32_t n)
{
    uint32_t P = 1, k, w;
    double *t, s;
    while (P < n) P <<= 1;
    t = (double *)calloc(P, sizeof(double));
    for (k = 0; k < n; ++k) t[k] = v[k];
    for (w = 1; w < P; w <<= 1)
        for (k = 0; k + w < P; k += 2 * w) t[k] = t[k] + t[k + w];
    s = t[0];
    free(t);
    return s;
}

static void measure(or_run *r, const uint32_t *counts, const uint64_t *f_rep, uint32_t Rprev,
                    double lnQ, uint64_t acc)
{
    uint32_t j;
    int N = r->N;
    uint64_t *fc = (uint64_t *)calloc(r->Rcap > r->R ? r->Rcap : r->R, sizeof(uint64_t));
    or_obs o;
    memset(&o, 0, sizeof(o));
    o.R_i = r->Rcur;
    o.lnQ = lnQ;
    o.sum_lnQ = r->sum_lnQ;
    for (j = 0; j < r->Rcur; ++j) {
        int64_t E = r->E[j];
        int64_t M = or_magnetisation(N, r->sig + (size_t)j * N);
        o.sumE += E;
        o.sumE2 += E * E;
        o.sumAbsM += M < 0 ? -M : M;
        o.sumM2 += M * M;
        fc[r->fam[j]] += 1;
    }
    /* family statistics: rho_t = R sum_k n_k^2 with n_k = c_k / R_i, read
     * with R_i in place of R, i.e. sum_k c_k^2 / R_i; entropy of {n_k}. */
    for (j = 0; j < r->R; ++j) {
        if (fc[j]) {
            double nk = (double)fc[j] / (double)r->Rcur;
            o.sumC2 += (int64_t)(fc[j] * fc[j]);
            o.entropy -= nk * log(nk);
        }
    }
    /* sampling variance, Eq. (sv), over the parents of the last resampling */
    if (counts && Rprev) {
        double s = 0.0;
        for (j = 0; j < Rprev; ++j) {
            double dlt = (double)counts[j] - ldexp((double)f_rep[j], -FRAC_BITS);
            s = s + dlt * dlt;
        }
        o.sv = s / (double)Rprev;
    }
    o.accepts = acc;
    /* weighted sums over the population (all weights 1 without partial
     * resampling) */
    {
        uint32_t n = r->Rcur;
        double *v = (double *)calloc(n ? n : 1, sizeof(double));
        const double *w = r->w;
        o.ess = r->ess;
        o.resampled = r->resampled;
        for (j = 0; j < n; ++j) v[j] = w ? w[j] : 1.0;
        o.wsum = tree_sum(v, n);
        for (j = 0; j < n; ++j) v[j] = (w ? w[j] : 1.0) * (double)r->E[j];
        o.wE = tree_sum(v, n);
        for (j = 0; j < n; ++j)
            v[j] = (w ? w[j] : 1.0) * ((double)r->E[j] * (double)r->E[j]);
        o.wE2 = tree_sum(v, n);
        for (j = 0; j < n; ++j) {
            double M = (double)or_magnetisation(N, r->sig + (size_t)j * N);
            v[j] = (w ? w[j] : 1.0) * (M < 0 ? -M : M);
        }
        o.wAM = tree_sum(v, n);
        for (j = 0; j < n; ++j) {
            double M = (double)or_magnetisation(N, r->sig + (size_t)j * N);
            v[j] = (w ? w[j] : 1.0) * (M * M);
        }
        o.wM2 = tree_sum(v, n);
        free(v);
    }
    r->obs = o;
    free(fc);
}

/*
 * Partial resampling (Sec. 3: resampling is needed only once the variance of
 * the importance weights grows too large).  Replicas carry weights w_j; the
 * step to beta_i multiplies them by the incremental weights
 * gamma_j ~ exp(-dbeta (E_j - E_min)) = q^l_j (l_j = (E_j - E_min)/4,
 * binary powering as for the level weights), giving wn_j, and
 *   ln Q_i = ln(sum_j wn_j) - ln(sum_j w_j) - dbeta E_min,
 *   ESS = (sum_j wn_j)^2 / sum_j wn_j^2   (sums: balanced binary trees).
 * If ESS < alpha R_{i-1} the population is resampled with expected copy
 * numbers R wn_j / sum wn (f_j = floor(2^40 R wn_j / S) as in the level
 * form) and all weights restart at 1; otherwise every replica is kept once
 * with its weight, rescaled by the power of two that puts the largest
 * weight in [1/2, 1).
 */
static int partial_weights(or_run *r, uint32_t Rprev, double dbeta, uint32_t step,
                           double *lnQ, uint64_t *Rnew, int *scale_exp)
{
    const int32_t *E = r->E;
    int32_t Emin = E[0];
    uint32_t j;
    double q, S_old, S_new, S2, mx = 0.0;
    double *sq = (double *)malloc(sizeof(double) * Rprev);
    int status = OR_OK;
    for (j = 1; j < Rprev; ++j)
        if (E[j] < Emin) Emin = E[j];
    q = exp(-(4.0 * dbeta));
    for (j = 0; j < Rprev; ++j) {
        r->wn[j] = r->w[j] * pow_bin(q, (uint32_t)((E[j] - Emin) / 4));
        sq[j] = r->wn[j] * r->wn[j];
        if (r->wn[j] > mx) mx = r->wn[j];
    }
    S_old = tree_sum(r->w, Rprev);
    S_new = tree_sum(r->wn, Rprev);
    S2 = tree_sum(sq, Rprev);
    free(sq);
    *lnQ = (log(S_new) - log(S_old)) - dbeta * (double)Emin;
    r->ess = (S_new * S_new) / S2;
    r->resampled = r->ess < r->alpha * (double)Rprev;
    frexp(mx, scale_exp);
    if (r->resampled) {
        for (j = 0; j < Rprev; ++j) {
            double a = (double)r->R * r->wn[j];
            a = a / S_new;
            a = ldexp(a, FRAC_BITS);
            r->f_rep[j] = (uint64_t)floor(a);
        }
        status = counts_from_f(r->f_rep, Rprev, r->R, r->method, r->seed, step, r->run_id,
                               r->counts, Rnew);
    } else {
        for (j = 0; j < Rprev; ++j) {
            r->f_rep[j] = 1ull << FRAC_BITS;
            r->counts[j] = 1u;
        }
        *Rnew = Rprev;
    }
    return status;
}

/* A run that is one of several advanced together: its replica slots are offset
 * by slot_base (a multiple of 32) in the sweep and initial draws, and its
 * resampling draws carry run_id.  slot_base = run_id = 0 is a lone run. */
or_run *or_run_create_ex(int d, int L, const int8_t *J, uint32_t R, uint32_t Rcap, int n_steps,
                         const double *beta, const uint32_t *theta, int method, uint64_t seed,
                         uint32_t slot_base, uint32_t run_id)
{
    or_run *r;
    uint32_t j;
    int N;
    if (d < 2 || d > 3 || L < 2 || (L & 1) || R == 0 || n_steps < 0 || (slot_base & 31u))
        return NULL;
    r = (or_run *)calloc(1, sizeof(or_run));
    N = npow(L, d);
    r->d = d; r->L = L; r->N = N;
    r->J = (int8_t *)malloc((size_t)d * N);
    memcpy(r->J, J, (size_t)d * N);
    r->R = R;
    r->Rcap = Rcap ? Rcap : R;
    r->n_steps = n_steps;
    r->beta = (double *)malloc(sizeof(double) * (n_steps + 1));
    memcpy(r->beta, beta, sizeof(double) * (n_steps + 1));
    r->theta = (uint32_t *)malloc(sizeof(uint32_t) * (n_steps > 0 ? n_steps : 1));
    if (n_steps > 0) memcpy(r->theta, theta, sizeof(uint32_t) * n_steps);
    r->method = method;
    r->seed = seed;
    r->slot_base = slot_base;
    r->run_id = run_id;
    r->sig = (int8_t *)malloc((size_t)r->Rcap * N);
    r->sig2 = (int8_t *)malloc((size_t)r->Rcap * N);
    r->E = (int32_t *)malloc(sizeof(int32_t) * r->Rcap);
    r->E2 = (int32_t *)malloc(sizeof(int32_t) * r->Rcap);
    r->fam = (uint32_t *)malloc(sizeof(uint32_t) * r->Rcap);
    r->fam2 = (uint32_t *)malloc(sizeof(uint32_t) * r->Rcap);
    r->counts = (uint32_t *)calloc(r->Rcap, sizeof(uint32_t));
    r->f_rep = (uint64_t *)calloc(r->Rcap, sizeof(uint64_t));
    r->anc = (uint32_t *)calloc(r->Rcap, sizeof(uint32_t));
    /* step 1 */
    for (j = 0; j < R; ++j) {
        or_init_replica(d, L, seed, slot_base + j, r->sig + (size_t)j * N);
        r->E[j] = or_energy(d, L, r->J, r->sig + (size_t)j * N);
        r->fam[j] = j;
    }
    r->Rcur = R;
    r->Rprev = R;
    r->step = 0;
    r->sum_lnQ = 0.0;
    r->alpha = -1.0;
    measure(r, NULL, NULL, 0, 0.0, 0);
    return r;
}

/* switch on partial resampling with threshold alpha in [0, 1] before the first
 * step: all weights start at 1 */
int or_run_set_partial(or_run *r, double alpha)
{
    uint32_t j;
    if (!r || r->step != 0 || !(alpha >= 0.0 && alpha <= 1.0) || r->w) return OR_ERR_ARG;
    r->alpha = alpha;
    r->w = (double *)malloc(sizeof(double) * r->Rcap);
    r->w2 = (double *)malloc(sizeof(double) * r->Rcap);
    r->wn = (double *)malloc(sizeof(double) * r->Rcap);
    for (j = 0; j < r->Rcap; ++j) r->w[j] = 1.0;
    /* the initial population is unweighted, as after a resampling */
    r->ess = (double)r->Rcur;
    r->resampled = 1;
    measure(r, NULL, NULL, 0, 0.0, 0);
    return OR_OK;
}

or_run *or_run_create(int d, int L, const int8_t *J, uint32_t R, uint32_t Rcap, int n_steps,
                      const double *beta, const uint32_t *theta, int method, uint64_t seed)
{
    return or_run_create_ex(d, L, J, R, Rcap, n_steps, beta, theta, method, seed, 0u, 0u);
}

void or_run_destroy(or_run *r)
{
    if (!r) return;
    free(r->J); free(r->beta); free(r->theta);
    free(r->sig); free(r->sig2); free(r->E); free(r->E2);
    free(r->fam); free(r->fam2); free(r->counts); free(r->f_rep); free(r->anc);
    free(r->w); free(r->w2); free(r->wn);
    free(r);
}

/* one temperature step i = step + 1: steps 2, 3 and 4 of Sec. 2 */
int or_run_step(or_run *r)
{
    int i, N = r->N, st;
    uint32_t j, d, Rprev = r->Rcur;
    uint64_t Rnew = 0, acc = 0;
    int scale_exp = 0;
    double dbeta, lnQ = 0.0;
    uint32_t thr[4];
    int8_t *ts;
    int32_t *te;
    uint32_t *tf;
    if (r->status) return r->status;
    if (r->step >= r->n_steps) return OR_ERR_ARG;
    i = r->step + 1;
    dbeta = r->beta[i] - r->beta[i - 1];
    /* step 2: resample (every step, or when the weights' ESS is too small) */
    if (r->alpha >= 0.0)
        st = partial_weights(r, Rprev, dbeta, (uint32_t)i, &lnQ, &Rnew, &scale_exp);
    else
        st = or_resample(r->E, Rprev, r->R, dbeta, r->method, r->seed, (uint32_t)i, r->run_id,
                         r->counts, r->f_rep, &lnQ, &Rnew);
    if (st) { r->status = st; return st; }
    /* a population that outgrows its capacity, or dies out, stops the run */
    if (Rnew > r->Rcap || Rnew == 0) { r->status = OR_ERR_CAP; return OR_ERR_CAP; }
    d = 0;
    for (j = 0; j < Rprev; ++j) {
        uint32_t c;
        for (c = 0; c < r->counts[j]; ++c) {
            r->anc[d] = j;
            memcpy(r->sig2 + (size_t)d * N, r->sig + (size_t)j * N, (size_t)N);
            r->E2[d] = r->E[j];
            r->fam2[d] = r->fam[j];
            if (r->w) r->w2[d] = r->resampled ? 1.0 : ldexp(r->wn[j], -scale_exp);
            ++d;
        }
    }
    if (r->w) {
        double *tw = r->w; r->w = r->w2; r->w2 = tw;
    }
    ts = r->sig; r->sig = r->sig2; r->sig2 = ts;
    te = r->E; r->E = r->E2; r->E2 = te;
    tf = r->fam; r->fam = r->fam2; r->fam2 = tf;
    r->Rprev = Rprev;
    r->Rcur = (uint32_t)Rnew;
    r->sum_lnQ += lnQ;
    /* step 3: theta_i sweeps at beta_i.  The replicas are independent single-
     * replica chains; built with -fopenmp (the multi-core CPU baseline) the loop
     * is shared among the host cores, with the same result. */
    or_thresholds(r->beta[i], thr);
    {
        long jj, nrep = (long)r->Rcur;
#pragma omp parallel for reduction(+ : acc) schedule(static)
        for (jj = 0; jj < nrep; ++jj)
            acc += or_sweeps(r->d, r->L, r->J, r->sig + (size_t)jj * N, &r->E[jj], r->seed,
                             (uint32_t)i, r->slot_base + (uint32_t)jj, r->theta[i - 1], thr);
    }
    r->step = i;
    /* step 4: measure */
    measure(r, r->counts, r->f_rep, Rprev, lnQ, acc);
    return OR_OK;
}

/* accessors */
int or_run_status(const or_run *r) { return r->status; }
int or_run_step_index(const or_run *r) { return r->step; }
uint32_t or_run_size(const or_run *r) { return r->Rcur; }
uint32_t or_run_prev_size(const or_run *r) { return r->Rprev; }
double or_run_sum_lnQ(const or_run *r) { return r->sum_lnQ; }
void or_run_obs(const or_run *r, or_obs *o) { *o = r->obs; }
const int8_t *or_run_spins(const or_run *r) { return r->sig; }
const int32_t *or_run_energies(const or_run *r) { return r->E; }
const uint32_t *or_run_families(const or_run *r) { return r->fam; }
const uint32_t *or_run_counts(const or_run *r) { return r->counts; }
const uint64_t *or_run_fixed_weights(const or_run *r) { return r->f_rep; }
const uint32_t *or_run_ancestors(const or_run *r) { return r->anc; }
const double *or_run_weights(const or_run *r) { return r->w; }
/* -beta F = ln Z_0 + sum ln Q, ln Z_0 = N ln 2 (Eq. free-energy-estimator) */
double or_run_minus_beta_F(const or_run *r) { return (double)r->N * log(2.0) + r->sum_lnQ; }
