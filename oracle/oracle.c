/*
 * FP64 CPU oracle for the randomized mini-batch operator (Gargiani, Martinelli, Ruts Martinez,
 * Lygeros, "Parallel and Flexible Dynamic Programming via the Randomized Mini-Batch Operator").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header, table or helper with the CUDA path; it is
 * written to be read against the paper, not to be fast.  Values are promoted exactly from the
 * FP32 problem arrays and every sum, product and comparison is done in double precision.
 *
 * Problem layout (row r = s*m + a holds P(.|s,a)):
 *   dense: P[(s*m + a)*n + j]
 *   CSR:   row_ptr[r] .. row_ptr[r+1]-1 index col[] / prob[]
 *   cost[r] = g(s,a); +inf marks an action outside U(s) (Sec. II-A).
 *
 * Pinned by the tests against: Philox known-answer vectors, brute force over all deterministic
 * policies with direct linear solves, closed-form policy values, the monotonicity / shift /
 * contraction / fixed-point properties (Sec. III-B.1), the batch-size comparison theorem and its
 * corollary (Sec. III-B.2), the set-based definition of M_m(i) (eq. M(i) definition) and the
 * b=n / b=1 reductions (Sec. III-A).  The batch selection with replacement (Sec. V extension) is
 * pinned against its draw rule written with Python integers, constant weights against uniform
 * draws, draw frequencies, a batch-by-batch definition with repeated states, and J* through the
 * full-residual stop rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;             /* number of states */
    int32_t m;             /* actions per state (fixed; inadmissible ones carry cost +inf) */
    int32_t dense;         /* 1: dense P, 0: CSR */
    const float *P;        /* dense [n*m*n] */
    const int64_t *row_ptr;/* CSR [n*m+1] */
    const int32_t *col;    /* CSR [nnz] */
    const float *prob;     /* CSR [nnz] */
    const float *cost;     /* [n*m] */
    double gamma;          /* discount alpha in (0,1) */
} orc_mdp;

/* ------------------------------------------------------------------------------------------ *
 * Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2): ten rounds of
 *   (x0,x1,x2,x3) -> (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
 * with the key bumped by the Weyl constants (W0, W1) between rounds.
 * ------------------------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------------------------ *
 * Random re-indexing of the states for sweep k (Sec. III-A: states get random indexes and are
 * processed in ascending order, re-drawn every iteration; Sec. IV-A: shuffled before every
 * evaluation of the operator; Sec. V: uniform sampling without replacement).
 *
 * sigma_{seed,k} : [0,n) -> [0,n) is a bijection; sigma(p) is the state processed at position p.
 * Construction: an 8-round balanced Feistel network on 2h-bit words (h = max(1, ceil(ceil(log2 n)/2))),
 * round function F_r(R) = Philox4x32-10(ctr={R, r, k_lo, k_hi}, key={seed_lo, seed_hi}).x0 mod 2^h,
 * round (L,R) -> (R, L ^ F_r(R)); cycle-walking re-applies the network until the value is < n.
 * ------------------------------------------------------------------------------------------ */
int orc_perm_half_bits(int64_t n)
{
    int lg = 0;
    while (lg < 62 && ((int64_t)1 << lg) < n) lg++;
    int h = (lg + 1) / 2;
    return h < 1 ? 1 : h;
}

static uint64_t feistel_once(uint64_t x, int h, uint64_t seed, uint64_t sweep)
{
    uint64_t mask = ((uint64_t)1 << h) - 1;
    uint64_t L = x >> h, R = x & mask;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (uint32_t r = 0; r < 8; ++r) {
        uint32_t ctr[4] = { (uint32_t)R, r, (uint32_t)sweep, (uint32_t)(sweep >> 32) };
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        uint64_t F = (uint64_t)out[0] & mask;
        uint64_t newL = R;
        uint64_t newR = L ^ F;
        L = newL;
        R = newR;
    }
    return (L << h) | R;
}

int64_t orc_perm(int64_t n, uint64_t seed, uint64_t sweep, int64_t p)
{
    int h = orc_perm_half_bits(n);
    uint64_t domain = (uint64_t)1 << (2 * h);
    uint64_t x = (uint64_t)p, steps = 0;
    do {
        x = feistel_once(x, h, seed, sweep);
        /* a bijection of the domain returns to [0,n) within domain-n+1 steps */
        if (++steps > domain) return -1;
    } while (x >= (uint64_t)n);
    return (int64_t)x;
}

void orc_perm_all(int64_t n, uint64_t seed, uint64_t sweep, int64_t *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p)
        out[p] = orc_perm(n, seed, sweep, p);
}

/* ------------------------------------------------------------------------------------------ *
 * Batch selection with replacement (Sec. V names sampling with replacement and non-uniform /
 * importance-sampled selection as extensions; the paper gives no rule, the one below is ours).
 * Position p of sweep k draws x = Philox4x32-10(ctr = {p, 2^31, k_lo, k_hi}, key = {seed_lo,
 * seed_hi}) (the second counter word never takes the Feistel round numbers 0..7) and reads the
 * 64-bit integer u = x0 * 2^32 + x1.  Then, in exact integer arithmetic:
 *   select 1 (uniform):  state = floor(u * n / 2^64);
 *   select 2 (weighted, integer weights w with W = sum w > 0): r = floor(u * W / 2^64) and
 *     state = the smallest s with w_0 + ... + w_s > r, so P(state = s) = w_s / W up to 2^-64.
 * ------------------------------------------------------------------------------------------ */
static uint64_t draw_word(uint64_t seed, uint64_t sweep, int64_t p)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)p, 0x80000000u, (uint32_t)sweep, (uint32_t)(sweep >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return ((uint64_t)out[0] << 32) | out[1];
}

/* cumulative weights: cum[s] = w_0 + ... + w_s (plain running sum) */
static uint64_t *cumulative(int64_t n, const uint32_t *w)
{
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t run = 0;
    for (int64_t s = 0; s < n; ++s) {
        run += w[s];
        cum[s] = run;
    }
    return cum;
}

/* the state of position p; cum = NULL for select 1 */
static int64_t draw_state(int64_t n, uint64_t seed, uint64_t sweep, int64_t p, const uint64_t *cum)
{
    unsigned __int128 u = draw_word(seed, sweep, p);
    if (!cum) return (int64_t)((u * (unsigned __int128)(uint64_t)n) >> 64);
    uint64_t r = (uint64_t)((u * (unsigned __int128)cum[n - 1]) >> 64);
    /* smallest s with cum[s] > r (cum is nondecreasing and cum[n-1] > r) */
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cum[mid] > r) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* processing order of one sweep: sigma (select 0) or n draws (select 1, 2); weights for 2 */
int orc_sweep_order(int64_t n, uint64_t seed, uint64_t sweep, int32_t select, const uint32_t *weights,
                    int64_t *out)
{
    if (select == 0) {
        orc_perm_all(n, seed, sweep, out);
        return 0;
    }
    if ((select != 1 && select != 2) || n < 1) return -1;
    uint64_t *cum = NULL;
    if (select == 2) {
        cum = cumulative(n, weights);
        if (cum[n - 1] == 0) { free(cum); return -1; }
    }
    for (int64_t p = 0; p < n; ++p) out[p] = draw_state(n, seed, sweep, p, cum);
    free(cum);
    return 0;
}

/* ------------------------------------------------------------------------------------------ *
 * Q-factor of one state-action pair at a value function J (the bracket of eqs. (6)-(7), the
 * Bellman operators T_mu and T):  g(i,u) + alpha * sum_j p_ij(u) J(j).
 * ------------------------------------------------------------------------------------------ */
double orc_q(const orc_mdp *M, int64_t s, int32_t a, const double *J)
{
    int64_t r = s * (int64_t)M->m + a;
    double g = (double)M->cost[r];
    if (isinf(g) && g > 0) return INFINITY;   /* u not in U(s) */
    double acc = 0.0;
    if (M->dense) {
        const float *row = M->P + r * M->n;
        for (int64_t j = 0; j < M->n; ++j) acc += (double)row[j] * J[j];
    } else {
        for (int64_t e = M->row_ptr[r]; e < M->row_ptr[r + 1]; ++e)
            acc += (double)M->prob[e] * J[M->col[e]];
    }
    return g + M->gamma * acc;
}

/* min over u in U(s) of the Q-factor (eq. (7)); ties resolved to the lowest action index. */
static double backup_min(const orc_mdp *M, int64_t s, const double *J, int32_t *argmin, double *gap)
{
    double best = INFINITY, second = INFINITY;
    int32_t ba = 0;
    for (int32_t a = 0; a < M->m; ++a) {
        double q = orc_q(M, s, a, J);
        if (q < best) { second = best; best = q; ba = a; }
        else if (q < second) { second = q; }
    }
    if (argmin) *argmin = ba;
    if (gap) *gap = second - best;
    return best;
}

/* ------------------------------------------------------------------------------------------ *
 * Greedy / Bellman pass (eq. (7) for every state, and the policy-improvement step of Alg. 1):
 * TV(s) = min_u Q(s,u), pi(s) = lowest u attaining it, gap(s) = second smallest Q - smallest Q
 * (+inf when only one action is admissible).  Returns ||TV - V||_inf.
 * ------------------------------------------------------------------------------------------ */
double orc_greedy(const orc_mdp *M, const double *V, double *TV, int32_t *pi, double *gap)
{
    double res = 0.0;
    #pragma omp parallel for schedule(static) reduction(max:res)
    for (int64_t s = 0; s < M->n; ++s) {
        int32_t a; double gp;
        double t = backup_min(M, s, V, &a, &gp);
        if (TV) TV[s] = t;
        if (pi) pi[s] = a;
        if (gap) gap[s] = gp;
        double d = fabs(t - V[s]);
        if (d > res) res = d;
    }
    return res;
}

/* ------------------------------------------------------------------------------------------ *
 * One application of the mini-batch operator B_b (eq. B definition) or B_{pi,b} (eq. Bmu
 * definition), with the states re-indexed by sigma_{seed,k} (Sec. III-A).
 *
 * The processing order is sigma(0), sigma(1), ...; M_b(i) = {first b*floor((i-1)/b) states of
 * that order} (eq. M(i) definition), i.e. batch t holds positions [t*b, min(n,(t+1)b)).  A state in
 * batch t reads the new value of every state of batches < t and the old value of every other state,
 * including the states of its own batch.  So each batch first computes all its new values from V
 * and only then writes them back.
 *
 * pi == NULL: B_b (min over actions); else B_{pi,b} (the row of pi(s) only).
 * perm: caller-provided scratch of n entries (filled here).  W: scratch of b doubles.
 * Returns max_s |V_new(s) - V_old(s)|.
 * ------------------------------------------------------------------------------------------ */
/* one sweep over a given processing order (n positions in batches of b; entries may repeat) */
static double apply_order(const orc_mdp *M, const int32_t *pi, int64_t b, const int64_t *perm, double *V, double *W)
{
    int64_t n = M->n;
    double delta = 0.0;
    for (int64_t start = 0; start < n; start += b) {
        int64_t len = (n - start < b) ? (n - start) : b;
        /* compute every new value of the batch from the current V ... */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < len; ++i) {
            int64_t s = perm[start + i];
            if (pi) W[i] = orc_q(M, s, pi[s], V);
            else    W[i] = backup_min(M, s, V, NULL, NULL);
        }
        /* ... then write them all back */
        for (int64_t i = 0; i < len; ++i) {
            int64_t s = perm[start + i];
            double d = fabs(W[i] - V[s]);
            if (d > delta || isnan(d)) delta = d;
            V[s] = W[i];
        }
    }
    return delta;
}

double orc_mb_apply(const orc_mdp *M, const int32_t *pi, int64_t b, uint64_t seed, uint64_t sweep,
                    double *V, int64_t *perm, double *W)
{
    orc_perm_all(M->n, seed, sweep, perm);
    return apply_order(M, pi, b, perm, V, W);
}

/* ||T V - V||_inf (pi NULL) or ||T_pi V - V||_inf over all states */
static double full_residual(const orc_mdp *M, const int32_t *pi, const double *V)
{
    double r = 0.0;
    for (int64_t s = 0; s < M->n; ++s) {
        double t = pi ? orc_q(M, s, pi[s], V) : backup_min(M, s, V, NULL, NULL);
        double d = fabs(t - V[s]);
        if (d > r || isnan(d)) r = d;
    }
    return r;
}

/* ------------------------------------------------------------------------------------------ *
 * MB-VI (Sec. III-B: B_b in place of T in value iteration).  Sweep k = start_sweep, start_sweep+1,
 * ... applies B_b with sigma_{seed,k}; stops after the first sweep with delta_k <= eps or after
 * max_sweeps sweeps.  delta_trace[j] (optional) = delta of the j-th sweep; V_traj (optional,
 * [max_sweeps*n]) = V after each sweep.  Returns the number of sweeps done.
 * ------------------------------------------------------------------------------------------ */
int64_t orc_mbvi_select(const orc_mdp *M, const int32_t *pi, int64_t b, uint64_t seed, int64_t start_sweep,
                        double eps, int64_t max_sweeps, int32_t select, const uint32_t *weights, int32_t residual_kind,
                        double *V, double *delta_trace, double *V_traj, double *resid_out);

int64_t orc_mbvi(const orc_mdp *M, const int32_t *pi, int64_t b, uint64_t seed, int64_t start_sweep,
                 double eps, int64_t max_sweeps, double *V, double *delta_trace, double *V_traj)
{
    return orc_mbvi_select(M, pi, b, seed, start_sweep, eps, max_sweeps, 0, NULL, 0, V, delta_trace, V_traj, NULL);
}

/* ------------------------------------------------------------------------------------------ *
 * MB-VI / evaluation with a batch-selection rule (select 0: sigma, the paper's method; 1, 2: draws
 * with replacement as defined above) and a stop test (residual_kind 0: the sweep change delta_k;
 * 1: the Bellman residual).  With draws a sweep's change covers only the states drawn, so there,
 * and with residual_kind 1, a sweep with delta <= eps is followed by the full residual
 * ||TV - V||_inf (||T_pi V - V||_inf) and the solve stops only when that is <= eps too.
 * *resid_out (optional) = the last full residual when one was taken, else delta.  Returns sweeps
 * done, or -1 on a bad select / zero weights.
 * ------------------------------------------------------------------------------------------ */
int64_t orc_mbvi_select(const orc_mdp *M, const int32_t *pi, int64_t b, uint64_t seed, int64_t start_sweep,
                        double eps, int64_t max_sweeps, int32_t select, const uint32_t *weights, int32_t residual_kind,
                        double *V, double *delta_trace, double *V_traj, double *resid_out)
{
    int64_t n = M->n;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *W = (double *)malloc(sizeof(double) * (size_t)(b < n ? b : n));
    int64_t done = 0;
    double resid = 0.0;
    for (int64_t j = 0; j < max_sweeps; ++j) {
        if (orc_sweep_order(n, seed, (uint64_t)(start_sweep + j), select, weights, perm) != 0) {
            done = -1;
            break;
        }
        double delta = apply_order(M, pi, b, perm, V, W);
        if (delta_trace) delta_trace[j] = delta;
        if (V_traj) memcpy(V_traj + j * n, V, sizeof(double) * (size_t)n);
        done = j + 1;
        resid = delta;
        if (delta <= eps) {
            if (select == 0 && residual_kind == 0) break;
            resid = full_residual(M, pi, V);
            if (resid <= eps) break;
        }
    }
    if (resid_out) *resid_out = resid;
    free(perm);
    free(W);
    return done;
}

/* ------------------------------------------------------------------------------------------ *
 * MB-MPI (Alg. 1 with B_{mu,b} in place of T_mu in the evaluation step, Sec. III-B), with the
 * stopping rule and start read as: V starts from the caller's V; the policy starts greedy at V;
 * each outer iteration runs the improvement pass (TV, pi, ||TV-V||_inf), stops when that residual
 * is <= eps, else applies K evaluation sweeps of B_{pi,b} warm-started from V (the sweep counter
 * of sigma keeps running across all evaluation sweeps).  The improvement pass does not modify V.
 * resid_trace[it] (optional) = residual of outer iteration it.  Returns outer iterations done
 * (greedy passes); *sweeps_out = evaluation sweeps done.
 * ------------------------------------------------------------------------------------------ */
int64_t orc_mpi_select(const orc_mdp *M, int64_t b, int32_t K, uint64_t seed, int64_t start_sweep,
                       double eps, int64_t max_iters, int32_t select, const uint32_t *weights, double *V,
                       int32_t *pi, int64_t *sweeps_out, double *resid_trace);

int64_t orc_mpi(const orc_mdp *M, int64_t b, int32_t K, uint64_t seed, int64_t start_sweep,
                double eps, int64_t max_iters, double *V, int32_t *pi, int64_t *sweeps_out,
                double *resid_trace)
{
    return orc_mpi_select(M, b, K, seed, start_sweep, eps, max_iters, 0, NULL, V, pi, sweeps_out, resid_trace);
}

/* MB-MPI whose evaluation sweeps use a batch-selection rule (select 0, 1, 2 as above); the stop
   test is the improvement pass's full residual either way.  Returns -1 on a bad select. */
int64_t orc_mpi_select(const orc_mdp *M, int64_t b, int32_t K, uint64_t seed, int64_t start_sweep,
                       double eps, int64_t max_iters, int32_t select, const uint32_t *weights, double *V,
                       int32_t *pi, int64_t *sweeps_out, double *resid_trace)
{
    int64_t n = M->n;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *W = (double *)malloc(sizeof(double) * (size_t)(b < n ? b : n));
    int64_t sweep = start_sweep, it = 0;
    for (;;) {
        double res = orc_greedy(M, V, NULL, pi, NULL);
        if (resid_trace) resid_trace[it] = res;
        it++;
        if (res <= eps || it >= max_iters) break;
        for (int32_t j = 0; j < K; ++j) {
            if (orc_sweep_order(n, seed, (uint64_t)sweep, select, weights, perm) != 0) {
                free(perm);
                free(W);
                return -1;
            }
            apply_order(M, pi, b, perm, V, W);
            sweep++;
        }
    }
    if (sweeps_out) *sweeps_out = sweep - start_sweep;
    free(perm);
    free(W);
    return it;
}

/* ------------------------------------------------------------------------------------------ *
 * Independently written special cases used to pin the reductions stated after the definition
 * of B (Sec. III-A): b = n gives the Bellman operator T (eq. (7), all states from the same J) and
 * b = 1 gives the Gauss-Seidel operator F (Sec. II-D, one state at a time, in place, in the given
 * processing order).
 * ------------------------------------------------------------------------------------------ */
void orc_bellman_T(const orc_mdp *M, const double *J, double *out)
{
    for (int64_t s = 0; s < M->n; ++s) {
        double best = INFINITY;
        for (int32_t a = 0; a < M->m; ++a) {
            double q = orc_q(M, s, a, J);
            if (q < best) best = q;
        }
        out[s] = best;
    }
}

void orc_gauss_seidel_F(const orc_mdp *M, const int64_t *order, double *J)
{
    for (int64_t i = 0; i < M->n; ++i) {
        int64_t s = order[i];
        double best = INFINITY;
        for (int32_t a = 0; a < M->m; ++a) {
            double q = orc_q(M, s, a, J);
            if (q < best) best = q;
        }
        J[s] = best;
    }
}

/* Number of OpenMP threads the oracle runs on (1 when built without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
