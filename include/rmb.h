/*
 * rmb.h -- C ABI of librmb: the randomized mini-batch operator for finite discounted MDPs
 * (Gargiani, Martinelli, Ruts Martinez, Lygeros, "Parallel and Flexible Dynamic Programming via
 * the Randomized Mini-Batch Operator"), with value iteration, modified policy iteration and
 * policy evaluation built on it, on one NVIDIA B300 (sm_103a).
 *
 * Problem (Sec. II-A): states S = {0..n-1}, m actions per state, transition rows P(.|s,a),
 * stage costs g(s,a) (here "cost"), discount alpha (here "gamma") in (0,1).  An action outside
 * U(s) carries cost +inf; every state needs at least one finite cost.
 *
 * Row r = s*m + a holds P(.|s,a).  Layouts (all arrays in device memory, caller-owned):
 *   RMB_DENSE: P[n][m][n] float32, row-major (the m rows of a state are contiguous);
 *   RMB_CSR:   row_ptr[n*m+1] int64 (row_ptr[0] = 0, non-decreasing), col[nnz] int32 in [0,n),
 *              prob[nnz] float32 in [0,1];
 *   both:      cost[n*m] float32.
 * Rows should sum to 1 (checked to 1e-4 when opts.validate != 0).
 *
 * Values are float32 on the interface.  Inside a solve they are stored centred, V = mu + d, with
 * mu a double and d float32; the reported residuals are exact differences of the stored values.
 *
 * Conventions shared by every entry point:
 *   - Device pointers are caller-owned; the library never allocates device memory and never
 *     frees anything.  Scratch memory ("workspace") is caller-provided, sized by
 *     rmb_workspace_bytes, 256-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every call is
 *     asynchronous on that stream unless `stats` is non-NULL, in which case the call waits
 *     for the stream and fills *stats (then the return value is the device-side status).
 *   - Errors are returned as rmb_status codes; nothing aborts, exits or throws across the ABI.
 *     Argument errors are reported before anything is launched.  Every grid-wide wait inside a
 *     kernel gives up after opts.barrier_timeout_ns and reports RMB_ERR_BARRIER_TIMEOUT.
 *   - On any error the outputs are unspecified.
 */
#ifndef RMB_H
#define RMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RMB_OK = 0,
    RMB_ERR_ARG = -1,              /* invalid argument (host check; nothing launched) */
    RMB_ERR_CUDA = -2,             /* a CUDA runtime call or kernel launch failed */
    RMB_ERR_NOT_CONVERGED = -3,    /* max_sweeps / max outer iterations reached above eps */
    RMB_ERR_BARRIER_TIMEOUT = -4,  /* a grid-wide wait gave up; the kernel returned early */
    RMB_ERR_INVALID_MDP = -5,      /* device validation: bad probability, index, row sum or cost */
    RMB_ERR_WORKSPACE = -6,        /* workspace NULL, too small or not 256-byte aligned */
    RMB_ERR_UNSUPPORTED = -7,      /* a size this build does not handle (n >= 2^31, ...) */
    RMB_ERR_NONFINITE = -8,        /* a value became NaN during the solve */
    RMB_ERR_TOO_LARGE = -9         /* rmb_vi_noalloc: the solve needs more scratch than
                                      RMB_NOALLOC_SCRATCH_BYTES */
} rmb_status;

enum { RMB_DENSE = 0, RMB_CSR = 1 };

/* Storage of dense transition rows.  RMB_P_F32 rows are used as given.  RMB_P_BF16 / RMB_P_FP8E4M3
   rows are codes c_rj = p_rj / scale_r (rmb_quantize_rows); the kernels decode them to float32 and
   divide by the decoded row sum (taken from row_scale when given), so the quantisation scale cancels
   and every decoded row is a distribution. */
enum { RMB_P_F32 = 0, RMB_P_BF16 = 1, RMB_P_FP8E4M3 = 2 };

/* The MDP (Sec. II-A).  All pointers are device pointers. */
typedef struct {
    int64_t n;               /* number of states, 1 <= n < 2^31 */
    int32_t m;               /* actions per state, >= 1 */
    int32_t format;          /* RMB_DENSE or RMB_CSR */
    const void *P;           /* RMB_DENSE: [n*m*n] elements of p_dtype */
    const int64_t *row_ptr;  /* RMB_CSR: [n*m+1] */
    const int32_t *col;      /* RMB_CSR: [nnz] */
    const float *prob;       /* RMB_CSR: [nnz] */
    const float *cost;       /* [n*m]; +inf = action not admissible; NaN and -inf are invalid
                                (rmb_validate rejects them; unvalidated, a NaN cost drops its action
                                from the minimum like +inf) */
    double gamma;            /* discount, 0 < gamma < 1 */
    int32_t k_uniform;       /* RMB_CSR: k > 0 declares row_ptr[r] == r*k for every row (enables
                                the vectorised row path; checked when validate != 0); 0 = unknown */
    int32_t p_dtype;         /* RMB_DENSE: RMB_P_F32 / RMB_P_BF16 / RMB_P_FP8E4M3 */
    const float *row_scale;  /* RMB_DENSE coded rows: [n*m] = 1 / (sum of the row's decoded codes), as
                                written by rmb_quantize_rows; NULL = the kernels sum each row */
} rmb_mdp;

/* Options of a solve. */
typedef struct {
    int64_t batch;           /* mini-batch size b (the paper's m), 1 <= b; b >= n means b = n;
                                0 = chosen by the library's time model (stats->batch reports it) */
    uint64_t seed;           /* key of the per-sweep state permutation */
    double eps;              /* stop when the residual <= eps (VI / evaluation: sup-norm change of a
                                sweep; MPI: ||TV - V||_inf of the improvement pass) */
    int64_t max_sweeps;      /* VI / evaluation: sweep limit; MPI: limit on improvement passes */
    int64_t start_sweep;     /* index of the first sweep (the permutation of sweep k depends only on
                                (seed, k), so a solve resumes exactly from V and start_sweep) */
    int32_t eval_sweeps;     /* MPI: K evaluation sweeps per improvement (Alg. 1) */
    int32_t validate;        /* != 0: run the device validation pass first */
    int64_t barrier_timeout_ns; /* limit of every grid-wide wait; 0 = 2e9 (2 s) */
    int32_t grid_ctas;       /* 0 = occupancy-sized persistent grid; else the number of CTAs */
    int32_t flags;           /* RMB_FLAG_* */
    double *trace;           /* optional device [max_sweeps] doubles: per-sweep residual (VI /
                                evaluation) or per-improvement residual (MPI); NULL = none */
    int32_t select;          /* batch selection: RMB_SELECT_PERMUTATION (0, the paper's method),
                                RMB_SELECT_UNIFORM or RMB_SELECT_WEIGHTED (with replacement) */
    int32_t residual_kind;   /* stop test of rmb_vi: RMB_RESIDUAL_SWEEP (0: the sweep change
                                delta_k = ||V_k - V_{k-1}||_inf) or RMB_RESIDUAL_BELLMAN (1: a sweep
                                with delta_k <= eps is confirmed by a full Bellman pass and the solve
                                stops only if ||TV - V||_inf <= eps; stats->residual is that value).
                                MPI always stops on ||TV - V||_inf (Alg. 1); rmb_eval_policy and the
                                batched API support 0 only. */
    const uint32_t *weights; /* RMB_SELECT_WEIGHTED: device [n] integer weights, sum > 0; else NULL */
} rmb_opts;

/*
 * Batch selection with replacement (Sec. V proposes sampling with replacement and non-uniform /
 * importance-sampled selection; the paper fixes no rule, this one is the library's).  A sweep is
 * still n positions in batches of b, but position p of sweep k holds a drawn state instead of
 * sigma_{seed,k}(p):  u = x0 * 2^32 + x1 of Philox4x32-10(ctr = {p, 2^31, k_lo, k_hi},
 * key = {seed_lo, seed_hi}) (the Feistel rounds of sigma use counter words 0..7 there), then in
 * exact integer arithmetic
 *   RMB_SELECT_UNIFORM:  state = floor(u * n / 2^64);
 *   RMB_SELECT_WEIGHTED: r = floor(u * W / 2^64) with W = sum of the weights, state = the smallest
 *                        s with w_0 + ... + w_s > r (probability w_s / W; weight 0 = never drawn).
 * A state drawn twice in one batch gets the same value twice; a state not drawn keeps its value.
 * The sweep's change then covers only the drawn states, so a sweep whose change is <= eps is
 * followed by a full Bellman pass, and the solve stops only if ||TV - V||_inf <= eps as well
 * (stats->residual is that value).  Supported by rmb_vi, rmb_mpi (evaluation sweeps; MPI's stop
 * test is its improvement pass) and rmb_vi_noalloc; rmb_eval_policy and the batched API return
 * RMB_ERR_UNSUPPORTED.  A state drawn in two consecutive batches takes the later batch's value.
 * Workspace: + 16*n bytes of batch marks when b < n, and for RMB_SELECT_WEIGHTED another 8*n bytes
 * of cumulative weights (+ 8 per 8192 states).
 */
#define RMB_RESIDUAL_SWEEP 0
#define RMB_RESIDUAL_BELLMAN 1
#define RMB_SELECT_PERMUTATION 0
#define RMB_SELECT_UNIFORM 1
#define RMB_SELECT_WEIGHTED 2

/* Test-only fault injection: CTA 0 never arrives at the first grid-wide wait, so every wait runs
   out and the call must report RMB_ERR_BARRIER_TIMEOUT with the GPU context intact. */
#define RMB_FLAG_INJECT_BARRIER_STALL 1
/* Rows need not sum to 1 (used for the transposed chain of rmb_fixed_point_grad): values are kept
   uncentred (mu = 0) and the sweeps run in plain float32. */
#define RMB_FLAG_RAW_ROWS 2
/* Asynchronous sweeps (RMB_CSR only, single-MDP solves: rmb_vi, rmb_mpi, rmb_eval_policy,
   rmb_vi_noalloc; others return RMB_ERR_UNSUPPORTED. Sec. V suggests asynchronous MB-VI / MB-MPI): a
   sweep processes the whole random order of its permutation in one pass and writes every new value in
   place at once, with no grid-wide barrier between batches, so a state reads whatever updates of the
   same sweep have already landed (chaotic relaxation; b is ignored).  One barrier per sweep keeps
   the stop test.  Converges to the same fixed point; trajectories are not reproducible. */
#define RMB_FLAG_ASYNC 4
/* rmb_vi, rmb_mpi and rmb_eval_policy pick a one-cluster solve for small MDPs with small batches (MB-MPI:
   improvement passes and evaluation sweeps alike): up to 16 CTAs of one thread-block
   cluster each hold a copy of the values (and of the order) in shared memory, exchange every batch's
   new values through distributed shared memory and separate batches by the hardware cluster barrier
   instead of a grid-wide barrier through memory (stats->path = 4).  It is taken when n * 16 bytes fit
   in shared memory (n <= 14080), the sweep has >= 2 batches of at most 2 states per warp of the cluster
   (b <= 512 with 16 CTAs of 512 threads), rows are float32 dense or CSR (vectorisable uniform rows of
   <= 256 entries per state, other uniform rows of <= 32, or ragged rows), the order is sigma (RMB_SELECT_PERMUTATION),
   the stop test RMB_RESIDUAL_SWEEP, grid_ctas = 0 and neither RMB_FLAG_ASYNC nor
   RMB_FLAG_INJECT_BARRIER_STALL is set.  This flag keeps the grid-wide solve instead. */
#define RMB_FLAG_NO_CLUSTER 8

/* Results of a solve (filled only when a stats pointer is passed). */
typedef struct {
    int64_t sweeps;          /* applications of B_b / B_{pi,b} done */
    int64_t iters;           /* MPI: improvement passes done; else 0 */
    int64_t barriers;        /* grid-wide waits crossed */
    double residual;         /* last residual (see rmb_opts.eps) */
    double v_shift;          /* centring offset mu at exit */
    int32_t status;          /* device-side rmb_status */
    int32_t grid_ctas;       /* CTAs of the persistent launch */
    int32_t path;            /* 0 dense, 1 CSR vectorised rows, 2 CSR generic rows, 3 dense TMA pipeline,
                                4 one-cluster solve of a small MDP (RMB_FLAG_NO_CLUSTER) */
    int32_t lanes_per_state; /* CSR paths: lanes that share one state */
    float ms;                /* device time of the call (CUDA events on `stream`); batched solves: this
                                MDP's solve time (device clock, from its start to its group's first CTA
                                finishing it) */
    int32_t batch;           /* the mini-batch size b used (the model's choice when opts.batch = 0) */
    float start_ms;          /* batched solves: when this MDP started, after the first MDP of the launch
                                started (device clock); 0 otherwise */
} rmb_stats;

/*
 * opts.batch = 0: b from a model of one solve on a B300 whose constants come from the measured bench
 * workloads.  time(b) = sweeps(b) * ceil(n/b) * (max(stream time of one batch, waves of concurrent
 * states) + 6 us per batch), where sweeps(b) shrinks with b as fitted on the 2^20-state CSR MDP
 * (the comparison theorem of Sec. III-B.2 says smaller b never needs more sweeps).  CSR: one batch
 * gathers b * m * k successors at 244 G/s (k = 4 when rows are ragged), 2368 states at once, 1 us per
 * wave.  Dense: b * m * n element bytes at 6.5 TB/s, 148 states at once, m * n element bytes per
 * state at 44 GB/s per SM.  b runs over n, n/2, n/4, ..., >= 32.  The choice depends only on the MDP's
 * sizes, format, gamma and eps, so rmb_workspace_bytes and the solve agree.
 */

/* Bytes of workspace a call with this MDP and these options needs (0 on invalid arguments). */
size_t rmb_workspace_bytes(const rmb_mdp *mdp, const rmb_opts *opts);

/*
 * MB-VI (Sec. III-B: B_b of eq. (11) in place of T in value iteration).
 * Sweep k = start_sweep, start_sweep+1, ... re-indexes the states by a Philox-keyed permutation
 * sigma_{seed,k} (Sec. III-A, Sec. IV-A) and updates them in batches of b positions: every
 * state of batch t reads the new values of batches < t and the old values of the rest (its own
 * batch included), so b = 1 is Gauss-Seidel and b = n is the Bellman operator T.
 * Stops after the first sweep whose sup-norm change is <= eps (confirmed by ||TV - V||_inf <= eps
 * with residual_kind = RMB_RESIDUAL_BELLMAN or with draws), or after max_sweeps sweeps.  Options:
 * opts.flags = RMB_FLAG_ASYNC (asynchronous sweeps, CSR), opts.select / opts.weights (batches drawn
 * with replacement).
 *   V_inout  [n] float32: start values on entry (the paper uses 0), final values on exit.
 *   pi_out   [n] int32 or NULL: greedy policy at the final values (lowest action on ties).
 *   qgap_out [n] float32 or NULL: second smallest minus smallest Q-factor at the final values.
 */
int rmb_vi(const rmb_mdp *mdp, const rmb_opts *opts, float *V_inout, int32_t *pi_out,
           float *qgap_out, void *workspace, size_t workspace_bytes, rmb_stats *stats,
           void *stream);

/*
 * MB-MPI (Alg. 1 with B_{pi,b} of eq. (12) in the evaluation step, Sec. III-B), warm-started:
 * repeat { improvement pass: pi = greedy(V), r = ||TV - V||_inf (V unchanged); stop if r <= eps
 * or after max_sweeps passes; K = eval_sweeps sweeps V <- B_{pi,b} V }.  The permutation's
 * sweep counter runs on across all evaluation sweeps.
 *   V_inout [n]: start values / final values.  pi_out [n] (required): the final greedy policy.
 *   qgap_out [n] or NULL: Q-gap of the final improvement pass.
 */
int rmb_mpi(const rmb_mdp *mdp, const rmb_opts *opts, float *V_inout, int32_t *pi_out,
            float *qgap_out, void *workspace, size_t workspace_bytes, rmb_stats *stats,
            void *stream);

/*
 * Mini-batch policy evaluation: sweeps V <- B_{pi,b} V (eq. (12)) until the sup-norm change of a
 * sweep is <= eps or max_sweeps sweeps are done.  Converges to J_pi of eq. (4).
 *   pi [n] int32 in [0,m), admissible actions only.  V_inout [n]: start / final values.
 */
int rmb_eval_policy(const rmb_mdp *mdp, const int32_t *pi, const rmb_opts *opts, float *V_inout,
                    void *workspace, size_t workspace_bytes, rmb_stats *stats, void *stream);

/*
 * One full Bellman pass at V (eq. (7)) and the improvement step of Alg. 1:
 *   TV_out [n] or NULL, pi_out [n] or NULL (lowest action on ties), qgap_out [n] or NULL.
 * stats->residual = ||TV - V||_inf.  Only opts.validate, grid_ctas, barrier_timeout_ns and flags
 * are used.
 */
int rmb_greedy(const rmb_mdp *mdp, const rmb_opts *opts, const float *V, float *TV_out,
               int32_t *pi_out, float *qgap_out, void *workspace, size_t workspace_bytes,
               rmb_stats *stats, void *stream);

/*
 * The processing order of sweep k (Sec. III-A): out[p] = sigma_{seed,k}(p), p = 0..n-1, a
 * bijection of [0,n).  An 8-round balanced Feistel network on 2h-bit words with
 * h = max(1, ceil(ceil(log2 n)/2)) and round function Philox4x32-10(ctr = {R, round, k_lo, k_hi},
 * key = {seed_lo, seed_hi}).x0 mod 2^h (Salmon et al., SC'11), cycle-walked into [0,n).
 *   out [n] int32, device.
 */
int rmb_permutation(int64_t n, uint64_t seed, uint64_t sweep, int32_t *out, void *stream);

/*
 * One backup of an explicit list of states: W_out[i] = min_a c(s,a) + gamma sum_j P(j|s,a) V(j) with
 * s = states[i] (eq. (7) restricted to the list), or, with pi != NULL, the policy's backup
 * c(s,pi(s)) + gamma sum_j P(j|s,pi(s)) V(j) (T_pi of eq. (4)).  Float32 values as given (not
 * centred), one warp per listed state.  This is the step one rank takes in a row-partitioned
 * mini-batch sweep: the batch's states that it owns, read from its replica of V (eq. (11): every state
 * of a batch reads the values before the batch).
 *   V [n], states [count] int32 (entries outside [0,n) are clamped into it), pi [n] or NULL,
 *   W_out [count]: device.  RMB_DENSE with coded rows returns RMB_ERR_UNSUPPORTED.  Asynchronous.
 */
int rmb_backup_states(const rmb_mdp *mdp, const float *V, const int32_t *states, int64_t count,
                      const int32_t *pi, float *W_out, void *stream);

/*
 * Device validation of an MDP: probabilities finite and in [0,1], |row sum - 1| <= 1e-4,
 * indices in [0,n), row_ptr non-decreasing from 0 (and == r*k when k_uniform is declared),
 * costs not NaN and not -inf, at least one admissible action per state.
 * Synchronous: returns RMB_OK or RMB_ERR_INVALID_MDP (or an argument / CUDA error).
 *   workspace: at least 256 bytes (its first 256 bytes are used).
 */
int rmb_validate(const rmb_mdp *mdp, void *workspace, size_t workspace_bytes, void *stream);

/*
 * MB-VI exactly as rmb_vi, for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Who needs it: code that only ever receives device pointers for its inputs and outputs from a host
 * application that owns all device memory (a plugin inside a simulator, a solver embedded in a
 * serving process, a pure C caller with no allocator handle), and control loops that forbid device
 * allocation after start-up because cudaMalloc can synchronise the device and take unbounded time.
 *
 * Instead of a caller-provided workspace it uses one fixed scratch array of
 * RMB_NOALLOC_SCRATCH_BYTES (8 MiB) compiled into the library as a file-scope __device__ array;
 * every GPU that loads the library holds that array until the process exits.  A solve needs
 * rmb_workspace_bytes(mdp, opts) of scratch (about 8*n + 16*min(b,n) bytes, plus 4*n when the
 * permutation is precomputed: T = ceil(n/b) >= 16, or 2 <= T and n < T*65536); larger problems are
 * rejected with RMB_ERR_TOO_LARGE before anything is
 * launched.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine, no CUDA events.
 *
 * Set-up: the first call on a device (with that device current) looks up the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream capture.
 * Sharing: every call on a device uses the same array, which keeps the previous call's contents
 * (each call clears the parts that must start at zero).  Calls that overlap on the GPU -- on
 * different streams or from different host threads -- race on the array and give wrong results;
 * serialise them.
 * stats (optional): as for rmb_vi (batch included) except ms = 0, grid_ctas = 0, path = -1,
 * lanes_per_state = 0.
 */
#define RMB_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
int rmb_vi_noalloc(const rmb_mdp *mdp, const rmb_opts *opts, float *V_inout, int32_t *pi_out,
                   float *qgap_out, rmb_stats *stats, void *stream);

/*
 * Importance weights for RMB_SELECT_WEIGHTED from the Bellman residual (Sec. V suggests importance
 * sampling and epsilon-greedy selection of the batch states; the rule is the library's): one
 * Bellman pass at V gives r(s) = |TV(s) - V(s)| (float32, from TV and V as floats) and R = max r;
 *   weights_out[s] = floor(2^20 * (floor_frac + (1 - floor_frac) * r(s) / R))   (2^20 if R = 0),
 * so every state keeps probability >= floor_frac / (2^20 n) of the total when floor_frac > 0 (the
 * epsilon-greedy part) and the rest goes in proportion to the residual.
 *   V [n] float32, weights_out [n] uint32, device; floor_frac in [0, 1].
 *   workspace: rmb_residual_weights_workspace_bytes(mdp) bytes, 256-byte aligned.
 * Asynchronous on `stream`; argument errors return before any launch.  MDPs as for rmb_greedy.
 */
size_t rmb_residual_weights_workspace_bytes(const rmb_mdp *mdp);
int rmb_residual_weights(const rmb_mdp *mdp, const float *V, float floor_frac, uint32_t *weights_out,
                         void *workspace, size_t workspace_bytes, void *stream);

/*
 * MB-VI with importance-sampled batches (Sec. V suggests importance sampling and epsilon-greedy
 * selection of the batch states; the refresh rule is the library's): in rounds,
 *   weights = rmb_residual_weights(V, floor_frac);
 *   up to `refresh` sweeps of MB-VI whose batches are drawn with RMB_SELECT_WEIGHTED by those weights
 *   (the sweep counter of the draws runs on across rounds);
 * until a sweep's change <= opts->eps is confirmed by ||TV - V||_inf <= opts->eps (the stop rule of
 * draws), or opts->max_sweeps sweeps in all (then RMB_ERR_NOT_CONVERGED).  opts->select, weights,
 * residual_kind and trace are ignored; RMB_FLAG_ASYNC is unsupported.  refresh >= 1, floor_frac in
 * [0, 1].  V_inout, pi_out, qgap_out as for rmb_vi.
 *   workspace: rmb_vi_prioritized_workspace_bytes(mdp, opts) bytes, 256-byte aligned.
 * Synchronous: each round's status is read on the host.  stats (optional): sweeps in all,
 * iters = rounds, barriers in all, ms = device time of the whole call, the rest from the last round.
 */
size_t rmb_vi_prioritized_workspace_bytes(const rmb_mdp *mdp, const rmb_opts *opts);
int rmb_vi_prioritized(const rmb_mdp *mdp, const rmb_opts *opts, int32_t refresh, float floor_frac,
                       float *V_inout, int32_t *pi_out, float *qgap_out, void *workspace,
                       size_t workspace_bytes, rmb_stats *stats, void *stream);

/*
 * P(.|s,a) = softmax of the row's logits over its k successors (RMB_CSR with k_uniform = k > 0):
 * the parametrisation whose gradient rmb_fixed_point_grad returns.  logits, prob_out: [n*m*k], device.
 */
int rmb_softmax_rows(const rmb_mdp *mdp, const float *logits, float *prob_out, void *stream);

/* Workspace bytes of rmb_fixed_point_grad (0 on invalid arguments or non-uniform CSR rows). */
size_t rmb_fixed_point_grad_workspace_bytes(const rmb_mdp *mdp, const rmb_opts *opts);

/*
 * Gradient of L = w . V* with respect to the stage costs and the transition logits, through the
 * Bellman equation (eq. (5)) at the greedy policy pi (implicit function theorem, valid away from
 * action ties): V* = g_pi + gamma P_pi V*, so the adjoint lambda solves (I - gamma P_pi)^T lambda = w
 * and
 *   dL/dcost(s,a)    = lambda(s) [a = pi(s)],
 *   dL/dlogit(s,a,t) = gamma lambda(s) [a = pi(s)] p_t (V*(j_t) - sum_u p_u V*(j_u)).
 * lambda is computed by mini-batch sweeps (b = opts.batch >= 1, the permutation of opts.seed) of
 * lambda <- w + gamma P_pi^T lambda on the transposed greedy chain, built on the device (rows sorted
 * by predecessor, so the result is deterministic), starting from lambda = w, until the sup-norm
 * change of a sweep is <= opts.eps or opts.max_sweeps.  RMB_CSR with k_uniform > 0 only.
 *   pi [n] (the greedy policy of V*), V [n] (= V*), w [n]: device inputs.
 *   lambda_out [n]; grad_cost [n*m] or NULL; grad_logits [n*m*k] or NULL: device outputs.
 */
int rmb_fixed_point_grad(const rmb_mdp *mdp, const int32_t *pi, const float *V, const float *w,
                         const rmb_opts *opts, float *lambda_out, float *grad_cost, float *grad_logits,
                         void *workspace, size_t workspace_bytes, rmb_stats *stats, void *stream);

/*
 * Batched MB-VI: many independent MDPs (RMB_CSR) solved in one persistent launch (the paper has one
 * MDP per solve; this runs its MB-VI, eq. (11), on each).  A host-side autotuner picks every MDP's
 * batch size b (unless fixed) and the number of CTAs that solve it from a cost model.  MDPs solved by
 * a single CTA are taken at run time from one shared queue, longest estimate first, by whichever CTA
 * is free (a group's CTAs join once their MDP is solved); the workspace's first 4 bytes hold the
 * queue cursor, which rmb_batched_run resets.  Results per MDP are identical to rmb_vi with the same
 * b, seed and options and RMB_FLAG_NO_CLUSTER (the grid-wide solve, whose sums run in the same order).
 *
 * 1. rmb_batched_workspace_bytes(items, count, opts): workspace size for this plan.
 * 2. rmb_batched_plan(...): plans, writes the kernel parameters into the workspace (synchronous) and
 *    fills *handle (plain data; keep it with the workspace).  plan_out (host, [count]) may be NULL.
 * 3. rmb_batched_run(handle, stream): asynchronous solve of every MDP (capturable in a CUDA graph);
 *    rmb_batched_graph_create / _launch / _destroy capture it once and replay it.
 * 4. rmb_batched_results(handle, out[count], stream): waits, returns per-MDP stats and the first
 *    non-OK status.
 * Options: eps, max_sweeps, seed, start_sweep, barrier_timeout_ns and flags apply to every MDP.
 */
typedef struct {
    rmb_mdp mdp;           /* RMB_CSR */
    int64_t batch;         /* b for this MDP; 0 = autotuned */
    float *V;              /* [n] device: start values in, solution out */
    int32_t *pi;           /* [n] device greedy policy out, or NULL */
    float *qgap;           /* [n] device Q-gap out, or NULL */
} rmb_batch_item;

typedef struct {
    int64_t batch;         /* chosen b */
    int32_t group_ctas;    /* CTAs solving this MDP together (1 = alone: taken from a shared queue,
                              longest estimate first, by whichever CTA is free) */
    int32_t first_cta;     /* first CTA of the group; -1 for an MDP solved alone (queue) */
    double est_ms;         /* cost-model estimate of this MDP's solve time */
} rmb_batch_plan_item;

typedef struct {
    void *workspace;
    int32_t count, grid_ctas, ntasks, nqueue;   /* nqueue: single-CTA MDPs in the shared queue */
    int64_t ctrl_offset, kp_offset, toff_offset, tasks_offset;
    double est_ms;         /* cost-model makespan */
} rmb_batch_handle;

size_t rmb_batched_workspace_bytes(const rmb_batch_item *items, int count, const rmb_opts *opts);
int rmb_batched_plan(const rmb_batch_item *items, int count, const rmb_opts *opts, void *workspace,
                     size_t workspace_bytes, rmb_batch_handle *handle, rmb_batch_plan_item *plan_out,
                     void *stream);
int rmb_batched_run(const rmb_batch_handle *handle, void *stream);
int rmb_batched_results(const rmb_batch_handle *handle, rmb_stats *out, void *stream);
/* stream must be a created (non-default) stream; graph_exec receives a cudaGraphExec_t */
int rmb_batched_graph_create(const rmb_batch_handle *handle, void *stream, void **graph_exec);
int rmb_batched_graph_launch(void *graph_exec, void *stream);
int rmb_batched_graph_destroy(void *graph_exec);

/*
 * Row quantiser: codes[r][j] = round-to-nearest-even(P[r][j] / s_r) in p_dtype, with
 * s_r = max_j P[r][j] / F (F = 1 for bf16, 448 = the largest finite e4m3 value for fp8, so no code
 * saturates; a zero row gets s_r = 1), and row_scale[r] = 1 / sum_j decode(codes[r][j]) (float32
 * warp-order sum), the factor that turns decoded codes into the row's probabilities.
 * P [rows*cols] float32, codes [rows*cols] 2- or 1-byte elements, row_scale [rows] or NULL: device.
 */
int rmb_quantize_rows(const float *P, int64_t rows, int64_t cols, int32_t p_dtype, void *codes,
                      float *row_scale, void *stream);

/*
 * MB-VI with low-precision transition storage and float32 refinement: first MB-VI on `lowp`
 * (coded rows) until the sweep residual is <= eps_low (or opts.max_sweeps), then MB-VI sweeps on
 * `ref` (the same MDP with float32 rows) from those values until the residual is <= opts.eps; the
 * greedy policy and Q-gap come from the final float32 pass.  lowp and ref must agree in n, m, cost
 * and gamma.  stats_low / stats_ref (optional) receive each phase's results (then the call waits).
 */
int rmb_vi_refined(const rmb_mdp *lowp, const rmb_mdp *ref, const rmb_opts *opts, double eps_low,
                   float *V_inout, int32_t *pi_out, float *qgap_out, void *workspace,
                   size_t workspace_bytes, rmb_stats *stats_low, rmb_stats *stats_ref, void *stream);

/* Static text for a status code. */
const char *rmb_status_string(int status);

/* Number of kernels this library has launched in this process (all devices, all threads). */
uint64_t rmb_kernel_launches(void);

/* ABI version: (major << 16) | minor. */
int rmb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RMB_H */
