// librmb: the randomized mini-batch operator (Gargiani et al., Sec. III) and the VI / MPI /
// policy-evaluation schemes built on it, as persistent sm_103a kernels behind the C ABI of rmb.h.
//
// One launch runs a whole solve.  Every CTA walks the same sequence of phases and all control
// decisions (stop, re-centre) are taken from values every CTA reads after the same grid-wide wait,
// so the grid stays in step without host round trips.
//
// Mini-batch semantics (eq. (11)): within sweep k, positions [t*b, (t+1)*b) of the order
// sigma_{seed,k} form batch t; a state of batch t must read the new values of batches < t and the
// old values of every other state, its own batch included.  Two value buffers make that hold with
// one grid-wide wait per batch: batch t reads buffer A_t = d[(c+t)&1] and writes its new values
// into B_t = d[(c+t+1)&1], together with the new values of batch t-1 (kept in a small position-
// indexed cache), so that before batch t the buffer A_t holds exactly "batches < t new, rest old".
// At the end of a sweep with two or more batches the last batch is copied once more, so both
// buffers agree when the next sweep (with a new permutation) starts.
//
// Values are stored centred: V = mu + d with mu a double shared by the grid and d float32, so the
// float32 arithmetic works on differences of size ~ the spread of V instead of |V|.  With rows
// summing to 1, V'(s) = min_a [c + gamma sum p (mu + d)] gives d'(s) = min_a [c + gamma sum p d]
// - (1 - gamma) mu.  mu moves (and every d with it) only between sweeps, when the midpoint of the
// values drifts by more than a quarter of their spread.

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "rmb.h"
#include "rmb_device.cuh"

namespace rmb {

enum Mode { MODE_VI = 0, MODE_EVAL = 1, MODE_MPI = 2, MODE_GREEDY = 3 };
enum Path { PATH_DENSE = 0, PATH_CSR_VEC = 1, PATH_CSR_GEN = 2, PATH_DENSE_TMA = 3 };
enum Kind { K_MIN = 0, K_POLICY = 1, K_GREEDY = 2 };

constexpr int kCsrThreads = 512;
// cumulative weights of RMB_SELECT_WEIGHTED: tiles of 8192 weights (1024 threads x 8)
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanPer;
constexpr int kDenseThreads = 256;
constexpr int kDenseMaxM = 256;
constexpr int kDenseMB = 8;               // actions accumulated per pass in the dense path
constexpr int kDenseMaxStage = 40960;     // floats of V staged at once (160 KB of shared memory)

struct KP {
    // problem
    int n, m, k, path;
    int p_dtype;            // dense: RMB_P_F32 / RMB_P_BF16 / RMB_P_FP8E4M3
    const float* row_scale; // dense coded rows: 1 / (sum of the row's decoded codes), or null
    const void* P;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* prob;
    const float* cost;
    float gamma;
    double gamma_d;
    // schedule
    int mode, b, T, last_len, K;
    long long start_sweep, max_sweeps;
    double eps;
    uint32_t seed_lo, seed_hi, h;
    int lps_all, lps_one;   // CSR: lanes sharing one state (all actions / one row)
    int nc_all, nc_one;     // CSR vectorised: float4 chunks per lane per state (0 = general loop)
    int k4_log2;            // CSR vectorised: log2(k/4)
    int32_t* perm_buf;      // non-null when the order is precomputed (see use_perm_buf): that of the coming sweep
    int select;             // RMB_SELECT_*: sigma, or draws with replacement (uniform / by weight)
    int residual_kind;      // RMB_RESIDUAL_*: stop test of MB-VI (sweep change / confirmed Bellman residual)
    const uint64_t* cdf;    // RMB_SELECT_WEIGHTED: cumulative weights [n] (in the workspace)
    uint64_t* mark;         // draws with T >= 2: [2][n], mark[t & 1][s] = stamp of batch t if it updates s
    int stage;              // dense: floats of V staged per chunk
    // buffers
    const float* Vin;
    float* Vout;
    float* TVout;
    int32_t* pi;            // VI / MPI / greedy: policy output (MPI: also the evaluated policy)
    float* qgap;
    const int32_t* pi_in;   // evaluation: the policy
    float* d[2];
    int32_t* S[2];
    float* W[2];
    Ctrl* ctrl;
    double* trace;
    long long timeout_ns;
    int flags;
};

struct Best {
    float q;
    int a;
    float q2;
};

__device__ __forceinline__ Best better(const Best& x, const Best& y)
{
    const bool xf = (x.q < y.q) || (x.q == y.q && x.a < y.a);
    Best w = xf ? x : y;
    const float lq = xf ? y.q : x.q;
    w.q2 = fminf(w.q2, lq);
    return w;
}

template <bool ARG>
__device__ __forceinline__ Best shfl_xor_best(Best v, int off)
{
    Best o;
    o.q = __shfl_xor_sync(0xffffffffu, v.q, off);
    if (ARG) {
        o.a = __shfl_xor_sync(0xffffffffu, v.a, off);
        o.q2 = __shfl_xor_sync(0xffffffffu, v.q2, off);
    } else {
        o.a = 0;
        o.q2 = kInf;
    }
    return o;
}

__device__ __forceinline__ float gather(const float* __restrict__ A, int j, uint32_t nm1)
{
    // clamp keeps an unvalidated bad index inside the buffer (validation reports it).  The read
    // buffer does not change within a batch, and plain L1-cached loads issued after the grid-wide
    // barrier's acquire observe every value released before it, so the gathers may hit in L1.
    return __ldca(A + min((uint32_t)j, nm1));
}

// Q-factors of one state on the vectorised CSR path (every row has k entries, k % 4 == 0).
// `lps` lanes share the state: cpr lanes per row, each reading whole float4/int4 chunks; rows
// are combined with xor-shuffles.  Inactive groups still take part in the shuffles.
template <bool ARG>
__device__ __forceinline__ Best csr_vec_state(const KP& p, int s, int pi_s, bool act,
                                              const float* __restrict__ A, int lps, int lane_g)
{
    const int k4 = p.k >> 2;
    const int cpr = k4 < lps ? k4 : lps;
    const int cpl = k4 / cpr;
    const int rpi = lps / cpr;
    const int slot = lane_g / cpr, ch = lane_g - slot * cpr;
    const int nrows = pi_s >= 0 ? 1 : p.m;
    const uint32_t nm1 = (uint32_t)(p.n - 1);
    Best best = {kInf, 0x7fffffff, kInf};
    for (int a0 = 0; a0 < nrows; a0 += rpi) {
        const int ai = a0 + slot;
        const bool valid = act && ai < nrows;
        const int a = pi_s >= 0 ? pi_s : ai;
        const int64_t r = (int64_t)s * p.m + a;
        float part = 0.f;
        if (valid) {
            const float4* pr = reinterpret_cast<const float4*>(p.prob + r * p.k) + ch;
            const int4* cr = reinterpret_cast<const int4*>(p.col + r * p.k) + ch;
            for (int c = 0; c < cpl; ++c) {
                const float4 pv = __ldcs(pr + c * cpr);
                const int4 cv = __ldcs(cr + c * cpr);
                part = fmaf(pv.x, gather(A, cv.x, nm1), part);
                part = fmaf(pv.y, gather(A, cv.y, nm1), part);
                part = fmaf(pv.z, gather(A, cv.z, nm1), part);
                part = fmaf(pv.w, gather(A, cv.w, nm1), part);
            }
        }
        for (int off = 1; off < cpr; off <<= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        Best cur = {kInf, valid ? a : 0x7fffffff, kInf};
        if (valid) {
            const float c = __ldg(p.cost + r);
            cur.q = (c == kInf) ? kInf : fmaf(p.gamma, part, c);
        }
        for (int off = cpr; off < lps; off <<= 1) cur = better(cur, shfl_xor_best<ARG>(cur, off));
        best = better(best, cur);
    }
    return best;
}

// Q-factors of one state on the generic CSR path, walking each row in turn with the whole warp
// (states whose rows hold more than 32 entries, or m >= 32; the others take the one-pass form of
// gen_eval below).
template <bool ARG>
__device__ __forceinline__ Best csr_gen_state(const KP& p, int s, int pi_s, bool act,
                                              const float* __restrict__ A, int lane)
{
    const int nrows = pi_s >= 0 ? 1 : p.m;
    const uint32_t nm1 = (uint32_t)(p.n - 1);
    Best best = {kInf, 0x7fffffff, kInf};
    for (int ai = 0; ai < nrows; ++ai) {
        const int a = pi_s >= 0 ? pi_s : ai;
        const int64_t r = (int64_t)s * p.m + a;
        float part = 0.f;
        int64_t e0 = 0, e1 = 0;
        if (act) {
            e0 = __ldg(p.row_ptr + r);
            e1 = __ldg(p.row_ptr + r + 1);
        }
        for (int64_t e = e0 + lane; e < e1; e += 32)
            part = fmaf(__ldcs(p.prob + e), gather(A, __ldcs(p.col + e), nm1), part);
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        Best cur = {kInf, act ? a : 0x7fffffff, kInf};
        if (act) {
            const float c = __ldg(p.cost + r);
            cur.q = (c == kInf) ? kInf : fmaf(p.gamma, part, c);
        }
        best = better(best, cur);
    }
    return best;
}

struct Acc {
    float dmax, vlo, vhi;
};

struct Centre {
    double mu;
    float kap_hi, kap_lo;   // (1 - gamma) mu split in two floats
    float gmu;              // gamma * mu (float; only for TV output)
};

__device__ __forceinline__ Centre make_centre(double mu, double gamma)
{
    Centre c;
    c.mu = mu;
    const double kap = (1.0 - gamma) * mu;
    c.kap_hi = (float)kap;
    c.kap_lo = (float)(kap - (double)c.kap_hi);
    c.gmu = (float)(gamma * mu);
    return c;
}

__device__ __forceinline__ float new_value(float q, const Centre& C) { return (q - C.kap_hi) - C.kap_lo; }

// Per-state epilogue shared by the CSR and dense paths.
template <int KIND>
__device__ __forceinline__ void state_epilogue_old(const KP& p, const Best& r, int s, int i, float old, float* B,
                                                   int32_t* Sout, float* Wout, const Centre& C, Acc& acc);

template <int KIND>
__device__ __forceinline__ void state_epilogue(const KP& p, const Best& r, int s, int i, const float* A,
                                               float* B, int32_t* Sout, float* Wout, const Centre& C,
                                               Acc& acc)
{
    state_epilogue_old<KIND>(p, r, s, i, ld_l2(A + s), B, Sout, Wout, C, acc);
}

// the same with the state's value before the batch already loaded
template <int KIND>
__device__ __forceinline__ void state_epilogue_old(const KP& p, const Best& r, int s, int i, float old, float* B,
                                                   int32_t* Sout, float* Wout, const Centre& C, Acc& acc)
{
    const float v = new_value(r.q, C);
    if (v != v) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
    if (KIND == K_GREEDY) {
        acc.dmax = fmaxf(acc.dmax, fabsf(v - old));          // ||TV - V||_inf
        if (p.pi) st_l2(p.pi + s, r.a);
        if (p.qgap) p.qgap[s] = r.q2 - r.q;
        if (p.TVout) p.TVout[s] = (float)((double)r.q + p.gamma_d * C.mu);
        if (p.Vout) p.Vout[s] = (float)(C.mu + (double)old);
    } else {
        acc.dmax = fmaxf(acc.dmax, fabsf(v - old));
        acc.vlo = fminf(acc.vlo, v);
        acc.vhi = fmaxf(acc.vhi, v);
        if (Sout) {
            st_l2(Sout + i, s);
            st_l2(Wout + i, v);
        }
        st_l2(B + s, v);
    }
}

// ------------------------------------------------------------------------------------------------
// One batch (or, for K_GREEDY, the full state set in natural order) on the CSR paths.
// Unit = a group of lps lanes; position i of the batch goes to unit (i mod U), step (i div U).
// ------------------------------------------------------------------------------------------------
template <int KIND, bool VEC>
__device__ void csr_batch(const KP& p, const GroupView& gv, int lps, const float* __restrict__ A, float* B, int pos0,
                          int len, const PermKey* K, int32_t* Sout, float* Wout, const Centre& C, Acc& acc,
                          bool* perm_ok)
{
    constexpr bool ARG = (KIND == K_GREEDY);
    const int lane = threadIdx.x & 31;
    const int warp = (gv.rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
    const int nwarps = (gv.size * (int)blockDim.x) >> 5;
    const int spw = 32 / lps;
    const int g = lane / lps, lane_g = lane - g * lps;
    const int U = nwarps * spw;
    const int first = warp * spw;
    for (int j0 = 0; first + j0 * U < len; j0 += 32 / spw) {
        // each lane resolves the state of one (group, step) pair of the next 32/spw steps
        const int my_pos = first + (lane % spw) + (j0 + lane / spw) * U;
        int my_state = -1;
        if (my_pos < len) my_state = K ? state_at((uint32_t)(pos0 + my_pos), *K, perm_ok) : pos0 + my_pos;
        for (int jj = 0; jj < 32 / spw; ++jj) {
            const int j = j0 + jj;
            if (first + j * U >= len) break;
            const int s = __shfl_sync(0xffffffffu, my_state, jj * spw + g);
            const bool act = s >= 0;
            const int ss = act ? s : 0;
            const int pi_s = (KIND == K_POLICY)
                                 ? (act ? (int)min((uint32_t)ld_l2(p.pi_in ? p.pi_in + ss : p.pi + ss), (uint32_t)(p.m - 1)) : 0)
                                 : -1;
            const Best r = VEC ? csr_vec_state<ARG>(p, ss, pi_s, act, A, lps, lane_g)
                               : csr_gen_state<ARG>(p, ss, pi_s, act, A, lane);
            if (act && lane_g == 0) state_epilogue<KIND>(p, r, s, first + g + j * U, A, B, Sout, Wout, C, acc);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Generic CSR path (ragged rows), one warp per state, software-pipelined: while state j gathers its
// successor values and reduces, the entries of state j+1 and the row pointers of state j+2 load.
// The m rows of a state are contiguous; when they hold at most 32 entries in all (and m < 32), lane e
// holds entry e of the state, a segmented warp scan sums every row and the row ends combine to the
// minimum.  With a policy only that row's lanes load, at the same lanes and through the same scan,
// so T_pi and the improvement pass's Q-factor round identically.
// ------------------------------------------------------------------------------------------------
struct GenRegs {
    int s;          // state (-1: none); the same in every lane of the warp
    int pi_s;       // K_POLICY: its action, else -1
    long long rp;   // lane l <= m: start of row l (lane m: end of the last row)
    float c;        // lane l < m: cost of row l
    float pr;       // lane e: entry e of the state's rows (one-pass form)
    int col;
    bool has;       // this lane holds an entry
    bool has_old;   // old holds the state's value before the batch (loaded with the rows)
    float old;
};

// A: the batch's read buffer, or nullptr when its value may still change before the evaluation
// (across a barrier, or in place in an asynchronous sweep): the epilogue then loads it
template <int KIND>
__device__ __forceinline__ void gen_stage1(const KP& p, int s, int lane, GenRegs& R, const float* A)
{
    R.s = s;
    R.has_old = A != nullptr && s >= 0;
    R.old = R.has_old && lane == 0 ? ld_l2(A + s) : 0.f;
    R.pi_s = -1;
    R.rp = 0;
    R.c = kInf;
    R.pr = 0.f;
    R.col = 0;
    R.has = false;
    if (s < 0) return;
    if (KIND == K_POLICY) R.pi_s = (int)min((uint32_t)ld_l2(p.pi_in ? p.pi_in + s : p.pi + s), (uint32_t)(p.m - 1));
    if (p.m < 32) {
        const int64_t r0 = (int64_t)s * p.m;
        if (lane <= p.m) R.rp = __ldg(p.row_ptr + r0 + lane);
        if (lane < p.m) R.c = __ldg(p.cost + r0 + lane);
    }
}

__device__ __forceinline__ void gen_stage2(const KP& p, int lane, GenRegs& R)
{
    if (R.s < 0 || p.m >= 32) return;
    const long long E0 = __shfl_sync(0xffffffffu, R.rp, 0);
    const long long E1 = __shfl_sync(0xffffffffu, R.rp, p.m);
    if (E1 - E0 > 32) return;
    int lo = 0, hi = (int)(E1 - E0);
    if (R.pi_s >= 0) {
        lo = (int)(__shfl_sync(0xffffffffu, R.rp, R.pi_s) - E0);
        hi = (int)(__shfl_sync(0xffffffffu, R.rp, R.pi_s + 1) - E0);
    }
    if (lane >= lo && lane < hi) {
        R.pr = __ldcs(p.prob + E0 + lane);
        R.col = __ldcs(p.col + E0 + lane);
        R.has = true;
    }
}

template <bool ARG>
__device__ __forceinline__ Best gen_eval(const KP& p, const GenRegs& R, const float* __restrict__ A, int lane)
{
    Best cur = {kInf, 0x7fffffff, kInf};
    if (R.s < 0) return cur;
    if (p.m < 32) {
        const long long E0 = __shfl_sync(0xffffffffu, R.rp, 0);
        const long long E1 = __shfl_sync(0xffffffffu, R.rp, p.m);
        if (E1 - E0 <= 32) {
            const uint32_t nm1 = (uint32_t)(p.n - 1);
            const long long nxt = __shfl_down_sync(0xffffffffu, R.rp, 1);
            const int len = lane < p.m ? (int)(nxt - R.rp) : 0;
            uint32_t starts = len > 0 ? (1u << (int)(R.rp - E0)) : 0u;   // heads of non-empty rows
            for (int off = 16; off > 0; off >>= 1) starts |= __shfl_xor_sync(0xffffffffu, starts, off);
            float x = R.has ? R.pr * gather(A, R.col, nm1) : 0.f;
            // inclusive scan within rows: add the value d lanes down unless a row starts in between
            for (int d = 1; d < 32; d <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d && ((starts >> (lane - d + 1)) & ((1u << d) - 1u)) == 0u) x += y;
            }
            const float sum = __shfl_sync(0xffffffffu, x, len > 0 ? (int)(nxt - E0) - 1 : 0);
            if (R.pi_s >= 0 ? lane == R.pi_s : lane < p.m) {
                cur.a = lane;
                cur.q = (R.c == kInf) ? kInf : fmaf(p.gamma, len > 0 ? sum : 0.f, R.c);
            }
            for (int off = 16; off > 0; off >>= 1) cur = better(cur, shfl_xor_best<ARG>(cur, off));
            return cur;
        }
    }
    return csr_gen_state<ARG>(p, R.s, R.pi_s, true, A, lane);
}

struct GenCarry {
    GenRegs R0;         // first step of the warp: rows and entries loaded
    GenRegs R1;         // second step: rows loaded
    int block_states;   // this lane's state for step `lane` of the first block
    bool valid;
};

// the states of steps j0 .. j0+31 of this warp (lane L: step j0 + L)
__device__ __forceinline__ int gen_resolve(int warp, int U, int j0, int lane, int pos0, int len, const PermKey* K,
                                           bool* perm_ok)
{
    const int pos = warp + (j0 + lane) * U;
    if (pos >= len) return -1;
    return K ? state_at((uint32_t)(pos0 + pos), *K, perm_ok) : pos0 + pos;
}

// between the arrival at and the wait on a barrier: load this warp's first two steps of a batch
template <int KIND>
__device__ __forceinline__ void gen_prefetch_first(const KP& p, const GroupView& gv, int pos0, int len,
                                                   const PermKey* K, GenCarry& carry, bool* perm_ok)
{
    const int lane = threadIdx.x & 31;
    const int warp = (gv.rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
    const int U = (gv.size * (int)blockDim.x) >> 5;
    carry.valid = false;
    if (warp >= len) return;
    carry.block_states = gen_resolve(warp, U, 0, lane, pos0, len, K, perm_ok);
    gen_stage1<KIND>(p, __shfl_sync(0xffffffffu, carry.block_states, 0), lane, carry.R0, nullptr);
    gen_stage1<KIND>(p, __shfl_sync(0xffffffffu, carry.block_states, 1), lane, carry.R1, nullptr);
    gen_stage2(p, lane, carry.R0);
    carry.valid = true;
}

template <int KIND>
__device__ void csr_batch_gen(const KP& p, const GroupView& gv, const float* __restrict__ A, float* B, int pos0,
                              int len, const PermKey* K, int32_t* Sout, float* Wout, const Centre& C, Acc& acc,
                              bool* perm_ok, GenCarry& carry)
{
    constexpr bool ARG = (KIND == K_GREEDY);
    const int lane = threadIdx.x & 31;
    const int warp = (gv.rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
    const int U = (gv.size * (int)blockDim.x) >> 5;
    if (warp >= len) { carry.valid = false; return; }
    // the old values can load with the rows unless the batch writes where it reads (asynchronous)
    const float* Aold = (A == B) ? nullptr : A;
    int block_states;
    GenRegs r0, r1, r2;
    if (carry.valid) {
        block_states = carry.block_states;
        r0 = carry.R0;
        r1 = carry.R1;
    } else {
        block_states = gen_resolve(warp, U, 0, lane, pos0, len, K, perm_ok);
        gen_stage1<KIND>(p, __shfl_sync(0xffffffffu, block_states, 0), lane, r0, Aold);
        gen_stage1<KIND>(p, __shfl_sync(0xffffffffu, block_states, 1), lane, r1, Aold);
        gen_stage2(p, lane, r0);
    }
    carry.valid = false;
    for (int j = 0; warp + j * U < len; ++j) {
        const int j2 = j + 2;
        int s2 = -1;
        if (warp + j2 * U < len) {
            if ((j2 & 31) == 0) block_states = gen_resolve(warp, U, j2, lane, pos0, len, K, perm_ok);
            s2 = __shfl_sync(0xffffffffu, block_states, j2 & 31);
        }
        gen_stage1<KIND>(p, s2, lane, r2, Aold);
        gen_stage2(p, lane, r1);
        const Best r = gen_eval<ARG>(p, r0, A, lane);
        if (r0.s >= 0 && lane == 0)
            state_epilogue_old<KIND>(p, r, r0.s, warp + j * U, r0.has_old ? r0.old : ld_l2(A + r0.s), B, Sout,
                                     Wout, C, acc);
        r0 = r1;
        r1 = r2;
    }
}

// ------------------------------------------------------------------------------------------------
// Fast CSR path (k/4 <= lanes per state, at most 4 float4 chunks per lane and state).  Every lane
// loads all its chunks of a state at once, and the next state's rows are prefetched while the
// current state's successor gathers resolve.  The first state of the next batch is prefetched
// between the arrival at and the wait on the grid-wide barrier (its rows and position in the
// permutation do not depend on the values being written), so small batches do not pay the
// permutation and HBM latency after every barrier.
// ------------------------------------------------------------------------------------------------
template <int NC>
struct StateRegs {
    float4 p[NC];
    int4 c[NC];
    float cost[NC];
};

template <int NC>
struct Carry {
    StateRegs<NC> R;
    int block_states;   // this lane's state for (group, step) of the first permutation block
    int s;              // the group's first state (-1 = none)
    bool valid;
};

template <int KIND, int NC>
__device__ __forceinline__ void fast_load(const KP& p, int s, bool act, int lps, int lane_g, StateRegs<NC>& R)
{
    int pi_s = -1;
    if (KIND == K_POLICY && act)
        pi_s = (int)min((uint32_t)ld_l2(p.pi_in ? p.pi_in + s : p.pi + s), (uint32_t)(p.m - 1));
    const int total = (KIND == K_POLICY ? 1 : p.m) << p.k4_log2;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int ci = c * lps + lane_g;
        const bool v = act && ci < total;
        const int row = ci >> p.k4_log2;
        const int ch = ci - (row << p.k4_log2);
        const int a = KIND == K_POLICY ? pi_s : row;
        const int64_t r = (int64_t)s * p.m + a;
        if (v) {
            R.p[c] = __ldcs(reinterpret_cast<const float4*>(p.prob + r * p.k) + ch);
            R.c[c] = __ldcs(reinterpret_cast<const int4*>(p.col + r * p.k) + ch);
            R.cost[c] = __ldg(p.cost + r);
        } else {
            R.p[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            R.c[c] = make_int4(0, 0, 0, 0);
            R.cost[c] = kInf;
        }
    }
}

// min (and, with ARG, the lowest arg-min and the second smallest value) over the state's rows of
// c + gamma * sum p * A[col]; every lane of the group gets the result
template <bool ARG, int NC>
__device__ __forceinline__ Best fast_eval(const KP& p, const StateRegs<NC>& R, const float* __restrict__ A, int lps,
                                          int lane_g)
{
    const uint32_t nm1 = (uint32_t)(p.n - 1);
    float part[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float g0 = gather(A, R.c[c].x, nm1), g1 = gather(A, R.c[c].y, nm1);
        const float g2 = gather(A, R.c[c].z, nm1), g3 = gather(A, R.c[c].w, nm1);
        part[c] = fmaf(R.p[c].x, g0, fmaf(R.p[c].y, g1, fmaf(R.p[c].z, g2, R.p[c].w * g3)));
    }
    const int k4 = 1 << p.k4_log2;
    for (int off = 1; off < k4; off <<= 1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) part[c] += __shfl_xor_sync(0xffffffffu, part[c], off);
    }
    Best b = {kInf, 0x7fffffff, kInf};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float q = R.cost[c] == kInf ? kInf : fmaf(p.gamma, part[c], R.cost[c]);
        if (ARG) b = better(b, Best{q, (c * lps + lane_g) >> p.k4_log2, kInf});
        else b.q = fminf(b.q, q);
    }
    for (int off = k4; off < lps; off <<= 1) {
        if (ARG) b = better(b, shfl_xor_best<true>(b, off));
        else b.q = fminf(b.q, __shfl_xor_sync(0xffffffffu, b.q, off));
    }
    return b;
}

struct FastGeom {
    int lane, spw, per_block, g, lane_g, U, first, my_off, my_step;
    __device__ FastGeom(int lps, const GroupView& gv)
    {
        lane = threadIdx.x & 31;
        const int warp = (gv.rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
        const int nwarps = (gv.size * (int)blockDim.x) >> 5;
        spw = 32 / lps;
        per_block = 32 / spw;          // steps covered by one permutation evaluation per lane
        g = lane / lps;
        lane_g = lane - g * lps;
        U = nwarps * spw;
        first = warp * spw;
        my_off = first + (lane % spw);
        my_step = lane / spw;
    }
    __device__ int resolve(int j0, int pos0, int len, const PermKey* K, bool* ok) const
    {
        const int pos = my_off + (j0 + my_step) * U;
        if (pos >= len) return -1;
        return K ? state_at((uint32_t)(pos0 + pos), *K, ok) : pos0 + pos;
    }
};

// resolve and load this warp's first state of a batch ahead of time
template <int KIND, int NC>
__device__ __forceinline__ void fast_prefetch_first(const KP& p, const GroupView& gv, int lps, int pos0, int len,
                                                    const PermKey* K, Carry<NC>& carry, bool* perm_ok)
{
    const FastGeom G(lps, gv);
    carry.valid = false;
    if (G.first >= len) return;
    carry.block_states = G.resolve(0, pos0, len, K, perm_ok);
    carry.s = __shfl_sync(0xffffffffu, carry.block_states, G.g);
    fast_load<KIND, NC>(p, carry.s < 0 ? 0 : carry.s, carry.s >= 0, lps, G.lane_g, carry.R);
    carry.valid = true;
}

template <int KIND, int NC>
__device__ void csr_batch_fast(const KP& p, const GroupView& gv, int lps, const float* __restrict__ A, float* B,
                               int pos0, int len, const PermKey* K, int32_t* Sout, float* Wout, const Centre& C,
                               Acc& acc, bool* perm_ok, Carry<NC>& carry)
{
    constexpr bool ARG = (KIND == K_GREEDY);
    constexpr int LK = (KIND == K_POLICY) ? K_POLICY : K_MIN;   // which rows to load
    const FastGeom G(lps, gv);
    if (G.first >= len) { carry.valid = false; return; }
    int block_states, s_cur;
    StateRegs<NC> cur, nxt;
    if (carry.valid) {
        block_states = carry.block_states;
        s_cur = carry.s;
        cur = carry.R;
    } else {
        block_states = G.resolve(0, pos0, len, K, perm_ok);
        s_cur = __shfl_sync(0xffffffffu, block_states, G.g);
        fast_load<LK, NC>(p, s_cur < 0 ? 0 : s_cur, s_cur >= 0, lps, G.lane_g, cur);
    }
    carry.valid = false;
    for (int j = 0; G.first + j * G.U < len; ++j) {
        const int jn = j + 1;
        int s_nxt = -1;
        if (G.first + jn * G.U < len) {
            if (jn % G.per_block == 0) block_states = G.resolve(jn, pos0, len, K, perm_ok);
            s_nxt = __shfl_sync(0xffffffffu, block_states, (jn % G.per_block) * G.spw + G.g);
        }
        fast_load<LK, NC>(p, s_nxt < 0 ? 0 : s_nxt, s_nxt >= 0, lps, G.lane_g, nxt);
        const bool lead = s_cur >= 0 && G.lane_g == 0;
        const float old = lead ? ld_l2(A + s_cur) : 0.f;
        const Best r = fast_eval<ARG, NC>(p, cur, A, lps, G.lane_g);
        if (lead) {
            const float v = new_value(r.q, C);
            if (v != v) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
            acc.dmax = fmaxf(acc.dmax, fabsf(v - old));
            if (KIND == K_GREEDY) {
                if (p.pi) st_l2(p.pi + s_cur, r.a);
                if (p.qgap) p.qgap[s_cur] = r.q2 - r.q;
                if (p.TVout) p.TVout[s_cur] = (float)((double)r.q + p.gamma_d * C.mu);
                if (p.Vout) p.Vout[s_cur] = (float)(C.mu + (double)old);
            } else {
                acc.vlo = fminf(acc.vlo, v);
                acc.vhi = fmaxf(acc.vhi, v);
                const int i = G.first + G.g + j * G.U;
                if (Sout) {
                    st_l2(Sout + i, s_cur);
                    st_l2(Wout + i, v);
                }
                st_l2(B + s_cur, v);
            }
        }
        cur = nxt;
        s_cur = s_nxt;
    }
}

// ------------------------------------------------------------------------------------------------
// Dense path: one CTA per state, the current values staged in shared memory by a bulk async copy.
// ------------------------------------------------------------------------------------------------
struct DenseSmem {
    uint64_t mbar;
    uint32_t phase;
    int ok;
    float red[kDenseThreads / 32][kDenseMB];
    float red2[kDenseThreads / 32][kDenseMB];
    float q[kDenseMaxM];
    int perm[32];
};

__device__ __forceinline__ int try_wait_bounded(uint32_t mb, uint32_t parity, long long timeout_ns)
{
    uint32_t done = 0, spins = 0;
    const uint64_t t0 = globaltimer_ns();
    while (!done) {
        asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                     : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (!done && (++spins & 63u) == 0 && (int64_t)(globaltimer_ns() - t0) > timeout_ns) return 0;
    }
    return 1;
}

// bulk copy of nfl floats into shared memory (issued by thread 0); stage_wait completes it
__device__ __forceinline__ void stage_issue(DenseSmem& sm, float* dst, const float* src, int nfl)
{
    // nfl is a multiple of 4 floats (16 bytes), src and dst 16-byte aligned
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const uint32_t bytes = (uint32_t)nfl * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(d), "l"(src), "r"(bytes), "r"(mb) : "memory");
    }
}

// every thread of the CTA: wait (bounded) for the copy issued by stage_issue
__device__ __forceinline__ bool stage_wait(const KP& p, DenseSmem& sm)
{
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
    const uint32_t parity = sm.phase & 1u;
    if (threadIdx.x == 0) {
        // bounded wait; after a timeout wait (bounded again) for the copy in flight to land
        int ok = try_wait_bounded(mb, parity, p.timeout_ns);
        if (!ok) {
            atomicCAS(&p.ctrl->error, 0, RMB_ERR_BARRIER_TIMEOUT);
            try_wait_bounded(mb, parity, p.timeout_ns);
        }
        sm.ok = ok;
    }
    __syncthreads();
    const bool ok = sm.ok != 0;
    if (ok && threadIdx.x != 0) try_wait_bounded(mb, parity, p.timeout_ns);   // completes at once
    __syncthreads();
    if (threadIdx.x == 0) sm.phase++;
    return ok;
}

__device__ __forceinline__ bool stage_values(const KP& p, DenseSmem& sm, float* dst, const float* src, int nfl)
{
    stage_issue(sm, dst, src, nfl);
    return stage_wait(p, sm);
}

// Dense row elements: float32, or bf16 / fp8-e4m3 codes.  Coded rows are renormalised by the sum of
// their decoded entries (the per-row scale cancels), so a decoded row is an exact distribution and
// gamma * row sum never exceeds gamma.
template <int DT>
struct Elem {
    static constexpr int bytes = DT == RMB_P_F32 ? 4 : (DT == RMB_P_BF16 ? 2 : 1);
    static constexpr int per16 = 16 / bytes;   // elements in one 16-byte load
};

template <int DT>
__device__ __forceinline__ void decode16(const uint4 w, float* d)
{
    if (DT == RMB_P_F32) {
        d[0] = __uint_as_float(w.x);
        d[1] = __uint_as_float(w.y);
        d[2] = __uint_as_float(w.z);
        d[3] = __uint_as_float(w.w);
    } else if (DT == RMB_P_BF16) {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            d[2 * i] = __uint_as_float(u[i] << 16);
            d[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
        }
    } else {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u[i] & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u[i] >> 16), __NV_E4M3);
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
            d[4 * i] = a.x;
            d[4 * i + 1] = a.y;
            d[4 * i + 2] = b.x;
            d[4 * i + 3] = b.y;
        }
    }
}

template <int DT>
__device__ __forceinline__ float decode1(const unsigned char* row, int64_t j)
{
    if (DT == RMB_P_F32) return __ldcs(reinterpret_cast<const float*>(row) + j);
    if (DT == RMB_P_BF16) return __uint_as_float((uint32_t)__ldcs(reinterpret_cast<const unsigned short*>(row) + j) << 16);
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)__ldcs(reinterpret_cast<const unsigned char*>(row) + j),
                                                __NV_E4M3);
    return __half2float(*reinterpret_cast<const __half*>(&h));
}

template <int KIND, int DT, bool VEC>
__device__ Best dense_state(const KP& p, DenseSmem& sm, float* stage, bool whole, const float* A, int s,
                            int pi_s, bool* ok)
{
    constexpr int EB = Elem<DT>::bytes;
    constexpr int E = Elem<DT>::per16;
    // coded rows are normalised by the decoded row sum: read from row_scale when the quantiser
    // stored it, accumulated here otherwise
    const bool NORM = DT != RMB_P_F32 && p.row_scale == nullptr;
    const int n = p.n;
    const int nrows = pi_s >= 0 ? 1 : p.m;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned char* P = static_cast<const unsigned char*>(p.P);
    for (int a0 = 0; a0 < nrows; a0 += kDenseMB) {
        float acc[kDenseMB], sum[kDenseMB];
#pragma unroll
        for (int u = 0; u < kDenseMB; ++u) acc[u] = sum[u] = 0.f;
        const unsigned char* rows[kDenseMB];
#pragma unroll
        for (int u = 0; u < kDenseMB; ++u) {
            const int a = pi_s >= 0 ? pi_s : min(a0 + u, p.m - 1);
            rows[u] = P + ((int64_t)s * p.m + a) * (int64_t)n * EB;
        }
        for (int c0 = 0; c0 < n; c0 += p.stage) {
            const int clen = min(p.stage, n - c0);
            if (!whole) {
                __syncthreads();
                if (!stage_values(p, sm, stage, A + c0, (clen + 3) & ~3)) { *ok = false; return Best{kInf, 0, kInf}; }
            }
            if (VEC) {
                for (int jv = tid; jv < clen / E; jv += blockDim.x) {
                    float v[E];
#pragma unroll
                    for (int q = 0; q < E / 4; ++q) {
                        const float4 f = reinterpret_cast<const float4*>(stage)[jv * (E / 4) + q];
                        v[4 * q] = f.x;
                        v[4 * q + 1] = f.y;
                        v[4 * q + 2] = f.z;
                        v[4 * q + 3] = f.w;
                    }
#pragma unroll
                    for (int u = 0; u < kDenseMB; ++u) {
                        if (a0 + u < nrows) {
                            const uint4 w = __ldcs(reinterpret_cast<const uint4*>(rows[u] + (int64_t)c0 * EB) + jv);
                            float d[E];
                            decode16<DT>(w, d);
                            // two partial chains per row (even / odd entries) keep the FMA chains short
                            float x0 = 0.f, x1 = 0.f;
#pragma unroll
                            for (int e = 0; e < E; e += 2) {
                                x0 = fmaf(d[e], v[e], x0);
                                x1 = fmaf(d[e + 1], v[e + 1], x1);
                            }
                            acc[u] += x0 + x1;
                            if (NORM) {
                                float y0 = 0.f, y1 = 0.f;
#pragma unroll
                                for (int e = 0; e < E; e += 2) {
                                    y0 += d[e];
                                    y1 += d[e + 1];
                                }
                                sum[u] += y0 + y1;
                            }
                        }
                    }
                }
            } else {
                for (int j = tid; j < clen; j += blockDim.x) {
                    const float v = stage[j];
#pragma unroll
                    for (int u = 0; u < kDenseMB; ++u) {
                        if (a0 + u < nrows) {
                            const float d = decode1<DT>(rows[u], c0 + j);
                            acc[u] = fmaf(d, v, acc[u]);
                            if (NORM) sum[u] += d;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kDenseMB; ++u) {
            float x = acc[u], y = sum[u];
            for (int off = 16; off > 0; off >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, off);
                if (NORM) y += __shfl_xor_sync(0xffffffffu, y, off);
            }
            if (lane == 0) {
                sm.red[wid][u] = x;
                sm.red2[wid][u] = y;
            }
        }
        __syncthreads();
        if (tid < kDenseMB && a0 + tid < nrows) {
            float tot = 0.f, tsum = 0.f;
            for (int w = 0; w < nw; ++w) {
                tot += sm.red[w][tid];
                tsum += sm.red2[w][tid];
            }
            const int a = pi_s >= 0 ? pi_s : a0 + tid;
            if (NORM) tot = tsum > 0.f ? tot / tsum : 0.f;
            else if (DT != RMB_P_F32) tot *= __ldg(p.row_scale + (int64_t)s * p.m + a);
            const float c = __ldg(p.cost + (int64_t)s * p.m + a);
            sm.q[a0 + tid] = (c == kInf) ? kInf : fmaf(p.gamma, tot, c);
        }
        __syncthreads();
    }
    Best best = {kInf, 0x7fffffff, kInf};
    if (tid == 0) {
        for (int ai = 0; ai < nrows; ++ai) {
            const Best cur = {sm.q[ai], pi_s >= 0 ? pi_s : ai, kInf};
            best = better(best, cur);
        }
    }
    return best;
}

template <int KIND, int DT, bool VEC>
__device__ bool dense_batch(const KP& p, const GroupView& gv, DenseSmem& sm, float* stage, const float* A, float* B,
                            int pos0, int len, const PermKey* K, int32_t* Sout, float* Wout, const Centre& C,
                            Acc& acc, bool* perm_ok)
{
    const bool whole = p.n <= p.stage;
    const int G = gv.size;
    const int me = gv.rank;
    if (me >= len) return true;
    bool ok = true;
    if (whole && !stage_values(p, sm, stage, A, (p.n + 3) & ~3)) return false;
    for (int j0 = 0; me + j0 * G < len; j0 += 32) {
        __syncthreads();
        if (threadIdx.x < 32) {
            const int pos = me + (j0 + (int)threadIdx.x) * G;
            int st = -1;
            if (pos < len) st = K ? state_at((uint32_t)(pos0 + pos), *K, perm_ok) : pos0 + pos;
            sm.perm[threadIdx.x] = st;
        }
        __syncthreads();
        for (int jj = 0; jj < 32; ++jj) {
            const int s = sm.perm[jj];
            if (s < 0) break;
            const int pi_s = (KIND == K_POLICY)
                                 ? (int)min((uint32_t)ld_l2(p.pi_in ? p.pi_in + s : p.pi + s), (uint32_t)(p.m - 1))
                                 : -1;
            const Best r = dense_state<KIND, DT, VEC>(p, sm, stage, whole, A, s, pi_s, &ok);
            if (!ok) return false;
            if (threadIdx.x == 0)
                state_epilogue<KIND>(p, r, s, me + (j0 + jj) * G, A, B, Sout, Wout, C, acc);
        }
    }
    return true;
}

// ------------------------------------------------------------------------------------------------
// Dense path with a TMA pipeline: one producer warp streams the transition rows of the CTA's states,
// row group by row group and column tile by column tile, into a ring of shared-memory stages with
// cp.async.bulk (mbarrier transaction counts); eight consumer warps decode them and multiply with the
// current values, staged once per batch.  Memory-level parallelism is the ring (kRingStages x
// kStageBytes per SM), not registers, so coded rows (bf16 / fp8) stream as fast as float32 rows.
// Every wait is bounded; after a timeout all threads still pass the same barriers (abort flag).
// ------------------------------------------------------------------------------------------------
constexpr int kTmaConsumers = 8;                    // consumer warps
constexpr int kTmaThreads = (kTmaConsumers + 1) * 32;
constexpr int kRingStages = 4;
constexpr int kStageBytes = 32768;
constexpr int kTmaRowGroup = 8;                     // rows per stage (all-action passes)
constexpr int kTmaMaxStates = 512;                  // states per chunk of a batch

struct TmaSmem {
    uint64_t full[kRingStages];
    uint64_t empty[kRingStages];
    uint64_t vbar;
    uint32_t vphase;
    int abort;
    int ids[kTmaMaxStates];
    int pis[kTmaMaxStates];
    float red[kTmaConsumers][kTmaRowGroup];
    float q[kDenseMaxM];
};

__device__ __forceinline__ bool mb_try(uint32_t mb, uint32_t parity)
{
    uint32_t done;
    asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                 : "=r"(done) : "r"(mb), "r"(parity) : "memory");
    return done != 0;
}

// bounded wait; returns false (and raises the abort flag and the error) on timeout or abort
__device__ __forceinline__ bool mb_wait(uint32_t mb, uint32_t parity, const KP& p, volatile int* abort_flag)
{
    if (*abort_flag) return false;
    const uint64_t t0 = globaltimer_ns();
    uint32_t spins = 0;
    while (!mb_try(mb, parity)) {
        if ((++spins & 63u) == 0) {
            if (*abort_flag) return false;
            if ((int64_t)(globaltimer_ns() - t0) > p.timeout_ns) {
                *abort_flag = 1;
                atomicCAS(&p.ctrl->error, 0, RMB_ERR_BARRIER_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTmaConsumers * 32) : "memory"); }

template <int KIND, int DT>
__device__ bool dense_batch_tma(const KP& p, const GroupView& gv, TmaSmem& sm, float* vst, unsigned char* ring,
                                uint32_t& ring_it, const float* A, float* B, int pos0, int len, const PermKey* K,
                                int32_t* Sout, float* Wout, const Centre& C, Acc& acc, bool* perm_ok)
{
    constexpr int EB = Elem<DT>::bytes;
    constexpr int E = Elem<DT>::per16;
    const int n = p.n;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const bool producer = wid == kTmaConsumers;
    const int RG = KIND == K_POLICY ? 1 : kTmaRowGroup;
    const int nrows = KIND == K_POLICY ? 1 : p.m;
    const int TC = min(n, (kStageBytes / (RG * EB)) & ~15);       // columns per tile
    const int ntiles = (n + TC - 1) / TC;
    const int ngroups = (nrows + RG - 1) / RG;
    const int G = gv.size, me = gv.rank;
    if (me >= len) return true;
    volatile int* abort_flag = &sm.abort;
    // stage the current values once per batch (bulk copy into this CTA's shared memory)
    const uint32_t vb = (uint32_t)__cvta_generic_to_shared(&sm.vbar);
    if (tid == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const uint32_t bytes = (uint32_t)((n + 3) & ~3) * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vb), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"((uint32_t)__cvta_generic_to_shared(vst)), "l"(A), "r"(bytes), "r"(vb) : "memory");
    }
    const bool v_ok = mb_wait(vb, sm.vphase & 1u, p, abort_flag);
    __syncthreads();
    if (tid == 0) sm.vphase++;
    if (!v_ok || *abort_flag) return false;
    const unsigned char* P = static_cast<const unsigned char*>(p.P);
    const int total = (len - me + G - 1) / G;                     // this CTA's states in the batch
    for (int c0 = 0; c0 < total; c0 += kTmaMaxStates) {
        const int cnt = min(kTmaMaxStates, total - c0);
        __syncthreads();
        for (int i = tid; i < cnt; i += blockDim.x) {
            const int pos = me + (c0 + i) * G;
            const int st = K ? state_at((uint32_t)(pos0 + pos), *K, perm_ok) : pos0 + pos;
            sm.ids[i] = st;
            sm.pis[i] = KIND == K_POLICY
                            ? (int)min((uint32_t)ld_l2(p.pi_in ? p.pi_in + st : p.pi + st), (uint32_t)(p.m - 1))
                            : 0;
        }
        __syncthreads();
        if (producer) {
            if (lane == 0) {
                uint32_t it = ring_it;
                for (int i = 0; i < cnt; ++i) {
                    const int s = sm.ids[i];
                    for (int g = 0; g < ngroups; ++g) {
                        const int a0 = g * RG;
                        const int rg = min(RG, nrows - a0);
                        for (int t = 0; t < ntiles; ++t, ++it) {
                            const int slot = it % kRingStages;
                            const uint32_t use = it / kRingStages;
                            const uint32_t fb = (uint32_t)__cvta_generic_to_shared(&sm.full[slot]);
                            if (use > 0 && !mb_wait((uint32_t)__cvta_generic_to_shared(&sm.empty[slot]), (use - 1) & 1u, p,
                                                    abort_flag))
                                continue;
                            const int width = min(TC, n - t * TC);
                            const uint32_t bytes = (uint32_t)(rg * width * EB);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes)
                                         : "memory");
                            unsigned char* dst = ring + (size_t)slot * kStageBytes;
                            for (int r = 0; r < rg; ++r) {
                                const int a = KIND == K_POLICY ? sm.pis[i] : a0 + r;
                                const unsigned char* src = P + (((int64_t)s * p.m + a) * n + (int64_t)t * TC) * EB;
                                asm volatile(
                                    "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                    ::"r"((uint32_t)__cvta_generic_to_shared(dst + (size_t)r * width * EB)), "l"(src),
                                    "r"((uint32_t)(width * EB)), "r"(fb) : "memory");
                            }
                        }
                    }
                }
                // on abort, let the copies already issued land before the CTA moves on
                if (*abort_flag) {
                    const uint32_t first = it > (uint32_t)kRingStages ? it - kRingStages : 0u;
                    for (uint32_t k = first; k < it; ++k) {
                        const uint32_t fb = (uint32_t)__cvta_generic_to_shared(&sm.full[k % kRingStages]);
                        const uint64_t t0 = globaltimer_ns();
                        while (!mb_try(fb, (k / kRingStages) & 1u) &&
                               (int64_t)(globaltimer_ns() - t0) < p.timeout_ns) {
                        }
                    }
                }
            }
        } else {
            uint32_t it = ring_it;
            for (int i = 0; i < cnt; ++i) {
                const int s = sm.ids[i];
                for (int g = 0; g < ngroups; ++g) {
                    const int a0 = g * RG;
                    const int rg = min(RG, nrows - a0);
                    float accv[kTmaRowGroup];
#pragma unroll
                    for (int r = 0; r < kTmaRowGroup; ++r) accv[r] = 0.f;
                    for (int t = 0; t < ntiles; ++t, ++it) {
                        const int slot = it % kRingStages;
                        const bool ok = mb_wait((uint32_t)__cvta_generic_to_shared(&sm.full[slot]),
                                                (it / kRingStages) & 1u, p, abort_flag);
                        if (ok) {
                            const int width = min(TC, n - t * TC);
                            const unsigned char* st = ring + (size_t)slot * kStageBytes;
                            const float* vt = vst + (size_t)t * TC;
                            for (int jv = tid; jv < width / E; jv += kTmaConsumers * 32) {
                                float v[E];
#pragma unroll
                                for (int q = 0; q < E / 4; ++q) {
                                    const float4 f = reinterpret_cast<const float4*>(vt)[jv * (E / 4) + q];
                                    v[4 * q] = f.x;
                                    v[4 * q + 1] = f.y;
                                    v[4 * q + 2] = f.z;
                                    v[4 * q + 3] = f.w;
                                }
#pragma unroll
                                for (int r = 0; r < kTmaRowGroup; ++r) {
                                    if (r < rg) {
                                        const uint4 w = reinterpret_cast<const uint4*>(st + (size_t)r * width * EB)[jv];
                                        float d[E];
                                        decode16<DT>(w, d);
                                        float x0 = 0.f, x1 = 0.f;
#pragma unroll
                                        for (int e = 0; e < E; e += 2) {
                                            x0 = fmaf(d[e], v[e], x0);
                                            x1 = fmaf(d[e + 1], v[e + 1], x1);
                                        }
                                        accv[r] += x0 + x1;
                                    }
                                }
                            }
                        }
                        __syncwarp();
                        if (lane == 0 && ok)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                                         ::"r"((uint32_t)__cvta_generic_to_shared(&sm.empty[slot])) : "memory");
                    }
                    // row sums over the consumer warps
#pragma unroll
                    for (int r = 0; r < kTmaRowGroup; ++r) {
                        float x = accv[r];
                        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                        if (lane == 0) sm.red[wid][r] = x;
                    }
                    consumer_sync();
                    if (tid < rg) {
                        float tot = 0.f;
                        for (int w = 0; w < kTmaConsumers; ++w) tot += sm.red[w][tid];
                        const int a = KIND == K_POLICY ? sm.pis[i] : a0 + tid;
                        const int64_t r = (int64_t)s * p.m + a;
                        if (DT != RMB_P_F32) tot *= __ldg(p.row_scale + r);
                        const float c = __ldg(p.cost + r);
                        sm.q[KIND == K_POLICY ? 0 : a0 + tid] = (c == kInf) ? kInf : fmaf(p.gamma, tot, c);
                    }
                    consumer_sync();
                }
                if (tid == 0 && !*abort_flag) {
                    Best best = {kInf, 0x7fffffff, kInf};
                    for (int ai = 0; ai < nrows; ++ai)
                        best = better(best, Best{sm.q[ai], KIND == K_POLICY ? sm.pis[i] : ai, kInf});
                    state_epilogue<KIND>(p, best, s, me + (c0 + i) * G, A, B, Sout, Wout, C, acc);
                }
            }
        }
        // every thread advances the ring counter by the tiles of this chunk
        ring_it += (uint32_t)(cnt * ngroups * ntiles);
    }
    __syncthreads();
    return *abort_flag == 0;
}

// ------------------------------------------------------------------------------------------------
// The persistent driver.
// ------------------------------------------------------------------------------------------------
struct RedSmem {
    float v[3][32];
    float bc[4];
};

__device__ __forceinline__ void publish(Ctrl* c, int slot, Acc a, RedSmem& rs)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        a.dmax = fmaxf(a.dmax, __shfl_xor_sync(0xffffffffu, a.dmax, off));
        a.vlo = fminf(a.vlo, __shfl_xor_sync(0xffffffffu, a.vlo, off));
        a.vhi = fmaxf(a.vhi, __shfl_xor_sync(0xffffffffu, a.vhi, off));
    }
    __syncthreads();
    if (lane == 0) {
        rs.v[0][wid] = a.dmax;
        rs.v[1][wid] = a.vlo;
        rs.v[2][wid] = a.vhi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {   // thread 0 already holds warp 0's values
            a.dmax = fmaxf(a.dmax, rs.v[0][w]);
            a.vlo = fminf(a.vlo, rs.v[1][w]);
            a.vhi = fmaxf(a.vhi, rs.v[2][w]);
        }
        atomicMax(&c->red_delta[slot], __float_as_uint(a.dmax));
        atomicMax(&c->red_hi[slot], okey(a.vhi));
        atomicMax(&c->red_nlo[slot], okey(-a.vlo));
    }
}

// read a reduction slot after a grid-wide wait; every thread of the CTA gets the same values
__device__ __forceinline__ void read_slot(Ctrl* c, int slot, RedSmem& rs, float& dmax, float& lo, float& hi)
{
    if (threadIdx.x == 0) {
        rs.bc[0] = __uint_as_float(ld_l2((const int*)&c->red_delta[slot]));
        rs.bc[1] = -okey_inv((uint32_t)ld_l2((const int*)&c->red_nlo[slot]));
        rs.bc[2] = okey_inv((uint32_t)ld_l2((const int*)&c->red_hi[slot]));
    }
    __syncthreads();
    dmax = rs.bc[0];
    lo = rs.bc[1];
    hi = rs.bc[2];
    __syncthreads();
}

template <int PATH, int NCA = 0, int NCO = 0>
struct Runner {
    const KP& p;
    Ctrl* c;
    unsigned long long target;
    long long barriers;
    bool stall;
    int cur;
    int red_epoch;
    Centre C;
    RedSmem& rs;
    DenseSmem* dsm;
    float* stage;
    bool perm_ok;
    GroupView gv;
    bool lead;   // thread 0 of the group's first CTA
    TmaSmem* tsm = nullptr;        // dense TMA path: barriers, state lists
    unsigned char* ring = nullptr; // dense TMA path: stage ring
    uint32_t ring_it = 0;          // dense TMA path: tiles streamed so far (same in every thread)

    __device__ Runner(const KP& kp, RedSmem& r, DenseSmem* d, float* st, GroupView g)
        : p(kp), c(kp.ctrl), target(0), barriers(0), stall(false), cur(0), red_epoch(0), rs(r), dsm(d),
          stage(st), perm_ok(true), gv(g), lead(g.rank == 0 && threadIdx.x == 0)
    {
        carry_a.valid = false;
        carry_o.valid = false;
        carry_g.valid = false;
    }

    __device__ bool sync(int site)
    {
        arrive();
        return wait(site);
    }
    // split grid-wide barrier: work between arrive() and wait() must not read what other CTAs
    // write before their arrival
    __device__ void arrive()
    {
        const bool skip = stall;
        stall = false;
        if (!perm_ok) atomicCAS(&c->error, 0, RMB_ERR_UNSUPPORTED);
        ++barriers;
        grid_arrive(c, target, skip, gv.size);
    }
    __device__ bool wait(int site) { return grid_wait_arrived(c, target, p.timeout_ns, site, gv.size); }

    __device__ size_t gtid() const { return (size_t)gv.rank * blockDim.x + threadIdx.x; }
    __device__ size_t gthreads() const { return (size_t)gv.size * blockDim.x; }

    static constexpr int NCA_ = NCA > 0 ? NCA : 1;
    static constexpr int NCO_ = NCO > 0 ? NCO : 1;
    Carry<NCA_> carry_a;    // prefetched first state of the next min-over-actions batch
    GenCarry carry_g;       // generic path: prefetched first steps of the next batch
    Carry<NCO_> carry_o;    // ... of the next policy-row batch
    uint64_t wtot = 0;      // RMB_SELECT_WEIGHTED: sum of the weights (read at set-up)

    template <int KIND>
    __device__ bool batch(const float* A, float* B, int pos0, int len, const PermKey* K, int32_t* So, float* Wo,
                          Acc& acc)
    {
        if (PATH == PATH_DENSE_TMA) {
            constexpr int DT = NCA;
            return dense_batch_tma<KIND, DT>(p, gv, *tsm, stage, ring, ring_it, A, B, pos0, len, K, So, Wo, C, acc,
                                             &perm_ok);
        }
        if (PATH == PATH_DENSE) {
            // dense kernels are instantiated per storage type: NCA carries the element type
            constexpr int DT = NCA;
            const bool vec = (((uintptr_t)p.P) & 15) == 0 && p.n % Elem<DT>::per16 == 0;
            if (vec) return dense_batch<KIND, DT, true>(p, gv, *dsm, stage, A, B, pos0, len, K, So, Wo, C, acc, &perm_ok);
            return dense_batch<KIND, DT, false>(p, gv, *dsm, stage, A, B, pos0, len, K, So, Wo, C, acc, &perm_ok);
        } else {
            const int lps = (KIND == K_POLICY) ? p.lps_one : p.lps_all;
            if (PATH == PATH_CSR_VEC && KIND == K_POLICY && NCO > 0) {
                csr_batch_fast<K_POLICY, NCO_>(p, gv, lps, A, B, pos0, len, K, So, Wo, C, acc, &perm_ok, carry_o);
                return true;
            }
            if (PATH == PATH_CSR_VEC && KIND != K_POLICY && NCA > 0) {
                carry_a.valid = carry_a.valid && KIND == K_MIN;
                csr_batch_fast<KIND == K_GREEDY ? K_GREEDY : K_MIN, NCA_>(p, gv, lps, A, B, pos0, len, K, So, Wo, C,
                                                                         acc, &perm_ok, carry_a);
                return true;
            }
            if (PATH == PATH_CSR_GEN) {
                carry_g.valid = carry_g.valid && KIND != K_GREEDY;
                csr_batch_gen<KIND>(p, gv, A, B, pos0, len, K, So, Wo, C, acc, &perm_ok, carry_g);
                return true;
            }
            csr_batch<KIND, true>(p, gv, lps, A, B, pos0, len, K, So, Wo, C, acc, &perm_ok);
            return true;
        }
    }

    // between arrive() and wait(): load the first state of the next batch of the same sweep
    template <int KIND>
    __device__ void prefetch_next(int pos0, int len, const PermKey* K)
    {
        if (PATH == PATH_CSR_GEN && KIND != K_GREEDY) {
            gen_prefetch_first<KIND>(p, gv, pos0, len, K, carry_g, &perm_ok);
            return;
        }
        if (PATH != PATH_CSR_VEC) return;
        if (KIND == K_POLICY && NCO > 0)
            fast_prefetch_first<K_POLICY, NCO_>(p, gv, p.lps_one, pos0, len, K, carry_o, &perm_ok);
        if (KIND == K_MIN && NCA > 0) fast_prefetch_first<K_MIN, NCA_>(p, gv, p.lps_all, pos0, len, K, carry_a, &perm_ok);
    }

    __device__ void copy_batch(const int32_t* S, const float* Wv, int len, float* B, size_t skip = 0,
                               uint64_t stamp = 0, const uint64_t* mk = nullptr)
    {
        for (size_t i = gtid() + skip; i < (size_t)len; i += gthreads()) {
            const int s = ld_l2(S + i);
            if (stamp && ld_l2(mk + s) == stamp) continue;   // the current batch updates s itself
            st_l2(B + s, ld_l2(Wv + i));
        }
    }

    // Draws with replacement can put a state in two consecutive batches t and t+1; batch t+1 then
    // writes its own value of s into the buffer that also receives batch t's values, so that copy
    // must skip s.  The states of batch t+1 are marked during batch t (before its barrier), in the
    // other half of the mark array than the one batch t's copy is reading.
    __device__ void mark_batch(const PermKey& K, int pos0, int len, uint64_t stamp, uint64_t* mk)
    {
        bool ok = true;
        for (size_t i = gtid(); i < (size_t)len; i += gthreads())
            st_l2(mk + state_at((uint32_t)(pos0 + (int)i), K, &ok), stamp);
        if (!ok) perm_ok = false;
    }

    // Re-centre between sweeps when the midpoint of the values moved by more than a quarter of
    // their spread: mu += shift, d -= shift in the buffer that holds the complete values (and the
    // other buffer gets the same, which also completes the end-of-sweep copy).
    __device__ float shift_for(float lo, float hi) const
    {
        if (p.flags & RMB_FLAG_RAW_ROWS) return 0.f;
        const float mid = 0.5f * (lo + hi);
        const float spread = hi - lo;
        const float floor_ = 1e-6f * (float)(fabs(C.mu) + 1.0);
        if (!(fabsf(mid) > fmaxf(0.25f * spread, floor_))) return 0.f;
        return mid;
    }

    __device__ PermKey key_for(long long k) const
    {
        PermKey K;
        K.n = (uint32_t)p.n;
        K.h = p.h;
        K.mask = (1u << p.h) - 1u;
        K.k0 = p.seed_lo;
        K.k1 = p.seed_hi;
        K.s_lo = (uint32_t)(unsigned long long)k;
        K.s_hi = (uint32_t)((unsigned long long)k >> 32);
        K.buf = nullptr;
        K.select = (uint32_t)p.select;
        K.wtot = wtot;
        K.cdf = p.cdf;
        return K;
    }

    // the order of sweep k (sigma or the draws) for every position, by the whole grid, into the
    // order buffer (done in a phase that ends with a grid-wide barrier, before sweep k starts)
    __device__ void compute_perm(long long k)
    {
        if (!p.perm_buf) return;
        const PermKey K = key_for(k);
        for (size_t i = gtid(); i < (size_t)p.n; i += gthreads())
            st_l2(p.perm_buf + i, order_at((uint32_t)i, K, &perm_ok));
    }

    // One sweep of B_b (KIND K_MIN) or B_{pi,b} (K_POLICY).  Returns false on failure; sets stop.
    // can_stop: VI / evaluation (may end after this sweep); MPI evaluation sweeps always complete
    template <int KIND>
    __device__ bool sweep(long long k, long long j, bool can_stop, bool is_last, bool& stop, float& delta)
    {
        PermKey K = key_for(k);
        K.buf = p.perm_buf;
        const int slot = red_epoch % 3;
        if (lead) {
            const int nxt = (red_epoch + 1) % 3;
            c->red_delta[nxt] = 0u;
            c->red_hi[nxt] = 0u;
            c->red_nlo[nxt] = 0u;
        }
        ++red_epoch;
        Acc acc = {0.f, kInf, -kInf};
        const bool async = (p.flags & RMB_FLAG_ASYNC) != 0;
        if (async) {
            // asynchronous sweep: the whole order in one pass, every new value written in place at once
            // (no barrier between batches: later states read whatever updates have landed)
            float* A = p.d[cur];
            K.buf = nullptr;
            if (!batch<KIND>(A, A, 0, p.n, &K, nullptr, nullptr, acc)) return false;
            publish(c, slot, acc, rs);
            if (!sync(12)) return false;
        }
        // one batch (b >= n) of sigma is the Bellman operator T: every state reads old values only,
        // so the order is immaterial and sigma is not evaluated (nor the position / value caches
        // written).  Draws with replacement choose which states update, so they are always taken.
        const bool ordered = p.T > 1 || p.select != RMB_SELECT_PERMUTATION;
        for (int t = 0; t < (async ? 0 : p.T); ++t) {
            float* A = p.d[(cur + t) & 1];
            float* B = p.d[(cur + t + 1) & 1];
            const int len = (t == p.T - 1) ? p.last_len : p.b;
            // B must also receive batch t-1's new values before the next batch reads it: the first
            // item of each thread is loaded before the batch's compute and stored after it
            int c_s = -1;
            float c_v = 0.f;
            const size_t c0 = gtid();
            if (t >= 1 && c0 < (size_t)p.b) {
                c_s = ld_l2(p.S[(t - 1) & 1] + c0);
                c_v = ld_l2(p.W[(t - 1) & 1] + c0);
            }
            if (!batch<KIND>(A, B, t * p.b, len, ordered ? &K : nullptr, ordered ? p.S[t & 1] : nullptr,
                             ordered ? p.W[t & 1] : nullptr, acc))
                return false;
            // stamps are unique within the solve (mark is cleared at set-up)
            const uint64_t stamp = p.mark ? (uint64_t)(k - p.start_sweep) * (uint64_t)p.T + (uint64_t)t + 1u : 0u;
            uint64_t* mk = p.mark ? p.mark + (size_t)(t & 1) * (size_t)p.n : nullptr;
            if (c_s >= 0 && !(stamp && ld_l2(mk + c_s) == stamp)) st_l2(B + c_s, c_v);
            if (t >= 1) copy_batch(p.S[(t - 1) & 1], p.W[(t - 1) & 1], p.b, B, gthreads(), stamp, mk);
            if (p.mark && t + 1 < p.T)
                mark_batch(K, (t + 1) * p.b, (t + 2 == p.T) ? p.last_len : p.b, stamp + 1u,
                           p.mark + (size_t)((t + 1) & 1) * (size_t)p.n);
            if (t == p.T - 1) publish(c, slot, acc, rs);
            arrive();
            if (t + 1 < p.T) prefetch_next<KIND>((t + 1) * p.b, (t + 2 == p.T) ? p.last_len : p.b, &K);
            if (!wait(10 + (t & 1))) return false;
        }
        float lo, hi;
        read_slot(c, slot, rs, delta, lo, hi);
        const int newcur = async ? cur : (cur + p.T) & 1;
        if (lead && p.trace && j >= 0) p.trace[j] = (double)delta;
        stop = can_stop && ((double)delta <= p.eps || is_last);
        if (delta != delta) {
            atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
            return false;
        }
        cur = newcur;
        // a solve that ends here skips the closing phase; with draws the caller may still go on
        // (its full-residual check can fail), so the buffers and the next order must be completed
        if (stop && ((p.select == RMB_SELECT_PERMUTATION && p.residual_kind == RMB_RESIDUAL_SWEEP) || is_last))
            return true;
        const float shift = shift_for(lo, hi);
        if (shift != 0.f) {
            float* F = p.d[cur];
            float* O = p.d[cur ^ 1];
            for (size_t i = gtid(); i < (size_t)p.n; i += gthreads()) {
                const float v = ld_l2(F + i) - shift;
                st_l2(F + i, v);
                if (!async) st_l2(O + i, v);
            }
            C = make_centre(C.mu + (double)shift, p.gamma_d);
            compute_perm(k + 1);
            if (!sync(20)) return false;
        } else if ((p.T >= 2 || p.select != RMB_SELECT_PERMUTATION) && !async) {
            // (one batch of draws leaves the states not drawn to be carried over as well)
            copy_batch(p.S[(p.T - 1) & 1], p.W[(p.T - 1) & 1], p.last_len, p.d[cur ^ 1]);
            compute_perm(k + 1);
            if (!sync(21)) return false;
        }
        return true;
    }

    // Full Bellman pass at the current values: greedy policy, Q-gap, TV, ||TV - V||_inf, V out.
    // next_k >= 0: also prepare the permutation of sweep next_k (MPI: the evaluation sweep that may
    // follow).
    __device__ bool greedy_pass(float& resid, long long next_k = -1)
    {
        const int slot = red_epoch % 3;
        if (lead) {
            const int nxt = (red_epoch + 1) % 3;
            c->red_delta[nxt] = 0u;
            c->red_hi[nxt] = 0u;
            c->red_nlo[nxt] = 0u;
        }
        ++red_epoch;
        Acc acc = {0.f, kInf, -kInf};
        const float* A = p.d[cur];
        carry_a.valid = false;
        carry_g.valid = false;
        if (!batch<K_GREEDY>(A, nullptr, 0, p.n, nullptr, nullptr, nullptr, acc)) return false;
        if (next_k >= 0) compute_perm(next_k);
        publish(c, slot, acc, rs);
        if (!sync(30)) return false;
        float lo, hi;
        read_slot(c, slot, rs, resid, lo, hi);
        if (resid != resid) {
            atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
            return false;
        }
        return true;
    }

    __device__ void write_values()
    {
        const float* F = p.d[cur];
        for (size_t i = gtid(); i < (size_t)p.n; i += gthreads()) p.Vout[i] = (float)(C.mu + (double)ld_l2(F + i));
    }

    __device__ void run()
    {
        stall = (p.flags & RMB_FLAG_INJECT_BARRIER_STALL) && gv.rank == 0;
        if (PATH == PATH_DENSE_TMA && threadIdx.x == 0) {
            for (int i = 0; i < kRingStages; ++i) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&tsm->full[i])) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&tsm->empty[i])),
                             "r"(kTmaConsumers) : "memory");
            }
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&tsm->vbar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            tsm->vphase = 0;
            tsm->abort = 0;
        }
        if (PATH == PATH_DENSE && threadIdx.x == 0) {
            const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&dsm->mbar);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            dsm->phase = 0;
        }
        __syncthreads();
        if (ld_volatile(&c->error) != 0) return;   // the validation pass rejected the MDP

        if (p.select == RMB_SELECT_WEIGHTED) {
            wtot = __ldg(p.cdf + (p.n - 1));
            if (wtot == 0 && lead) atomicCAS(&c->error, 0, RMB_ERR_ARG);
        }
        // set-up: centre on the midpoint of the start values
        Acc a0 = {0.f, kInf, -kInf};
        for (size_t i = gtid(); i < (size_t)p.n; i += gthreads()) {
            const float v = p.Vin[i];
            a0.vlo = fminf(a0.vlo, v);
            a0.vhi = fmaxf(a0.vhi, v);
            if (v != v || fabsf(v) == kInf) atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
        }
        publish(c, 3, a0, rs);
        if (!sync(1)) return finish(false, 0, 0, 0.0);
        if (ld_volatile(&c->error) != 0) return finish(false, 0, 0, 0.0);   // e.g. all weights zero
        float dm, lo, hi;
        read_slot(c, 3, rs, dm, lo, hi);
        // rows that need not sum to 1 (RMB_FLAG_RAW_ROWS) keep the values uncentred: mu = 0
        const double mu0 = (p.flags & RMB_FLAG_RAW_ROWS) ? 0.0 : (double)(float)(0.5 * ((double)lo + (double)hi));
        C = make_centre(mu0, p.gamma_d);
        for (size_t i = gtid(); i < (size_t)p.n; i += gthreads()) {
            const float v = (float)((double)p.Vin[i] - mu0);
            st_l2(p.d[0] + i, v);
            st_l2(p.d[1] + i, v);
            if (p.mark) {
                st_l2(p.mark + i, (uint64_t)0);
                st_l2(p.mark + p.n + i, (uint64_t)0);
            }
        }
        if (p.mode == MODE_VI || p.mode == MODE_EVAL) compute_perm(p.start_sweep);
        if (!sync(2)) return finish(false, 0, 0, 0.0);
        cur = 0;

        long long sweeps = 0, iters = 0;
        double residual = 0.0;
        bool converged = false;
        if (p.mode == MODE_GREEDY) {
            float r;
            if (!greedy_pass(r)) return finish(false, 0, 0, 0.0);
            return finish(true, 0, 0, (double)r, true);
        }
        if (p.mode == MODE_VI || p.mode == MODE_EVAL) {
            for (long long j = 0; j < p.max_sweeps; ++j) {
                bool stop = false;
                float delta = 0.f;
                const bool last = j + 1 == p.max_sweeps;
                const bool ok = (p.mode == MODE_VI)
                                    ? sweep<K_MIN>(p.start_sweep + j, j, true, last, stop, delta)
                                    : sweep<K_POLICY>(p.start_sweep + j, j, true, last, stop, delta);
                if (!ok) return finish(false, sweeps, 0, 0.0);
                ++sweeps;
                residual = (double)delta;
                if (stop) {
                    converged = (double)delta <= p.eps;
                    if (converged && (p.select != RMB_SELECT_PERMUTATION || p.residual_kind == RMB_RESIDUAL_BELLMAN)) {
                        // draws (the change covers only the drawn states) or the Bellman stop test:
                        // confirm with a full pass
                        float r;
                        if (!greedy_pass(r)) return finish(false, sweeps, 0, residual);   // also writes V
                        residual = (double)r;
                        converged = (double)r <= p.eps;
                        if (converged) return finish(true, sweeps, 0, residual, true);
                        if (!last) continue;
                    }
                    break;
                }
            }
            if (p.mode == MODE_VI && (p.pi || p.qgap)) {
                float r;
                if (!greedy_pass(r)) return finish(false, sweeps, 0, residual);   // also writes V
            } else {
                write_values();
            }
            return finish(true, sweeps, 0, residual, converged);
        }
        // MODE_MPI (Alg. 1): improvement pass, stop test, K evaluation sweeps of B_{pi,b}
        for (;;) {
            float r;
            if (!greedy_pass(r, p.start_sweep + sweeps)) return finish(false, sweeps, iters, residual);   // also writes V
            residual = (double)r;
            if (lead && p.trace) p.trace[iters] = residual;
            ++iters;
            if (residual <= p.eps) { converged = true; break; }
            if (iters >= p.max_sweeps) break;
            for (int e = 0; e < p.K; ++e) {
                bool stop = false;
                float delta = 0.f;
                if (!sweep<K_POLICY>(p.start_sweep + sweeps, -1, false, false, stop, delta))
                    return finish(false, sweeps, iters, residual);
                ++sweeps;
            }
        }
        return finish(true, sweeps, iters, residual, converged);
    }

    __device__ void finish(bool ok, long long sweeps, long long iters, double residual, bool converged = false)
    {
        if (lead) {
            c->sweeps = sweeps;
            c->iters = iters;
            c->barriers = barriers;
            c->residual = residual;
            c->mu = C.mu;
            int st = ld_volatile(&c->error);
            if (ok && st == 0 && !converged) st = RMB_ERR_NOT_CONVERGED;
            c->status = st;
        }
    }
};

// CSR rows with k % 4 == 0: NCA / NCO = float4 chunks per lane in the min-over-actions sweeps and in
// the policy-row sweeps (0 = the general row loop).
template <int NCA, int NCO>
__global__ void __launch_bounds__(kCsrThreads, 1) rmb_csr_vec_kernel(KP p)
{
    __shared__ RedSmem rs;
    Runner<PATH_CSR_VEC, NCA, NCO> R(p, rs, nullptr, nullptr, GroupView{(int)blockIdx.x, (int)gridDim.x});
    R.run();
}

__global__ void __launch_bounds__(kCsrThreads, 1) rmb_csr_gen_kernel(KP p)
{
    __shared__ RedSmem rs;
    Runner<PATH_CSR_GEN> R(p, rs, nullptr, nullptr, GroupView{(int)blockIdx.x, (int)gridDim.x});
    R.run();
}

// Dense rows streamed by the TMA pipeline; DT = element type of P.  Dynamic shared memory: the
// staged values (vst_floats) followed by the stage ring.
template <int DT>
__global__ void __launch_bounds__(kTmaThreads, 1) rmb_dense_tma_kernel(KP p)
{
    __shared__ RedSmem rs;
    __shared__ __align__(16) TmaSmem tsm;
    extern __shared__ __align__(128) unsigned char dyn[];
    float* vst = reinterpret_cast<float*>(dyn);
    Runner<PATH_DENSE_TMA, DT> R(p, rs, nullptr, vst, GroupView{(int)blockIdx.x, (int)gridDim.x});
    R.tsm = &tsm;
    R.ring = dyn + (size_t)p.stage * 4;
    R.run();
}

// Dense rows; DT = element type of P (RMB_P_F32 / RMB_P_BF16 / RMB_P_FP8E4M3).
template <int DT>
__global__ void __launch_bounds__(kDenseThreads, 2) rmb_dense_kernel(KP p)
{
    __shared__ RedSmem rs;
    __shared__ __align__(16) DenseSmem dsm;
    extern __shared__ __align__(128) float stage[];
    Runner<PATH_DENSE, DT> R(p, rs, &dsm, stage, GroupView{(int)blockIdx.x, (int)gridDim.x});
    R.run();
}

// ------------------------------------------------------------------------------------------------
// Batched solves: many independent MDPs in one persistent launch.  Every CTA runs a list of tasks; a
// task is one MDP solved by a group of CTAs (its own barrier counter and control block) or by this
// CTA alone (barriers are then CTA barriers).  CTAs of a multi-CTA group run the same task list.
// ------------------------------------------------------------------------------------------------
struct BatchTask {
    int item, rank, size, pad;
};

__global__ void __launch_bounds__(kCsrThreads, 1)
rmb_batched_kernel(const KP* __restrict__ kps, const int* __restrict__ task_off, const BatchTask* __restrict__ tasks)
{
    __shared__ RedSmem rs;
    __shared__ KP s_kp;
    const int t0 = task_off[blockIdx.x], t1 = task_off[blockIdx.x + 1];
    for (int t = t0; t < t1; ++t) {
        const BatchTask bt = tasks[t];
        __syncthreads();
        if (threadIdx.x == 0) s_kp = kps[bt.item];
        __syncthreads();
        const GroupView gv{bt.rank, bt.size};
        if (s_kp.path == PATH_CSR_VEC && s_kp.nc_all == 1 && s_kp.nc_one == 1) {
            Runner<PATH_CSR_VEC, 1, 1> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        } else if (s_kp.path == PATH_CSR_VEC && s_kp.nc_all == 2 && s_kp.nc_one == 1) {
            Runner<PATH_CSR_VEC, 2, 1> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        } else {
            Runner<PATH_CSR_GEN> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Differentiable fixed point (gradient of L = w . V* through the Bellman equation at the greedy
// policy): row softmax, transposed greedy chain, gradient assembly.  The adjoint system
// lambda = w + gamma P_pi^T lambda is solved by the persistent kernel's policy-row sweeps on the
// transposed chain (one action per "state", rows = columns of P_pi).
// ------------------------------------------------------------------------------------------------
__global__ void rmb_softmax_kernel(int64_t rows, int k, const float* __restrict__ z, float* __restrict__ p)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nw) {
        const float* zr = z + r * k;
        float mx = -kInf;
        for (int e = lane; e < k; e += 32) mx = fmaxf(mx, zr[e]);
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        float sum = 0.f;
        for (int e = lane; e < k; e += 32) sum += expf(zr[e] - mx);
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        const float inv = 1.f / sum;
        for (int e = lane; e < k; e += 32) p[r * k + e] = expf(zr[e] - mx) * inv;
    }
}

// in-degree of every state in the greedy chain (rows r = s*m + pi(s), k entries each)
__global__ void rmb_tr_count_kernel(int n, int m, int k, const int32_t* __restrict__ pi, const int32_t* __restrict__ col,
                                    int32_t* __restrict__ cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / k), t = (int)(e - (int64_t)s * k);
        const int a = min((uint32_t)pi[s], (uint32_t)(m - 1));
        const int j = col[((int64_t)s * m + a) * k + t];
        atomicAdd(cnt + min((uint32_t)j, (uint32_t)(n - 1)), 1);
    }
}

// exclusive scan of the counts into row_ptr (one CTA: runs once per gradient call)
__global__ void rmb_tr_scan_kernel(int n, const int32_t* __restrict__ cnt, int64_t* __restrict__ row_ptr,
                                   int32_t* __restrict__ cursor)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t per = ((int64_t)n + T - 1) / T;
    const int64_t a = (int64_t)t * per, b = min((int64_t)n, a + per);
    int64_t sum = 0;
    for (int64_t i = a; i < b; ++i) sum += cnt[i];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < T; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        row_ptr[n] = run;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t i = a; i < b; ++i) {
        const int32_t c = cnt[i];   // cursor may alias cnt: read before writing
        row_ptr[i] = run;
        cursor[i] = (int32_t)run;
        run += c;
    }
}

__global__ void rmb_tr_scatter_kernel(int n, int m, int k, const int32_t* __restrict__ pi, const int32_t* __restrict__ col,
                                      const float* __restrict__ prob, int32_t* __restrict__ cursor,
                                      int32_t* __restrict__ colT, float* __restrict__ probT)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / k), t = (int)(e - (int64_t)s * k);
        const int a = min((uint32_t)pi[s], (uint32_t)(m - 1));
        const int64_t src = ((int64_t)s * m + a) * k + t;
        const int j = min((uint32_t)col[src], (uint32_t)(n - 1));
        const int pos = atomicAdd(cursor + j, 1);
        colT[pos] = s;
        probT[pos] = prob[src];
    }
}

// order each transposed row by source state, so sums run in a fixed order (deterministic results)
__global__ void rmb_tr_sort_kernel(int n, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ colT,
                                   float* __restrict__ probT)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[j], b = row_ptr[j + 1];
        for (int64_t i = a + 1; i < b; ++i) {
            const int32_t c = colT[i];
            const float pv = probT[i];
            int64_t q = i - 1;
            while (q >= a && colT[q] > c) {
                colT[q + 1] = colT[q];
                probT[q + 1] = probT[q];
                --q;
            }
            colT[q + 1] = c;
            probT[q + 1] = pv;
        }
    }
}

// dL/dcost(s, pi(s)) = lambda(s); dL/dz(s, pi(s), t) = gamma lambda(s) p_t (V(j_t) - sum_u p_u V(j_u))
__global__ void rmb_grad_kernel(int n, int m, int k, float gamma, const int32_t* __restrict__ pi,
                                const int32_t* __restrict__ col, const float* __restrict__ prob,
                                const float* __restrict__ V, const float* __restrict__ lam,
                                float* __restrict__ grad_cost, float* __restrict__ grad_z)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < n; s += nw) {
        const int a = min((uint32_t)pi[s], (uint32_t)(m - 1));
        const int64_t r = s * m + a;
        const float l = lam[s];
        if (grad_cost && lane == 0) grad_cost[r] = l;
        if (!grad_z) continue;
        float mean = 0.f;
        for (int t = lane; t < k; t += 32) mean = fmaf(prob[r * k + t], V[min((uint32_t)col[r * k + t], (uint32_t)(n - 1))], mean);
        for (int off = 16; off > 0; off >>= 1) mean += __shfl_xor_sync(0xffffffffu, mean, off);
        for (int t = lane; t < k; t += 32) {
            const float pv = prob[r * k + t];
            const float vj = V[min((uint32_t)col[r * k + t], (uint32_t)(n - 1))];
            grad_z[r * k + t] = gamma * l * pv * (vj - mean);
        }
    }
}

// Gather-rate probe: every thread streams 16-byte chunks of an index array and gathers src at those
// indices (L1-cached, as the successor gathers), accumulating a checksum per thread.  Measures the
// attainable rate of random 4-byte gathers from a table of a given size (the CSR kernel's L2 bound).
// ------------------------------------------------------------------------------------------------
// Cumulative weights of RMB_SELECT_WEIGHTED (exact: 64-bit integer sums), in three launches:
// per-tile sums, an exclusive scan of the tile sums by one CTA, then every tile's running sums.
// ------------------------------------------------------------------------------------------------
__device__ uint64_t block_exscan_u64(uint64_t v, uint64_t* total)
{
    __shared__ uint64_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint64_t t = lane < nw ? warp_tot[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const uint64_t ex = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    *total = warp_tot[nw - 1];
    __syncthreads();                          // warp_tot is reused by the next call
    return ex;
}

__global__ void __launch_bounds__(kScanThreads) rmb_wsum_kernel(const uint32_t* __restrict__ w, int64_t n,
                                                               uint64_t* __restrict__ parts)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) sum += w[base + i];
    uint64_t tot;
    block_exscan_u64(sum, &tot);
    if (threadIdx.x == 0) parts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) rmb_wparts_kernel(uint64_t* __restrict__ parts, int64_t tiles)
{
    uint64_t carry = 0;
    for (int64_t c0 = 0; c0 < tiles; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const uint64_t v = i < tiles ? parts[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_exscan_u64(v, &tot);
        if (i < tiles) parts[i] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) rmb_wcdf_kernel(const uint32_t* __restrict__ w, int64_t n,
                                                               const uint64_t* __restrict__ parts,
                                                               uint64_t* __restrict__ cdf)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint64_t v[kScanPer];
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = base + i < n ? w[base + i] : 0;
        sum += v[i];
    }
    uint64_t tot;
    uint64_t run = parts[blockIdx.x] + block_exscan_u64(sum, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        run += v[i];
        if (base + i < n) cdf[base + i] = run;
    }
}

// ------------------------------------------------------------------------------------------------
// Importance weights from the Bellman residual: r(s) = |TV(s) - V(s)|, R = max r, then
// w(s) = floor(2^20 (f + (1 - f) r(s) / R)).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rmb_resid_max_kernel(const float* __restrict__ TV, const float* __restrict__ V,
                                                            int64_t n, uint32_t* __restrict__ rmax)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(TV[i] - V[i]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(rmax, __float_as_uint(m));   // non-negative floats order as their bits
}

__global__ void __launch_bounds__(256) rmb_resid_weights_kernel(const float* __restrict__ TV,
                                                                const float* __restrict__ V, int64_t n, float f,
                                                                const uint32_t* __restrict__ rmax,
                                                                uint32_t* __restrict__ w)
{
    const float R = __uint_as_float(*rmax);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = R > 0.f ? fminf(fabsf(TV[i] - V[i]) / R, 1.f) : 1.f;
        w[i] = (uint32_t)floorf(1048576.f * (f + (1.f - f) * x));
    }
}

__global__ void __launch_bounds__(512, 1) rmb_gather_probe_kernel(const float* __restrict__ src, uint32_t nm1,
                                                                  const int4* __restrict__ idx, int64_t n4, int reps,
                                                                  float* __restrict__ out)
{
    float acc = 0.f;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t i = t; i < n4; i += T) {
            const int4 c = __ldcs(idx + i);
            acc += __ldca(src + min((uint32_t)c.x, nm1)) + __ldca(src + min((uint32_t)c.y, nm1)) +
                   __ldca(src + min((uint32_t)c.z, nm1)) + __ldca(src + min((uint32_t)c.w, nm1));
        }
    }
    out[t] = acc;
}

// Row quantiser (low-precision storage of dense rows): one warp per row.
__global__ void rmb_quantize_kernel(const float* __restrict__ P, int64_t rows, int64_t cols, int dt,
                                    void* __restrict__ codes, float* __restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nw) {
        const float* row = P + r * cols;
        float mx = 0.f;
        for (int64_t j = lane; j < cols; j += 32) mx = fmaxf(mx, row[j]);
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        const float sc = mx > 0.f ? (dt == RMB_P_FP8E4M3 ? mx / 448.f : mx) : 1.f;
        float dsum = 0.f;   // sum of the decoded codes
        if (dt == RMB_P_BF16) {
            __nv_bfloat16* out = static_cast<__nv_bfloat16*>(codes) + r * cols;
            for (int64_t j = lane; j < cols; j += 32) {
                const __nv_bfloat16 c = __float2bfloat16_rn(row[j] / sc);
                out[j] = c;
                dsum += __bfloat162float(c);
            }
        } else {
            __nv_fp8_storage_t* out = static_cast<__nv_fp8_storage_t*>(codes) + r * cols;
            for (int64_t j = lane; j < cols; j += 32) {
                const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(row[j] / sc, __NV_SATFINITE, __NV_E4M3);
                out[j] = c;
                const __half_raw h = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
                dsum += __half2float(*reinterpret_cast<const __half*>(&h));
            }
        }
        for (int off = 16; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
        if (lane == 0 && scale) scale[r] = dsum > 0.f ? 1.f / dsum : 0.f;
    }
}

// ------------------------------------------------------------------------------------------------
// Permutation and validation kernels.
// ------------------------------------------------------------------------------------------------
__global__ void rmb_perm_kernel(uint32_t n, uint32_t h, uint32_t k0, uint32_t k1, uint32_t s_lo, uint32_t s_hi,
                                int32_t* out)
{
    PermKey K{n, h, (1u << h) - 1u, k0, k1, s_lo, s_hi, nullptr};
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        bool ok = true;
        const uint32_t x = perm_at((uint32_t)p, K, &ok);
        out[p] = ok ? (int32_t)x : -1;   // -1 cannot occur for a bijection; marks a broken walk
    }
}

struct VP {
    int n, m, k, fmt, p_dtype;
    const void* P;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* prob;
    const float* cost;
    int* err;
};

__global__ void rmb_validate_kernel(VP v)
{
    const int lane = threadIdx.x & 31;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t rows = (size_t)v.n * v.m;
    bool bad = false;
    for (size_t r = warp; r < rows; r += nwarps) {
        const float c = v.cost[r];
        if (c != c || c == -kInf) bad = true;
        const bool admissible = c != kInf;
        float sum = 0.f;
        if (v.fmt == RMB_CSR) {
            const int64_t e0 = v.row_ptr[r], e1 = v.row_ptr[r + 1];
            if (e0 < 0 || e1 < e0) { bad = true; continue; }
            if (v.k > 0 && (e0 != (int64_t)r * v.k || e1 != (int64_t)(r + 1) * v.k)) bad = true;
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                const float pr = v.prob[e];
                const int j = v.col[e];
                if (!(pr >= 0.f && pr <= 1.f)) bad = true;
                if (j < 0 || j >= v.n) bad = true;
                sum += pr;
            }
        } else {
            const unsigned char* row = static_cast<const unsigned char*>(v.P) +
                                       r * (size_t)v.n * (v.p_dtype == RMB_P_F32 ? 4 : (v.p_dtype == RMB_P_BF16 ? 2 : 1));
            for (int j = lane; j < v.n; j += 32) {
                float pr;
                if (v.p_dtype == RMB_P_BF16) pr = decode1<RMB_P_BF16>(row, j);
                else if (v.p_dtype == RMB_P_FP8E4M3) pr = decode1<RMB_P_FP8E4M3>(row, j);
                else pr = decode1<RMB_P_F32>(row, j);
                // coded rows only need to be finite and non-negative (they are renormalised)
                if (!(pr >= 0.f && (v.p_dtype != RMB_P_F32 ? pr <= 3.4e38f : pr <= 1.f))) bad = true;
                sum += pr;
            }
        }
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (admissible && v.fmt == RMB_CSR && !(fabsf(sum - 1.f) <= 1e-4f)) bad = true;
        if (admissible && v.fmt == RMB_DENSE && v.p_dtype == RMB_P_F32 && !(fabsf(sum - 1.f) <= 1e-4f)) bad = true;
        if (admissible && v.fmt == RMB_DENSE && v.p_dtype != RMB_P_F32 && !(sum > 0.f)) bad = true;
    }
    // every state needs one admissible action
    for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < (size_t)v.n;
         s += (size_t)gridDim.x * blockDim.x) {
        bool any = false;
        for (int a = 0; a < v.m; ++a) any |= (v.cost[s * v.m + a] != kInf);
        if (!any) bad = true;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && v.fmt == RMB_CSR && v.row_ptr[0] != 0) bad = true;
    if (bad) atomicCAS(v.err, 0, RMB_ERR_INVALID_MDP);
}

}  // namespace rmb

// ==================================================================================================
// Host side
// ==================================================================================================
using namespace rmb;

namespace {

std::atomic<uint64_t> g_launches{0};

struct DevInfo {
    int sms = 0;
    bool init = false;
};
DevInfo g_dev[64];
std::mutex g_mu;

int dev_info(DevInfo** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RMB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DevInfo& d = g_dev[dev];
    if (!d.init) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RMB_ERR_CUDA;
        d.init = true;
    }
    *out = &d;
    return RMB_OK;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t ctrl, d0, d1, s0, s1, w0, w1, pb, mark, cdf, parts, total;
    bool perm_buf;
};


// A sweep with at least this many batches precomputes its permutation into the workspace ...
constexpr int64_t kPermBufMinBatches = 16;
// ... and so does one with 2..15 batches when n < batches * 65536: evaluating sigma for all n
// positions once per sweep (about n / 65536 evaluations per thread of a full grid) then costs less
// than one evaluation, with its cycle-walking tail, on the path of every batch.
constexpr int64_t kPermBufPerBatch = 65536;

bool use_perm_buf(int64_t n, int64_t b)
{
    const int64_t T = (n + b - 1) / b;
    return T >= kPermBufMinBatches || (T >= 2 && n < T * kPermBufPerBatch);
}

Layout layout(int64_t n, int64_t b, int select = RMB_SELECT_PERMUTATION)
{
    Layout L;
    const size_t nb = align_up((size_t)n * 4, 256);
    const size_t bb = align_up((size_t)b * 4, 256);
    L.ctrl = 0;
    L.d0 = align_up(sizeof(Ctrl), 256);
    L.d1 = L.d0 + nb;
    L.s0 = L.d1 + nb;
    L.s1 = L.s0 + bb;
    L.w0 = L.s1 + bb;
    L.w1 = L.w0 + bb;
    L.pb = L.w1 + bb;
    L.perm_buf = use_perm_buf(n, b);
    L.mark = L.pb + (L.perm_buf ? nb : 0);
    const bool draws = select == RMB_SELECT_UNIFORM || select == RMB_SELECT_WEIGHTED;
    L.cdf = L.mark + (draws && b < n ? align_up((size_t)n * 16, 256) : 0);
    const bool w = select == RMB_SELECT_WEIGHTED;
    L.parts = L.cdf + (w ? align_up((size_t)n * 8, 256) : 0);
    L.total = L.parts + (w ? align_up((size_t)((n + kScanTile - 1) / kScanTile) * 8, 256) : 0);
    return L;
}

struct GradLayout {
    size_t rowT, colT, probT, cnt, zpi, eval, total;
};

GradLayout grad_layout(int64_t n, int64_t k, int64_t b)
{
    GradLayout G;
    const int64_t nnzT = n * k;
    G.rowT = 0;
    G.colT = align_up((size_t)(n + 1) * 8, 256);
    G.probT = G.colT + align_up((size_t)nnzT * 4, 256);
    G.cnt = G.probT + align_up((size_t)nnzT * 4, 256);
    G.zpi = G.cnt + align_up((size_t)n * 4, 256);
    G.eval = G.zpi + align_up((size_t)n * 4, 256);
    G.total = G.eval + layout(n, b).total;
    return G;
}

int check_mdp(const rmb_mdp* M)
{
    if (!M) return RMB_ERR_ARG;
    if (M->n < 1 || M->m < 1) return RMB_ERR_ARG;
    if (M->n >= ((int64_t)1 << 31)) return RMB_ERR_UNSUPPORTED;
    if (!(M->gamma > 0.0 && M->gamma < 1.0)) return RMB_ERR_ARG;
    if (!M->cost) return RMB_ERR_ARG;
    if (M->format == RMB_DENSE) {
        if (!M->P) return RMB_ERR_ARG;
        if (M->m > kDenseMaxM) return RMB_ERR_UNSUPPORTED;
        if (M->p_dtype < RMB_P_F32 || M->p_dtype > RMB_P_FP8E4M3) return RMB_ERR_ARG;
    } else if (M->format == RMB_CSR) {
        if (!M->row_ptr || !M->col || !M->prob) return RMB_ERR_ARG;
        if (M->k_uniform < 0) return RMB_ERR_ARG;
    } else {
        return RMB_ERR_ARG;
    }
    return RMB_OK;
}

int effective_batch(const rmb_mdp* M, const rmb_opts* O, int64_t* b)
{
    if (!O || O->batch < 1) return RMB_ERR_ARG;
    *b = O->batch > M->n ? M->n : O->batch;
    return RMB_OK;
}

bool csr_vec_ok(const rmb_mdp* M)
{
    if (M->format != RMB_CSR || M->k_uniform <= 0 || (M->k_uniform & 3)) return false;
    const int k4 = M->k_uniform >> 2;
    const bool pow2 = (k4 & (k4 - 1)) == 0;
    if (!(pow2 || k4 % 32 == 0)) return false;
    if (((uintptr_t)M->prob & 15) || ((uintptr_t)M->col & 15)) return false;
    return true;
}

const void* csr_vec_kernel_for(int nca, int nco)
{
    const int a = (nca == 1 || nca == 2 || nca == 4) ? nca : 0;
    const int o = nco == 1 ? 1 : 0;
#define RMB_K(A_, O_) if (a == A_ && o == O_) return reinterpret_cast<const void*>(rmb_csr_vec_kernel<A_, O_>);
    RMB_K(0, 0) RMB_K(1, 0) RMB_K(2, 0) RMB_K(4, 0) RMB_K(0, 1) RMB_K(1, 1) RMB_K(2, 1) RMB_K(4, 1)
#undef RMB_K
    return reinterpret_cast<const void*>(rmb_csr_vec_kernel<0, 0>);
}

int pow2ceil(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct Call {
    int mode;
    const rmb_mdp* M;
    const rmb_opts* O;
    const float* Vin;
    float* Vout;
    float* TV;
    int32_t* pi;
    float* qgap;
    const int32_t* pi_in;
    void* ws;
    size_t ws_bytes;
    rmb_stats* stats;
    cudaStream_t stream;
};

int launch_validate(const rmb_mdp* M, int* err, cudaStream_t st, int sms)
{
    VP v;
    v.n = (int)M->n;
    v.m = M->m;
    v.k = M->format == RMB_CSR ? M->k_uniform : 0;
    v.fmt = M->format;
    v.p_dtype = M->format == RMB_DENSE ? M->p_dtype : RMB_P_F32;
    v.P = M->P;
    v.row_ptr = M->row_ptr;
    v.col = M->col;
    v.prob = M->prob;
    v.cost = M->cost;
    v.err = err;
    rmb_validate_kernel<<<sms * 4, 256, 0, st>>>(v);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

// Kernel parameters of one solve: problem, schedule, workspace buffers at `ws` (laid out as L), the
// control block `ctrl`.  The caller sets the value / policy pointers.  Returns the row path.
int fill_kp(int mode, const rmb_mdp* M, const rmb_opts* O, int64_t b, char* ws, const Layout& L, Ctrl* ctrl, KP& p)
{
    std::memset(&p, 0, sizeof(p));
    p.n = (int)M->n;
    p.m = M->m;
    p.k = M->format == RMB_CSR ? M->k_uniform : 0;
    p.P = M->P;
    p.p_dtype = M->format == RMB_DENSE ? M->p_dtype : RMB_P_F32;
    p.row_scale = (M->format == RMB_DENSE && M->p_dtype != RMB_P_F32) ? M->row_scale : nullptr;
    p.row_ptr = M->row_ptr;
    p.col = M->col;
    p.prob = M->prob;
    p.cost = M->cost;
    p.gamma = (float)M->gamma;
    p.gamma_d = M->gamma;
    p.mode = mode;
    p.b = (int)b;
    p.T = (int)((M->n + b - 1) / b);
    p.last_len = (int)(M->n - (int64_t)(p.T - 1) * b);
    p.K = O->eval_sweeps;
    p.start_sweep = O->start_sweep;
    p.max_sweeps = mode == MODE_GREEDY ? 0 : O->max_sweeps;
    p.eps = O->eps;
    p.seed_lo = (uint32_t)O->seed;
    p.seed_hi = (uint32_t)(O->seed >> 32);
    p.h = perm_half_bits(M->n);
    p.d[0] = reinterpret_cast<float*>(ws + L.d0);
    p.d[1] = reinterpret_cast<float*>(ws + L.d1);
    p.S[0] = reinterpret_cast<int32_t*>(ws + L.s0);
    p.S[1] = reinterpret_cast<int32_t*>(ws + L.s1);
    p.W[0] = reinterpret_cast<float*>(ws + L.w0);
    p.W[1] = reinterpret_cast<float*>(ws + L.w1);
    // asynchronous sweeps have no barrier before a sweep's first read, so sigma is computed on the fly
    const bool async = (O->flags & RMB_FLAG_ASYNC) != 0;
    p.perm_buf = (L.perm_buf && mode != MODE_GREEDY && !async) ? reinterpret_cast<int32_t*>(ws + L.pb) : nullptr;
    p.select = RMB_SELECT_PERMUTATION;   // solve() sets the selection rule and stop test of a single-MDP call
    p.residual_kind = RMB_RESIDUAL_SWEEP;
    p.cdf = nullptr;
    p.mark = nullptr;
    p.ctrl = ctrl;
    p.trace = mode == MODE_GREEDY ? nullptr : O->trace;
    p.timeout_ns = O->barrier_timeout_ns > 0 ? O->barrier_timeout_ns : 2000000000LL;
    p.flags = O->flags;

    int path;
    if (M->format == RMB_DENSE) path = PATH_DENSE;
    else if (csr_vec_ok(M)) path = PATH_CSR_VEC;
    else path = PATH_CSR_GEN;
    p.path = path;
    if (path == PATH_CSR_VEC) {
        const int k4 = p.k >> 2;
        const int cpr = k4 < 32 ? k4 : 32;
        p.lps_one = cpr;
        int all = pow2ceil(cpr * p.m);
        p.lps_all = all > 32 ? 32 : all;
        int lg = 0;
        while ((1 << lg) < k4) ++lg;
        p.k4_log2 = lg;
        // fast path: a row's chunks fit in one lane group and a lane holds <= 4 chunks of a state
        auto nc_of = [&](int rows, int lps) {
            if (k4 > lps || (k4 & (k4 - 1))) return 0;
            const int nc = (rows * k4 + lps - 1) / lps;
            return (nc == 1 || nc == 2 || nc == 4) ? nc : (nc == 3 ? 4 : 0);
        };
        p.nc_all = nc_of(p.m, p.lps_all);
        p.nc_one = nc_of(1, p.lps_one) == 1 ? 1 : 0;
    } else {
        p.lps_one = 32;
        p.lps_all = 32;
    }

    return path;
}

int solve(const Call& q)
{
    int st = check_mdp(q.M);
    if (st) return st;
    const rmb_mdp* M = q.M;
    const rmb_opts* O = q.O;
    if (!O) return RMB_ERR_ARG;
    int64_t b = M->n;
    if (q.mode != MODE_GREEDY) {
        if ((st = effective_batch(M, O, &b))) return st;
        if (O->max_sweeps < 1) return RMB_ERR_ARG;
        if (!(O->eps >= 0.0) || std::isinf(O->eps)) return RMB_ERR_ARG;
        if (q.mode == MODE_MPI && (O->eval_sweeps < 1 || !q.pi)) return RMB_ERR_ARG;
        if (q.mode == MODE_EVAL && !q.pi_in) return RMB_ERR_ARG;
        if (O->start_sweep < 0) return RMB_ERR_ARG;
    }
    if (!q.Vin) return RMB_ERR_ARG;
    if (O->grid_ctas < 0 || O->barrier_timeout_ns < 0) return RMB_ERR_ARG;
    if ((O->flags & RMB_FLAG_ASYNC) && M->format != RMB_CSR) return RMB_ERR_UNSUPPORTED;
    // batch selection (rmb_greedy has no order and ignores it)
    const int select = q.mode == MODE_GREEDY ? RMB_SELECT_PERMUTATION : O->select;
    if (select < RMB_SELECT_PERMUTATION || select > RMB_SELECT_WEIGHTED) return RMB_ERR_ARG;
    if (select == RMB_SELECT_WEIGHTED && !O->weights) return RMB_ERR_ARG;
    if (select != RMB_SELECT_PERMUTATION && q.mode == MODE_EVAL) return RMB_ERR_UNSUPPORTED;
    const int rkind = q.mode == MODE_VI ? O->residual_kind : RMB_RESIDUAL_SWEEP;
    if (q.mode != MODE_GREEDY && (O->residual_kind < RMB_RESIDUAL_SWEEP || O->residual_kind > RMB_RESIDUAL_BELLMAN))
        return RMB_ERR_ARG;
    if (O->residual_kind != RMB_RESIDUAL_SWEEP && q.mode == MODE_EVAL) return RMB_ERR_UNSUPPORTED;
    const Layout L = layout(M->n, b, select);
    if (!q.ws || ((uintptr_t)q.ws & 255)) return RMB_ERR_WORKSPACE;
    if (q.ws_bytes < L.total) return RMB_ERR_WORKSPACE;

    DevInfo* D = nullptr;
    if ((st = dev_info(&D))) return st;

    char* ws = static_cast<char*>(q.ws);
    KP p;
    int path = fill_kp(q.mode, M, O, b, ws, L, reinterpret_cast<Ctrl*>(ws + L.ctrl), p);
    p.select = select;
    p.residual_kind = rkind;
    p.cdf = select == RMB_SELECT_WEIGHTED ? reinterpret_cast<const uint64_t*>(ws + L.cdf) : nullptr;
    // consecutive batches may share states only with draws, and only an asynchronous sweep has no copies
    p.mark = (L.cdf > L.mark && !(O->flags & RMB_FLAG_ASYNC)) ? reinterpret_cast<uint64_t*>(ws + L.mark) : nullptr;
    p.Vin = q.Vin;
    p.Vout = q.Vout;
    p.TVout = q.TV;
    p.pi = q.pi;
    p.qgap = q.qgap;
    p.pi_in = q.pi_in;

    const void* fn;
    int threads, per_sm;
    size_t smem = 0;
    if (path == PATH_DENSE) {
        // large rows stream through the TMA pipeline when the staged values and the ring fit
        const int e16 = p.p_dtype == RMB_P_F32 ? 4 : (p.p_dtype == RMB_P_BF16 ? 8 : 16);
        const size_t vbytes = align_up((size_t)((M->n + 3) & ~3LL) * 4, 128);
        const size_t tma_smem = vbytes + (size_t)kRingStages * kStageBytes;
        const bool tma_ok = M->n >= 2048 && M->n % e16 == 0 && (((uintptr_t)M->P) & 15) == 0 &&
                            (p.p_dtype == RMB_P_F32 || p.row_scale) && tma_smem + sizeof(TmaSmem) + 2048 <= 227 * 1024 &&
                            !std::getenv("RMB_DENSE_NO_TMA");
        if (tma_ok) {
            path = PATH_DENSE_TMA;
            p.path = path;
            fn = p.p_dtype == RMB_P_BF16      ? reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_BF16>)
                 : p.p_dtype == RMB_P_FP8E4M3 ? reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_FP8E4M3>)
                                              : reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_F32>);
            threads = kTmaThreads;
            p.stage = (int)(vbytes / 4);
            smem = tma_smem;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return RMB_ERR_CUDA;
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess) return RMB_ERR_CUDA;
            per_sm = occ < 2 ? occ : 2;
        }
    }
    if (path == PATH_DENSE) {
        fn = p.p_dtype == RMB_P_BF16      ? reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_BF16>)
             : p.p_dtype == RMB_P_FP8E4M3 ? reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_FP8E4M3>)
                                          : reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_F32>);
        threads = kDenseThreads;
        int max_stage = kDenseMaxStage;
        if (const char* e = std::getenv("RMB_DENSE_STAGE")) {   // tuning / test knob: floats staged at once
            const int v = std::atoi(e);
            if (v >= 16 && v <= kDenseMaxStage) max_stage = v & ~15;
        }
        p.stage = M->n <= max_stage ? (int)((M->n + 3) & ~3LL) : max_stage;
        smem = (size_t)p.stage * 4;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return RMB_ERR_CUDA;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess)
            return RMB_ERR_CUDA;
        per_sm = occ < 2 ? occ : 2;
    } else if (path != PATH_DENSE_TMA) {
        fn = path == PATH_CSR_VEC ? csr_vec_kernel_for(p.nc_all, p.nc_one)
                                  : reinterpret_cast<const void*>(rmb_csr_gen_kernel);
        threads = kCsrThreads;
        // the CSR kernels use almost no shared memory: give the unified L1 as much as possible for
        // the successor gathers
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess) return RMB_ERR_CUDA;
        per_sm = occ < 4 ? occ : 4;
    }
    if (per_sm < 1) return RMB_ERR_CUDA;
    const int max_grid = per_sm * D->sms;
    int grid = O->grid_ctas > 0 ? O->grid_ctas : max_grid;
    if (grid > max_grid) grid = max_grid;
    // dense rows take one CTA per state: with batches smaller than the grid, one CTA per SM is enough
    // (fewer CTAs at every grid barrier, no two sharing an SM)
    if (O->grid_ctas == 0 && path == PATH_DENSE && b < grid) grid = (int)std::max<int64_t>(b, D->sms);

    cudaStream_t s = q.stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (q.stats) {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RMB_ERR_CUDA;
        cudaEventRecord(e0, s);
    }
    if (cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return RMB_ERR_CUDA;
    if (O->validate && (st = launch_validate(M, &p.ctrl->error, s, D->sms))) return st;
    if (select == RMB_SELECT_WEIGHTED) {
        const int64_t tiles = (M->n + kScanTile - 1) / kScanTile;
        uint64_t* parts = reinterpret_cast<uint64_t*>(ws + L.parts);
        uint64_t* cdf = reinterpret_cast<uint64_t*>(ws + L.cdf);
        rmb_wsum_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(O->weights, M->n, parts);
        rmb_wparts_kernel<<<1, kScanThreads, 0, s>>>(parts, tiles);
        rmb_wcdf_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(O->weights, M->n, parts, cdf);
        g_launches += 3;
        if (cudaGetLastError() != cudaSuccess) return RMB_ERR_CUDA;
    }
    void* args[] = {&p};
    cudaError_t ce = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    g_launches++;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return RMB_ERR_CUDA;
    }
    if (!q.stats) return RMB_OK;
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    Ctrl h;
    if (cudaMemcpy(&h, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return RMB_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::memset(q.stats, 0, sizeof(rmb_stats));
    q.stats->sweeps = h.sweeps;
    q.stats->iters = h.iters;
    q.stats->barriers = h.barriers;
    q.stats->residual = h.residual;
    q.stats->v_shift = h.mu;
    q.stats->status = h.status != 0 ? h.status : h.error;
    q.stats->grid_ctas = grid;
    q.stats->path = path;
    q.stats->lanes_per_state = path == PATH_DENSE ? threads : p.lps_all;
    q.stats->ms = ms;
    return q.stats->status;
}

// Fixed scratch of rmb_vi_noalloc: a file-scope device array, one per GPU that loads the library.
// In host code its name is only a host-side stand-in, never a device address: the address is
// looked up once per device with cudaGetSymbolAddress (with that device current) and cached.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RMB_NOALLOC_SCRATCH_BYTES];
void* g_noalloc_ptr[64];

int noalloc_scratch(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RMB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RMB_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RMB_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched solves: autotuner and plan.
//
// Cost model of one MDP solved by G CTAs with batch b (times in microseconds):
//   sweeps(b)  = 0.85 ln(eps) / ln(gamma) * (0.65 + 0.35 (b/n)^0.835)   (VI from V = 0, costs in [0,1];
//                the b-dependence is the fit to the measured sweeps-to-1e-6 of the n = 2^20 CSR MDP)
//   batch time = latency(G) + max(steps * 2.0, b * bytes_per_state / (13000 * G))
//                latency(1) = 1.2 (CTA barrier), latency(G > 1) = 5.0 (grid-group barrier);
//                steps = ceil(b / (states a group processes at once)); 13 GB/s = one SM's share of the
//                measured P-stream rate
//   time       = sweeps(b) * ceil(n/b) * batch time
// Each MDP gets the b minimising its time (unless the caller fixed b).  The makespan target M is
// found by bisection: MDPs whose single-CTA time exceeds M get the smallest group that meets M, the
// others are packed onto the remaining CTAs longest-first (LPT); M is feasible if every CTA meets it.
// ------------------------------------------------------------------------------------------------
struct ItemCost {
    int64_t n;
    double bytes_per_state, gamma;
    int concurrency_per_cta;   // states one CTA processes at once
};

double est_sweeps(double gamma, double eps, double frac)
{
    const double e = eps > 1e-12 ? eps : 1e-12;
    const double base = 0.85 * std::log(e) / std::log(gamma);
    const double s = base * (0.65 + 0.35 * std::pow(frac, 0.835));
    return s > 1.0 ? s : 1.0;
}

double est_time_us(const ItemCost& c, int64_t b, int G, double eps)
{
    const double T = (double)((c.n + b - 1) / b);
    const double conc = (double)c.concurrency_per_cta * G;
    const double steps = std::ceil((double)b / conc);
    const double lat = G == 1 ? 1.2 : 5.0;
    const double stream = (double)b * c.bytes_per_state / (13000.0 * G);
    const double per_batch = lat + (steps * 2.0 > stream ? steps * 2.0 : stream);
    return est_sweeps(c.gamma, eps, (double)b / (double)c.n) * T * per_batch;
}

struct ItemPlan {
    int64_t b;
    int G;
    double t;
};

ItemPlan best_b(const ItemCost& c, int G, double eps, int64_t fixed_b)
{
    ItemPlan best{c.n, G, 1e300};
    if (fixed_b > 0) {
        best.b = fixed_b > c.n ? c.n : fixed_b;
        best.t = est_time_us(c, best.b, G, eps);
        return best;
    }
    for (int64_t b = c.n;; b = (b + 1) / 2) {
        const double t = est_time_us(c, b, G, eps);
        if (t < best.t) best = ItemPlan{b, G, t};
        if (b <= 32) break;
    }
    return best;
}

struct BatchPlan {
    std::vector<ItemPlan> items;
    std::vector<int> first_cta;
    std::vector<int> task_off;
    std::vector<BatchTask> tasks;
    double makespan;
};

bool try_makespan(const std::vector<ItemCost>& cs, const std::vector<int64_t>& fixed, int ctas, double eps, double M,
                  BatchPlan* out)
{
    const int N = (int)cs.size();
    std::vector<ItemPlan> ip(N);
    std::vector<int> big, small;
    int used = 0;
    for (int i = 0; i < N; ++i) {
        const ItemPlan one = best_b(cs[i], 1, eps, fixed[i]);
        if (one.t <= M) {
            ip[i] = one;
            small.push_back(i);
            continue;
        }
        bool ok = false;
        for (int G = 2; G <= ctas; G = G < 8 ? G + 1 : G + G / 4) {
            const ItemPlan pg = best_b(cs[i], G, eps, fixed[i]);
            if (pg.t <= M) {
                ip[i] = pg;
                ok = true;
                break;
            }
        }
        if (!ok) return false;
        used += ip[i].G;
        big.push_back(i);
    }
    const int free_ctas = ctas - used;
    if (free_ctas < 0 || (free_ctas == 0 && !small.empty())) return false;
    std::sort(small.begin(), small.end(), [&](int a, int b) { return ip[a].t > ip[b].t; });
    std::vector<double> load(free_ctas > 0 ? free_ctas : 0, 0.0);
    std::vector<std::vector<int>> bins(load.size());
    for (int i : small) {
        int best = 0;
        for (int c = 1; c < (int)load.size(); ++c)
            if (load[c] < load[best]) best = c;
        load[best] += ip[i].t;
        bins[best].push_back(i);
        if (load[best] > M) return false;
    }
    if (!out) return true;
    out->items = ip;
    out->first_cta.assign(N, -1);
    out->task_off.assign(ctas + 1, 0);
    out->tasks.clear();
    std::vector<std::vector<BatchTask>> per(ctas);
    int cta = 0;
    double mk = 0.0;
    for (int i : big) {
        out->first_cta[i] = cta;
        for (int r = 0; r < ip[i].G; ++r) per[cta + r].push_back(BatchTask{i, r, ip[i].G, 0});
        cta += ip[i].G;
        mk = ip[i].t > mk ? ip[i].t : mk;
    }
    for (size_t bI = 0; bI < bins.size(); ++bI) {
        for (int i : bins[bI]) {
            out->first_cta[i] = cta + (int)bI;
            per[cta + bI].push_back(BatchTask{i, 0, 1, 0});
        }
        mk = load[bI] > mk ? load[bI] : mk;
    }
    for (int c = 0; c < ctas; ++c) {
        out->task_off[c + 1] = out->task_off[c] + (int)per[c].size();
        for (const BatchTask& t : per[c]) out->tasks.push_back(t);
    }
    out->makespan = mk;
    return true;
}

int make_batch_plan(const rmb_batch_item* items, int count, const rmb_opts* O, int ctas, BatchPlan* plan)
{
    std::vector<ItemCost> cs(count);
    std::vector<int64_t> fixed(count);
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < count; ++i) {
        const rmb_mdp* M = &items[i].mdp;
        const int64_t nnz_row = M->format == RMB_CSR ? (M->k_uniform > 0 ? M->k_uniform : 16) : M->n;
        cs[i].n = M->n;
        cs[i].gamma = M->gamma;
        cs[i].bytes_per_state = (double)M->m * (double)nnz_row * 8.0 + 4.0 * M->m;
        int lps = 32;
        if (csr_vec_ok(M)) {
            const int k4 = M->k_uniform >> 2;
            const int cpr = k4 < 32 ? k4 : 32;
            const int all = pow2ceil(cpr * M->m);
            lps = all > 32 ? 32 : all;
        }
        cs[i].concurrency_per_cta = (kCsrThreads / 32) * (32 / lps);
        fixed[i] = items[i].batch;
        const ItemPlan one = best_b(cs[i], 1, O->eps, fixed[i]);
        lo += one.t;
        hi = one.t > hi ? one.t : hi;
    }
    lo /= ctas;
    if (hi < lo) hi = lo;
    hi *= 2.0;
    if (!try_makespan(cs, fixed, ctas, O->eps, hi, nullptr)) {
        // even the slowest single-CTA time is infeasible with these CTAs: grow until feasible
        int guard = 0;
        while (!try_makespan(cs, fixed, ctas, O->eps, hi, nullptr) && guard++ < 60) hi *= 2.0;
        if (guard >= 60) return RMB_ERR_UNSUPPORTED;
    }
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (try_makespan(cs, fixed, ctas, O->eps, mid, nullptr)) hi = mid;
        else lo = mid;
        if (hi - lo < 1e-3 * hi) break;
    }
    return try_makespan(cs, fixed, ctas, O->eps, hi, plan) ? RMB_OK : RMB_ERR_UNSUPPORTED;
}

struct BatchLayout {
    size_t ctrl, kps, toff, tasks, items0, total;
    std::vector<size_t> item_off;
};

BatchLayout batch_layout(const rmb_batch_item* items, int count, const BatchPlan& plan, int ctas)
{
    BatchLayout B;
    B.ctrl = 256;
    B.kps = B.ctrl + align_up((size_t)count * sizeof(Ctrl), 256);
    B.toff = B.kps + align_up((size_t)count * sizeof(KP), 256);
    B.tasks = B.toff + align_up((size_t)(ctas + 1) * sizeof(int), 256);
    B.items0 = B.tasks + align_up((size_t)plan.tasks.size() * sizeof(BatchTask) + 16, 256);
    size_t off = B.items0;
    B.item_off.resize(count);
    for (int i = 0; i < count; ++i) {
        B.item_off[i] = off;
        off += layout(items[i].mdp.n, plan.items[i].b).total;
    }
    B.total = off;
    return B;
}

int check_batch(const rmb_batch_item* items, int count, const rmb_opts* O)
{
    if (!items || count < 1 || !O) return RMB_ERR_ARG;
    if (O->max_sweeps < 1 || !(O->eps >= 0.0) || std::isinf(O->eps) || O->start_sweep < 0) return RMB_ERR_ARG;
    if ((O->flags & RMB_FLAG_ASYNC) || O->select != RMB_SELECT_PERMUTATION || O->residual_kind != RMB_RESIDUAL_SWEEP)
        return RMB_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i) {
        const int st = check_mdp(&items[i].mdp);
        if (st) return st;
        if (items[i].mdp.format != RMB_CSR) return RMB_ERR_UNSUPPORTED;
        if (!items[i].V || items[i].batch < 0) return RMB_ERR_ARG;
    }
    return RMB_OK;
}

int batched_ctas(int* ctas)
{
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    cudaFuncSetAttribute(rmb_batched_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rmb_batched_kernel, kCsrThreads, 0) != cudaSuccess || occ < 1)
        return RMB_ERR_CUDA;
    *ctas = D->sms;   // one CTA per SM (the kernel is register-bound to one 512-thread CTA per SM)
    return RMB_OK;
}

}  // namespace

extern "C" {

size_t rmb_batched_workspace_bytes(const rmb_batch_item* items, int count, const rmb_opts* opts)
{
    if (check_batch(items, count, opts)) return 0;
    int ctas = 0;
    if (batched_ctas(&ctas)) return 0;
    BatchPlan plan;
    if (make_batch_plan(items, count, opts, ctas, &plan)) return 0;
    return batch_layout(items, count, plan, ctas).total;
}

int rmb_batched_plan(const rmb_batch_item* items, int count, const rmb_opts* opts, void* workspace,
                     size_t workspace_bytes, rmb_batch_handle* handle, rmb_batch_plan_item* plan_out, void* stream)
{
    int st = check_batch(items, count, opts);
    if (st) return st;
    if (!handle) return RMB_ERR_ARG;
    int ctas = 0;
    if ((st = batched_ctas(&ctas))) return st;
    BatchPlan plan;
    if ((st = make_batch_plan(items, count, opts, ctas, &plan))) return st;
    const BatchLayout B = batch_layout(items, count, plan, ctas);
    if (!workspace || ((uintptr_t)workspace & 255)) return RMB_ERR_WORKSPACE;
    if (workspace_bytes < B.total) return RMB_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    std::vector<KP> kps(count);
    for (int i = 0; i < count; ++i) {
        const rmb_mdp* M = &items[i].mdp;
        const Layout L = layout(M->n, plan.items[i].b);
        rmb_opts oi = *opts;
        oi.batch = plan.items[i].b;
        oi.trace = nullptr;
        fill_kp(MODE_VI, M, &oi, plan.items[i].b, ws + B.item_off[i], L,
                reinterpret_cast<Ctrl*>(ws + B.ctrl) + i, kps[i]);
        if (kps[i].path == PATH_CSR_VEC && !((kps[i].nc_all == 1 || kps[i].nc_all == 2) && kps[i].nc_one == 1)) {
            if (!M->row_ptr) return RMB_ERR_UNSUPPORTED;
            kps[i].path = PATH_CSR_GEN;
            kps[i].lps_all = kps[i].lps_one = 32;
        }
        kps[i].Vin = items[i].V;
        kps[i].Vout = items[i].V;
        kps[i].pi = items[i].pi;
        kps[i].qgap = items[i].qgap;
        if (plan_out) {
            plan_out[i].batch = plan.items[i].b;
            plan_out[i].group_ctas = plan.items[i].G;
            plan_out[i].first_cta = plan.first_cta[i];
            plan_out[i].est_ms = plan.items[i].t / 1e3;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(ws + B.kps, kps.data(), kps.size() * sizeof(KP), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + B.toff, plan.task_off.data(), plan.task_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(ws + B.tasks, plan.tasks.data(), plan.tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return RMB_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    std::memset(handle, 0, sizeof(*handle));
    handle->workspace = workspace;
    handle->count = count;
    handle->grid_ctas = ctas;
    handle->ntasks = (int32_t)plan.tasks.size();
    handle->ctrl_offset = (int64_t)B.ctrl;
    handle->kp_offset = (int64_t)B.kps;
    handle->toff_offset = (int64_t)B.toff;
    handle->tasks_offset = (int64_t)B.tasks;
    handle->est_ms = plan.makespan / 1e3;
    return RMB_OK;
}

int rmb_batched_run(const rmb_batch_handle* h, void* stream)
{
    if (!h || !h->workspace || h->count < 1 || h->grid_ctas < 1) return RMB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(h->workspace);
    if (cudaMemsetAsync(ws + h->ctrl_offset, 0, (size_t)h->count * sizeof(Ctrl), s) != cudaSuccess) return RMB_ERR_CUDA;
    const KP* kps = reinterpret_cast<const KP*>(ws + h->kp_offset);
    const int* toff = reinterpret_cast<const int*>(ws + h->toff_offset);
    const BatchTask* tasks = reinterpret_cast<const BatchTask*>(ws + h->tasks_offset);
    void* args[] = {(void*)&kps, (void*)&toff, (void*)&tasks};
    const cudaError_t ce = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(rmb_batched_kernel),
                                                       dim3(h->grid_ctas), dim3(kCsrThreads), args, 0, s);
    g_launches++;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return RMB_ERR_CUDA;
    }
    return RMB_OK;
}

int rmb_batched_results(const rmb_batch_handle* h, rmb_stats* out, void* stream)
{
    if (!h || !h->workspace || !out || h->count < 1) return RMB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    std::vector<Ctrl> c(h->count);
    if (cudaMemcpy(c.data(), static_cast<char*>(h->workspace) + h->ctrl_offset, c.size() * sizeof(Ctrl),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return RMB_ERR_CUDA;
    int worst = RMB_OK;
    for (int i = 0; i < h->count; ++i) {
        std::memset(&out[i], 0, sizeof(rmb_stats));
        out[i].sweeps = c[i].sweeps;
        out[i].iters = c[i].iters;
        out[i].barriers = c[i].barriers;
        out[i].residual = c[i].residual;
        out[i].v_shift = c[i].mu;
        out[i].status = c[i].status != 0 ? c[i].status : c[i].error;
        out[i].path = -1;
        if (out[i].status != RMB_OK && worst == RMB_OK) worst = out[i].status;
    }
    return worst;
}

int rmb_batched_graph_create(const rmb_batch_handle* h, void* stream, void** graph_exec)
{
    if (!h || !graph_exec || !stream) return RMB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RMB_ERR_CUDA;
    const int st = rmb_batched_run(h, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != RMB_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != RMB_OK ? st : RMB_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        return RMB_ERR_CUDA;
    }
    *graph_exec = ex;
    return RMB_OK;
}

int rmb_batched_graph_launch(void* graph_exec, void* stream)
{
    if (!graph_exec) return RMB_ERR_ARG;
    g_launches++;
    return cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? RMB_OK
               : RMB_ERR_CUDA;
}

int rmb_batched_graph_destroy(void* graph_exec)
{
    if (!graph_exec) return RMB_ERR_ARG;
    return cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec)) == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}


size_t rmb_workspace_bytes(const rmb_mdp* mdp, const rmb_opts* opts)
{
    if (check_mdp(mdp)) return 0;
    int64_t b = mdp->n;
    if (opts && opts->batch >= 1) b = opts->batch > mdp->n ? mdp->n : opts->batch;
    return layout(mdp->n, b, opts ? opts->select : RMB_SELECT_PERMUTATION).total;
}

int rmb_vi(const rmb_mdp* mdp, const rmb_opts* opts, float* V_inout, int32_t* pi_out, float* qgap_out,
           void* workspace, size_t workspace_bytes, rmb_stats* stats, void* stream)
{
    Call q{MODE_VI, mdp, opts, V_inout, V_inout, nullptr, pi_out, qgap_out, nullptr,
           workspace, workspace_bytes, stats, static_cast<cudaStream_t>(stream)};
    return solve(q);
}

int rmb_mpi(const rmb_mdp* mdp, const rmb_opts* opts, float* V_inout, int32_t* pi_out, float* qgap_out,
            void* workspace, size_t workspace_bytes, rmb_stats* stats, void* stream)
{
    Call q{MODE_MPI, mdp, opts, V_inout, V_inout, nullptr, pi_out, qgap_out, nullptr,
           workspace, workspace_bytes, stats, static_cast<cudaStream_t>(stream)};
    return solve(q);
}

int rmb_eval_policy(const rmb_mdp* mdp, const int32_t* pi, const rmb_opts* opts, float* V_inout,
                    void* workspace, size_t workspace_bytes, rmb_stats* stats, void* stream)
{
    Call q{MODE_EVAL, mdp, opts, V_inout, V_inout, nullptr, nullptr, nullptr, pi,
           workspace, workspace_bytes, stats, static_cast<cudaStream_t>(stream)};
    return solve(q);
}

int rmb_greedy(const rmb_mdp* mdp, const rmb_opts* opts, const float* V, float* TV_out, int32_t* pi_out,
               float* qgap_out, void* workspace, size_t workspace_bytes, rmb_stats* stats, void* stream)
{
    Call q{MODE_GREEDY, mdp, opts, V, nullptr, TV_out, pi_out, qgap_out, nullptr,
           workspace, workspace_bytes, stats, static_cast<cudaStream_t>(stream)};
    return solve(q);
}

int rmb_permutation(int64_t n, uint64_t seed, uint64_t sweep, int32_t* out, void* stream)
{
    if (n < 1 || !out) return RMB_ERR_ARG;
    if (n >= ((int64_t)1 << 31)) return RMB_ERR_UNSUPPORTED;
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)D->sms * 8);
    rmb_perm_kernel<<<blocks, 256, 0, s>>>((uint32_t)n, perm_half_bits(n), (uint32_t)seed, (uint32_t)(seed >> 32),
                                           (uint32_t)sweep, (uint32_t)(sweep >> 32), out);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

int rmb_validate(const rmb_mdp* mdp, void* workspace, size_t workspace_bytes, void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < 256) return RMB_ERR_WORKSPACE;
    DevInfo* D = nullptr;
    if ((st = dev_info(&D))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = static_cast<int*>(workspace);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return RMB_ERR_CUDA;
    if ((st = launch_validate(mdp, err, s, D->sms))) return st;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RMB_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    return h;
}

int rmb_softmax_rows(const rmb_mdp* mdp, const float* logits, float* prob_out, void* stream)
{
    if (!mdp || !logits || !prob_out) return RMB_ERR_ARG;
    if (mdp->format != RMB_CSR || mdp->k_uniform <= 0 || mdp->n < 1 || mdp->m < 1) return RMB_ERR_ARG;
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    const int64_t rows = mdp->n * (int64_t)mdp->m;
    const int blocks = (int)std::min<int64_t>((rows + 7) / 8, (int64_t)D->sms * 16);
    rmb_softmax_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, mdp->k_uniform, logits, prob_out);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

size_t rmb_residual_weights_workspace_bytes(const rmb_mdp* mdp)
{
    if (check_mdp(mdp)) return 0;
    // one Bellman pass (b = n) + TV [n] + the maximum
    return layout(mdp->n, mdp->n).total + align_up((size_t)mdp->n * 4, 256) + 256;
}

int rmb_residual_weights(const rmb_mdp* mdp, const float* V, float floor_frac, uint32_t* weights_out,
                         void* workspace, size_t workspace_bytes, void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (!V || !weights_out || !(floor_frac >= 0.f && floor_frac <= 1.f)) return RMB_ERR_ARG;
    const size_t need = rmb_residual_weights_workspace_bytes(mdp);
    if (!workspace || ((uintptr_t)workspace & 255)) return RMB_ERR_WORKSPACE;
    if (workspace_bytes < need) return RMB_ERR_WORKSPACE;
    const size_t g = layout(mdp->n, mdp->n).total;
    char* ws = static_cast<char*>(workspace);
    float* TV = reinterpret_cast<float*>(ws + g);
    uint32_t* rmax = reinterpret_cast<uint32_t*>(ws + g + align_up((size_t)mdp->n * 4, 256));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rmb_opts o;
    std::memset(&o, 0, sizeof(o));
    o.batch = mdp->n;
    o.max_sweeps = 1;
    Call q{MODE_GREEDY, mdp, &o, V, nullptr, TV, nullptr, nullptr, nullptr, ws, g, nullptr, s};
    if ((st = solve(q))) return st;
    DevInfo* D = nullptr;
    if ((st = dev_info(&D))) return st;
    if (cudaMemsetAsync(rmax, 0, sizeof(uint32_t), s) != cudaSuccess) return RMB_ERR_CUDA;
    const int grid = D->sms * 4;
    rmb_resid_max_kernel<<<grid, 256, 0, s>>>(TV, V, mdp->n, rmax);
    rmb_resid_weights_kernel<<<grid, 256, 0, s>>>(TV, V, mdp->n, floor_frac, rmax, weights_out);
    g_launches += 2;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

size_t rmb_fixed_point_grad_workspace_bytes(const rmb_mdp* mdp, const rmb_opts* opts)
{
    if (check_mdp(mdp) || mdp->format != RMB_CSR || mdp->k_uniform <= 0) return 0;
    int64_t b = mdp->n;
    if (opts && opts->batch >= 1) b = opts->batch > mdp->n ? mdp->n : opts->batch;
    return grad_layout(mdp->n, mdp->k_uniform, b).total;
}

int rmb_fixed_point_grad(const rmb_mdp* mdp, const int32_t* pi, const float* V, const float* w, const rmb_opts* opts,
                         float* lambda_out, float* grad_cost, float* grad_logits, void* workspace,
                         size_t workspace_bytes, rmb_stats* stats, void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (mdp->format != RMB_CSR || mdp->k_uniform <= 0) return RMB_ERR_UNSUPPORTED;
    if (mdp->n * (int64_t)mdp->k_uniform >= ((int64_t)1 << 31)) return RMB_ERR_UNSUPPORTED;
    if (!pi || !V || !w || !lambda_out || !opts) return RMB_ERR_ARG;
    if (opts->batch < 1 || opts->max_sweeps < 1 || !(opts->eps >= 0.0) || std::isinf(opts->eps)) return RMB_ERR_ARG;
    if (opts->select != RMB_SELECT_PERMUTATION) return RMB_ERR_UNSUPPORTED;
    const int64_t n = mdp->n;
    const int k = mdp->k_uniform;
    const int64_t b = opts->batch > n ? n : opts->batch;
    const GradLayout G = grad_layout(n, k, b);
    if (!workspace || ((uintptr_t)workspace & 255)) return RMB_ERR_WORKSPACE;
    if (workspace_bytes < G.total) return RMB_ERR_WORKSPACE;
    DevInfo* D = nullptr;
    if ((st = dev_info(&D))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    int64_t* rowT = reinterpret_cast<int64_t*>(ws + G.rowT);
    int32_t* colT = reinterpret_cast<int32_t*>(ws + G.colT);
    float* probT = reinterpret_cast<float*>(ws + G.probT);
    int32_t* cnt = reinterpret_cast<int32_t*>(ws + G.cnt);
    int32_t* zpi = reinterpret_cast<int32_t*>(ws + G.zpi);
    // 1. the transposed greedy chain: row j lists (i, p_ij(pi(i))) for every predecessor i
    if (cudaMemsetAsync(cnt, 0, (size_t)n * 4, s) != cudaSuccess) return RMB_ERR_CUDA;
    if (cudaMemsetAsync(zpi, 0, (size_t)n * 4, s) != cudaSuccess) return RMB_ERR_CUDA;
    const int eb = (int)std::min<int64_t>((n * k + 255) / 256, (int64_t)D->sms * 16);
    rmb_tr_count_kernel<<<eb, 256, 0, s>>>((int)n, mdp->m, k, pi, mdp->col, cnt);
    rmb_tr_scan_kernel<<<1, 1024, 0, s>>>((int)n, cnt, rowT, cnt);
    rmb_tr_scatter_kernel<<<eb, 256, 0, s>>>((int)n, mdp->m, k, pi, mdp->col, mdp->prob, cnt, colT, probT);
    const int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)D->sms * 8);
    rmb_tr_sort_kernel<<<nb, 256, 0, s>>>((int)n, rowT, colT, probT);
    g_launches += 4;
    if (cudaGetLastError() != cudaSuccess) return RMB_ERR_CUDA;
    // 2. adjoint sweeps lambda <- w + gamma P_pi^T lambda (mini-batch, one row per state), from lambda = w
    rmb_mdp mt;
    std::memset(&mt, 0, sizeof(mt));
    mt.n = n;
    mt.m = 1;
    mt.format = RMB_CSR;
    mt.row_ptr = rowT;
    mt.col = colT;
    mt.prob = probT;
    mt.cost = w;
    mt.gamma = mdp->gamma;
    rmb_opts o2 = *opts;
    o2.flags |= RMB_FLAG_RAW_ROWS;
    o2.validate = 0;
    if (cudaMemcpyAsync(lambda_out, w, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return RMB_ERR_CUDA;
    Call q{MODE_EVAL, &mt, &o2, lambda_out, lambda_out, nullptr, nullptr, nullptr, zpi,
           ws + G.eval, G.total - G.eval, stats, s};
    st = solve(q);
    if (st != RMB_OK && st != RMB_ERR_NOT_CONVERGED) return st;
    // 3. gradients
    if (grad_cost && cudaMemsetAsync(grad_cost, 0, (size_t)n * mdp->m * 4, s) != cudaSuccess) return RMB_ERR_CUDA;
    if (grad_logits && cudaMemsetAsync(grad_logits, 0, (size_t)n * mdp->m * k * 4, s) != cudaSuccess) return RMB_ERR_CUDA;
    if (grad_cost || grad_logits) {
        const int gb = (int)std::min<int64_t>((n + 7) / 8, (int64_t)D->sms * 16);
        rmb_grad_kernel<<<gb, 256, 0, s>>>((int)n, mdp->m, k, (float)mdp->gamma, pi, mdp->col, mdp->prob, V, lambda_out,
                                           grad_cost, grad_logits);
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return RMB_ERR_CUDA;
    }
    if (stats && cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    return st;
}

int rmb_quantize_rows(const float* P, int64_t rows, int64_t cols, int32_t p_dtype, void* codes, float* scale,
                      void* stream)
{
    if (!P || !codes || rows < 1 || cols < 1) return RMB_ERR_ARG;
    if (p_dtype != RMB_P_BF16 && p_dtype != RMB_P_FP8E4M3) return RMB_ERR_ARG;
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    const int blocks = (int)std::min<int64_t>((rows + 7) / 8, (int64_t)D->sms * 16);
    rmb_quantize_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(P, rows, cols, p_dtype, codes, scale);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

int rmb_vi_refined(const rmb_mdp* lowp, const rmb_mdp* ref, const rmb_opts* opts, double eps_low, float* V_inout,
                   int32_t* pi_out, float* qgap_out, void* workspace, size_t workspace_bytes, rmb_stats* stats_low,
                   rmb_stats* stats_ref, void* stream)
{
    int st = check_mdp(lowp);
    if (st) return st;
    if ((st = check_mdp(ref))) return st;
    if (!opts || !(eps_low >= 0.0) || std::isinf(eps_low)) return RMB_ERR_ARG;
    if (lowp->n != ref->n || lowp->m != ref->m || lowp->gamma != ref->gamma || lowp->cost != ref->cost)
        return RMB_ERR_ARG;
    rmb_opts o1 = *opts;
    o1.eps = eps_low;
    o1.trace = nullptr;
    Call q1{MODE_VI, lowp, &o1, V_inout, V_inout, nullptr, nullptr, nullptr, nullptr,
            workspace, workspace_bytes, stats_low, static_cast<cudaStream_t>(stream)};
    st = solve(q1);
    if (st != RMB_OK && st != RMB_ERR_NOT_CONVERGED) return st;
    rmb_opts o2 = *opts;
    o2.trace = nullptr;
    Call q2{MODE_VI, ref, &o2, V_inout, V_inout, nullptr, pi_out, qgap_out, nullptr,
            workspace, workspace_bytes, stats_ref, static_cast<cudaStream_t>(stream)};
    return solve(q2);
}

int rmb_gather_probe(const float* src, int64_t n_src, const int32_t* idx, int64_t n_idx, int reps, float* out,
                     void* stream)
{
    if (!src || !idx || !out || n_src < 1 || n_src >= ((int64_t)1 << 32) || n_idx < 4 || (n_idx & 3) || reps < 1)
        return RMB_ERR_ARG;
    if (((uintptr_t)idx) & 15) return RMB_ERR_ARG;
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    cudaFuncSetAttribute(rmb_gather_probe_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    rmb_gather_probe_kernel<<<D->sms, 512, 0, static_cast<cudaStream_t>(stream)>>>(
        src, (uint32_t)(n_src - 1), reinterpret_cast<const int4*>(idx), n_idx / 4, reps, out);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
}

const char* rmb_status_string(int status)
{
    switch (status) {
    case RMB_OK: return "ok";
    case RMB_ERR_ARG: return "invalid argument";
    case RMB_ERR_CUDA: return "CUDA runtime error";
    case RMB_ERR_NOT_CONVERGED: return "not converged within the sweep limit";
    case RMB_ERR_BARRIER_TIMEOUT: return "grid-wide wait timed out";
    case RMB_ERR_INVALID_MDP: return "invalid MDP (probability, index, row sum or cost)";
    case RMB_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case RMB_ERR_UNSUPPORTED: return "unsupported size or layout";
    case RMB_ERR_NONFINITE: return "non-finite value";
    case RMB_ERR_TOO_LARGE: return "problem needs more scratch than the fixed no-allocation array holds";
    default: return "unknown status";
    }
}

int rmb_vi_noalloc(const rmb_mdp* mdp, const rmb_opts* opts, float* V_inout, int32_t* pi_out, float* qgap_out,
                   rmb_stats* stats, void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (!opts) return RMB_ERR_ARG;
    const size_t need = rmb_workspace_bytes(mdp, opts);
    if (need == 0) return RMB_ERR_ARG;
    if (need > RMB_NOALLOC_SCRATCH_BYTES) return RMB_ERR_TOO_LARGE;
    void* ws = nullptr;
    if ((st = noalloc_scratch(&ws))) return st;
    st = rmb_vi(mdp, opts, V_inout, pi_out, qgap_out, ws, RMB_NOALLOC_SCRATCH_BYTES, nullptr, stream);
    if (st != RMB_OK || !stats) return st;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return RMB_ERR_CUDA;
    Ctrl h;
    if (cudaMemcpy(&h, ws, sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return RMB_ERR_CUDA;
    std::memset(stats, 0, sizeof(rmb_stats));
    stats->sweeps = h.sweeps;
    stats->iters = h.iters;
    stats->barriers = h.barriers;
    stats->residual = h.residual;
    stats->v_shift = h.mu;
    stats->status = h.status != 0 ? h.status : h.error;
    stats->path = -1;
    return stats->status;
}

uint64_t rmb_kernel_launches(void) { return g_launches.load(); }

int rmb_version(void) { return (1 << 16) | 0; }

}  // extern "C"
