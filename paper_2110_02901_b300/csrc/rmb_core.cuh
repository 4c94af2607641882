#pragma once
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
enum Path { PATH_DENSE = 0, PATH_CSR_VEC = 1, PATH_CSR_GEN = 2, PATH_DENSE_TMA = 3, PATH_CLUSTER = 4 };
enum Kind { K_MIN = 0, K_POLICY = 1, K_GREEDY = 2 };

constexpr int kCsrThreads = 512;
constexpr int kSoloMaxN = 57344;        // batched MDPs up to this n keep their values in shared memory
                                        // (SoloRun): 224 KB of the batched launch
constexpr int kSoloSplitMaxN = 81920;   // ... up to this n the first kSoloMaxN of them (SPLIT)
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
    // the loaded rows are contiguous, k = 4 k4 entries each: chunk ci of them starts 4 ci entries
    // after the first row's start, and belongs to row ci >> log2 k4
    const int64_t r0 = (int64_t)s * p.m + (KIND == K_POLICY ? pi_s : 0);
    const int64_t e0 = r0 * p.k;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int ci = c * lps + lane_g;
        const bool v = act && ci < total;
        const int64_t e = e0 + 4 * ci;
        const int64_t r = r0 + (ci >> p.k4_log2);
        if (v) {
            R.p[c] = __ldcs(reinterpret_cast<const float4*>(p.prob + e));
            R.c[c] = __ldcs(reinterpret_cast<const int4*>(p.col + e));
            R.cost[c] = __ldg(p.cost + r);
        } else {
            R.p[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            R.c[c] = make_int4(0, 0, 0, 0);
            R.cost[c] = kInf;
        }
    }
}

__device__ __forceinline__ float lds_f32(uint32_t saddr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(saddr));
    return v;
}

// Where the successor values live: global memory (L1-cached, see gather), this CTA's shared memory,
// or split: states [0, nsm) in shared memory and the rest in global memory H (read from L2).
enum ValueMem { VM_GLOBAL = 0, VM_SHARED = 1, VM_SPLIT = 2 };

template <int VM>
__device__ __forceinline__ float gather_v(const float* __restrict__ A, int j, uint32_t nm1, const float* H,
                                          uint32_t nsm)
{
    if (VM == VM_SHARED) return lds_f32((uint32_t)__cvta_generic_to_shared(A) + 4u * min((uint32_t)j, nm1));
    if (VM == VM_SPLIT) {
        // one generic load for either space (the cache operator applies to the global part only)
        const uint32_t jj = min((uint32_t)j, nm1);
        const float* q = (jj < nsm ? A : H) + jj;
        float v;
        asm volatile("ld.cg.f32 %0, [%1];" : "=f"(v) : "l"(q));
        return v;
    }
    return gather(A, j, nm1);
}

// min (and, with ARG, the lowest arg-min and the second smallest value) over the state's rows of
// c + gamma * sum p * A[col]; every lane of the group gets the result
template <bool ARG, int NC, int VM = VM_GLOBAL>
__device__ __forceinline__ Best fast_eval(const KP& p, const StateRegs<NC>& R, const float* __restrict__ A, int lps,
                                          int lane_g, const float* H = nullptr, uint32_t nsm = 0)
{
    const uint32_t nm1 = (uint32_t)(p.n - 1);
    float part[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float g0 = gather_v<VM>(A, R.c[c].x, nm1, H, nsm), g1 = gather_v<VM>(A, R.c[c].y, nm1, H, nsm);
        const float g2 = gather_v<VM>(A, R.c[c].z, nm1, H, nsm), g3 = gather_v<VM>(A, R.c[c].w, nm1, H, nsm);
        part[c] = fmaf(R.p[c].x, g0, fmaf(R.p[c].y, g1, fmaf(R.p[c].z, g2, R.p[c].w * g3)));
    }
    // the two butterfly stages as fixed five-level ladders with warp-uniform conditions (no loop
    // counters): sums within a row (offsets < k4), then the minimum over rows (k4 <= offset < lps)
    const int k4l = p.k4_log2;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        if (l < k4l) {
#pragma unroll
            for (int c = 0; c < NC; ++c) part[c] += __shfl_xor_sync(0xffffffffu, part[c], 1 << l);
        }
    }
    Best b = {kInf, 0x7fffffff, kInf};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float q = R.cost[c] == kInf ? kInf : fmaf(p.gamma, part[c], R.cost[c]);
        if (ARG) b = better(b, Best{q, (c * lps + lane_g) >> k4l, kInf});
        else b.q = fminf(b.q, q);
    }
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const int off = 1 << l;
        if (l >= k4l && off < lps) {
            if (ARG) b = better(b, shfl_xor_best<true>(b, off));
            else b.q = fminf(b.q, __shfl_xor_sync(0xffffffffu, b.q, off));
        }
    }
    return b;
}

struct FastGeom {
    int lane, spw, per_block, pb_mask, g, lane_g, U, first, my_off, my_step;
    __device__ FastGeom(int lps, const GroupView& gv)
    {
        lane = threadIdx.x & 31;
        const int warp = (gv.rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
        const int nwarps = (gv.size * (int)blockDim.x) >> 5;
        spw = 32 / lps;
        per_block = 32 / spw;          // steps covered by one permutation evaluation per lane (= lps)
        pb_mask = per_block - 1;       // lps is a power of two: j % per_block = j & pb_mask
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
            if ((jn & G.pb_mask) == 0) block_states = G.resolve(jn, pos0, len, K, perm_ok);
            s_nxt = __shfl_sync(0xffffffffu, block_states, (jn & G.pb_mask) * G.spw + G.g);
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
        // e4m3 pairs to f16 pairs (exact), then each f16 to f32 (exact): three conversions per 4 bytes
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t h01, h23;
            asm("{ .reg .b16 lo, hi;\n\t"
                "mov.b32 {lo, hi}, %2;\n\t"
                "cvt.rn.f16x2.e4m3x2 %0, lo;\n\t"
                "cvt.rn.f16x2.e4m3x2 %1, hi; }"
                : "=r"(h01), "=r"(h23) : "r"(u[i]));
            asm("{ .reg .b16 a, b, c, e;\n\t"
                "mov.b32 {a, b}, %4;\n\t"
                "mov.b32 {c, e}, %5;\n\t"
                "cvt.f32.f16 %0, a;\n\t"
                "cvt.f32.f16 %1, b;\n\t"
                "cvt.f32.f16 %2, c;\n\t"
                "cvt.f32.f16 %3, e; }"
                : "=f"(d[4 * i]), "=f"(d[4 * i + 1]), "=f"(d[4 * i + 2]), "=f"(d[4 * i + 3]) : "r"(h01), "r"(h23));
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
// cp.async.bulk (mbarrier transaction counts); consumer warps decode them and multiply with the
// current values, staged once per batch.  Memory-level parallelism is the ring (kRingStages x
// kStageBytes per SM), not registers, so coded rows (bf16 / fp8) stream as fast as float32 rows.
// The consumers never wait for each other: each writes its partial row sums of a row group into one of
// two slots and arrives on the slot's mbarrier; a reducer warp sums the slots, forms Q(s, a), and
// finishes each state (min over actions, new value), then frees the slot.
// Every wait is bounded; after a timeout all threads still pass the same barriers (abort flag).
// ------------------------------------------------------------------------------------------------
constexpr int kTmaConsumers = 16;                   // consumer warps
constexpr int kTmaThreads = (kTmaConsumers + 2) * 32;   // + the producer warp and the reducer warp
constexpr int kRingStages = 2;
constexpr int kStageBytes = 65536;
constexpr int kTmaRowGroup = 8;                     // rows per stage (all-action passes)
constexpr int kTmaMaxStates = 512;                  // states per chunk of a batch

struct TmaSmem {
    uint64_t full[kRingStages];
    uint64_t empty[kRingStages];
    uint64_t red_full[2];    // a slot's partial sums are written (one arrival per consumer warp)
    uint64_t red_empty[2];   // the reducer has read the slot
    uint64_t vbar;
    uint32_t vphase;
    int abort;
    int ids[kTmaMaxStates];
    int pis[kTmaMaxStates];
    float red[2][kTmaConsumers][kTmaRowGroup];
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


template <int KIND, int DT>
__device__ bool dense_batch_tma(const KP& p, const GroupView& gv, TmaSmem& sm, float* vst, unsigned char* ring,
                                uint32_t& ring_it, uint32_t& red_it, const float* A, float* B, int pos0, int len,
                                const PermKey* K, int32_t* Sout, float* Wout, const Centre& C, Acc& acc,
                                bool* perm_ok)
{
    constexpr int EB = Elem<DT>::bytes;
    constexpr int E = Elem<DT>::per16;
    const int n = p.n;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const bool producer = wid == kTmaConsumers;
    const bool reducer = wid == kTmaConsumers + 1;
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
        } else if (reducer) {
            uint32_t rit = red_it;
            for (int i = 0; i < cnt; ++i) {
                const int s = sm.ids[i];
                bool all_ok = true;
                for (int g = 0; g < ngroups; ++g, ++rit) {
                    const int a0 = g * RG;
                    const int rg = min(RG, nrows - a0);
                    const int slot = (int)(rit & 1u);
                    const bool ok = mb_wait((uint32_t)__cvta_generic_to_shared(&sm.red_full[slot]), (rit >> 1) & 1u, p,
                                            abort_flag);
                    all_ok = all_ok && ok;
                    if (ok && lane < rg) {
                        float tot = 0.f;
                        for (int w = 0; w < kTmaConsumers; ++w) tot += sm.red[slot][w][lane];
                        const int a = KIND == K_POLICY ? sm.pis[i] : a0 + lane;
                        const int64_t r = (int64_t)s * p.m + a;
                        if (DT != RMB_P_F32) tot *= __ldg(p.row_scale + r);
                        const float c = __ldg(p.cost + r);
                        sm.q[KIND == K_POLICY ? 0 : a0 + lane] = (c == kInf) ? kInf : fmaf(p.gamma, tot, c);
                    }
                    __syncwarp();
                    if (lane == 0 && ok)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                                     ::"r"((uint32_t)__cvta_generic_to_shared(&sm.red_empty[slot])) : "memory");
                }
                if (lane == 0 && all_ok && !*abort_flag) {
                    Best best = {kInf, 0x7fffffff, kInf};
                    for (int ai = 0; ai < nrows; ++ai)
                        best = better(best, Best{sm.q[ai], KIND == K_POLICY ? sm.pis[i] : ai, kInf});
                    state_epilogue<KIND>(p, best, s, me + (c0 + i) * G, A, B, Sout, Wout, C, acc);
                }
                __syncwarp();
            }
        } else {
            uint32_t rit = red_it;
            uint32_t it = ring_it;
            for (int i = 0; i < cnt; ++i) {
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
#pragma unroll 2
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
                    // this warp's row sums into the group's slot, once the reducer has freed it
#pragma unroll
                    for (int r = 0; r < kTmaRowGroup; ++r) {
                        float x = accv[r];
                        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                        accv[r] = x;
                    }
                    const int slot = (int)(rit & 1u);
                    const uint32_t use = rit >> 1;
                    const bool free_ok = use == 0 || mb_wait((uint32_t)__cvta_generic_to_shared(&sm.red_empty[slot]),
                                                             (use - 1) & 1u, p, abort_flag);
                    if (free_ok && lane == 0) {
#pragma unroll
                        for (int r = 0; r < kTmaRowGroup; ++r) sm.red[slot][wid][r] = accv[r];
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];"
                                     ::"r"((uint32_t)__cvta_generic_to_shared(&sm.red_full[slot])) : "memory");
                    }
                    ++rit;
                }
            }
        }
        // every thread advances the ring and slot counters by the tiles and row groups of this chunk
        ring_it += (uint32_t)(cnt * ngroups * ntiles);
        red_it += (uint32_t)(cnt * ngroups);
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
    uint32_t red_it = 0;           // dense TMA path: row groups reduced so far (same in every thread)

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
            return dense_batch_tma<KIND, DT>(p, gv, *tsm, stage, ring, ring_it, red_it, A, B, pos0, len, K, So, Wo, C, acc,
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
            for (int i = 0; i < 2; ++i) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&tsm->red_full[i])),
                             "r"(kTmaConsumers) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&tsm->red_empty[i]))
                             : "memory");
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

// ------------------------------------------------------------------------------------------------
// MB-VI of one CSR MDP (vectorised rows) by a group of CTAs of the batched launch, each CTA with a
// private copy of all n values in its shared memory.  The same state arithmetic as Runner (fast_load /
// fast_eval, the same lanes per state and the same split of a batch over the group, centred values,
// the same re-centring), so results equal rmb_vi's grid solve bit for bit; successor values come from
// shared memory instead of L2.  A batch's states read the values from before the batch (eq. (11)):
// their (state, value) pairs go to the workspace lists S / W[t & 1], and after the group's barrier
// every CTA writes the whole list into its copy.  The lists alternate from batch to batch, across
// sweeps too: a CTA writes a list again two batches later, after the barrier of the batch between,
// which every CTA reaches only after it has applied the list.  A one-CTA group uses CTA barriers only.
// SPLIT: n is larger than the shared memory holds; states [nsm, n) keep their values in global memory
// (read from L2), in one of two buffers.  Every CTA writes every entry of a list into that part too, so
// a CTA's own writes complete it before its next batch reads it, and the writes of other CTAs store
// the same values; a re-centring writes the shifted values into the other buffer (the same values
// from every CTA), which the next shift two sweeps later overwrites only after every CTA has crossed
// a barrier that follows its last read of it.
// ------------------------------------------------------------------------------------------------
template <int NCA, bool SPLIT = false>
struct SoloRun {
    const KP& p;
    RedSmem& rs;
    float* Vs;          // centred values of states [0, nsm) (shared memory)
    uint32_t nsm;       // states whose values are in shared memory (n unless SPLIT)
    int hb = 0;         // SPLIT: the global buffer p.d[hb] that holds states [nsm, n)
    GroupView gv;
    Ctrl* c;
    bool lead;          // thread 0 of the group's first CTA
    Centre C;
    long long syncs = 0;
    unsigned long long target = 0;
    int red_epoch = 0;
    bool perm_ok = true;

    __device__ SoloRun(const KP& kp, RedSmem& r, float* v, GroupView g)
        : p(kp), rs(r), Vs(v), nsm(SPLIT ? (uint32_t)kSoloMaxN : (uint32_t)kp.n), gv(g), c(kp.ctrl),
          lead(g.rank == 0 && threadIdx.x == 0) {}

    __device__ float val(int i) const { return (!SPLIT || (uint32_t)i < nsm) ? Vs[i] : ld_l2(p.d[hb] + i); }
    __device__ void set_val(int i, float v)
    {
        if (!SPLIT || (uint32_t)i < nsm) Vs[i] = v;
        else st_l2(p.d[hb] + i, v);
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
        K.select = 0;
        K.wtot = 0;
        K.cdf = nullptr;
        return K;
    }

    __device__ void bar()
    {
        ++syncs;
        __syncthreads();
    }

    // the group's barrier (a CTA barrier for a one-CTA group); false: a CTA reported an error or the
    // wait timed out
    __device__ bool gsync(int site)
    {
        ++syncs;
        if (!perm_ok) atomicCAS(&c->error, 0, RMB_ERR_UNSUPPORTED);
        grid_arrive(c, target, false, gv.size);
        return grid_wait_arrived(c, target, p.timeout_ns, site, gv.size);
    }

    __device__ int gtid() const { return gv.rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ int gthreads() const { return gv.size * (int)blockDim.x; }

    // block-wide max |change|, min, max of the accumulators (every thread gets them)
    __device__ void reduce(Acc& a)
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
            for (int w = 1; w < nw; ++w) {
                a.dmax = fmaxf(a.dmax, rs.v[0][w]);
                a.vlo = fminf(a.vlo, rs.v[1][w]);
                a.vhi = fmaxf(a.vhi, rs.v[2][w]);
            }
            rs.bc[0] = a.dmax;
            rs.bc[1] = a.vlo;
            rs.bc[2] = a.vhi;
        }
        __syncthreads();
        a.dmax = rs.bc[0];
        a.vlo = rs.bc[1];
        a.vhi = rs.bc[2];
        __syncthreads();
    }

    // the state of step j of this lane group (-1 past the end); bs caches the resolved block of steps
    __device__ int step_state(const FastGeom& G, int j, int pos0, int len, const PermKey* K, int& bs, int& bs_j0)
    {
        if (G.first + j * G.U >= len) return -1;
        const int j0 = j & ~G.pb_mask;
        if (j0 != bs_j0) {
            bs = G.resolve(j0, pos0, len, K, &perm_ok);
            bs_j0 = j0;
        }
        return __shfl_sync(0xffffffffu, bs, (j & G.pb_mask) * G.spw + G.g);
    }

    // this CTA's share of positions [pos0, pos0 + len) of the order K (K null: natural order): KIND
    // K_MIN writes (state, value) into S / W[i] (i: the position in the batch); K_GREEDY writes the
    // outputs.  Rows load two steps ahead.
    template <int KIND>
    __device__ void batch(int pos0, int len, const PermKey* K, int32_t* S, float* W, Acc& acc)
    {
        constexpr bool ARG = (KIND == K_GREEDY);
        const float* Hs = SPLIT ? p.d[hb] : nullptr;
        const int lps = p.lps_all;
        const FastGeom G(lps, gv);
        if (G.first >= len) return;
        int bs = 0, bs_j0 = -1;
        int s_cur = step_state(G, 0, pos0, len, K, bs, bs_j0);
        int s_n1 = step_state(G, 1, pos0, len, K, bs, bs_j0);
        StateRegs<NCA> cur, n1, n2;
        fast_load<K_MIN, NCA>(p, s_cur < 0 ? 0 : s_cur, s_cur >= 0, lps, G.lane_g, cur);
        fast_load<K_MIN, NCA>(p, s_n1 < 0 ? 0 : s_n1, s_n1 >= 0, lps, G.lane_g, n1);
        for (int j = 0; G.first + j * G.U < len; ++j) {
            const int s_n2 = step_state(G, j + 2, pos0, len, K, bs, bs_j0);
            fast_load<K_MIN, NCA>(p, s_n2 < 0 ? 0 : s_n2, s_n2 >= 0, lps, G.lane_g, n2);
            const Best r = SPLIT ? fast_eval<ARG, NCA, VM_SPLIT>(p, cur, Vs, lps, G.lane_g, Hs, nsm)
                                 : fast_eval<ARG, NCA, VM_SHARED>(p, cur, Vs, lps, G.lane_g);
            if (s_cur >= 0 && G.lane_g == 0) {
                const float old = val(s_cur);
                const float v = new_value(r.q, C);
                if (v != v) atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
                acc.dmax = fmaxf(acc.dmax, fabsf(v - old));
                if (KIND == K_GREEDY) {
                    if (p.pi) st_l2(p.pi + s_cur, r.a);
                    if (p.qgap) p.qgap[s_cur] = r.q2 - r.q;
                    p.Vout[s_cur] = (float)(C.mu + (double)old);
                } else {
                    acc.vlo = fminf(acc.vlo, v);
                    acc.vhi = fmaxf(acc.vhi, v);
                    const int i = G.first + G.g + j * G.U;
                    st_l2(S + i, s_cur);
                    st_l2(W + i, v);
                }
            }
            cur = n1;
            n1 = n2;
            s_cur = s_n1;
            s_n1 = s_n2;
        }
    }

    // write a batch's (state, value) list into this CTA's values: four pairs per thread in flight
    __device__ void apply_list(const int32_t* S, const float* W, int len)
    {
        const int nt = blockDim.x;
        for (int i0 = threadIdx.x; i0 < len; i0 += 4 * nt) {
            int st[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * nt;
                st[u] = i < len ? ld_l2(S + i) : -1;
                w[u] = i < len ? ld_l2(W + i) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (st[u] >= 0) set_val(st[u], w[u]);
        }
    }

    __device__ float shift_for(float lo, float hi) const
    {
        const float mid = 0.5f * (lo + hi);
        const float spread = hi - lo;
        const float floor_ = 1e-6f * (float)(fabs(C.mu) + 1.0);
        if (!(fabsf(mid) > fmaxf(0.25f * spread, floor_))) return 0.f;
        return mid;
    }

    __device__ void finish(long long sweeps, double residual, bool ok, bool converged)
    {
        if (!perm_ok) atomicCAS(&c->error, 0, RMB_ERR_UNSUPPORTED);
        __syncthreads();
        if (lead) {
            c->sweeps = sweeps;
            c->iters = 0;
            c->barriers = syncs;
            c->residual = residual;
            c->mu = C.mu;
            int st = ld_volatile(&c->error);
            if (st == 0 && ok && !converged) st = RMB_ERR_NOT_CONVERGED;
            c->status = st;
        }
    }

    __device__ void run()
    {
        if (ld_volatile(&c->error) != 0) return;
        // set-up: every CTA reads all start values (the same centre in each)
        Acc a0 = {0.f, kInf, -kInf};
        for (int i = threadIdx.x; i < p.n; i += blockDim.x) {
            const float v = p.Vin[i];
            a0.vlo = fminf(a0.vlo, v);
            a0.vhi = fmaxf(a0.vhi, v);
            if (v != v || fabsf(v) == kInf) atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
        }
        reduce(a0);
        const double mu0 = (double)(float)(0.5 * ((double)a0.vlo + (double)a0.vhi));
        C = make_centre(mu0, p.gamma_d);
        for (int i = threadIdx.x; i < p.n; i += blockDim.x) set_val(i, (float)((double)p.Vin[i] - mu0));
        bar();
        long long sweeps = 0;
        double residual = 0.0;
        bool converged = false, ok = ld_volatile(&c->error) == 0;
        const bool ordered = p.T > 1;
        const bool multi = gv.size > 1;
        unsigned nbatch = 0;   // batches done (the list parity)
        for (long long j = 0; ok && j < p.max_sweeps; ++j) {
            const long long k = p.start_sweep + j;
            PermKey K = key_for(k);
            if (p.perm_buf && ordered) {
                // the whole order of the sweep, then the batches read it (the group's last barrier of
                // the previous sweep ordered every read of the previous order before these writes)
                for (int i = gtid(); i < p.n; i += gthreads())
                    st_l2(p.perm_buf + i, order_at((uint32_t)i, K, &perm_ok));
                if (!gsync(40)) { ok = false; break; }
                K.buf = p.perm_buf;
            }
            const int slot = red_epoch % 3;
            if (multi && lead) {
                const int nxt = (red_epoch + 1) % 3;
                c->red_delta[nxt] = 0u;
                c->red_hi[nxt] = 0u;
                c->red_nlo[nxt] = 0u;
            }
            ++red_epoch;
            Acc acc = {0.f, kInf, -kInf};
            for (int t = 0; ok && t < p.T; ++t) {
                const int len = (t == p.T - 1) ? p.last_len : p.b;
                const int par = multi ? (int)(nbatch++ & 1u) : 0;
                int32_t* S = p.S[par];
                float* W = p.W[par];
                batch<K_MIN>(t * p.b, len, ordered ? &K : nullptr, S, W, acc);
                if (multi && t == p.T - 1) publish(c, slot, acc, rs);
                if (!gsync(41)) { ok = false; break; }
                apply_list(S, W, len);
                bar();
            }
            if (!ok) break;
            if (multi) {
                read_slot(c, slot, rs, acc.dmax, acc.vlo, acc.vhi);
            } else {
                reduce(acc);
            }
            ++sweeps;
            residual = (double)acc.dmax;
            if (lead && p.trace) p.trace[j] = residual;
            if (acc.dmax != acc.dmax) {
                atomicCAS(&c->error, 0, RMB_ERR_NONFINITE);
                ok = false;
                break;
            }
            if (ld_volatile(&c->error) != 0) {
                ok = false;
                break;
            }
            if ((double)acc.dmax <= p.eps) {
                converged = true;
                break;
            }
            // the grid solve ends its last sweep without re-centring; so does this one (same outputs)
            const float sh = j + 1 < p.max_sweeps ? shift_for(acc.vlo, acc.vhi) : 0.f;
            if (sh != 0.f) {
                for (int i = threadIdx.x; i < (int)nsm; i += blockDim.x) Vs[i] -= sh;
                if (SPLIT) {
                    for (int i = (int)nsm + threadIdx.x; i < p.n; i += blockDim.x)
                        st_l2(p.d[hb ^ 1] + i, ld_l2(p.d[hb] + i) - sh);
                    hb ^= 1;
                }
                C = make_centre(C.mu + (double)sh, p.gamma_d);
                bar();
            }
        }
        if (ok) {
            if (p.pi || p.qgap) {
                Acc g = {0.f, kInf, -kInf};
                batch<K_GREEDY>(0, p.n, nullptr, nullptr, nullptr, g);
            } else {
                for (int i = gtid(); i < p.n; i += gthreads()) p.Vout[i] = (float)(C.mu + (double)val(i));
            }
        }
        finish(sweeps, residual, ok, converged);
    }
};

// ------------------------------------------------------------------------------------------------
// Batched solves: many independent MDPs in one persistent launch.  Every CTA runs a list of tasks; a
// task is one MDP solved by a group of CTAs (its own barrier counter and control block) or by this
// CTA alone (barriers are then CTA barriers).  CTAs of a multi-CTA group run the same task list.
// ------------------------------------------------------------------------------------------------
struct BatchTask {
    int item, rank, size, pad;
};


// Addresses of the persistent kernels.  Each kernel family lives in its own translation unit
// (rmb_csr.cu: CSR and batched kernels, rmb_dense.cu) so that the library compiles in parallel; the host
// code launches them through these addresses.
const void* csr_vec_kernel_for(int nca, int nco);   // rmb_csr_vec_kernel<NCA, NCO>
const void* csr_gen_kernel_ptr();                    // rmb_csr_gen_kernel
const void* dense_kernel_ptr(int p_dtype);           // rmb_dense_kernel<DT>
const void* dense_tma_kernel_ptr(int p_dtype);       // rmb_dense_tma_kernel<DT>
const void* batched_kernel_ptr();                    // rmb_batched_kernel
const void* small_kernel_ptr(int nc);                // rmb_small_kernel<NC> (one cluster, values in shared memory)
constexpr int kSmallThreads = 512;
constexpr int kSmallMaxPer = 2;                      // states per warp and batch in rmb_small_kernel
constexpr int kSmallMaxDyn = 220 * 1024;             // its dynamic shared memory: 16 bytes per state + 16

}  // namespace rmb
