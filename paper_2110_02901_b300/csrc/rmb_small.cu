// librmb: MB-VI of a small MDP on one thread-block cluster (a translation unit of its own so that the
// library compiles in parallel).
//
// For MDPs whose values fit in shared memory and whose batches are small, a solve is bound by the
// latency of every batch (eq. (11) makes batch t+1 wait for batch t), and the grid-wide barrier through
// an L2 counter is most of that.  Here one cluster of C CTAs (C <= 16) runs the whole solve:
//   - every CTA holds its own copy of the (centred) values in shared memory, so successor reads are
//     shared-memory loads.  Batch t's positions are spread over the CTAs round robin; each CTA computes
//     its states of the batch from its copy, which holds the values from before the batch (eq. (11)),
//     and writes (state, new value) pairs into a small list in its shared memory;
//   - batches are separated by the hardware cluster barrier (arrive with release, wait with acquire at
//     cluster scope).  After it, every CTA reads all C lists of the batch (one distributed-shared-memory
//     load per thread) and writes their values into its copy, so every copy holds batches <= t new
//     before batch t+1 starts.  The lists alternate between two buffers by batch parity: a list is
//     rewritten only after every CTA has passed the barrier that follows its readers;
//   - between the arrival at and the wait on each barrier, every warp loads the transition rows of its
//     states of the next batch (rows do not depend on values; the order is computed per CTA for its own
//     positions during the previous sweep), so a batch costs shared-memory gathers, not L2 round trips;
//   - every control decision (stop, re-centre, abort) is taken from values every CTA reads after the
//     same barrier: an error is stored into every CTA's error word before a barrier and read after it,
//     so all CTAs leave the sweep loop at the same barrier and none waits for an arrival that never
//     comes.  Every CTA leaves through one more cluster barrier after its last remote access, so no
//     CTA's shared memory goes away while another may still read it.
// Results (values, stop sweep, greedy policy) are those of the grid solver; sums run in another order.

#include "rmb_core.cuh"

namespace rmb {

constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kDenseAhead = 16;   // float4 chunks per lane staged ahead: dense states of <= 2048 elements

// One state's rows, loaded ahead of its batch by the warp that computes it.  CSR (registers): lane
// l <= m holds row_ptr[s*m + l] (lane m: the end), lane l < m its cost, lane e entry e of the state's
// rows; taken when the state's m < 32 rows hold at most 32 entries.  Dense: the state's m*n values
// are copied by cp.async into the warp's 8 KB staging area of shared memory (n % 4 == 0,
// m*n <= 2048, m <= 16; lane l < m holds the costs).  Otherwise (fast = false) the rows are read when
// the state is computed.
struct Ahead {
    int s;
    int a;         // the only action taken (evaluation sweeps: the policy's), or -1 for the minimum over all
    bool fast;
    long long rp;
    float c, pr;
    int col;
};
template <int NC>
struct AheadVec {
    StateRegs<NC> R;
};
template <>
struct AheadVec<0> {
};

constexpr int kListSlots = kSmallWarps * kSmallMaxPer;   // (state, value) pairs one CTA writes per batch

struct SmallSmem {
    int2 list[2][kListSlots];   // this CTA's results of the last two batches: (state or -1, value bits)
    uint32_t err;               // cluster error word (every CTA holds a copy; errors are stored into all)
    uint32_t red[3][4];         // CTA 0's copy is the cluster's reduction ring: max |change|, okey(max), okey(-min)
    float wred[3][kSmallWarps];
    float bc[4];
};

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ int2 cl_ld_s32x2(uint32_t addr)
{
    int2 v;
    asm volatile("ld.shared::cluster.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void cl_red_max_u32(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cl_arrive()
{
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}

__device__ __forceinline__ void cl_wait()
{
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void cl_hw_barrier()
{
    // the non-.aligned form: threads of a warp need not have reconverged after divergent code
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// NC > 0: CSR rows of uniform length k (k % 4 == 0) read as float4 / int4 chunks, NC per lane with all 32
// lanes of a warp on one state (fast_load / fast_eval of the grid path, gathers from shared memory)
template <int NC>
struct SmallRun {
    const KP& p;
    SmallSmem& sm;
    float* V;          // this CTA's copy of the centred values
    int32_t* perm0;    // sigma of sweeps of even / odd parity, at this CTA's own positions
    int32_t* perm1;
    int32_t* rofs;     // CSR: rofs[s] = row_ptr[s*m] (saturated at 2^31 - 1), s = 0..n
    float* stage;      // dense rows staged ahead: kDenseAhead * 128 floats per warp (or null)
    uint32_t C, rank;
    long long syncs = 0;
    Centre Ce;
    int red_epoch = 0;
    bool perm_ok = true;

    __device__ SmallRun(const KP& kp, SmallSmem& s, float* v, int32_t* p0, int32_t* p1, int32_t* ro, float* st,
                        uint32_t c)
        : p(kp), sm(s), V(v), perm0(p0), perm1(p1), rofs(ro), stage(st), C(c), rank(cl_rank())
    {
    }

    // orders by parity, as a select (an indexed member array would live in local memory)
    __device__ int32_t* pbuf(long long k) const { return (k & 1) ? perm1 : perm0; }

    // position of a batch that this warp's r-th slot computes: round robin over the CTAs
    __device__ int my_pos(int r) const { return (int)rank + (int)C * ((int)(threadIdx.x >> 5) + kSmallWarps * r); }
    __device__ int batch_len(int t) const { return t == p.T - 1 ? p.last_len : p.b; }

    // an error seen by one thread: into every CTA's error word (read after the next barrier) and into
    // the status the host reads
    __device__ void raise(int code)
    {
        atomicCAS(&p.ctrl->error, 0, code);
        for (uint32_t r = 0; r < C; ++r) cl_red_max_u32(cl_map(&sm.err, r), 1u);
    }

    // cluster-wide barrier; false (in every thread of every CTA alike) once an error was raised
    __device__ bool sync()
    {
        ++syncs;
        cl_hw_barrier();
        return sm.err == 0u;
    }
    // the same, split: work between arrive() and wait() must not touch what other CTAs write before
    // they arrive (the rows of the next batch and its order do not: they are read-only or complete)
    __device__ void arrive()
    {
        ++syncs;
        cl_arrive();
    }
    __device__ bool wait()
    {
        cl_wait();
        return sm.err == 0u;
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

    // sigma_k at the positions this CTA computes in sweep k (all its slots of every batch)
    __device__ void compute_perm(long long k)
    {
        const PermKey K = key_for(k);
        int32_t* dst = pbuf(k);
        for (int j = threadIdx.x; j < p.T * kListSlots; j += kSmallThreads) {
            const int t = j / kListSlots, q = j - t * kListSlots;
            const int i = (int)rank + (int)C * q;
            if (i < batch_len(t)) dst[t * p.b + i] = (int)perm_at((uint32_t)(t * p.b + i), K, &perm_ok);
        }
    }

    // Q-factors of state s at the values A (shared memory): min (and arg-min, second smallest)
    template <bool ARG>
    __device__ Best eval(int s, const float* A, int a_only) const
    {
        const int lane = threadIdx.x & 31;
        const uint32_t nm1 = (uint32_t)(p.n - 1);
        Best best = {kInf, 0x7fffffff, kInf};
        if (p.path == PATH_DENSE) {
            const float* P = static_cast<const float*>(p.P);
            const bool vec = (p.n & 3) == 0 && (((uintptr_t)P) & 15) == 0;
            for (int a0 = 0; a0 < p.m; a0 += 8) {
                float part[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) part[u] = 0.f;
                if (vec) {
                    const int n4 = p.n >> 2;
                    for (int j4 = lane; j4 < n4; j4 += 32) {
                        const float4 av = reinterpret_cast<const float4*>(A)[j4];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (a0 + u < p.m) {
                                const float4 pv = __ldg(reinterpret_cast<const float4*>(P + ((int64_t)s * p.m + a0 + u) * p.n) + j4);
                                part[u] = fmaf(pv.x, av.x, fmaf(pv.y, av.y, fmaf(pv.z, av.z, fmaf(pv.w, av.w, part[u]))));
                            }
                        }
                    }
                } else {
                    for (int j = lane; j < p.n; j += 32) {
                        const float av = A[j];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (a0 + u < p.m) part[u] = fmaf(__ldg(P + ((int64_t)s * p.m + a0 + u) * p.n + j), av, part[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float x = part[u];
                    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                    if (a0 + u < p.m) {
                        float c = __ldg(p.cost + (int64_t)s * p.m + a0 + u);
                        if (a_only >= 0 && a0 + u != a_only) c = kInf;
                        const Best cur = {c == kInf ? kInf : fmaf(p.gamma, x, c), a0 + u, kInf};
                        best = better(best, cur);
                    }
                }
            }
            return best;
        }
        // CSR rows: the state's m rows are contiguous; lane e takes entry e of them when they hold at
        // most 32 entries (one load round trip for the row pointers, one for the entries), else rows
        // are walked one by one
        const int64_t r0 = (int64_t)s * p.m;
        long long rp = 0;
        float c = kInf;
        if (p.m < 32) {
            if (lane <= p.m) rp = __ldg(p.row_ptr + r0 + lane);
            if (lane < p.m) c = __ldg(p.cost + r0 + lane);
            if (a_only >= 0 && lane != a_only) c = kInf;
            const long long E0 = __shfl_sync(0xffffffffu, rp, 0), E1 = __shfl_sync(0xffffffffu, rp, p.m);
            if (E1 - E0 <= 32) {
                float x = 0.f;
                if (lane < E1 - E0) x = __ldg(p.prob + E0 + lane) * A[min((uint32_t)__ldg(p.col + E0 + lane), nm1)];
                const long long nxt = __shfl_down_sync(0xffffffffu, rp, 1);
                const int len = lane < p.m ? (int)(nxt - rp) : 0;
                uint32_t starts = len > 0 ? (1u << (int)(rp - E0)) : 0u;
                for (int off = 16; off > 0; off >>= 1) starts |= __shfl_xor_sync(0xffffffffu, starts, off);
                for (int dd = 1; dd < 32; dd <<= 1) {
                    const float y = __shfl_up_sync(0xffffffffu, x, dd);
                    if (lane >= dd && ((starts >> (lane - dd + 1)) & ((1u << dd) - 1u)) == 0u) x += y;
                }
                const float sum = __shfl_sync(0xffffffffu, x, len > 0 ? (int)(nxt - E0) - 1 : 0);
                Best cur = {kInf, 0x7fffffff, kInf};
                if (lane < p.m) {
                    cur.a = lane;
                    cur.q = (c == kInf) ? kInf : fmaf(p.gamma, len > 0 ? sum : 0.f, c);
                }
                for (int off = 16; off > 0; off >>= 1) cur = better(cur, shfl_xor_best<ARG>(cur, off));
                return cur;
            }
        }
        for (int a = 0; a < p.m; ++a) {
            const int64_t r = r0 + a;
            const long long e0 = __ldg(p.row_ptr + r), e1 = __ldg(p.row_ptr + r + 1);
            float x = 0.f;
            for (long long e = e0 + lane; e < e1; e += 32) x = fmaf(__ldg(p.prob + e), A[min((uint32_t)__ldg(p.col + e), nm1)], x);
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            const float cc = (a_only >= 0 && a != a_only) ? kInf : __ldg(p.cost + r);
            best = better(best, Best{cc == kInf ? kInf : fmaf(p.gamma, x, cc), a, kInf});
        }
        return best;
    }

    __device__ float* warp_stage() const { return stage + (size_t)(threadIdx.x >> 5) * (kDenseAhead * 128); }

    // rows of state s ahead of its batch (s < 0: none); with_stage: this slot may use the staging area;
    // a_only >= 0: only that action is taken (the other rows get cost +inf, so the minimum over the
    // rows is Q(s, a_only), the backup of B_{pi,b})
    __device__ void load(int s, Ahead& h, AheadVec<NC>& hv, bool with_stage, int a_only) const
    {
        const int lane = threadIdx.x & 31;
        h.s = s;
        h.a = a_only;
        h.fast = false;
        if (s < 0) return;
        if constexpr (NC > 0) {
            h.fast = true;
            fast_load<K_MIN, NC>(p, s, true, 32, lane, hv.R);
            if (a_only >= 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (((c * 32 + lane) >> p.k4_log2) != a_only) hv.R.cost[c] = kInf;
            }
            return;
        }
        if (p.path == PATH_DENSE) {
            if (!with_stage || !stage) return;
            h.fast = true;
            const int total = (p.m * p.n) >> 2;
            const float4* P4 = reinterpret_cast<const float4*>(static_cast<const float*>(p.P) + (int64_t)s * p.m * p.n);
            float* dst = warp_stage();
            __syncwarp();   // the previous state's staged rows have been read by every lane
#pragma unroll
            for (int i = 0; i < kDenseAhead; ++i) {
                const int q = lane + 32 * i;
                if (q < total)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                 ::"r"((uint32_t)__cvta_generic_to_shared(dst + 4 * q)), "l"(P4 + q) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            h.c = lane < p.m && (a_only < 0 || lane == a_only) ? __ldg(p.cost + (int64_t)s * p.m + lane) : kInf;
            return;
        }
        const int e0 = rofs[s], e1 = rofs[s + 1];
        if (p.m >= 32 || e1 == 0x7fffffff || e1 - e0 > 32) return;
        h.fast = true;
        const int64_t r0 = (int64_t)s * p.m;
        h.rp = lane <= p.m ? __ldg(p.row_ptr + r0 + lane) : 0;
        h.c = lane < p.m && (a_only < 0 || lane == a_only) ? __ldg(p.cost + r0 + lane) : kInf;
        h.pr = 0.f;
        h.col = 0;
        if (lane < e1 - e0) {
            h.pr = __ldg(p.prob + e0 + lane);
            h.col = __ldg(p.col + e0 + lane);
        }
    }

    // Q-factors of a state whose rows were loaded ahead (falls back to eval() otherwise)
    template <bool ARG>
    __device__ Best compute(const Ahead& h, const AheadVec<NC>& hv, const float* A) const
    {
        const int lane = threadIdx.x & 31;
        if constexpr (NC > 0) return fast_eval<ARG, NC, VM_SHARED>(p, hv.R, A, 32, lane);
        if (!h.fast) return eval<ARG>(h.s, A, h.a);
        Best cur = {kInf, 0x7fffffff, kInf};
        if (p.path == PATH_DENSE) {
            const int n4 = p.n >> 2;
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            const float4* st4 = reinterpret_cast<const float4*>(warp_stage());
            const float4* A4 = reinterpret_cast<const float4*>(A);
            // row a of the state is staged at chunks [a n4, (a+1) n4); four rows at a time, so that
            // their loads and their warp sums overlap
            for (int a0 = 0; a0 < p.m; a0 += 4) {
                float part[4] = {0.f, 0.f, 0.f, 0.f};
                for (int j4 = lane; j4 < n4; j4 += 32) {
                    const float4 av = A4[j4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (a0 + u < p.m) {
                            const float4 pv = st4[(a0 + u) * n4 + j4];
                            part[u] = fmaf(pv.x, av.x, fmaf(pv.y, av.y, fmaf(pv.z, av.z, fmaf(pv.w, av.w, part[u]))));
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], off);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float c = __shfl_sync(0xffffffffu, h.c, (a0 + u) & 31);
                    if (a0 + u < p.m) cur = better(cur, Best{c == kInf ? kInf : fmaf(p.gamma, part[u], c), a0 + u, kInf});
                }
            }
            return cur;
        }
        const uint32_t nm1 = (uint32_t)(p.n - 1);
        const long long E0 = __shfl_sync(0xffffffffu, h.rp, 0);
        const long long E1 = __shfl_sync(0xffffffffu, h.rp, p.m);
        float x = lane < E1 - E0 ? h.pr * A[min((uint32_t)h.col, nm1)] : 0.f;
        const long long nxt = __shfl_down_sync(0xffffffffu, h.rp, 1);
        const int len = lane < p.m ? (int)(nxt - h.rp) : 0;
        uint32_t starts = len > 0 ? (1u << (int)(h.rp - E0)) : 0u;
        for (int off = 16; off > 0; off >>= 1) starts |= __shfl_xor_sync(0xffffffffu, starts, off);
        for (int dd = 1; dd < 32; dd <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, x, dd);
            if (lane >= dd && ((starts >> (lane - dd + 1)) & ((1u << dd) - 1u)) == 0u) x += y;
        }
        const float sum = __shfl_sync(0xffffffffu, x, len > 0 ? (int)(nxt - E0) - 1 : 0);
        if (lane < p.m) {
            cur.a = lane;
            cur.q = (h.c == kInf) ? kInf : fmaf(p.gamma, len > 0 ? sum : 0.f, h.c);
        }
        for (int off = 16; off > 0; off >>= 1) cur = better(cur, shfl_xor_best<ARG>(cur, off));
        return cur;
    }

    // per-warp partials -> this CTA's maximum -> CTA 0's ring slot (remote max)
    __device__ void publish(int slot, Acc a)
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int off = 16; off > 0; off >>= 1) {
            a.dmax = fmaxf(a.dmax, __shfl_xor_sync(0xffffffffu, a.dmax, off));
            a.vlo = fminf(a.vlo, __shfl_xor_sync(0xffffffffu, a.vlo, off));
            a.vhi = fmaxf(a.vhi, __shfl_xor_sync(0xffffffffu, a.vhi, off));
        }
        if (lane == 0) {
            sm.wred[0][wid] = a.dmax;
            sm.wred[1][wid] = a.vlo;
            sm.wred[2][wid] = a.vhi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kSmallWarps; ++w) {
                a.dmax = fmaxf(a.dmax, sm.wred[0][w]);
                a.vlo = fminf(a.vlo, sm.wred[1][w]);
                a.vhi = fmaxf(a.vhi, sm.wred[2][w]);
            }
            cl_red_max_u32(cl_map(&sm.red[slot][0], 0), __float_as_uint(a.dmax));
            cl_red_max_u32(cl_map(&sm.red[slot][1], 0), okey(a.vhi));
            cl_red_max_u32(cl_map(&sm.red[slot][2], 0), okey(-a.vlo));
        }
    }

    // after the sync that follows publish(): every thread reads CTA 0's slot
    __device__ void read_slot(int slot, float& dmax, float& lo, float& hi)
    {
        if (threadIdx.x == 0) {
            sm.bc[0] = __uint_as_float(cl_ld_u32(cl_map(&sm.red[slot][0], 0)));
            sm.bc[1] = -okey_inv(cl_ld_u32(cl_map(&sm.red[slot][2], 0)));
            sm.bc[2] = okey_inv(cl_ld_u32(cl_map(&sm.red[slot][1], 0)));
        }
        __syncthreads();
        dmax = sm.bc[0];
        lo = sm.bc[1];
        hi = sm.bc[2];
        __syncthreads();
    }

    __device__ void clear_slot(int slot)
    {
        if (rank == 0 && threadIdx.x == 0) {
            sm.red[slot][0] = 0u;
            sm.red[slot][1] = 0u;
            sm.red[slot][2] = 0u;
        }
    }

    __device__ float shift_for(float lo, float hi) const
    {
        if (p.flags & RMB_FLAG_RAW_ROWS) return 0.f;
        const float mid = 0.5f * (lo + hi);
        const float spread = hi - lo;
        const float floor_ = 1e-6f * (float)(fabs(Ce.mu) + 1.0);
        if (!(fabsf(mid) > fmaxf(0.25f * spread, floor_))) return 0.f;
        return mid;
    }

    // every CTA writes the batch's (state, value) pairs from the C lists of buffer par into its own
    // copy: thread i reads the slot that holds position i of the batch (len <= 32 C <= 512 threads)
    __device__ void apply(int par, int len)
    {
        const int i = threadIdx.x;
        if (i < len) {
            const int q = i / (int)C;
            const int slot = (q % kSmallWarps) * kSmallMaxPer + q / kSmallWarps;
            const int2 e = cl_ld_s32x2(cl_map(&sm.list[par][slot], (uint32_t)(i - q * (int)C)));
            if (e.x >= 0) V[e.x] = __int_as_float(e.y);
        }
        __syncthreads();
    }

    __device__ void run()
    {
        const int lane = threadIdx.x & 31;
        if (threadIdx.x == 0) {
            sm.err = 0u;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 4; ++j) sm.red[i][j] = 0u;
        }
        cl_hw_barrier();   // every CTA's words are initialised before any remote access
        // the validation pass (a launch before this one) may have rejected the MDP: every CTA reads the
        // same word, so all skip the solve alike
        bool ok = ld_volatile(&p.ctrl->error) == 0;

        // set-up: centre on the midpoint of the start values (every CTA reads all of them)
        Acc a0 = {0.f, kInf, -kInf};
        for (int i = threadIdx.x; i < p.n; i += kSmallThreads) {
            const float v = p.Vin[i];
            a0.vlo = fminf(a0.vlo, v);
            a0.vhi = fmaxf(a0.vhi, v);
            if (v != v || fabsf(v) == kInf) a0.dmax = 1.f;   // every CTA scans all start values alike
        }
        for (int off = 16; off > 0; off >>= 1) {
            a0.dmax = fmaxf(a0.dmax, __shfl_xor_sync(0xffffffffu, a0.dmax, off));
            a0.vlo = fminf(a0.vlo, __shfl_xor_sync(0xffffffffu, a0.vlo, off));
            a0.vhi = fmaxf(a0.vhi, __shfl_xor_sync(0xffffffffu, a0.vhi, off));
        }
        if (lane == 0) {
            sm.wred[0][threadIdx.x >> 5] = a0.dmax;
            sm.wred[1][threadIdx.x >> 5] = a0.vlo;
            sm.wred[2][threadIdx.x >> 5] = a0.vhi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kSmallWarps; ++w) {
                a0.dmax = fmaxf(a0.dmax, sm.wred[0][w]);
                a0.vlo = fminf(a0.vlo, sm.wred[1][w]);
                a0.vhi = fmaxf(a0.vhi, sm.wred[2][w]);
            }
            sm.bc[0] = a0.dmax;
            sm.bc[1] = a0.vlo;
            sm.bc[2] = a0.vhi;
        }
        __syncthreads();
        if (sm.bc[0] != 0.f) {
            if (rank == 0 && threadIdx.x == 0) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
            ok = false;
        }
        const double mu0 = (p.flags & RMB_FLAG_RAW_ROWS) ? 0.0 : (double)(float)(0.5 * ((double)sm.bc[1] + (double)sm.bc[2]));
        __syncthreads();
        Ce = make_centre(mu0, p.gamma_d);
        for (int i = threadIdx.x; i < p.n; i += kSmallThreads) V[i] = (float)((double)p.Vin[i] - mu0);
        if (p.path != PATH_DENSE)
            for (int i = threadIdx.x; i <= p.n; i += kSmallThreads)
                rofs[i] = (int32_t)min(__ldg(p.row_ptr + (int64_t)i * p.m), (int64_t)0x7fffffff);
        if (ok) compute_perm(p.start_sweep);
        __syncthreads();
        long long sweeps = 0, iters = 0;
        double residual = 0.0;
        bool converged = false;
        const bool mpi = p.mode == MODE_MPI;
        // sweeps of B_{pi,b} (MB-MPI's evaluation sweeps, policy evaluation) take the policy's row only
        const bool pol_rows = p.mode != MODE_VI;
        const int32_t* pol = p.pi_in ? p.pi_in : p.pi;
        // rows of this warp's states of the next batch, loaded between the arrival at and the wait on
        // the barrier before it (dense: the first slot uses the warp's staging area)
        Ahead ah[kSmallMaxPer];
        AheadVec<NC> av[kSmallMaxPer];
        auto prefetch = [&](const int32_t* order, int t) {
            const int len = batch_len(t);
#pragma unroll
            for (int r = 0; r < kSmallMaxPer; ++r) {
                const int i = my_pos(r);
                const int s = i < len ? order[t * p.b + i] : -1;
                // the policy was written before a barrier this CTA has waited on (MB-MPI: the
                // improvement pass), and is read at L2
                const int a = (pol_rows && s >= 0) ? (int)min((uint32_t)ld_l2(pol + s), (uint32_t)(p.m - 1)) : -1;
                load(s, ah[r], av[r], r == 0, a);
            }
        };
        uint32_t bt = 0;   // batches done (list buffer parity)
        // sweep k over its order, whose first batch has been prefetched; next_sweep: the first batch of
        // sweep k + 1 may be prefetched at the last barrier (not when a pass that changes the policy
        // comes first).  Returns false on an error (the same in every CTA).
        auto sweep = [&](long long k, bool next_sweep, float& delta, float& lo, float& hi) -> bool {
            const int32_t* order = pbuf(k);
            const int slot = red_epoch % 3;
            clear_slot((red_epoch + 1) % 3);
            ++red_epoch;
            Acc acc = {0.f, kInf, -kInf};
            bool good = true;
            for (int t = 0; good && t < p.T; ++t, ++bt) {
                const int par = bt & 1;
#pragma unroll
                for (int r = 0; r < kSmallMaxPer; ++r) {
                    int2 e = make_int2(-1, 0);
                    if (ah[r].s >= 0) {
                        const int s = ah[r].s;
                        const Best q = compute<false>(ah[r], av[r], V);
                        const float v = new_value(q.q, Ce);
                        if (lane == 0) {
                            if (v != v) raise(RMB_ERR_NONFINITE);
                            const float old = V[s];
                            acc.dmax = fmaxf(acc.dmax, fabsf(v - old));
                            acc.vlo = fminf(acc.vlo, v);
                            acc.vhi = fmaxf(acc.vhi, v);
                        }
                        e = make_int2(s, __float_as_int(v));
                    }
                    if (lane == 0) sm.list[par][(threadIdx.x >> 5) * kSmallMaxPer + r] = e;
                }
                // the order of the next sweep (this CTA's positions) is computed during the first batch
                if (t == 0) compute_perm(k + 1);
                if (t == p.T - 1) publish(slot, acc);
                // arrive, then load the rows of the next batch (of this sweep, or the first batch of the
                // next, whose order was completed before this batch's barrier; T >= 2) while the others
                // arrive: loads issued before a release arrival would hold it back until they complete
                arrive();
                if (t + 1 < p.T) prefetch(order, t + 1);
                else if (next_sweep) prefetch(pbuf(k + 1), 0);
                good = wait();
                if (good) apply(par, batch_len(t));
            }
            if (!good) return false;
            read_slot(slot, delta, lo, hi);
            return true;
        };
        // MB-MPI's improvement pass (Alg. 1): the greedy policy and Q-gap at the current values, written
        // by the CTA that owns the state's range, and ||TV - V||_inf over the cluster; V is unchanged
        auto greedy_pass = [&](float& resid) -> bool {
            const int slot = red_epoch % 3;
            clear_slot((red_epoch + 1) % 3);
            ++red_epoch;
            Acc acc = {0.f, kInf, -kInf};
            const uint32_t per = ((uint32_t)p.n + C - 1) / C;
            const uint32_t lo = rank * per, hi = min((uint32_t)p.n, lo + per);
            for (uint32_t i = lo + (threadIdx.x >> 5); i < hi; i += kSmallWarps) {
                Ahead h;
                AheadVec<NC> hv;
                load((int)i, h, hv, false, -1);
                const Best q = compute<true>(h, hv, V);
                if (lane == 0) {
                    const float d = new_value(q.q, Ce) - V[i];
                    if (d != d) raise(RMB_ERR_NONFINITE);
                    acc.dmax = fmaxf(acc.dmax, fabsf(d));
                    st_l2(p.pi + i, q.a);
                    if (p.qgap) p.qgap[i] = q.q2 - q.q;
                }
            }
            publish(slot, acc);
            arrive();
            const bool good = wait();
            float l2, h2;
            if (good) read_slot(slot, resid, l2, h2);
            return good;
        };
        auto shift_values = [&](float lo, float hi) {
            const float sh = shift_for(lo, hi);
            if (sh != 0.f) {   // every CTA shifts its own copy; other CTAs read only its lists
                for (int i = threadIdx.x; i < p.n; i += kSmallThreads) V[i] -= sh;
                Ce = make_centre(Ce.mu + (double)sh, p.gamma_d);
                __syncthreads();
            }
        };
        if (ok && !mpi) {
            // MB-VI / policy evaluation: sweeps until the sweep change is <= eps
            prefetch(pbuf(p.start_sweep), 0);
            for (long long j = 0; ok && j < p.max_sweeps; ++j) {
                float delta, lo, hi;
                if (!sweep(p.start_sweep + j, true, delta, lo, hi)) {
                    ok = false;
                    break;
                }
                ++sweeps;
                residual = (double)delta;
                if (rank == 0 && threadIdx.x == 0 && p.trace) p.trace[j] = residual;
                if (delta != delta) {   // the same value in every CTA
                    if (rank == 0 && threadIdx.x == 0) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
                    ok = false;
                    break;
                }
                if ((double)delta <= p.eps) { converged = true; break; }
                shift_values(lo, hi);
            }
        }
        if (ok && mpi) {
            // MB-MPI (Alg. 1): improvement pass, stop test, K sweeps of B_{pi,b}; the sweep counter of
            // sigma runs on across the evaluation sweeps of all iterations
            for (;;) {
                float r = 0.f;
                if (!greedy_pass(r)) {
                    ok = false;
                    break;
                }
                residual = (double)r;
                if (rank == 0 && threadIdx.x == 0 && p.trace) p.trace[iters] = residual;
                ++iters;
                if (r != r) {
                    if (rank == 0 && threadIdx.x == 0) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
                    ok = false;
                    break;
                }
                if (residual <= p.eps) { converged = true; break; }
                if (iters >= p.max_sweeps) break;
                prefetch(pbuf(p.start_sweep + sweeps), 0);
                for (int e = 0; ok && e < p.K; ++e) {
                    float delta, lo, hi;
                    if (!sweep(p.start_sweep + sweeps, e + 1 < p.K, delta, lo, hi)) {
                        ok = false;
                        break;
                    }
                    ++sweeps;
                    if (delta != delta) {
                        if (rank == 0 && threadIdx.x == 0) atomicCAS(&p.ctrl->error, 0, RMB_ERR_NONFINITE);
                        ok = false;
                        break;
                    }
                    shift_values(lo, hi);
                }
                if (!ok) break;
            }
        }
        // outputs: values, and (MB-VI) the greedy policy / Q-gap at them (a full Bellman pass); MB-MPI's
        // last improvement pass wrote its policy and Q-gap already
        if (ok) {
            const uint32_t per = ((uint32_t)p.n + C - 1) / C;
            const uint32_t lo = rank * per, hi = min((uint32_t)p.n, lo + per);
            for (uint32_t i = lo + threadIdx.x; i < hi; i += kSmallThreads) p.Vout[i] = (float)(Ce.mu + (double)V[i]);
            if (!mpi && (p.pi || p.qgap)) {
                for (uint32_t i = lo + (threadIdx.x >> 5); i < hi; i += kSmallWarps) {
                    Ahead h;
                    AheadVec<NC> hv;
                    load((int)i, h, hv, false, -1);
                    const Best q = compute<true>(h, hv, V);
                    if (lane == 0) {
                        if (p.pi) p.pi[i] = q.a;
                        if (p.qgap) p.qgap[i] = q.q2 - q.q;
                    }
                }
            }
        }
        if (!perm_ok) atomicCAS(&p.ctrl->error, 0, RMB_ERR_UNSUPPORTED);
        if (rank == 0 && threadIdx.x == 0) {
            Ctrl* c = p.ctrl;
            c->sweeps = sweeps;
            c->iters = iters;
            c->barriers = syncs;
            c->residual = residual;
            c->mu = Ce.mu;
        }
        cl_hw_barrier();   // no CTA leaves while another may still read its shared memory
        if (rank == 0 && threadIdx.x == 0) {
            int st = ld_volatile(&p.ctrl->error);
            if (st == 0 && !converged) st = RMB_ERR_NOT_CONVERGED;
            p.ctrl->status = st;
        }
    }
};

template <int NC>
__global__ void __launch_bounds__(kSmallThreads, 1) rmb_small_kernel(KP p)
{
    __shared__ SmallSmem sm;
    extern __shared__ __align__(16) unsigned char dyn[];
    // dynamic shared memory: V [n] | sigma of even / odd sweeps [n] each | row offsets [n + 1] |
    // (dense rows that fit) the warps' staging areas, 16-byte aligned
    float* v = reinterpret_cast<float*>(dyn);
    int32_t* p0 = reinterpret_cast<int32_t*>(v + p.n);
    int32_t* p1 = p0 + p.n;
    int32_t* ro = p1 + p.n;
    const bool dense_stage = p.path == PATH_DENSE && (p.n & 3) == 0 && (((uintptr_t)p.P) & 15) == 0 && p.m <= 16 &&
                             p.m * p.n <= kDenseAhead * 128;
    float* st = dense_stage ? reinterpret_cast<float*>(dyn + (((size_t)p.n * 16 + 4 + 15) & ~(size_t)15)) : nullptr;
    uint32_t C;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
    SmallRun<NC> R(p, sm, v, p0, p1, ro, st, C);
    R.run();
}

const void* small_kernel_ptr(int nc)
{
    if (nc == 1) return reinterpret_cast<const void*>(rmb_small_kernel<1>);
    if (nc == 2) return reinterpret_cast<const void*>(rmb_small_kernel<2>);
    return reinterpret_cast<const void*>(rmb_small_kernel<0>);
}

}  // namespace rmb
