// Device primitives of librmb: counter-based permutation, bounded grid-wide wait, cache-policy
// loads/stores, ordered float keys for atomic min/max.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rmb {

constexpr float kInf = __builtin_huge_valf();

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the multiply-xor round with the
// key bumped by the Weyl increments between rounds.  The first two output words are used.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint2 philox_x01(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint2(c0, c1);
}

__device__ __forceinline__ uint32_t philox_x0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1)
{
    return philox_x01(c0, c1, c2, c3, k0, k1).x;
}

// Processing order of one sweep (Sec. III-A): sigma(p) by an 8-round balanced Feistel network on
// 2h-bit words, round function F_r(R) = Philox(ctr={R, r, sweep_lo, sweep_hi}, key=seed).x0 mod 2^h,
// cycle-walked into [0,n).  A Feistel network is a bijection of its domain, so the walk returns
// to [0,n) within (4^h - n + 1) steps; *ok is cleared if that bound is ever exceeded.
struct PermKey {
    uint32_t n, h, mask, k0, k1, s_lo, s_hi;
    const int32_t* buf;   // non-null: the order of this sweep is precomputed here (buf[p] = state)
    uint32_t select;      // 0: sigma; 1: uniform draws; 2: draws by weight (with replacement)
    uint64_t wtot;        // select 2: sum of the weights
    const uint64_t* cdf;  // select 2: cdf[s] = w_0 + ... + w_s
};

__device__ __forceinline__ uint32_t feistel8(uint32_t x, const PermKey& K)
{
    uint32_t L = x >> K.h, R = x & K.mask;
#pragma unroll
    for (uint32_t r = 0; r < 8; ++r) {
        const uint32_t F = philox_x0(R, r, K.s_lo, K.s_hi, K.k0, K.k1) & K.mask;
        const uint32_t nl = R;
        R = L ^ F;
        L = nl;
    }
    return (L << K.h) | R;
}

__device__ __forceinline__ uint32_t perm_at(uint32_t p, const PermKey& K, bool* ok)
{
    const uint64_t limit = (uint64_t)1 << (2 * K.h);
    uint32_t x = p;
    uint64_t steps = 0;
    do {
        x = feistel8(x, K);
        if (++steps > limit) { *ok = false; return 0; }
    } while (x >= K.n);
    return x;
}

// Batch selection with replacement (the Sec. V extension): u = x0 * 2^32 + x1 of
// Philox(ctr = {p, 2^31, sweep_lo, sweep_hi}, key = seed) -- a counter word the Feistel rounds
// (0..7) never use -- then floor(u n / 2^64) (uniform), or r = floor(u W / 2^64) and the first s
// with cdf[s] > r (by weight), all in integers.
__device__ __forceinline__ int draw_at(uint32_t p, const PermKey& K)
{
    const uint2 x = philox_x01(p, 0x80000000u, K.s_lo, K.s_hi, K.k0, K.k1);
    const uint64_t u = ((uint64_t)x.x << 32) | x.y;
    if (K.select == 1) return (int)__umul64hi(u, (uint64_t)K.n);
    const uint64_t r = __umul64hi(u, K.wtot);
    uint32_t lo = 0, hi = K.n - 1;
    while (lo < hi) {   // at most ceil(log2 n) steps: the interval halves every time
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(K.cdf + mid) > r) hi = mid;
        else lo = mid + 1;
    }
    return (int)lo;
}

// the state at position p of the sweep's order, evaluated here (no buffer)
__device__ __forceinline__ int order_at(uint32_t p, const PermKey& K, bool* ok)
{
    if (K.select) return draw_at(p, K);
    return (int)perm_at(p, K, ok);
}

// the state at position p: from the precomputed buffer when there is one, else evaluated here
__device__ __forceinline__ int state_at(uint32_t p, const PermKey& K, bool* ok)
{
    if (K.buf) return __ldcg(K.buf + p);
    return order_at(p, K, ok);
}

__host__ __device__ inline uint32_t perm_half_bits(int64_t n)
{
    uint32_t lg = 0;
    while (lg < 62 && ((int64_t)1 << lg) < n) ++lg;
    const uint32_t h = (lg + 1) / 2;
    return h < 1 ? 1 : h;
}

// ------------------------------------------------------------------------------------------------
// Loads / stores.  The transition stream is read once per sweep: evict-first (".cs").  Values that
// other CTAs write inside the same launch are read and written at L2 (".cg"): L1 is not coherent.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ int ld_l2(const int* p) { return __ldcg(p); }
__device__ __forceinline__ void st_l2(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void st_l2(int* p, int v) { __stcg(p, v); }
__device__ __forceinline__ uint64_t ld_l2(const uint64_t* p)
{
    return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ void st_l2(uint64_t* p, uint64_t v)
{
    __stcg(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

__device__ __forceinline__ int ld_volatile(const int* p)
{
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Order-preserving map float -> uint32 (for atomicMax on signed values); 0 is below every key.
__device__ __forceinline__ uint32_t okey(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float okey_inv(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// ------------------------------------------------------------------------------------------------
// Control block at the head of the workspace (zeroed by the host before every launch).
// ------------------------------------------------------------------------------------------------
struct Ctrl {
    unsigned long long bar;      // grid-wide wait arrivals
    int error;                   // first error status (0 = none)
    int wait_site;               // which wait gave up (diagnostics)
    uint32_t red_delta[4];       // ring of max |change| (non-negative float bits); slot 3 = setup
    uint32_t red_hi[4];          // ring of okey(max value)
    uint32_t red_nlo[4];         // ring of okey(-min value)
    long long sweeps, iters, barriers;
    double residual, mu;
    int status, pad;
    unsigned long long t_begin, t_end;   // batched solves: globaltimer at the MDP's start and end (ns)
};

// The CTAs that solve one MDP: all of the grid (single solves) or a group of it (batched solves).
struct GroupView {
    int rank;   // this CTA's index in the group
    int size;   // CTAs in the group
};

// Bounded grid-wide barrier, split in two: grid_arrive() publishes this CTA's arrival (a CTA barrier,
// then one release add by thread 0), grid_wait_arrived() spins with acquire loads until
// every CTA has arrived.  A wait gives up after timeout_ns, or as soon as another CTA reports an
// error, and then returns false in every thread of the CTA.
__device__ __forceinline__ void grid_arrive(Ctrl* c, unsigned long long& target, bool skip_arrive, int gsize)
{
    __syncthreads();
    if (gsize == 1) return;   // a one-CTA group synchronises with the CTA barrier alone
    if (threadIdx.x == 0) {
        target += gsize;
        // the release add publishes the CTA's writes: they are ordered before it by the CTA barrier
        // above, and release is cumulative, so no separate fence is needed
        if (!skip_arrive) red_release_add_u64(&c->bar, 1ull);
    }
}

__device__ __forceinline__ bool grid_wait_arrived(Ctrl* c, unsigned long long target, int64_t timeout_ns, int site,
                                                  int gsize)
{
    __shared__ int s_ok;
    if (gsize == 1) {
        if (threadIdx.x == 0) s_ok = ld_volatile(&c->error) == 0;
        __syncthreads();
        return s_ok != 0;
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        uint32_t spins = 0;
        while (ld_acquire_u64(&c->bar) < target) {
            if ((++spins & 31u) == 0) {
                if (ld_volatile(&c->error) != 0) { ok = 0; break; }
                if ((int64_t)(globaltimer_ns() - t0) > timeout_ns) {
                    if (atomicCAS(&c->error, 0, -4 /* RMB_ERR_BARRIER_TIMEOUT */) == 0)
                        c->wait_site = site;
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && ld_volatile(&c->error) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace rmb
