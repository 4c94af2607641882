// librmb host side and small kernels: the C ABI of rmb.h (argument checks, workspace layout, launch
// configuration, the batched planner, the adjoint pipeline) and the one-pass kernels (validation,
// permutation, quantisation, softmax, transposition, gradient, cumulative weights, residual
// weights, the gather-rate probe).  The persistent kernels and the device code they share live in
// rmb_core.cuh and the per-family translation units rmb_csr.cu (CSR and batched) and rmb_dense.cu.

#include <cuda.h>   // CUtensorMap and its enums (the encoder is reached through the runtime)

#include "rmb_core.cuh"
#include "rmb_diag.h"

namespace rmb {

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
// cursor may be cnt itself (the counts become the scatter cursors), so neither is declared __restrict__
__global__ void rmb_tr_scan_kernel(int n, const int32_t* cnt, int64_t* __restrict__ row_ptr, int32_t* cursor)
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

// ------------------------------------------------------------------------------------------------
// One backup of an explicit list of states (eq. (7) restricted to the list; with a policy, eq. (4)'s
// T_pi): W[i] = min_a c(s,a) + gamma sum_j P(j|s,a) V(j) for s = states[i], one warp per listed state,
// float32 values as given (not centred).  The step a rank of a row-partitioned batch takes for the
// states it owns.
// ------------------------------------------------------------------------------------------------
struct BL {
    int n, m, fmt;
    const float* P;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* prob;
    const float* cost;
    float gamma;
    const float* V;
    const int32_t* states;
    int64_t count;
    const int32_t* pi;
    float* W;
};

__global__ void rmb_backup_list_kernel(BL p)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t nm1 = (uint32_t)(p.n - 1);
    for (int64_t i = warp; i < p.count; i += nw) {
        const int s = (int)min((uint32_t)p.states[i], nm1);
        const int a0 = p.pi ? (int)min((uint32_t)p.pi[s], (uint32_t)(p.m - 1)) : 0;
        const int a1 = p.pi ? a0 + 1 : p.m;
        float best = kInf;
        for (int a = a0; a < a1; ++a) {
            const int64_t r = (int64_t)s * p.m + a;
            float part = 0.f;
            if (p.fmt == RMB_CSR) {
                const int64_t e0 = p.row_ptr[r], e1 = p.row_ptr[r + 1];
                for (int64_t e = e0 + lane; e < e1; e += 32)
                    part = fmaf(p.prob[e], p.V[min((uint32_t)p.col[e], nm1)], part);
            } else {
                const float* row = p.P + r * p.n;
                for (int j = lane; j < p.n; j += 32) part = fmaf(row[j], p.V[j], part);
            }
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            const float c = p.cost[r];
            best = fminf(best, c == kInf ? kInf : fmaf(p.gamma, part, c));
        }
        if (lane == 0) p.W[i] = best;
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

// The same gathers issued by the tensor-memory-access unit instead of the load/store path:
// cp.async.bulk.tensor tile::gather4 copies four 16-byte rows of src, viewed as [n/4][4] floats, at
// four arbitrary row coordinates into shared memory; the lane then picks the wanted float of each
// row.  Each warp owns a ring of kTgStages stages; a stage is one gather4 per lane (32 x 4 rows,
// 2048 bytes of payload) completing on one mbarrier.  Every wait is bounded; a warp whose wait runs
// out drains its copies in flight (bounded again) and writes NaN as its checksum.
constexpr int kTgWarps = 8;
constexpr int kTgStages = 4;
constexpr int kTgSlot = 128;                        // bytes per gather4 destination (64 used)
constexpr int kTgStageBytes = 32 * kTgSlot;
constexpr int kTgSmem = kTgWarps * kTgStages * kTgStageBytes;

__device__ __forceinline__ bool tg_wait(uint32_t bar, uint32_t parity, int64_t timeout_ns)
{
    const uint64_t t0 = globaltimer_ns();
    uint32_t spins = 0;
    while (!mb_try(bar, parity))
        if ((++spins & 63u) == 0 && (int64_t)(globaltimer_ns() - t0) > timeout_ns) return false;
    return true;
}

__global__ void __launch_bounds__(kTgWarps * 32, 1)
rmb_gather4_probe_kernel(const __grid_constant__ CUtensorMap map, uint32_t nm1, const int4* __restrict__ idx,
                         int64_t chunks, int reps, int64_t timeout_ns, float* __restrict__ out)
{
    extern __shared__ __align__(1024) unsigned char tg_ring[];
    __shared__ __align__(8) uint64_t bars[kTgWarps][kTgStages];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kTgWarps + w;
    const int64_t W = (int64_t)gridDim.x * kTgWarps;
    const uint32_t ring = (uint32_t)__cvta_generic_to_shared(tg_ring) + (uint32_t)(w * kTgStages * kTgStageBytes);
    if (lane == 0) {
        for (int s = 0; s < kTgStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bars[w][s]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // this warp's chunks (32 int4 of idx each): gw, gw + W, ... over reps passes of idx
    const int64_t total = (int64_t)reps * chunks;
    const int64_t mine = gw < total ? (total - 1 - gw) / W + 1 : 0;
    const uint64_t map_addr = reinterpret_cast<uint64_t>(&map);

    uint32_t sub[kTgStages], ph[kTgStages];
    uint32_t inflight = 0;
    float acc = 0.f;
    bool ok = true;
    auto issue = [&](int s, int64_t j) {
        const int64_t c = (gw + j * W) % chunks;
        const int4 v = __ldcs(idx + c * 32 + lane);
        const uint32_t x = min((uint32_t)v.x, nm1), y = min((uint32_t)v.y, nm1);
        const uint32_t z = min((uint32_t)v.z, nm1), q = min((uint32_t)v.w, nm1);
        sub[s] = (x & 3u) | ((y & 3u) << 2) | ((z & 3u) << 4) | ((q & 3u) << 6);
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[w][s]);
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(32 * 64) : "memory");
        __syncwarp();
        const uint32_t dst = ring + (uint32_t)(s * kTgStageBytes + lane * kTgSlot);
        // this lane's earlier reads of its slot come before the copy that overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                     ::"r"(dst), "l"(map_addr), "r"(0), "r"((int)(x >> 2)), "r"((int)(y >> 2)), "r"((int)(z >> 2)),
                       "r"((int)(q >> 2)), "r"(bar)
                     : "memory");
        inflight |= 1u << s;
    };
#pragma unroll
    for (int s = 0; s < kTgStages; ++s) {
        ph[s] = 0;
        if (s < mine) issue(s, s);
    }
    for (int64_t j0 = 0; j0 < mine && ok; j0 += kTgStages) {
#pragma unroll
        for (int s = 0; s < kTgStages; ++s) {
            const int64_t j = j0 + s;
            if (j < mine && ok) {
                const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[w][s]);
                // warp-uniform outcome: issue() below holds a __syncwarp
                if (!__all_sync(0xffffffffu, tg_wait(bar, ph[s], timeout_ns))) {
                    ok = false;
                } else {
                    ph[s] ^= 1u;
                    inflight &= ~(1u << s);
                    const float* slot = reinterpret_cast<const float*>(tg_ring + w * kTgStages * kTgStageBytes +
                                                                       s * kTgStageBytes + lane * kTgSlot);
                    acc += slot[sub[s] & 3u] + slot[4 + ((sub[s] >> 2) & 3u)] + slot[8 + ((sub[s] >> 4) & 3u)] +
                           slot[12 + ((sub[s] >> 6) & 3u)];
                    if (j + kTgStages < mine) issue(s, j + kTgStages);
                }
            }
        }
    }
    if (!ok) {
        // drain the copies still in flight before the shared memory goes away
#pragma unroll
        for (int s = 0; s < kTgStages; ++s)
            if (inflight & (1u << s)) tg_wait((uint32_t)__cvta_generic_to_shared(&bars[w][s]), ph[s], timeout_ns);
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = ok ? acc : __int_as_float(0x7fc00000);
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

int64_t auto_batch(const rmb_mdp* M, double eps);

// opts.batch: b in [1, n] (larger means n), or 0 for the time model's choice
int effective_batch(const rmb_mdp* M, const rmb_opts* O, int64_t* b)
{
    if (!O || O->batch < 0) return RMB_ERR_ARG;
    *b = O->batch == 0 ? auto_batch(M, O->eps) : (O->batch > M->n ? M->n : O->batch);
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

    const void* fn = nullptr;
    int threads = 0, per_sm = 0;
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
            fn = dense_tma_kernel_ptr(p.p_dtype);
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
        fn = dense_kernel_ptr(p.p_dtype);
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
        fn = path == PATH_CSR_VEC ? csr_vec_kernel_for(p.nc_all, p.nc_one) : csr_gen_kernel_ptr();
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

    // Small MDPs with small batches: one thread-block cluster runs the whole MB-VI solve with the values
    // in shared memory and cluster barriers between batches (rmb_small.cu), when the values, orders and
    // row offsets fit (16 bytes per state), every batch fits the cluster's warps (<= 2 states each) and the solve
    // is the paper's plain form (sigma order, sweep-change stop, float32 rows).
    int cluster = 0;
    const bool cluster_mode = q.mode == MODE_VI || q.mode == MODE_MPI ||
                              (q.mode == MODE_EVAL && !(O->flags & RMB_FLAG_RAW_ROWS));
    if (cluster_mode && O->grid_ctas == 0 && select == RMB_SELECT_PERMUTATION && rkind == RMB_RESIDUAL_SWEEP &&
        !(O->flags & (RMB_FLAG_ASYNC | RMB_FLAG_INJECT_BARRIER_STALL | RMB_FLAG_NO_CLUSTER)) && p.T >= 2 &&
        (M->format == RMB_CSR || p.p_dtype == RMB_P_F32) && !std::getenv("RMB_NO_CLUSTER")) {
        // dense rows of <= 2048 values (n % 4 == 0, m <= 16) are staged per warp: + 8 KB per warp
        const bool dstage = M->format == RMB_DENSE && (M->n & 3) == 0 && (((uintptr_t)M->P) & 15) == 0 && M->m <= 16 &&
                            (int64_t)M->m * M->n <= 2048;
        const size_t csmem = (((size_t)M->n * 16 + 4 + 15) & ~(size_t)15) + (dstage ? (size_t)(kSmallThreads / 32) * 8192 : 0);
        // vectorisable CSR rows are read as float4 / int4 chunks, <= 2 per lane of the state's warp;
        // larger uniform rows stay on the grid (the cluster would read them row by row)
        int cnc = 0;
        bool rows_ok = true;
        if (path == PATH_CSR_VEC) {
            const int64_t chunks = (int64_t)M->m * (M->k_uniform >> 2);
            const int k4 = M->k_uniform >> 2;
            cnc = chunks <= 32 ? 1 : (chunks <= 64 ? 2 : 0);
            rows_ok = cnc > 0 && k4 <= 32;
            if (!rows_ok) cnc = 0;
        } else if (M->format == RMB_CSR && M->k_uniform > 0) {
            rows_ok = (int64_t)M->m * M->k_uniform <= 32;   // uniform but not vectorisable: one entry per lane
        }
        const void* cfn = small_kernel_ptr(cnc);
        if (rows_ok && csmem <= (size_t)kSmallMaxDyn &&
            cudaFuncSetAttribute(cfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem) == cudaSuccess) {
            cudaFuncSetAttribute(cfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            for (int c : {16, 8, 4, 2}) {
                if (b > (int64_t)kSmallMaxPer * c * (kSmallThreads / 32)) break;
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)c;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)c);
                cfg.blockDim = dim3(kSmallThreads);
                cfg.dynamicSmemBytes = csmem;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int ncl = 0;
                if (cudaOccupancyMaxActiveClusters(&ncl, cfn, &cfg) == cudaSuccess && ncl >= 1) {
                    cluster = c;
                    break;
                }
                cudaGetLastError();
            }
            if (cluster) {
                fn = cfn;
                threads = kSmallThreads;
                smem = csmem;
                path = PATH_CLUSTER;
                // the row form the kernel reads: dense, vectorised CSR (cnc > 0) or one entry per lane
                p.path = M->format == RMB_DENSE ? PATH_DENSE : (cnc > 0 ? PATH_CSR_VEC : PATH_CSR_GEN);
            }
        }
    }
    if (cluster) grid = cluster;

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
    cudaError_t ce;
    if (cluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)cluster);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ce = cudaLaunchKernelExC(&cfg, fn, args);
    } else {
        ce = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, smem, s);
    }
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
    q.stats->lanes_per_state = path == PATH_DENSE ? threads : (path == PATH_CLUSTER ? 32 : p.lps_all);
    q.stats->ms = ms;
    q.stats->batch = (int32_t)b;
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
// MDPs with vectorised CSR rows and n <= kSoloSplitMaxN are solved with a copy of the values in every
// CTA of the group (the first kSoloMaxN in shared memory, the rest in L2), where a step of the group's
// lane groups costs the latency of its row loads.  Fitted to the per-MDP times of the 256-MDP bench
// launch (one CTA per SM, all SMs busy): in state order (b = n) 0.84 us, 1.14 us with two chunks of a
// state's rows per lane; in sigma's order 1.1 us, 1.37 us with two chunks, 1.5 us with two states per
// warp; x(1 + 8 f) when a fraction f of the values is in L2, as nearly every step then waits for an
// L2 gather.  A batch adds its barriers and the list exchange, 3 us (b = n) or 4 us:
//   batch time = latency + steps * step_us
// Each MDP gets the b minimising its time (unless the caller fixed b).  The makespan target M is
// found by bisection: MDPs whose single-CTA time exceeds M get the smallest group that meets M, the
// others are packed longest-first (LPT) onto the CTA that frees first, as the run-time queue does:
// free CTAs from time 0, a group's CTAs from the end of its MDP; M is feasible if every CTA meets it.
// ------------------------------------------------------------------------------------------------
struct ItemCost {
    int64_t n;
    double bytes_per_state, gamma;
    int concurrency_per_cta;   // states one CTA processes at once
    bool shared_values;        // solved with the values in shared memory (SoloRun)
    bool two_chunks;           // a lane holds two chunks of a state's rows
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
    if (c.shared_values) {
        // states beyond kSoloMaxN read their values from L2
        const double hi = c.n > kSoloMaxN ? (double)(c.n - kSoloMaxN) / (double)c.n : 0.0;
        const double base = T > 1.0 ? (c.two_chunks ? 1.37 : (c.concurrency_per_cta > kCsrThreads / 32 ? 1.5 : 1.1))
                                    : (c.two_chunks ? 1.14 : 0.84);
        const double step_us = base * (1.0 + 8.0 * hi);
        const double per_batch = (T > 1.0 ? 4.0 : 3.0) + steps * step_us;
        return est_sweeps(c.gamma, eps, (double)b / (double)c.n) * T * per_batch;
    }
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

// The single-solve time model of opts.batch = 0 (constants measured on this library's bench workloads on
// a B300: the random-gather rate of the CSR kernel, the dense TMA stream rate, the per-batch barrier
// and epilogue latency); sweeps(b) is est_sweeps' factor.  Independent of the device and of the mode,
// so the workspace size and the solve always agree on b.
int64_t auto_batch(const rmb_mdp* M, double eps)
{
    const double n = (double)M->n;
    double per_state_us, conc, wave_us;
    if (M->format == RMB_CSR) {
        const double k = M->k_uniform > 0 ? (double)M->k_uniform : 4.0;
        per_state_us = (double)M->m * k / 244.0e3;          // 244 G random gathers/s over the grid
        conc = 148.0 * 16.0;
        wave_us = 1.0;
    } else {
        const double eb = M->p_dtype == RMB_P_F32 ? 4.0 : (M->p_dtype == RMB_P_BF16 ? 2.0 : 1.0);
        per_state_us = (double)M->m * n * eb / 6.5e6;        // 6.5 TB/s over the grid
        conc = 148.0;
        wave_us = (double)M->m * n * eb / 44.0e3;            // 44 GB/s per SM
    }
    const double gamma = M->gamma;
    int64_t best = M->n;
    double best_t = 1e300;
    for (int64_t b = M->n;; b = (b + 1) / 2) {
        const double T = std::ceil(n / (double)b);
        const double stream = (double)b * per_state_us;
        const double waves = std::ceil((double)b / conc) * wave_us;
        const double t = est_sweeps(gamma, eps, (double)b / n) * T * ((stream > waves ? stream : waves) + 6.0);
        if (t < best_t * (1.0 - 1e-9)) {   // ties keep the larger b
            best_t = t;
            best = b;
        }
        if (b <= 32) break;
    }
    return best;
}

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
    std::vector<BatchTask> tasks;   // per-CTA static tasks (task_off), then the queue of single-CTA MDPs
    int nqueue = 0;
    double makespan;
};

constexpr double kAloneMargin = 1.2;

bool try_makespan(const std::vector<ItemCost>& cs, const std::vector<int64_t>& fixed, int ctas, double eps, double M,
                  BatchPlan* out)
{
    const int N = (int)cs.size();
    std::vector<ItemPlan> ip(N);
    std::vector<int> big, small;
    int used = 0;
    for (int i = 0; i < N; ++i) {
        const ItemPlan one = best_b(cs[i], 1, eps, fixed[i]);
        // an MDP must meet M with a margin: the long solves (single CTAs and groups) start with the
        // launch, while every SM streams rows, and measured up to ~1.2x their estimates there
        if (one.t * kAloneMargin <= M) {
            ip[i] = one;
            small.push_back(i);
            continue;
        }
        bool ok = false;
        for (int G = 2; G <= ctas; G = G < 8 ? G + 1 : G + G / 4) {
            const ItemPlan pg = best_b(cs[i], G, eps, fixed[i]);
            if (pg.t * kAloneMargin <= M) {
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
    if (free_ctas < 0) return false;
    std::sort(small.begin(), small.end(), [&](int a, int b) { return ip[a].t > ip[b].t; });
    // the run-time queue is list scheduling: the CTA that frees first takes the next MDP, longest
    // first.  Free CTAs start at 0; a group's CTAs join once their MDP is solved.
    std::vector<double> load(free_ctas, 0.0);
    for (int i : big)
        for (int r = 0; r < ip[i].G; ++r) load.push_back(ip[i].t);
    if (load.empty() && !small.empty()) return false;
    for (int i : small) {
        int best = 0;
        for (int c = 1; c < (int)load.size(); ++c)
            if (load[c] < load[best]) best = c;
        load[best] += ip[i].t;
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
    // the bins only prove M feasible: single-CTA MDPs are dispatched at run time from one queue,
    // longest first, to whichever CTA is free (the groups' CTAs too, once their MDP is solved), so
    // errors of the cost model do not leave CTAs idle
    for (double l : load) mk = l > mk ? l : mk;
    for (int c = 0; c < ctas; ++c) {
        out->task_off[c + 1] = out->task_off[c] + (int)per[c].size();
        for (const BatchTask& t : per[c]) out->tasks.push_back(t);
    }
    for (int i : small) out->tasks.push_back(BatchTask{i, 0, 1, 0});   // sorted longest first above
    out->nqueue = (int)small.size();
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
        cs[i].shared_values = false;
        cs[i].two_chunks = false;
        if (csr_vec_ok(M)) {
            const int k4 = M->k_uniform >> 2;
            const int cpr = k4 < 32 ? k4 : 32;
            const int all = pow2ceil(cpr * M->m);
            lps = all > 32 ? 32 : all;
            // the batched kernel's fast rows (one or two chunks per lane, rows within one lane group)
            const int nc = (k4 <= lps && (k4 & (k4 - 1)) == 0) ? (M->m * k4 + lps - 1) / lps : 0;
            cs[i].shared_values = (nc == 1 || nc == 2) && M->n <= kSoloSplitMaxN;
            cs[i].two_chunks = nc == 2;
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
    // MDPs of up to kSoloMaxN states keep their values in kSoloMaxN * 4 bytes of dynamic shared memory
    // of every CTA that solves them (SoloRun); the rest of the unified L1 stays cache
    if (cudaFuncSetAttribute(batched_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, kSoloMaxN * 4) !=
        cudaSuccess)
        return RMB_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel_ptr(), kCsrThreads, kSoloMaxN * 4) !=
            cudaSuccess || occ < 1)
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
    handle->nqueue = plan.nqueue;
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
    if (h->nqueue < 0 || h->nqueue > h->count) return RMB_ERR_ARG;
    // control blocks and the queue cursor (the first 4 bytes of the workspace)
    if (cudaMemsetAsync(ws + h->ctrl_offset, 0, (size_t)h->count * sizeof(Ctrl), s) != cudaSuccess ||
        cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess)
        return RMB_ERR_CUDA;
    const KP* kps = reinterpret_cast<const KP*>(ws + h->kp_offset);
    const int* toff = reinterpret_cast<const int*>(ws + h->toff_offset);
    const BatchTask* tasks = reinterpret_cast<const BatchTask*>(ws + h->tasks_offset);
    int nqueue = h->nqueue;
    int* qnext = reinterpret_cast<int*>(ws);
    void* args[] = {(void*)&kps, (void*)&toff, (void*)&tasks, (void*)&nqueue, (void*)&qnext};
    const cudaError_t ce = cudaLaunchCooperativeKernel(batched_kernel_ptr(), dim3(h->grid_ctas), dim3(kCsrThreads),
                                                       args, (size_t)kSoloMaxN * 4, s);
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
    unsigned long long t0 = ~0ull;
    for (int i = 0; i < h->count; ++i) t0 = c[i].t_begin < t0 ? c[i].t_begin : t0;
    for (int i = 0; i < h->count; ++i) {
        std::memset(&out[i], 0, sizeof(rmb_stats));
        out[i].sweeps = c[i].sweeps;
        out[i].iters = c[i].iters;
        out[i].barriers = c[i].barriers;
        out[i].residual = c[i].residual;
        out[i].v_shift = c[i].mu;
        out[i].status = c[i].status != 0 ? c[i].status : c[i].error;
        out[i].path = -1;
        out[i].ms = (float)((double)(c[i].t_end - c[i].t_begin) * 1e-6);
        out[i].start_ms = (float)((double)(c[i].t_begin - t0) * 1e-6);
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
    if (opts && opts->batch == 0) b = auto_batch(mdp, opts->eps);
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

int rmb_backup_states(const rmb_mdp* mdp, const float* V, const int32_t* states, int64_t count, const int32_t* pi,
                      float* W_out, void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (count < 0 || (count > 0 && (!V || !states || !W_out))) return RMB_ERR_ARG;
    if (mdp->format == RMB_DENSE && mdp->p_dtype != RMB_P_F32) return RMB_ERR_UNSUPPORTED;
    if (count == 0) return RMB_OK;
    DevInfo* D = nullptr;
    if ((st = dev_info(&D))) return st;
    BL b;
    b.n = (int)mdp->n;
    b.m = mdp->m;
    b.fmt = mdp->format;
    b.P = static_cast<const float*>(mdp->P);
    b.row_ptr = mdp->row_ptr;
    b.col = mdp->col;
    b.prob = mdp->prob;
    b.cost = mdp->cost;
    b.gamma = (float)mdp->gamma;
    b.V = V;
    b.states = states;
    b.count = count;
    b.pi = pi;
    b.W = W_out;
    const int64_t warps_needed = count;
    const int64_t blocks = std::min<int64_t>((warps_needed + 7) / 8, (int64_t)D->sms * 8);
    rmb_backup_list_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(b);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? RMB_OK : RMB_ERR_CUDA;
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

// workspace of rmb_vi_prioritized: weights [n] | the residual-weights pass | the weighted MB-VI solve
static size_t prioritized_parts(const rmb_mdp* mdp, const rmb_opts* opts, size_t* off_rw, size_t* off_vi)
{
    if (check_mdp(mdp) || !opts) return 0;
    rmb_opts o = *opts;
    o.select = RMB_SELECT_WEIGHTED;
    const size_t vi = rmb_workspace_bytes(mdp, &o);
    const size_t rw = rmb_residual_weights_workspace_bytes(mdp);
    if (vi == 0 || rw == 0) return 0;
    *off_rw = align_up((size_t)mdp->n * 4, 256);
    *off_vi = *off_rw + align_up(rw, 256);
    return *off_vi + vi;
}

size_t rmb_vi_prioritized_workspace_bytes(const rmb_mdp* mdp, const rmb_opts* opts)
{
    size_t a, b;
    return prioritized_parts(mdp, opts, &a, &b);
}

int rmb_vi_prioritized(const rmb_mdp* mdp, const rmb_opts* opts, int32_t refresh, float floor_frac, float* V_inout,
                       int32_t* pi_out, float* qgap_out, void* workspace, size_t workspace_bytes, rmb_stats* stats,
                       void* stream)
{
    int st = check_mdp(mdp);
    if (st) return st;
    if (!opts || !V_inout || refresh < 1 || !(floor_frac >= 0.f && floor_frac <= 1.f)) return RMB_ERR_ARG;
    if (opts->max_sweeps < 1 || !(opts->eps >= 0.0) || std::isinf(opts->eps) || opts->start_sweep < 0)
        return RMB_ERR_ARG;
    if (opts->flags & RMB_FLAG_ASYNC) return RMB_ERR_UNSUPPORTED;
    size_t off_rw = 0, off_vi = 0;
    const size_t need = prioritized_parts(mdp, opts, &off_rw, &off_vi);
    if (need == 0) return RMB_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return RMB_ERR_WORKSPACE;
    if (workspace_bytes < need) return RMB_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    uint32_t* w = reinterpret_cast<uint32_t*>(ws);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RMB_ERR_CUDA;
        cudaEventRecord(e0, s);
    }
    rmb_opts o = *opts;
    o.select = RMB_SELECT_WEIGHTED;
    o.weights = w;
    o.residual_kind = RMB_RESIDUAL_SWEEP;   // draws always confirm with the full residual
    o.trace = nullptr;
    int64_t sweeps = 0, rounds = 0, barriers = 0;
    rmb_stats r;
    std::memset(&r, 0, sizeof(r));
    int status = RMB_ERR_NOT_CONVERGED;
    while (sweeps < opts->max_sweeps) {
        // one round: weights from the residual at the current values, then up to `refresh` sweeps of
        // weighted draws (the solve stops early once its change and ||TV - V||_inf are <= eps)
        if ((st = rmb_residual_weights(mdp, V_inout, floor_frac, w, ws + off_rw, off_vi - off_rw, stream))) return st;
        o.start_sweep = opts->start_sweep + sweeps;
        o.max_sweeps = std::min<int64_t>(refresh, opts->max_sweeps - sweeps);
        o.validate = rounds == 0 ? opts->validate : 0;
        st = rmb_vi(mdp, &o, V_inout, pi_out, qgap_out, ws + off_vi, workspace_bytes - off_vi, &r, stream);
        ++rounds;
        sweeps += r.sweeps;
        barriers += r.barriers;
        if (st == RMB_OK) { status = RMB_OK; break; }
        if (st != RMB_ERR_NOT_CONVERGED) { status = st; break; }
        if (r.sweeps == 0) break;
    }
    if (!stats) return status;
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMB_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *stats = r;
    stats->sweeps = sweeps;
    stats->iters = rounds;
    stats->barriers = barriers;
    stats->status = status;
    stats->ms = ms;
    return status;
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
    // batch = 0: one b for both solves, the model's choice for the reference rows (the workspace is
    // sized by rmb_workspace_bytes(ref, opts))
    if (opts->batch == 0) o1.batch = auto_batch(ref, opts->eps);
    o1.eps = eps_low;
    o1.trace = nullptr;
    Call q1{MODE_VI, lowp, &o1, V_inout, V_inout, nullptr, nullptr, nullptr, nullptr,
            workspace, workspace_bytes, stats_low, static_cast<cudaStream_t>(stream)};
    st = solve(q1);
    if (st != RMB_OK && st != RMB_ERR_NOT_CONVERGED) return st;
    rmb_opts o2 = *opts;
    o2.batch = o1.batch;
    o2.trace = nullptr;
    Call q2{MODE_VI, ref, &o2, V_inout, V_inout, nullptr, pi_out, qgap_out, nullptr,
            workspace, workspace_bytes, stats_ref, static_cast<cudaStream_t>(stream)};
    return solve(q2);
}

int rmb_diag_gather_probe(const float* src, int64_t n_src, const int32_t* idx, int64_t n_idx, int reps, float* out,
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

int rmb_diag_gather_probe_tma(const float* src, int64_t n_src, const int32_t* idx, int64_t n_idx, int reps, float* out,
                         void* stream)
{
    if (!src || !idx || !out || n_src < 4 || (n_src & 3) || n_src >= ((int64_t)1 << 32) || n_idx < 128 ||
        (n_idx % 128) || reps < 1)
        return RMB_ERR_ARG;
    if ((((uintptr_t)idx) & 15) || (((uintptr_t)src) & 15)) return RMB_ERR_ARG;
    DevInfo* D = nullptr;
    int st = dev_info(&D);
    if (st) return st;
    using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return RMB_ERR_UNSUPPORTED;
    // src as [n/4][4] floats: 16-byte rows, a box of one row (the form gather4 takes)
    alignas(64) CUtensorMap map;
    const cuuint64_t dims[2] = {4, (cuuint64_t)(n_src / 4)};
    const cuuint64_t strides[1] = {16};
    const cuuint32_t box[2] = {4, 1};
    const cuuint32_t estr[2] = {1, 1};
    if (reinterpret_cast<EncodeTiled>(fn)(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(src), dims,
                                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                          CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return RMB_ERR_ARG;
    if (cudaFuncSetAttribute(rmb_gather4_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTgSmem) !=
        cudaSuccess)
        return RMB_ERR_CUDA;
    rmb_gather4_probe_kernel<<<D->sms, kTgWarps * 32, kTgSmem, static_cast<cudaStream_t>(stream)>>>(
        map, (uint32_t)(n_src - 1), reinterpret_cast<const int4*>(idx), n_idx / 128, reps, (int64_t)1000000000, out);
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
    int64_t b = mdp->n;
    if (effective_batch(mdp, opts, &b) == RMB_OK) stats->batch = (int32_t)b;
    return stats->status;
}

uint64_t rmb_kernel_launches(void) { return g_launches.load(); }

int rmb_version(void) { return (1 << 16) | 0; }

}  // extern "C"
