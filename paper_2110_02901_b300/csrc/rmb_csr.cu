// librmb: the persistent CSR kernels (vectorised rows, ragged rows) and the batched kernel, which
// runs the same CSR runners (a translation unit of its own so that the library compiles in parallel).

#include "rmb_core.cuh"

namespace rmb {

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


const void* csr_vec_kernel_for(int nca, int nco)
{
    const int a = (nca == 1 || nca == 2 || nca == 4) ? nca : 0;
    const int o = nco == 1 ? 1 : 0;
#define RMB_K(A_, O_) if (a == A_ && o == O_) return reinterpret_cast<const void*>(rmb_csr_vec_kernel<A_, O_>);
    RMB_K(0, 0) RMB_K(1, 0) RMB_K(2, 0) RMB_K(4, 0) RMB_K(0, 1) RMB_K(1, 1) RMB_K(2, 1) RMB_K(4, 1)
#undef RMB_K
    return reinterpret_cast<const void*>(rmb_csr_vec_kernel<0, 0>);
}

const void* csr_gen_kernel_ptr() { return reinterpret_cast<const void*>(rmb_csr_gen_kernel); }

__global__ void __launch_bounds__(kCsrThreads, 1)
rmb_batched_kernel(const KP* __restrict__ kps, const int* __restrict__ task_off, const BatchTask* __restrict__ tasks,
                   int nqueue, int* __restrict__ qnext)
{
    __shared__ RedSmem rs;
    __shared__ KP s_kp;
    __shared__ int s_next;
    extern __shared__ __align__(16) float solo_values[];   // kSoloMaxN floats: SoloRun's values
    // this CTA's own tasks (its share of the multi-CTA groups) first, then single-CTA MDPs from the
    // shared queue (longest first, after the last static task) until it is empty
    const int t0 = task_off[blockIdx.x], t1 = task_off[blockIdx.x + 1];
    const int nstatic = task_off[gridDim.x];
    for (int t = t0;; ++t) {
        BatchTask bt;
        if (t < t1) {
            bt = tasks[t];
        } else {
            __syncthreads();   // every thread has read the previous s_next
            if (threadIdx.x == 0) s_next = atomicAdd(qnext, 1);
            __syncthreads();
            if (s_next >= nqueue) break;
            bt = tasks[nstatic + s_next];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_kp = kps[bt.item];
        __syncthreads();
        const GroupView gv{bt.rank, bt.size};
        const unsigned long long t_begin = globaltimer_ns();
        // every CTA of the group keeps a copy of the values in its shared memory when they fit (the
        // launch is MB-VI over sigma with the sweep stop test only)
        // (the first kSoloMaxN values when they do not)
        const bool solo = s_kp.path == PATH_CSR_VEC && s_kp.n <= kSoloSplitMaxN && s_kp.mode == MODE_VI &&
                          s_kp.select == 0 && s_kp.residual_kind == 0 && (s_kp.flags & RMB_FLAG_ASYNC) == 0;
        const bool split = s_kp.n > kSoloMaxN;
        if (solo && !split && s_kp.nc_all == 1) {
            SoloRun<1> R(s_kp, rs, solo_values, gv);
            R.run();
        } else if (solo && !split && s_kp.nc_all == 2) {
            SoloRun<2> R(s_kp, rs, solo_values, gv);
            R.run();
        } else if (solo && s_kp.nc_all == 1) {
            SoloRun<1, true> R(s_kp, rs, solo_values, gv);
            R.run();
        } else if (solo && s_kp.nc_all == 2) {
            SoloRun<2, true> R(s_kp, rs, solo_values, gv);
            R.run();
        } else if (s_kp.path == PATH_CSR_VEC && s_kp.nc_all == 1 && s_kp.nc_one == 1) {
            Runner<PATH_CSR_VEC, 1, 1> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        } else if (s_kp.path == PATH_CSR_VEC && s_kp.nc_all == 2 && s_kp.nc_one == 1) {
            Runner<PATH_CSR_VEC, 2, 1> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        } else {
            Runner<PATH_CSR_GEN> R(s_kp, rs, nullptr, nullptr, gv);
            R.run();
        }
        if (threadIdx.x == 0 && bt.rank == 0) {
            s_kp.ctrl->t_begin = t_begin;
            s_kp.ctrl->t_end = globaltimer_ns();
        }
    }
}


const void* batched_kernel_ptr() { return reinterpret_cast<const void*>(rmb_batched_kernel); }

}  // namespace rmb
