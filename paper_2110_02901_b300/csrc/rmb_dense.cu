// librmb: the persistent dense kernels (TMA ring, register-staged rows) (a translation unit of its own so that the library compiles in parallel).

#include "rmb_core.cuh"

namespace rmb {

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


const void* dense_kernel_ptr(int p_dtype)
{
    if (p_dtype == RMB_P_BF16) return reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_BF16>);
    if (p_dtype == RMB_P_FP8E4M3) return reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_FP8E4M3>);
    return reinterpret_cast<const void*>(rmb_dense_kernel<RMB_P_F32>);
}

const void* dense_tma_kernel_ptr(int p_dtype)
{
    if (p_dtype == RMB_P_BF16) return reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_BF16>);
    if (p_dtype == RMB_P_FP8E4M3) return reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_FP8E4M3>);
    return reinterpret_cast<const void*>(rmb_dense_tma_kernel<RMB_P_F32>);
}

}  // namespace rmb
