/*
 * rmb_diag.h -- diagnostic kernels of librmb.  They are not part of the method or of its boundary
 * (include/rmb.h): they measure ceilings of the hardware that bound the CSR sweeps, and the bench
 * reports the mini-batch kernels against them.  Same conventions as rmb.h: device pointers are
 * caller-owned, calls are asynchronous on `stream`, errors come back as rmb_status codes.
 */
#ifndef RMB_DIAG_H
#define RMB_DIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Diagnostic (not part of the method): the attainable rate of random 4-byte gathers.  One CTA of 512
 * threads per SM streams idx (int32, 16-byte aligned, n_idx a multiple of 4) and gathers src[idx]
 * through L1, reps times; out receives one checksum per thread (grid_size * 512 floats, grid_size =
 * number of SMs).  With src sized like the value vector and uniformly random idx this measures the
 * L1->L2 request ceiling that bounds the CSR sweeps.
 */
int rmb_diag_gather_probe(const float *src, int64_t n_src, const int32_t *idx, int64_t n_idx, int reps,
                     float *out, void *stream);

/*
 * Diagnostic (not part of the method): the same gathers issued through the tensor-memory-access unit
 * (cp.async.bulk.tensor tile::gather4: four 16-byte rows of src, viewed as [n_src/4][4] floats, per
 * instruction), to compare with the load path of rmb_diag_gather_probe.  src: 16-byte aligned, n_src a
 * multiple of 4 (< 2^32); idx: int32, 16-byte aligned, n_idx a multiple of 128; out: grid_size * 256
 * floats (one checksum per thread, grid_size = number of SMs); a NaN checksum means a wait for a copy
 * ran out (1 s).  Returns RMB_ERR_UNSUPPORTED when the driver has no tensor-map encoder.
 */
int rmb_diag_gather_probe_tma(const float *src, int64_t n_src, const int32_t *idx, int64_t n_idx, int reps,
                         float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RMB_DIAG_H */
