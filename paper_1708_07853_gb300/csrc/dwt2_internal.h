// dwt2_internal.h -- host-side interface between the C ABI (dwt2_api.cu) and the kernel
// launchers (one translation unit per wavelet family, compiled in parallel).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "dwt2_persist.cuh"

namespace dwt2 {

// dtype codes of the C ABI
enum { DT_I32 = 0, DT_F32 = 1, DT_BF16 = 2, DT_F16 = 3 };

// Forward level launch.  ti = input-plane dtype, tb = band dtype (LL output is int32 / fp32).
// Returns cudaErrorNotSupported for a combination that has no kernel.
// a.tma selects TMA loads (tm valid) or plain loads.
cudaError_t launch_fwd_i53(int mode, const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_fwd_f53(int mode, int ti, int tb, const CUtensorMap& tm, const FwdArgs& a,
                           cudaStream_t s);
cudaError_t launch_fwd_f97(int mode, int ti, int tb, const CUtensorMap& tm, const FwdArgs& a,
                           cudaStream_t s);
// The Deslauriers-Dubuc wavelets (WV_DD97, WV_DD137): the non-separable scheme only.
cudaError_t launch_fwd_dd(int wavelet, int mode, int ti, int tb, const CUtensorMap& tm,
                          const FwdArgs& a, cudaStream_t s);
// Inverse level launch.  tb = band dtype, to = output-plane dtype; tm = LL, HL, LH, HH maps.
cudaError_t launch_inv(int wavelet, int tb, int to, const CUtensorMap* tm, const InvArgs& a,
                       cudaStream_t s);
cudaError_t launch_inv_dd(int wavelet, int tb, int to, const CUtensorMap* tm, const InvArgs& a,
                          cudaStream_t s);

// Adjoint levels (float wavelets, fp32): W_j^T with the inverse kernel's data flow, W_j^-T with
// the forward kernel's.
cudaError_t launch_adj_fwd(int wavelet, const CUtensorMap* tm, const InvArgs& a, cudaStream_t s);
cudaError_t launch_adj_inv(int wavelet, const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s);

// Persistent batched kernels (one launch for every level of every image of a plan).
// ctas_per_sm <= 0 uses the occupancy limit; *occ (if non-null) receives that limit and nothing
// is launched.  Forward data flow: mode MODE_NONSEP or MODE_ADJ_INV; inverse data flow: adj
// selects the transpose of the forward.
cudaError_t launch_fwd_persistent(int wavelet, int mode, int tb, const PersistArgs<FwdUnit>& p,
                                  int ctas_per_sm, cudaStream_t st, int* occ);
cudaError_t launch_inv_persistent(int wavelet, bool adj, int tb, const PersistArgs<InvUnit>& p,
                                  int ctas_per_sm, cudaStream_t st, int* occ);
// The Deslauriers-Dubuc wavelets' persistent kernels (forward and inverse; no adjoints).
cudaError_t launch_fwd_persistent_dd(int wavelet, int mode, int tb, const PersistArgs<FwdUnit>& p,
                                     int ctas_per_sm, cudaStream_t st, int* occ);
cudaError_t launch_inv_persistent_dd(int wavelet, bool adj, int tb, const PersistArgs<InvUnit>& p,
                                     int ctas_per_sm, cudaStream_t st, int* occ);

// dwt2_forward with the status header of the workspace cleared after the argument checks (the
// built-in scratch of dwt2_forward_static).
int forward_into_scratch(const void* img, int64_t img_pitch, int H, int W, int img_dtype,
                         void* coeffs, void* scratch, size_t scratch_bytes, int wavelet, int J,
                         int band_dtype, cudaStream_t st);

}  // namespace dwt2
