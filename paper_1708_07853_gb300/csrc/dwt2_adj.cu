// Adjoint-level kernels (gradients) of the float wavelets, fp32 storage.
#include "dwt2_internal.h"

namespace dwt2 {

cudaError_t launch_adj_fwd(int wavelet, const CUtensorMap* tm, const InvArgs& a, cudaStream_t s) {
    switch (wavelet) {
    case WV_CDF53: return launch_inverse_t<WV_CDF53, float, float, float, true>(tm, a, s);
    case WV_CDF97: return launch_inverse_t<WV_CDF97, float, float, float, true>(tm, a, s);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_adj_inv(int wavelet, const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s) {
    switch (wavelet) {
    case WV_CDF53: return launch_forward_t<WV_CDF53, MODE_ADJ_INV, float, float, float>(tm, a, s);
    case WV_CDF97: return launch_forward_t<WV_CDF97, MODE_ADJ_INV, float, float, float>(tm, a, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace dwt2
