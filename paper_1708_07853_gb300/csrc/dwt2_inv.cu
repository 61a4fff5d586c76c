// Inverse-level kernels of all wavelets.
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int WV, typename TB, typename TL, typename TO>
cudaError_t go(const CUtensorMap* tm, const InvArgs& a, cudaStream_t s) {
    return launch_inverse_t<WV, TB, TL, TO>(tm, a, s);
}

template <int WV>
cudaError_t go_float(int tb, int to, const CUtensorMap* tm, const InvArgs& a,
                     cudaStream_t s) {
    if (tb == DT_F32 && to == DT_F32) return go<WV, float, float, float>(tm, a, s);
    if (tb == DT_BF16 && to == DT_F32) return go<WV, __nv_bfloat16, float, float>(tm, a, s);
    if (tb == DT_BF16 && to == DT_BF16)
        return go<WV, __nv_bfloat16, float, __nv_bfloat16>(tm, a, s);
    if (tb == DT_F16 && to == DT_F32) return go<WV, __half, float, float>(tm, a, s);
    if (tb == DT_F16 && to == DT_F16) return go<WV, __half, float, __half>(tm, a, s);
    return cudaErrorNotSupported;
}
}  // namespace

cudaError_t launch_inv(int wavelet, int tb, int to, const CUtensorMap* tm,
                       const InvArgs& a, cudaStream_t s) {
    switch (wavelet) {
    case WV_CDF53_INT:
        if (tb != DT_I32 || to != DT_I32) return cudaErrorNotSupported;
        return go<WV_CDF53_INT, int32_t, int32_t, int32_t>(tm, a, s);
    case WV_CDF53: return go_float<WV_CDF53>(tb, to, tm, a, s);
    case WV_CDF97: return go_float<WV_CDF97>(tb, to, tm, a, s);
    case WV_DD97:
    case WV_DD137: return launch_inv_dd(wavelet, tb, to, tm, a, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace dwt2
