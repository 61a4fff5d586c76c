// Forward and inverse level kernels of the Deslauriers-Dubuc 9/7 and 13/7 wavelets (fp32
// arithmetic; fp32 / bf16 / fp16 storage; the non-separable scheme of Eq. 5 only).
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int WV>
cudaError_t fwd(int ti, int tb, const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s) {
    if (ti == DT_F32 && tb == DT_F32)
        return launch_forward_t<WV, MODE_NONSEP, float, float, float>(tm, a, s);
    if (ti == DT_F32 && tb == DT_BF16)
        return launch_forward_t<WV, MODE_NONSEP, float, __nv_bfloat16, float>(tm, a, s);
    if (ti == DT_F32 && tb == DT_F16)
        return launch_forward_t<WV, MODE_NONSEP, float, __half, float>(tm, a, s);
    if (ti == DT_BF16 && tb == DT_BF16)
        return launch_forward_t<WV, MODE_NONSEP, __nv_bfloat16, __nv_bfloat16, float>(tm, a, s);
    if (ti == DT_F16 && tb == DT_F16)
        return launch_forward_t<WV, MODE_NONSEP, __half, __half, float>(tm, a, s);
    return cudaErrorNotSupported;
}

template <int WV>
cudaError_t inv(int tb, int to, const CUtensorMap* tm, const InvArgs& a, cudaStream_t s) {
    if (tb == DT_F32 && to == DT_F32) return launch_inverse_t<WV, float, float, float>(tm, a, s);
    if (tb == DT_BF16 && to == DT_F32)
        return launch_inverse_t<WV, __nv_bfloat16, float, float>(tm, a, s);
    if (tb == DT_BF16 && to == DT_BF16)
        return launch_inverse_t<WV, __nv_bfloat16, float, __nv_bfloat16>(tm, a, s);
    if (tb == DT_F16 && to == DT_F32) return launch_inverse_t<WV, __half, float, float>(tm, a, s);
    if (tb == DT_F16 && to == DT_F16) return launch_inverse_t<WV, __half, float, __half>(tm, a, s);
    return cudaErrorNotSupported;
}
}  // namespace

// The two-pass separable comparator: the row pass and the column pass (fp32 only).
template <int WV>
cudaError_t twopass(int mode, int ti, int tb, const CUtensorMap& tm, const FwdArgs& a,
                    cudaStream_t s) {
    if (ti != DT_F32 || tb != DT_F32) return cudaErrorNotSupported;
    if (mode == MODE_ROWS) return launch_forward_t<WV, MODE_ROWS, float, float, float>(tm, a, s);
    return launch_forward_t<WV, MODE_COLS, float, float, float>(tm, a, s);
}

cudaError_t launch_fwd_dd(int wavelet, int mode, int ti, int tb, const CUtensorMap& tm,
                          const FwdArgs& a, cudaStream_t s) {
    if (mode == MODE_ROWS || mode == MODE_COLS) {
        if (wavelet == WV_DD97) return twopass<WV_DD97>(mode, ti, tb, tm, a, s);
        if (wavelet == WV_DD137) return twopass<WV_DD137>(mode, ti, tb, tm, a, s);
        return cudaErrorNotSupported;
    }
    if (mode != MODE_NONSEP) return cudaErrorNotSupported;
    if (wavelet == WV_DD97) return fwd<WV_DD97>(ti, tb, tm, a, s);
    if (wavelet == WV_DD137) return fwd<WV_DD137>(ti, tb, tm, a, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_inv_dd(int wavelet, int tb, int to, const CUtensorMap* tm, const InvArgs& a,
                          cudaStream_t s) {
    if (wavelet == WV_DD97) return inv<WV_DD97>(tb, to, tm, a, s);
    if (wavelet == WV_DD137) return inv<WV_DD137>(tb, to, tm, a, s);
    return cudaErrorNotSupported;
}

}  // namespace dwt2
