// Forward-level kernels of the float CDF 5/3 (fp32 arithmetic; fp32 / bf16 / fp16 storage).
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int MODE, typename TI, typename TB>
cudaError_t go(const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s) {
    return launch_forward_t<WV_CDF53, MODE, TI, TB, float>(tm, a, s);
}
}  // namespace

cudaError_t launch_fwd_f53(int mode, int ti, int tb, const CUtensorMap& tm,
                           const FwdArgs& a, cudaStream_t s) {
    if (mode == MODE_NONSEP) {
        if (ti == DT_F32 && tb == DT_F32) return go<MODE_NONSEP, float, float>(tm, a, s);
        if (ti == DT_F32 && tb == DT_BF16) return go<MODE_NONSEP, float, __nv_bfloat16>(tm, a, s);
        if (ti == DT_F32 && tb == DT_F16) return go<MODE_NONSEP, float, __half>(tm, a, s);
        if (ti == DT_BF16 && tb == DT_BF16)
            return go<MODE_NONSEP, __nv_bfloat16, __nv_bfloat16>(tm, a, s);
        if (ti == DT_F16 && tb == DT_F16) return go<MODE_NONSEP, __half, __half>(tm, a, s);
        return cudaErrorNotSupported;
    }
    if (ti != DT_F32 || tb != DT_F32) return cudaErrorNotSupported;
    switch (mode) {
    case MODE_SEP: return go<MODE_SEP, float, float>(tm, a, s);
    case MODE_ROWS: return go<MODE_ROWS, float, float>(tm, a, s);
    case MODE_COLS: return go<MODE_COLS, float, float>(tm, a, s);
    case MODE_ADAPTED: return go<MODE_ADAPTED, float, float>(tm, a, s);
    case MODE_CONV: return go<MODE_CONV, float, float>(tm, a, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace dwt2
