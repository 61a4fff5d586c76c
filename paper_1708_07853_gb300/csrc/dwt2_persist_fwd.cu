// Persistent batched kernels with the forward data flow (forward transform and the transpose
// of the inverse).
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int WV, int MODE, typename TI, typename TB, typename TL>
cudaError_t go(const PersistArgs<FwdUnit>& p, int ctas_per_sm, cudaStream_t st, int* occ_out) {
    auto k = k_forward_persistent<WV, MODE, TI, TB, TL>;
    constexpr size_t smem = fwd_smem_bytes<TI, persist_fwd_stages<WV>()>();
    static const int occ = configure(k, cta_threads<kPersistFwdNW>(), smem);
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    const int c = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    k<<<device_sm_count() * c, cta_threads<kPersistFwdNW>(), smem, st>>>(p);
    return cudaGetLastError();
}

template <int WV>
cudaError_t go_float(int mode, int tb, const PersistArgs<FwdUnit>& p, int c, cudaStream_t st,
                     int* occ) {
    if (mode == MODE_ADJ_INV)
        return tb == DT_F32 ? go<WV, MODE_ADJ_INV, float, float, float>(p, c, st, occ)
                            : cudaErrorNotSupported;
    switch (tb) {
    case DT_F32: return go<WV, MODE_NONSEP, float, float, float>(p, c, st, occ);
    case DT_BF16: return go<WV, MODE_NONSEP, float, __nv_bfloat16, float>(p, c, st, occ);
    case DT_F16: return go<WV, MODE_NONSEP, float, __half, float>(p, c, st, occ);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace

cudaError_t launch_fwd_persistent(int wavelet, int mode, int tb, const PersistArgs<FwdUnit>& p,
                                  int ctas_per_sm, cudaStream_t st, int* occ) {
    switch (wavelet) {
    case WV_CDF53_INT:
        if (mode != MODE_NONSEP || tb != DT_I32) return cudaErrorNotSupported;
        return go<WV_CDF53_INT, MODE_NONSEP, int32_t, int32_t, int32_t>(p, ctas_per_sm, st, occ);
    case WV_CDF53: return go_float<WV_CDF53>(mode, tb, p, ctas_per_sm, st, occ);
    case WV_CDF97: return go_float<WV_CDF97>(mode, tb, p, ctas_per_sm, st, occ);
    case WV_DD97:
    case WV_DD137: return launch_fwd_persistent_dd(wavelet, mode, tb, p, ctas_per_sm, st, occ);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace dwt2
