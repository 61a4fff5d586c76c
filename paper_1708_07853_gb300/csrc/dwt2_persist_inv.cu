// Persistent batched kernels with the inverse data flow (inverse transform and the transpose
// of the forward).
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int WV, typename TB, typename TL, typename TO, bool ADJ>
cudaError_t go(const PersistArgs<InvUnit>& p, int ctas_per_sm, cudaStream_t st, int* occ_out) {
    auto k = k_inverse_persistent<WV, TB, TL, TO, ADJ>;
    constexpr size_t smem = inv_smem_bytes<TL, TB, kPersistStages>();
    static const int occ = configure(k, cta_threads<persist_inv_nw<TB, TL>()>(), smem);
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    const int c = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    k<<<device_sm_count() * c, cta_threads<persist_inv_nw<TB, TL>()>(), smem, st>>>(p);
    return cudaGetLastError();
}

template <int WV>
cudaError_t go_float(bool adj, int tb, const PersistArgs<InvUnit>& p, int c, cudaStream_t st,
                     int* occ) {
    if (adj)
        return tb == DT_F32 ? go<WV, float, float, float, true>(p, c, st, occ)
                            : cudaErrorNotSupported;
    switch (tb) {
    case DT_F32: return go<WV, float, float, float, false>(p, c, st, occ);
    case DT_BF16: return go<WV, __nv_bfloat16, float, float, false>(p, c, st, occ);
    case DT_F16: return go<WV, __half, float, float, false>(p, c, st, occ);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace

cudaError_t launch_inv_persistent(int wavelet, bool adj, int tb, const PersistArgs<InvUnit>& p,
                                  int ctas_per_sm, cudaStream_t st, int* occ) {
    switch (wavelet) {
    case WV_CDF53_INT:
        if (adj || tb != DT_I32) return cudaErrorNotSupported;
        return go<WV_CDF53_INT, int32_t, int32_t, int32_t, false>(p, ctas_per_sm, st, occ);
    case WV_CDF53: return go_float<WV_CDF53>(adj, tb, p, ctas_per_sm, st, occ);
    case WV_CDF97: return go_float<WV_CDF97>(adj, tb, p, ctas_per_sm, st, occ);
    case WV_DD97:
    case WV_DD137: return launch_inv_persistent_dd(wavelet, adj, tb, p, ctas_per_sm, st, occ);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace dwt2
