// Persistent batched kernels of the Deslauriers-Dubuc 9/7 and 13/7 wavelets (forward and
// inverse transforms; fp32 arithmetic, fp32 / bf16 / fp16 bands; no adjoints).
#include "dwt2_internal.h"

namespace dwt2 {

namespace {
template <int WV, typename TB>
cudaError_t fwd(const PersistArgs<FwdUnit>& p, int ctas_per_sm, cudaStream_t st, int* occ_out) {
    auto k = k_forward_persistent<WV, MODE_NONSEP, float, TB, float>;
    constexpr size_t smem = fwd_smem_bytes<float, kPersistStages>();
    static const int occ = configure(k, cta_threads<kPersistFwdNW>(), smem);
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    const int c = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    k<<<device_sm_count() * c, cta_threads<kPersistFwdNW>(), smem, st>>>(p);
    return cudaGetLastError();
}

template <int WV, typename TB>
cudaError_t inv(const PersistArgs<InvUnit>& p, int ctas_per_sm, cudaStream_t st, int* occ_out) {
    auto k = k_inverse_persistent<WV, TB, float, float, false>;
    constexpr size_t smem = inv_smem_bytes<float, TB, kPersistStages>();
    static const int occ = configure(k, cta_threads<persist_inv_nw<TB, float>()>(), smem);
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    const int c = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    k<<<device_sm_count() * c, cta_threads<persist_inv_nw<TB, float>()>(), smem, st>>>(p);
    return cudaGetLastError();
}

template <int WV>
cudaError_t fwd_t(int tb, const PersistArgs<FwdUnit>& p, int c, cudaStream_t st, int* occ) {
    switch (tb) {
    case DT_F32: return fwd<WV, float>(p, c, st, occ);
    case DT_BF16: return fwd<WV, __nv_bfloat16>(p, c, st, occ);
    case DT_F16: return fwd<WV, __half>(p, c, st, occ);
    default: return cudaErrorNotSupported;
    }
}

template <int WV>
cudaError_t inv_t(int tb, const PersistArgs<InvUnit>& p, int c, cudaStream_t st, int* occ) {
    switch (tb) {
    case DT_F32: return inv<WV, float>(p, c, st, occ);
    case DT_BF16: return inv<WV, __nv_bfloat16>(p, c, st, occ);
    case DT_F16: return inv<WV, __half>(p, c, st, occ);
    default: return cudaErrorNotSupported;
    }
}
}  // namespace

cudaError_t launch_fwd_persistent_dd(int wavelet, int mode, int tb, const PersistArgs<FwdUnit>& p,
                                     int ctas_per_sm, cudaStream_t st, int* occ) {
    if (mode != MODE_NONSEP) return cudaErrorNotSupported;
    if (wavelet == WV_DD97) return fwd_t<WV_DD97>(tb, p, ctas_per_sm, st, occ);
    if (wavelet == WV_DD137) return fwd_t<WV_DD137>(tb, p, ctas_per_sm, st, occ);
    return cudaErrorNotSupported;
}

cudaError_t launch_inv_persistent_dd(int wavelet, bool adj, int tb, const PersistArgs<InvUnit>& p,
                                     int ctas_per_sm, cudaStream_t st, int* occ) {
    if (adj) return cudaErrorNotSupported;
    if (wavelet == WV_DD97) return inv_t<WV_DD97>(tb, p, ctas_per_sm, st, occ);
    if (wavelet == WV_DD137) return inv_t<WV_DD137>(tb, p, ctas_per_sm, st, occ);
    return cudaErrorNotSupported;
}

}  // namespace dwt2
