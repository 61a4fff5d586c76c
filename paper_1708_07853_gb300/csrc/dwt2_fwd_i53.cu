// Forward-level kernels of the reversible integer CDF 5/3.
#include "dwt2_internal.h"

namespace dwt2 {

cudaError_t launch_fwd_i53(int mode, const CUtensorMap& tm, const FwdArgs& a, cudaStream_t s) {
#define I53(M) return launch_forward_t<WV_CDF53_INT, M, int32_t, int32_t, int32_t>(tm, a, s)
    switch (mode) {
    case MODE_NONSEP: I53(MODE_NONSEP);
    case MODE_SEP: I53(MODE_SEP);
    case MODE_ROWS: I53(MODE_ROWS);
    case MODE_COLS: I53(MODE_COLS);
    default: return cudaErrorNotSupported;
    }
#undef I53
}

}  // namespace dwt2
