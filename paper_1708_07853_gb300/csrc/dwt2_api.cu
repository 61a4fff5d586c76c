// dwt2_api.cu -- the C ABI of libdwt2.so: argument validation, the coefficient-buffer layout,
// workspace planning, TMA tensor maps and the per-level launch sequence.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/dwt2.h"
#include "dwt2_internal.h"

#define DWT2_EXPORT extern "C" __attribute__((visibility("default")))

namespace dwt2 {

// ------------------------------------------------------------------------------ utilities
static thread_local std::string g_last_error;

// Records a message for dwt2_last_error() (used by entry points in other translation units).
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

static int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return DWT2_ECUDA;
}

int device_sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 1;
        return v;
    }();
    return n;
}

// L2 bytes a level may ask to keep for the next one: its LL output, stored evict_last, if the
// planes of all images of the launch fit in three quarters of the device's L2 (the LL_1 of an
// 8192^2 fp32 image, 64 MiB, does) and the next level streams (the direct kernels of small
// planes read from L2 anyway).
static int64_t l2_keep_budget() {
    static int64_t n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess) v = 0;
        return int64_t(v) / 4 * 3;
    }();
    return n;
}

static size_t esize(int dt) { return dt == DT_BF16 || dt == DT_F16 ? 2 : 4; }
static int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
static int64_t plane_pitch(int w, int dt) { return align_up(std::max<int64_t>(1, w) * esize(dt), 16); }

static int max_levels(int H, int W) {
    if (H < 1 || W < 1) return 0;
    int n = H > W ? H : W, L = 0;
    while (n > 1) {
        n = (n + 1) / 2;
        ++L;
    }
    return L < 1 ? 1 : L;
}

struct Layout {
    int J = 0;
    int h[34], w[34];      // plane size entering level j + 1 (index 0 = image)
    dwt2_band band[1 + 3 * 33];
    int64_t bytes = 0;
};

static const dwt2_band& band_of(const Layout& L, int level, int kind /*0 HL 1 LH 2 HH*/) {
    return L.band[1 + 3 * (L.J - level) + kind];
}

static int make_layout(int H, int W, int J, int band_dtype, Layout* L) {
    if (H < 1 || W < 1 || J < 1 || J > max_levels(H, W) || J > 32) return DWT2_EINVAL;
    if (band_dtype < DT_I32 || band_dtype > DT_F16) return DWT2_EINVAL;
    L->J = J;
    L->h[0] = H;
    L->w[0] = W;
    for (int j = 1; j <= J; ++j) {
        L->h[j] = (L->h[j - 1] + 1) / 2;
        L->w[j] = (L->w[j - 1] + 1) / 2;
    }
    int64_t off = 0;
    auto add = [&](int idx, int h, int w, int dt, int level, char kind) {
        dwt2_band& b = L->band[idx];
        b.offset_bytes = off;
        b.h = h;
        b.w = w;
        b.pitch_bytes = int32_t(plane_pitch(w, dt));
        b.dtype = dt;
        b.level = level;
        b.kind = kind;
        b.reserved[0] = b.reserved[1] = b.reserved[2] = 0;
        off = align_up(off + (h > 0 && w > 0 ? int64_t(h) * b.pitch_bytes : 0), 256);
    };
    const int ll_dt = band_dtype == DT_I32 ? DT_I32 : DT_F32;
    add(0, L->h[J], L->w[J], ll_dt, J, 'A');
    for (int j = J; j >= 1; --j) {
        const int h = L->h[j - 1], w = L->w[j - 1];
        const int base = 1 + 3 * (J - j);
        add(base + 0, (h + 1) / 2, w / 2, band_dtype, j, 'H');
        add(base + 1, h / 2, (w + 1) / 2, band_dtype, j, 'V');
        add(base + 2, h / 2, w / 2, band_dtype, j, 'D');
    }
    L->bytes = off;
    return DWT2_OK;
}

// Workspace: [0, 256) status header; then LL ping-pong planes A (LL_1, LL_3, ...) and
// B (LL_2, LL_4, ...); then, for the two-pass comparator, a full-size plane.
static constexpr int64_t kHeader = 256;
struct WsPlan {
    int64_t off[3] = {0, 0, 0};
    int64_t pitch[3] = {0, 0, 0};
    int64_t bytes = 0;
};

static WsPlan plan_workspace(int H, int W, int J, int wavelet, int scheme) {
    WsPlan p;
    const int dt = wavelet == WV_CDF53_INT ? DT_I32 : DT_F32;
    int64_t off = kHeader;
    int h = H, w = W;
    for (int k = 0; k < 2; ++k) {
        h = (h + 1) / 2;
        w = (w + 1) / 2;
        p.off[k] = off;
        p.pitch[k] = plane_pitch(w, dt);
        if (J >= k + 2) off = align_up(off + int64_t(h) * p.pitch[k], 256);
    }
    if (scheme == DWT2_SCHEME_SEP_TWOPASS) {
        p.off[2] = off;
        p.pitch[2] = plane_pitch(W, dt);
        off = align_up(off + int64_t(H) * p.pitch[2], 256);
    }
    p.bytes = off;
    return p;
}

// ------------------------------------------------------------------------------ tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

static CUtensorMapDataType tm_type(int dt) {
    switch (dt) {
    case DT_I32: return CU_TENSOR_MAP_DATA_TYPE_INT32;
    case DT_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    case DT_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    }
}

// A 3-D map over n planes of h x w (image z at base + z * bstride) with 1-row boxes of box_w
// elements; n = 1 for a single plane.
// MAP_OK: use TMA.  MAP_INELIGIBLE: the planes cannot be addressed by TMA (base, pitch or batch
// stride not 16-byte aligned, empty plane): use the plain-load path.  MAP_ERROR: an eligible
// plane was rejected by the driver, which is a library bug and is reported, never silently
// worked around.
enum MapResult { MAP_OK = 0, MAP_INELIGIBLE = 1, MAP_ERROR = 2 };

static MapResult make_map(CUtensorMap* m, const void* base, int64_t pitch, int64_t bstride, int h,
                          int w, int n, int dt, int box_w) {
    std::memset(m, 0, sizeof(*m));
    if (n <= 1) bstride = int64_t(h) * pitch;
    if (h < 1 || w < 1 || n < 1 || !aligned(base, 16) || pitch % 16 != 0 || bstride % 16 != 0)
        return MAP_INELIGIBLE;
    auto fn = encode_fn();
    if (!fn) {
        g_last_error = "cuTensorMapEncodeTiled is not available from the driver";
        return MAP_ERROR;
    }
    cuuint64_t dims[3] = {cuuint64_t(w), cuuint64_t(h), cuuint64_t(n)};
    cuuint64_t strides[2] = {cuuint64_t(pitch), cuuint64_t(bstride)};
    cuuint32_t box[3] = {cuuint32_t(box_w), 1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, tm_type(dt), 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        g_last_error = "cuTensorMapEncodeTiled failed (CUresult " + std::to_string(int(r)) +
                       ") for " + std::to_string(n) + " planes of " + std::to_string(h) + "x" +
                       std::to_string(w) + ", box " + std::to_string(box_w);
        return MAP_ERROR;
    }
    return MAP_OK;
}

// ------------------------------------------------------------------------------ validation
static int check_types(int wavelet, int img_dtype, int band_dtype) {
    if (wavelet < WV_CDF53_INT || wavelet > WV_DD137) return DWT2_EINVAL;
    if (img_dtype < DT_I32 || img_dtype > DT_F16 || band_dtype < DT_I32 || band_dtype > DT_F16)
        return DWT2_EINVAL;
    if (wavelet == WV_CDF53_INT)
        return (img_dtype == DT_I32 && band_dtype == DT_I32) ? DWT2_OK : DWT2_EUNSUPPORTED;
    if (band_dtype == DT_I32 || img_dtype == DT_I32) return DWT2_EUNSUPPORTED;
    if (img_dtype != DT_F32 && img_dtype != band_dtype) return DWT2_EUNSUPPORTED;
    return DWT2_OK;
}

static int check_image(const void* img, int64_t pitch, int W, int dt) {
    if (!img) return DWT2_EINVAL;
    const size_t es = esize(dt);
    if (!aligned(img, es) || pitch < int64_t(W) * int64_t(es) || pitch % int64_t(es) != 0)
        return DWT2_EINVAL;
    return DWT2_OK;
}

static FwdArgs level_args(const void* in, int64_t in_pitch, int64_t in_bstride, int h, int w,
                          int n, int* status) {
    FwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = in;
    a.in_pitch = in_pitch;
    a.in_bstride = in_bstride;
    a.H = h;
    a.W = w;
    a.ner = (h + 1) / 2;
    a.ndr = h / 2;
    a.nec = (w + 1) / 2;
    a.ndc = w / 2;
    a.status = status;
    a.nbatch = n;
    return a;
}

static cudaError_t launch_fwd(int wavelet, int mode, int ti, int tb, bool tma,
                              const CUtensorMap& tm, FwdArgs a, cudaStream_t s) {
    a.tma = tma ? 1 : 0;
    switch (wavelet) {
    case WV_CDF53_INT: return launch_fwd_i53(mode, tm, a, s);
    case WV_CDF53: return launch_fwd_f53(mode, ti, tb, tm, a, s);
    case WV_DD97:
    case WV_DD137: return launch_fwd_dd(wavelet, mode, ti, tb, tm, a, s);
    default: return launch_fwd_f97(mode, ti, tb, tm, a, s);
    }
}

// Per-level band scales of the CDF 9/7 normalisation (1 for CDF 5/3): per axis low 1/K, high
// K/2, and 1 on an axis of length 1 (that axis passes through).
static Scale4 level_scale(int wavelet, int h, int w) {
    const double K = 1.230174104914001;
    const bool s97 = wavelet == WV_CDF97;
    const double vl = (s97 && h > 1) ? 1.0 / K : 1.0, vh = (s97 && h > 1) ? K / 2 : 1.0;
    const double hl = (s97 && w > 1) ? 1.0 / K : 1.0, hh = (s97 && w > 1) ? K / 2 : 1.0;
    return Scale4{float(vl * hl), float(vl * hh), float(vh * hl), float(vh * hh)};
}

static Scale4 reciprocal(Scale4 s) { return Scale4{1.f / s.ll, 1.f / s.hl, 1.f / s.lh, 1.f / s.hh}; }

// A batch of N images (N = 1 for the single-image entry points): image z of the input at
// img + z * img_bstride, its coefficients at coeffs + z * coeff_bstride, and its intermediate LL
// planes in workspace region z (after the shared 256-byte status header).
struct Batch {
    int N;
    int64_t img_bstride, coeff_bstride;
};

static int check_batch(const Batch& b, int H, int64_t img_pitch, int img_dtype, const Layout& L) {
    if (b.N < 1 || b.N > 65535) return DWT2_EINVAL;
    if (b.N == 1) return DWT2_OK;
    if (b.img_bstride < int64_t(H) * img_pitch || b.img_bstride % int64_t(esize(img_dtype)) != 0 ||
        b.coeff_bstride < L.bytes || b.coeff_bstride % 16 != 0)
        return DWT2_EINVAL;
    return DWT2_OK;
}

// Bytes between the workspace regions of consecutive images of a batch.
static int64_t ws_region(const WsPlan& wp) { return align_up(wp.bytes - kHeader, 256); }

// The DC level shift of a float transform (ShiftSrc in dwt2_stream.cuh): c is sampled from the
// plane p (the image for a forward transform, LL_J for an inverse), taken off at the first
// level and put back at the last.  mode: kShiftIn and / or kShiftOut for this level.
static ShiftSrc shift_from(const void* p, int64_t pitch, int64_t bstride, int h, int w, int dt,
                           int mode) {
    ShiftSrc s;
    s.ptr = mode ? p : nullptr;
    s.pitch = pitch;
    s.bstride = bstride;
    s.h = h;
    s.w = w;
    s.dt = dt;
    s.mode = mode;
    return s;
}

// adjoint = true: W^-T, the transpose of the inverse (image-shaped gradient in, band gradients
// out), level by level 1..J with the forward kernel's data flow.
// clear_status: zero the workspace's status header on st once the arguments have passed every
// check (the built-in scratch of dwt2_forward_static, which no caller can initialise).
static int forward_impl(const void* img, int64_t img_pitch, int H, int W, int img_dtype,
                        void* coeffs, void* ws, size_t ws_bytes, int wavelet, int J,
                        int band_dtype, int scheme, cudaStream_t st, bool adjoint = false,
                        Batch bt = Batch{1, 0, 0}, bool clear_status = false) {
    int rc = check_types(wavelet, img_dtype, band_dtype);
    if (rc) return rc;
    if (adjoint && (wavelet == WV_CDF53_INT || is_dd(wavelet) || img_dtype != DT_F32 ||
                    band_dtype != DT_F32))
        return DWT2_EUNSUPPORTED;
    if (scheme < DWT2_SCHEME_NONSEP || scheme > DWT2_SCHEME_CONV) return DWT2_EINVAL;
    if (is_dd(wavelet) && scheme != DWT2_SCHEME_NONSEP && scheme != DWT2_SCHEME_SEP_TWOPASS)
        return DWT2_EUNSUPPORTED;
    if (scheme != DWT2_SCHEME_NONSEP && (img_dtype != band_dtype || bt.N != 1))
        return DWT2_EUNSUPPORTED;
    if ((scheme == DWT2_SCHEME_ADAPTED || scheme == DWT2_SCHEME_CONV) &&
        (wavelet == WV_CDF53_INT || adjoint))
        return DWT2_EUNSUPPORTED;
    Layout L;
    if ((rc = make_layout(H, W, J, band_dtype, &L))) return rc;
    if ((rc = check_image(img, img_pitch, W, img_dtype))) return rc;
    if ((rc = check_batch(bt, H, img_pitch, img_dtype, L))) return rc;
    if (!coeffs || !ws || !aligned(coeffs, 16) || !aligned(ws, 16)) return DWT2_EINVAL;
    const WsPlan wp = plan_workspace(H, W, J, wavelet, scheme);
    const int64_t region = ws_region(wp);
    if (int64_t(ws_bytes) < kHeader + bt.N * region) return DWT2_ENOMEM;
    const int64_t cbs = bt.N > 1 ? bt.coeff_bstride : 0;
    if (clear_status) {
        const cudaError_t e = cudaMemsetAsync(ws, 0, kHeader, st);
        if (e != cudaSuccess) return cuda_fail(e, "status header");
    }

    char* cb = static_cast<char*>(coeffs);
    char* wb = static_cast<char*>(ws);
    int* status = reinterpret_cast<int*>(wb);
    const int ll_dt = wavelet == WV_CDF53_INT ? DT_I32 : DT_F32;

    const void* in = img;
    int64_t in_pitch = img_pitch, in_bstride = bt.N > 1 ? bt.img_bstride : 0;
    int in_dt = img_dtype;
    // float lifting takes the DC level shift; the adjoint and the convolution scheme do not
    const bool shifted = wavelet != WV_CDF53_INT && !adjoint && scheme != DWT2_SCHEME_CONV;
    bool in_kept = false;  // the previous level stored this level's input evict_last
    for (int j = 1; j <= J; ++j) {
        const int h = L.h[j - 1], w = L.w[j - 1];
        FwdArgs a = level_args(in, in_pitch, in_bstride, h, w, bt.N, status);
        const int smode = shifted ? (j == 1 ? kShiftIn : 0) | (j == J ? kShiftOut : 0) : 0;
        a.shift = shift_from(img, img_pitch, bt.N > 1 ? bt.img_bstride : 0, H, W, img_dtype, smode);
        const dwt2_band &bhl = band_of(L, j, 0), &blh = band_of(L, j, 1), &bhh = band_of(L, j, 2);
        a.hl = {cb + bhl.offset_bytes, bhl.pitch_bytes, cbs};
        a.lh = {cb + blh.offset_bytes, blh.pitch_bytes, cbs};
        a.hh = {cb + bhh.offset_bytes, bhh.pitch_bytes, cbs};
        if (j == J) a.ll = {cb + L.band[0].offset_bytes, L.band[0].pitch_bytes, cbs};
        else a.ll = {wb + wp.off[(j - 1) % 2], wp.pitch[(j - 1) % 2], region};
        // LL_j stays in L2 for level j + 1 when it fits and that level streams
        const bool next_direct = scheme == DWT2_SCHEME_NONSEP && !adjoint &&
                                 takes_direct(L.h[j], L.w[j], esize(ll_dt), bt.N);
        a.ll_keep = keeps_ll_in_l2(wavelet) && j < J && !next_direct &&
                    a.ll.pitch * int64_t(L.h[j]) * bt.N <= l2_keep_budget();
        a.in_kept = in_kept;

        cudaError_t e;
        if (scheme == DWT2_SCHEME_SEP_TWOPASS) {
            // row pass into the full-size plane, then the column pass into the bands
            CUtensorMap tm;
            MapResult mr = make_map(&tm, in, in_pitch, 0, h, w, 1, in_dt, kBoxW);
            if (mr == MAP_ERROR) return DWT2_EINTERNAL;
            bool tma = mr == MAP_OK;
            FwdArgs r = a;
            r.ll = {wb + wp.off[2], wp.pitch[2], 0};
            r.shift.mode &= kShiftIn;  // the row pass takes the shift off the image
            if (!r.shift.mode) r.shift.ptr = nullptr;
            e = launch_fwd(wavelet, MODE_ROWS, in_dt, band_dtype, tma, tm, r, st);
            if (e != cudaSuccess) return cuda_fail(e, "row pass");
            FwdArgs c = level_args(wb + wp.off[2], wp.pitch[2], 0, h, w, 1, status);
            c.ll = a.ll;
            c.ll_keep = a.ll_keep;
            c.hl = a.hl;
            c.lh = a.lh;
            c.hh = a.hh;
            c.shift = a.shift;  // the column pass puts it back onto LL_J
            c.shift.mode &= kShiftOut;
            if (!c.shift.mode) c.shift.ptr = nullptr;
            mr = make_map(&tm, wb + wp.off[2], wp.pitch[2], 0, h, w, 1, ll_dt, kBoxW);
            if (mr == MAP_ERROR) return DWT2_EINTERNAL;
            tma = mr == MAP_OK;
            e = launch_fwd(wavelet, MODE_COLS, ll_dt, band_dtype, tma, tm, c, st);
            if (e != cudaSuccess) return cuda_fail(e, "column pass");
        } else {
            CUtensorMap tm;
            const MapResult mr = make_map(&tm, in, in_pitch, in_bstride, h, w, bt.N, in_dt, kBoxW);
            if (mr == MAP_ERROR) return DWT2_EINTERNAL;
            const bool tma = mr == MAP_OK;
            const int mode = scheme == DWT2_SCHEME_NONSEP    ? MODE_NONSEP
                             : scheme == DWT2_SCHEME_ADAPTED ? MODE_ADAPTED
                             : scheme == DWT2_SCHEME_CONV    ? MODE_CONV
                                                             : MODE_SEP;
            if (adjoint) {
                a.scale = reciprocal(level_scale(wavelet, h, w));
                a.tma = tma ? 1 : 0;
                e = launch_adj_inv(wavelet, tm, a, st);
            } else {
                e = launch_fwd(wavelet, mode, in_dt, band_dtype, tma, tm, a, st);
            }
            if (e == cudaErrorNotSupported) return DWT2_EUNSUPPORTED;
            if (e != cudaSuccess) return cuda_fail(e, "forward level");
        }
        in = a.ll.ptr;
        in_pitch = a.ll.pitch;
        in_bstride = a.ll.bstride;
        in_dt = ll_dt;
        in_kept = a.ll_keep != 0;
    }
    return DWT2_OK;
}

// adjoint = true: W^T, the transpose of the forward (band gradients in, image-shaped gradient
// out), level by level J..1 with the inverse kernel's data flow.
static int inverse_impl(const void* coeffs, void* img, int64_t img_pitch, int H, int W,
                        int img_dtype, void* ws, size_t ws_bytes, int wavelet, int J,
                        int band_dtype, cudaStream_t st, bool adjoint = false,
                        Batch bt = Batch{1, 0, 0}) {
    int rc = check_types(wavelet, img_dtype, band_dtype);
    if (rc) return rc;
    if (adjoint && (wavelet == WV_CDF53_INT || is_dd(wavelet) || img_dtype != DT_F32 ||
                    band_dtype != DT_F32))
        return DWT2_EUNSUPPORTED;
    Layout L;
    if ((rc = make_layout(H, W, J, band_dtype, &L))) return rc;
    if ((rc = check_image(img, img_pitch, W, img_dtype))) return rc;
    if ((rc = check_batch(bt, H, img_pitch, img_dtype, L))) return rc;
    if (!coeffs || !ws || !aligned(coeffs, 16) || !aligned(ws, 16)) return DWT2_EINVAL;
    const WsPlan wp = plan_workspace(H, W, J, wavelet, DWT2_SCHEME_NONSEP);
    const int64_t region = ws_region(wp);
    if (int64_t(ws_bytes) < kHeader + bt.N * region) return DWT2_ENOMEM;
    const int64_t cbs = bt.N > 1 ? bt.coeff_bstride : 0;
    const int64_t ibs = bt.N > 1 ? bt.img_bstride : 0;

    const char* cb = static_cast<const char*>(coeffs);
    char* wb = static_cast<char*>(ws);
    int* status = reinterpret_cast<int*>(wb);
    const int ll_dt = wavelet == WV_CDF53_INT ? DT_I32 : DT_F32;

    const bool shifted = wavelet != WV_CDF53_INT && !adjoint;
    bool ll_kept = false;  // the previous level stored this level's LL evict_last
    for (int j = J; j >= 1; --j) {
        const int h = L.h[j - 1], w = L.w[j - 1];
        InvArgs a;
        std::memset(&a, 0, sizeof(a));
        const int smode = shifted ? (j == J ? kShiftIn : 0) | (j == 1 ? kShiftOut : 0) : 0;
        a.shift = shift_from(cb + L.band[0].offset_bytes, L.band[0].pitch_bytes, cbs, L.h[J],
                             L.w[J], DT_F32, smode);
        a.H = h;
        a.W = w;
        a.ner = (h + 1) / 2;
        a.ndr = h / 2;
        a.nec = (w + 1) / 2;
        a.ndc = w / 2;
        a.status = status;
        a.nbatch = bt.N;
        if (j == J) {
            a.band[0] = cb + L.band[0].offset_bytes;
            a.band_pitch[0] = L.band[0].pitch_bytes;
            a.band_bstride[0] = cbs;
        } else {
            a.band[0] = wb + wp.off[(j - 1) % 2];
            a.band_pitch[0] = wp.pitch[(j - 1) % 2];
            a.band_bstride[0] = region;
        }
        for (int k = 0; k < 3; ++k) {
            const dwt2_band& b = band_of(L, j, k);
            a.band[1 + k] = cb + b.offset_bytes;
            a.band_pitch[1 + k] = b.pitch_bytes;
            a.band_bstride[1 + k] = cbs;
        }
        int out_dt;
        if (j == 1) {
            a.out = {img, img_pitch, ibs};
            out_dt = img_dtype;
        } else {
            a.out = {wb + wp.off[(j - 2) % 2], wp.pitch[(j - 2) % 2], region};
            out_dt = ll_dt;
        }
        const size_t vbytes = 4 * esize(out_dt);
        a.out_vec = aligned(a.out.ptr, vbytes) && a.out.pitch % int64_t(vbytes) == 0 &&
                    a.out.bstride % int64_t(vbytes) == 0;
        // LL_(j-1) stays in L2 for level j - 1 when it fits and that level streams
        const bool next_direct =
            j > 1 && !adjoint && takes_direct(L.h[j - 2], L.w[j - 2], esize(ll_dt), bt.N);
        a.out_keep = keeps_ll_in_l2(wavelet) && j > 1 && !next_direct &&
                     a.out.pitch * int64_t(h) * bt.N <= l2_keep_budget();
        a.ll_kept = ll_kept;
        ll_kept = a.out_keep != 0;

        // TMA needs all four band planes non-empty (h, w >= 2); the plain-load path covers the
        // rest (and planes whose base, pitch or batch stride TMA cannot address).
        CUtensorMap tm[4];
        bool tma = h >= 2 && w >= 2;
        if (tma) {
            const int dims[4][2] = {{a.ner, a.nec}, {a.ner, a.ndc}, {a.ndr, a.nec}, {a.ndr, a.ndc}};
            for (int k = 0; k < 4; ++k) {
                const MapResult r = make_map(&tm[k], a.band[k], a.band_pitch[k], a.band_bstride[k],
                                             dims[k][0], dims[k][1], bt.N, k == 0 ? ll_dt : band_dtype,
                                             kBoxW);
                if (r == MAP_ERROR) return DWT2_EINTERNAL;
                if (r != MAP_OK) tma = false;
            }
        }
        if (!tma) std::memset(tm, 0, sizeof(tm));
        a.tma = tma ? 1 : 0;
        cudaError_t e;
        if (adjoint) {
            a.scale = level_scale(wavelet, h, w);
            e = launch_adj_fwd(wavelet, tm, a, st);
        } else {
            e = launch_inv(wavelet, band_dtype, out_dt, tm, a, st);
        }
        if (e == cudaErrorNotSupported) return DWT2_EUNSUPPORTED;
        if (e != cudaSuccess) return cuda_fail(e, "inverse level");
    }
    return DWT2_OK;
}

// The forward transform of dwt2_forward_static: dwt2_forward into the built-in scratch, whose
// status header is cleared once the arguments are known to be valid.
int forward_into_scratch(const void* img, int64_t img_pitch, int H, int W, int img_dtype,
                         void* coeffs, void* scratch, size_t scratch_bytes, int wavelet, int J,
                         int band_dtype, cudaStream_t st) {
    return forward_impl(img, img_pitch, H, W, img_dtype, coeffs, scratch, scratch_bytes, wavelet,
                        J, band_dtype, DWT2_SCHEME_NONSEP, st, false, Batch{1, 0, 0}, true);
}

// ------------------------------------------------------------------ helpers for batched plans
Scale4 plan_level_scale(int wavelet, int h, int w) { return level_scale(wavelet, h, w); }

// Bytes of one image's LL ping-pong planes and their offsets / pitches within that region.
int64_t plan_image_scratch(int H, int W, int J, int wavelet, int64_t offs[2], int64_t pitch[2]) {
    const WsPlan wp = plan_workspace(H, W, J, wavelet, DWT2_SCHEME_NONSEP);
    for (int k = 0; k < 2; ++k) {
        offs[k] = wp.off[k] - kHeader;
        pitch[k] = wp.pitch[k];
    }
    return wp.bytes - kHeader;
}

int plan_layout(int H, int W, int J, int band_dtype, dwt2_band* bands, size_t* bytes) {
    Layout L;
    const int rc = make_layout(H, W, J, band_dtype, &L);
    if (rc) return rc;
    std::memcpy(bands, L.band, sizeof(dwt2_band) * (1 + 3 * J));
    *bytes = size_t(L.bytes);
    return DWT2_OK;
}

int plan_prepare_fwd_unit(FwdUnit* u, const void* in, int64_t in_pitch, int h, int w, int in_dt,
                          int tb, int* status) {
    (void)tb;
    u->a = level_args(in, in_pitch, 0, h, w, 1, status);
    const MapResult mr = make_map(&u->tm, in, in_pitch, 0, h, w, 1, in_dt, kBoxW);
    if (mr == MAP_ERROR) return DWT2_EINTERNAL;
    u->a.tma = mr == MAP_OK ? 1 : 0;
    return DWT2_OK;
}

int plan_prepare_inv_unit(InvUnit* u, const void* const bands[4], const int64_t pitches[4], int h,
                          int w, int tl, int tb, void* out, int64_t out_pitch, int out_dt,
                          int* status) {
    InvArgs& a = u->a;
    std::memset(&a, 0, sizeof(a));
    a.H = h;
    a.W = w;
    a.ner = (h + 1) / 2;
    a.ndr = h / 2;
    a.nec = (w + 1) / 2;
    a.ndc = w / 2;
    a.status = status;
    a.nbatch = 1;
    for (int k = 0; k < 4; ++k) {
        a.band[k] = bands[k];
        a.band_pitch[k] = pitches[k];
    }
    a.out = {out, out_pitch, 0};
    const size_t vbytes = 4 * esize(out_dt);
    a.out_vec = aligned(out, vbytes) && out_pitch % int64_t(vbytes) == 0;
    bool tma = h >= 2 && w >= 2;
    if (tma) {
        const int dims[4][2] = {{a.ner, a.nec}, {a.ner, a.ndc}, {a.ndr, a.nec}, {a.ndr, a.ndc}};
        for (int k = 0; k < 4; ++k) {
            const MapResult r = make_map(&u->tm[k], bands[k], pitches[k], 0, dims[k][0], dims[k][1],
                                         1, k == 0 ? tl : tb, kBoxW);
            if (r == MAP_ERROR) return DWT2_EINTERNAL;
            if (r != MAP_OK) tma = false;
        }
    }
    a.tma = tma ? 1 : 0;
    return DWT2_OK;
}

}  // namespace dwt2

using namespace dwt2;

// ==================================================================================== C ABI
DWT2_EXPORT const char* dwt2_status_string(int status) {
    switch (status) {
    case DWT2_OK: return "ok";
    case DWT2_EINVAL: return "invalid argument";
    case DWT2_EUNSUPPORTED: return "unsupported combination";
    case DWT2_ENOMEM: return "workspace or buffer too small";
    case DWT2_ECUDA: return "CUDA error";
    case DWT2_ETIMEOUT: return "device-side wait timed out";
    case DWT2_EINTERNAL: return "internal error";
    default: return "unknown status";
    }
}

DWT2_EXPORT const char* dwt2_last_error(void) { return g_last_error.c_str(); }

DWT2_EXPORT int dwt2_max_levels(int H, int W) { return max_levels(H, W); }

DWT2_EXPORT int dwt2_layout(int H, int W, int levels, int band_dtype, dwt2_band* bands,
                            size_t* coeff_bytes) {
    Layout L;
    const int rc = make_layout(H, W, levels, band_dtype, &L);
    if (rc) return rc;
    if (bands) std::memcpy(bands, L.band, sizeof(dwt2_band) * (1 + 3 * levels));
    if (coeff_bytes) *coeff_bytes = size_t(L.bytes);
    return DWT2_OK;
}

DWT2_EXPORT size_t dwt2_workspace_bytes_scheme(int H, int W, int levels, int wavelet,
                                               int band_dtype, int scheme) {
    Layout L;
    if (make_layout(H, W, levels, band_dtype, &L) || wavelet < 0 || wavelet > WV_DD137 ||
        scheme < DWT2_SCHEME_NONSEP || scheme > DWT2_SCHEME_CONV)
        return 0;
    return size_t(plan_workspace(H, W, levels, wavelet, scheme).bytes);
}

DWT2_EXPORT size_t dwt2_workspace_bytes(int H, int W, int levels, int wavelet, int band_dtype) {
    return dwt2_workspace_bytes_scheme(H, W, levels, wavelet, band_dtype, DWT2_SCHEME_NONSEP);
}

DWT2_EXPORT int dwt2_workspace_init(void* workspace, size_t ws_bytes, void* stream) {
    if (!workspace || ws_bytes < size_t(kHeader)) return DWT2_EINVAL;
    cudaError_t e = cudaMemsetAsync(workspace, 0, kHeader, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DWT2_OK : cuda_fail(e, "workspace init");
}

DWT2_EXPORT int dwt2_check_status(void* workspace, void* stream) {
    if (!workspace) return DWT2_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, workspace, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "check status");
    if (v != 0) {
        e = cudaMemsetAsync(workspace, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "check status");
    }
    return v == 0 ? DWT2_OK : v;
}

DWT2_EXPORT int dwt2_forward_scheme(const void* img, int64_t img_pitch_bytes, int H, int W,
                                    int img_dtype, void* coeffs, void* workspace, size_t ws_bytes,
                                    int wavelet, int levels, int band_dtype, int scheme,
                                    void* stream) {
    return forward_impl(img, img_pitch_bytes, H, W, img_dtype, coeffs, workspace, ws_bytes,
                        wavelet, levels, band_dtype, scheme, static_cast<cudaStream_t>(stream));
}

DWT2_EXPORT int dwt2_forward(const void* img, int64_t img_pitch_bytes, int H, int W,
                             int img_dtype, void* coeffs, void* workspace, size_t ws_bytes,
                             int wavelet, int levels, int band_dtype, void* stream) {
    return forward_impl(img, img_pitch_bytes, H, W, img_dtype, coeffs, workspace, ws_bytes,
                        wavelet, levels, band_dtype, DWT2_SCHEME_NONSEP,
                        static_cast<cudaStream_t>(stream));
}

DWT2_EXPORT int dwt2_inverse(const void* coeffs, void* img, int64_t img_pitch_bytes, int H, int W,
                             int img_dtype, void* workspace, size_t ws_bytes, int wavelet,
                             int levels, int band_dtype, void* stream) {
    return inverse_impl(coeffs, img, img_pitch_bytes, H, W, img_dtype, workspace, ws_bytes,
                        wavelet, levels, band_dtype, static_cast<cudaStream_t>(stream));
}

DWT2_EXPORT int dwt2_forward_adjoint(const void* g_coeffs, void* g_img, int64_t g_img_pitch_bytes,
                                     int H, int W, int img_dtype, void* workspace, size_t ws_bytes,
                                     int wavelet, int levels, int band_dtype, void* stream) {
    return inverse_impl(g_coeffs, g_img, g_img_pitch_bytes, H, W, img_dtype, workspace, ws_bytes,
                        wavelet, levels, band_dtype, static_cast<cudaStream_t>(stream), true);
}

DWT2_EXPORT int dwt2_inverse_adjoint(const void* g_img, int64_t g_img_pitch_bytes, int H, int W,
                                     int img_dtype, void* g_coeffs, void* workspace,
                                     size_t ws_bytes, int wavelet, int levels, int band_dtype,
                                     void* stream) {
    return forward_impl(g_img, g_img_pitch_bytes, H, W, img_dtype, g_coeffs, workspace, ws_bytes,
                        wavelet, levels, band_dtype, DWT2_SCHEME_NONSEP,
                        static_cast<cudaStream_t>(stream), true);
}

DWT2_EXPORT size_t dwt2_workspace_bytes_batch(int N, int H, int W, int levels, int wavelet,
                                              int band_dtype) {
    Layout L;
    if (N < 1 || make_layout(H, W, levels, band_dtype, &L) || wavelet < 0 || wavelet > WV_DD137)
        return 0;
    return size_t(kHeader + N * ws_region(plan_workspace(H, W, levels, wavelet, DWT2_SCHEME_NONSEP)));
}

DWT2_EXPORT int dwt2_forward_batch(const void* img, int64_t img_pitch_bytes, int64_t img_batch_bytes,
                                   int N, int H, int W, int img_dtype, void* coeffs,
                                   int64_t coeff_batch_bytes, void* workspace, size_t ws_bytes,
                                   int wavelet, int levels, int band_dtype, void* stream) {
    return forward_impl(img, img_pitch_bytes, H, W, img_dtype, coeffs, workspace, ws_bytes, wavelet,
                        levels, band_dtype, DWT2_SCHEME_NONSEP, static_cast<cudaStream_t>(stream),
                        false, Batch{N, img_batch_bytes, coeff_batch_bytes});
}

DWT2_EXPORT int dwt2_inverse_batch(const void* coeffs, int64_t coeff_batch_bytes, void* img,
                                   int64_t img_pitch_bytes, int64_t img_batch_bytes, int N, int H,
                                   int W, int img_dtype, void* workspace, size_t ws_bytes,
                                   int wavelet, int levels, int band_dtype, void* stream) {
    return inverse_impl(coeffs, img, img_pitch_bytes, H, W, img_dtype, workspace, ws_bytes, wavelet,
                        levels, band_dtype, static_cast<cudaStream_t>(stream), false,
                        Batch{N, img_batch_bytes, coeff_batch_bytes});
}

DWT2_EXPORT int dwt2_forward_adjoint_batch(const void* g_coeffs, int64_t coeff_batch_bytes,
                                           void* g_img, int64_t g_img_pitch_bytes,
                                           int64_t g_img_batch_bytes, int N, int H, int W,
                                           int img_dtype, void* workspace, size_t ws_bytes,
                                           int wavelet, int levels, int band_dtype, void* stream) {
    return inverse_impl(g_coeffs, g_img, g_img_pitch_bytes, H, W, img_dtype, workspace, ws_bytes,
                        wavelet, levels, band_dtype, static_cast<cudaStream_t>(stream), true,
                        Batch{N, g_img_batch_bytes, coeff_batch_bytes});
}

DWT2_EXPORT int dwt2_inverse_adjoint_batch(const void* g_img, int64_t g_img_pitch_bytes,
                                           int64_t g_img_batch_bytes, int N, int H, int W,
                                           int img_dtype, void* g_coeffs, int64_t coeff_batch_bytes,
                                           void* workspace, size_t ws_bytes, int wavelet,
                                           int levels, int band_dtype, void* stream) {
    return forward_impl(g_img, g_img_pitch_bytes, H, W, img_dtype, g_coeffs, workspace, ws_bytes,
                        wavelet, levels, band_dtype, DWT2_SCHEME_NONSEP,
                        static_cast<cudaStream_t>(stream), true,
                        Batch{N, g_img_batch_bytes, coeff_batch_bytes});
}
