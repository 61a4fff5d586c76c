// dwt2_stream.cuh -- the per-level kernels: a producer warp streams quad rows of the input into
// a ring of shared-memory stages (TMA 2-D tiles, or plain loads for unaligned inputs); four
// consumer warps run the lifting pipeline of dwt2_lifting.cuh in registers and write the
// results with vector stores.  One HBM read of the input and one write of the output per level.
//
// Geometry (all in polyphase quads; a quad is 2 x 2 pixels):
//   CTA   = a strip of cta_q<NW>() output quad columns (NW = 3 or 4 consumer warps x 30 lanes
//           x kQ) x rpc quad rows, plus one producer warp;
//   warp  = a window of 32 x kQ quad columns (kQ adjacent quads per lane); lanes 0 and 31 are halo
//           (they compute but never store: the lifting reaches 2 quads to each side);
//   rows  = the CTA streams its rpc rows plus halo quad rows above and below (one per lifting
//           pair: 1 for the 5/3 wavelets, 2 for the 9/7; the adjoints take 2).
// Boundaries: the producer maps every (extended) row to its whole-sample-symmetric source row;
// warps whose window crosses the left or right image edge read each column from its mirrored
// source column.  The lifting then runs on the symmetric extension with no boundary rule.
#pragma once

#include <algorithm>

#include "dwt2_lifting.cuh"

namespace dwt2 {

constexpr int kHQ = kQ;                  // halo quads on each side of a warp window (one lane)
constexpr int kWarpQ = 32 * kQ;          // quads in a warp window
constexpr int kWarpOut = kWarpQ - 2 * kHQ;  // output quads per warp (30 lanes)
// Consumer warps per CTA: 4 (a 240-quad strip, 5 warps with the producer) or 3 (a 180-quad strip,
// 4 warps).  At 80 registers an SM holds 24 warps: four 5-warp CTAs (16 consumer warps) or six
// 4-warp CTAs (18).  The wide CTA is faster on planes it divides well (8192^2 9/7 forward 1.5%,
// inverse 5%, int 5/3 forward 3% on GB300); the narrow one where the wide strips leave warps
// idle: a 1024-pixel row is 512 quads, 2 strips of 240 and one of 32 (9 of 12 warp windows
// busy) but 3 strips of 180 (9 of 9), and the batched 3-level transforms of 192 such images ran
// 21% faster with it (pick_nw chooses per launch).  The stage rows are sized for the wide CTA.
constexpr int kMaxNW = 4;
// Halo quads on each side of a warp window: the reach of one level.  The CDF wavelets and the
// Deslauriers-Dubuc 9/7 reach two quads each way (9/7: the four-tap predict m-1 .. m+2, then the
// two-tap update m-1, m), one halo lane; the 13/7's four-tap update (m-2 .. m+1) makes three, so
// its windows keep two halo lanes on each side (56 output quads per warp instead of 60).
template <int WV>
constexpr int halo_q() {
    return WV == WV_DD137 ? 2 * kQ : kHQ;
}
template <int WV>
constexpr int warp_out() {  // output quads per warp
    return kWarpQ - 2 * halo_q<WV>();
}
template <int NW, int WV = WV_CDF97>
constexpr int cta_q() {  // output quads per CTA strip
    return NW * warp_out<WV>();
}
template <int NW>
constexpr int cta_threads() {
    return 32 * (NW + 1);
}
constexpr int kMaxCtaQ = cta_q<kMaxNW>();
// Resident CTAs per SM the kernels are compiled for.  Measured on GB300: holding the cheap
// wavelets (integer and float CDF 5/3) to 64 registers for 6 CTAs per SM was 7% faster with an
// 8-stage ring (their 12-stage ring now holds them to 4 CTAs per SM by shared memory, which is
// faster still).  The CDF 9/7 kernels are left free (78-80 registers, 4 CTAs per SM): bound to
// 5 CTAs per SM (72 registers, no spills) the forward measured 6% and the inverse 9% slower.
// The Deslauriers-Dubuc 13/7 kernels are bound to 4 CTAs per SM (96 registers, no spills; 108
// and 3 CTAs per SM unbound): together with the unrolled row loop below its 8192^2 forward took
// 190 -> 172 us and its inverse 191 -> 169 us on GB300.
template <int WV, int NW>
constexpr int min_ctas() {  // the 5/3 kernels at 64 registers (6 wide or 8 narrow CTAs per SM)
    return (WV == WV_CDF97 || WV == WV_DD97) ? 1 : WV == WV_DD137 ? 4 : (NW == 3 ? 8 : 6);
}
// Consumer row loop unrolled by 2 for the 5/3 wavelets: the compiler then renames the row
// pipeline's registers instead of rotating them (int 5/3 forward 4.7% faster on GB300).  The 9/7
// kernels stay rolled: unrolled they measured 2% slower, and a hand-written loop over row pairs
// executed 19% more instructions (ALU and uniform-pipe work for the pair bookkeeping).
// The Deslauriers-Dubuc kernels are unrolled by 2 as well (their three-row windows rotate more
// registers per row; the 9/7 DD inverse took 148.5 -> 142.3 us with it).
template <int WV>
constexpr int row_unroll() {
    return WV == WV_CDF97 ? 1 : 2;
}
// Ring depth (quad rows in flight per CTA) per wavelet and data flow, from same-box A/B runs
// at 8192^2 over depths 6, 8 and 12: the 5/3 kernels are 2-3% faster with 12 (shared memory
// then holds them to 4 CTAs per SM, which still beats 6 CTAs with 8 stages), the 9/7 forward is
// 0.9% faster with 6 than with 8 (4, 5 and 7 are no better), and the 9/7 inverse is fastest
// with 8.
template <int WV>
constexpr int fwd_stages() {
    return WV == WV_CDF97 ? 6 : is_dd(WV) ? 8 : 12;
}
template <int WV>
constexpr int inv_stages() {
    return (WV == WV_CDF97 || is_dd(WV)) ? 8 : 12;
}
constexpr int kVHalo = 2;                // halo quad rows above and below a CTA's rows (adjoints)

// Halo quad rows above and below a CTA's rows.  A level's output quad row n depends on its input
// quad rows n - kLag .. n + kLag (the reach of kLag lifting pairs along the columns: 1 for the
// 5/3 wavelets, 2 for the 9/7), and its pipeline returns row n when row n + kLag is pushed, so
// the forward and inverse levels load exactly kLag halo rows on each side.  The adjoint levels
// keep kVHalo.
template <typename Pipe, bool kAdjoint>
constexpr int vhalo() {
    return kAdjoint ? kVHalo : Pipe::kLag;
}

// Forward: a stage holds 2 pixel rows of the strip's pixel columns [2*qx0 - kXL, +kSRow), loaded
// as 256-wide boxes (every TMA destination starts on a 128-byte boundary).
constexpr int kXL = 8;
constexpr int kBoxW = 256;
constexpr int kBoxes = (kXL + 2 * kMaxCtaQ + 2 * kHQ + kBoxW - 1) / kBoxW;
constexpr int kSRow = kBoxes * kBoxW;
// Inverse: a stage holds one row of each band, quad columns [qx0 - kXLB, +kBRow).
constexpr int kXLB = 8;
constexpr int kBBoxes = (kXLB + kMaxCtaQ + kHQ + kBoxW - 1) / kBoxW;
constexpr int kBRow = kBBoxes * kBoxW;
static_assert(kSRow >= kXL + 2 * kMaxCtaQ + 2 * kHQ, "forward stage row too short");
static_assert(kBRow >= kXLB + kMaxCtaQ + kHQ, "inverse stage row too short");

// A TMA copy must start on a 16-byte boundary in x.  The forward loads x = 2 qx0 - kXL + kBoxW b
// input elements, the inverse x = qx0 - kXLB + kBoxW b band elements, qx0 a multiple of the CTA
// strip: every term must be a multiple of 16 bytes.  The narrow strip (180 quads) fails this for
// 16-bit bands in the inverse (odd strips would start 8 bytes off), so those keep the wide CTA.
template <int NW, typename T, int WV = WV_CDF97>
constexpr bool fwd_tma_x_aligned() {
    return (2 * cta_q<NW, WV>() * sizeof(T)) % 16 == 0 && (kXL * sizeof(T)) % 16 == 0 &&
           (kBoxW * sizeof(T)) % 16 == 0 && 2 * halo_q<WV>() <= kXL;
}
template <int NW, typename T, int WV = WV_CDF97>
constexpr bool inv_tma_x_aligned() {
    return (cta_q<NW, WV>() * sizeof(T)) % 16 == 0 && (kXLB * sizeof(T)) % 16 == 0 &&
           (kBoxW * sizeof(T)) % 16 == 0 && halo_q<WV>() <= kXLB;
}
// The narrowest CTA whose inverse band loads stay aligned: band type TB, LL type TL.
template <typename TB, typename TL>
constexpr int inv_narrow_nw() {
    return inv_tma_x_aligned<3, TB>() && inv_tma_x_aligned<3, TL>() ? 3 : kMaxNW;
}

// A plane (or a batch of equally shaped planes): image z, row r starts at
// ptr + z * bstride + r * pitch (bytes).
struct PlaneOut {
    void* ptr;
    int64_t pitch;
    int64_t bstride;
};

// DC level shift of the float transforms.  The lifting intermediates of CDF 9/7 reach several
// times the signal level (the first predict leaves d = (1 + 2 alpha) x ~ -2.2 x on smooth
// content, its 2-D HH term (1 + 2 alpha)^2 x ~ 4.7 x), and fp32 rounds them at that magnitude.
// A transform of x - c with c added back to LL_J computes the same coefficients in exact
// arithmetic (LL has DC gain 1, the high-pass bands vanish on a constant), but its intermediates
// scale with |x - c|: on [0, 255] content about three times smaller errors.  c is one number per
// image, sampled from the data so that every tile, launch shape and entry point (single image,
// uniform batch, plan) uses the same value: the median of a 3 x 3 grid of samples of the source
// plane (the image for the forward, LL_J for the inverse; non-finite samples count as 0), rounded
// to an integer.  The median of 9 ignores up to 4 outlying samples.
enum ShiftType { SHIFT_F32 = 1, SHIFT_BF16 = 2, SHIFT_F16 = 3 };  // the C ABI's dtype codes
struct ShiftSrc {
    const void* ptr;  // plane the shift is sampled from; nullptr: no shift
    int64_t pitch;    // bytes
    int64_t bstride;  // bytes between the images of a batch
    int h, w;
    int dt;           // ShiftType
    int mode;         // bit 0: subtract c from the level's input; bit 1: add c to its output
};
constexpr int kShiftIn = 1;
constexpr int kShiftOut = 2;

struct FwdArgs {
    const void* in;     // input plane (used by the plain-load path)
    int64_t in_pitch;   // bytes
    int64_t in_bstride; // bytes between the images of a batch
    int H, W;           // input plane size in pixels
    int ner, ndr, nec, ndc;  // even/odd row and column counts = band sizes
    PlaneOut ll, hl, lh, hh;  // band planes (ll is the interleaved output plane in MODE_ROWS)
    int rpc;            // output quad rows per CTA
    int* status;        // workspace status word
    Scale4 scale;       // MODE_ADJ_INV: the reciprocal band scales applied last
    int tma;            // 1: load the input plane with TMA (16-byte aligned base and pitch)
    int nbatch;         // images in the batch (grid z)
    ShiftSrc shift;     // DC level shift: kShiftIn at level 1, kShiftOut (onto LL) at level J
    int ll_keep;        // 1: store LL evict_last (the next level reads it back from L2)
    int in_kept;        // 1: the input was stored evict_last; read it back with evict_normal
};

struct InvArgs {
    const void* band[4];  // LL, HL, LH, HH (used by the plain-load path)
    int64_t band_pitch[4];
    int64_t band_bstride[4];
    int H, W;             // output plane size in pixels
    int ner, ndr, nec, ndc;
    PlaneOut out;         // output plane
    int out_vec;          // output rows may use 4-element vector stores
    int rpc;
    int* status;
    Scale4 scale;         // adjoint: the band scales applied first
    int tma;              // 1: load the band planes with TMA
    int nbatch;           // images in the batch (grid z)
    ShiftSrc shift;       // DC level shift: kShiftIn (from LL) at level J, kShiftOut at level 1
    int out_keep;         // 1: store the output (the next level's LL) evict_last
    int ll_kept;          // 1: LL was stored evict_last; read it back with evict_normal
};

// The level shift c of image z (0 when none): see ShiftSrc.
__device__ __forceinline__ float shift_sample(const char* row, int c, int dt) {
    float v;
    if (dt == SHIFT_BF16) v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[c]);
    else if (dt == SHIFT_F16) v = __half2float(reinterpret_cast<const __half*>(row)[c]);
    else v = reinterpret_cast<const float*>(row)[c];
    return isfinite(v) ? v : 0.f;
}
__device__ __forceinline__ float level_shift(const ShiftSrc& s, int z) {
    if (s.ptr == nullptr || s.mode == 0 || s.h < 1 || s.w < 1) return 0.f;
    const char* base = static_cast<const char*>(s.ptr) + int64_t(z) * s.bstride;
    float v[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const char* row = base + (int64_t(2 * i + 1) * s.h / 6) * s.pitch;
#pragma unroll
        for (int j = 0; j < 3; ++j)
            v[3 * i + j] = shift_sample(row, int(int64_t(2 * j + 1) * s.w / 6), s.dt);
    }
    // the 5th smallest: a partial selection sort
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i + 1; j < 9; ++j) {
            const float lo = fminf(v[i], v[j]), hi = fmaxf(v[i], v[j]);
            v[i] = lo;
            v[j] = hi;
        }
    return rintf(v[4]);
}

// The values a level adds to its input (-c at the first level, else +0) and to its output
// (+c at the last level, else -0).  x + 0 with the sign that leaves every x unchanged, -0
// included, so an unshifted level computes exactly what it would without the shift.
struct LevelShift {
    float in_add, out_add;
    __device__ __forceinline__ void init(const ShiftSrc& s, int z) {
        const float c = level_shift(s, z);
        in_add = (s.mode & kShiftIn) && c != 0.f ? -c : -0.f;
        out_add = (s.mode & kShiftOut) && c != 0.f ? c : -0.f;
    }
};

template <typename T>
__device__ __forceinline__ T* row_ptr(const PlaneOut& p, int r, int z) {
    return reinterpret_cast<T*>(static_cast<char*>(p.ptr) + int64_t(z) * p.bstride +
                                static_cast<int64_t>(r) * p.pitch);
}

// Stores N consecutive values of an output row starting at column c0 (an aligned vector store
// when allowed and wholly inside the row, else element by element, clipped at the width).
template <int N, typename T, typename C>
__device__ __forceinline__ void putN(T* p, const C (&v)[N], int c0, int width, bool vec) {
    if (vec && c0 + N - 1 < width) {
        stN<N>(p, v);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (c0 + k >= 0 && c0 + k < width) p[k] = from_c<T>(v[k]);
    }
}

// putN with an L2 eviction policy on the vector stores (the clipped edge stores are plain).
template <int N, typename T, typename C>
__device__ __forceinline__ void putN_hint(T* p, const C (&v)[N], int c0, int width, bool vec,
                                          uint64_t pol) {
    static_assert(N == 2 || N == 4, "vector width");
    if (vec && c0 + N - 1 < width) {
        if constexpr (N == 2) st2_hint(p, v[0], v[1], pol);
        else st4_hint(p, v[0], v[1], v[2], v[3], pol);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (c0 + k >= 0 && c0 + k < width) p[k] = from_c<T>(v[k]);
    }
}

// Bytes of dynamic shared memory of the kernels with NS ring stages (+128 to align the base to
// 128 bytes).
template <typename TI, int NS>
constexpr size_t fwd_smem_bytes() {
    return size_t(NS) * 2 * kSRow * sizeof(TI) + 2 * NS * sizeof(uint64_t) + 4 * (2 * NS + 4) +
           128;
}
template <typename TL, typename TB, int NS>
constexpr size_t inv_smem_bytes() {
    return size_t(NS) * kBRow * (sizeof(TL) + 3 * sizeof(TB)) + 2 * NS * sizeof(uint64_t) +
           4 * (2 * NS + 4) + 128;
}

__device__ __forceinline__ uint8_t* align128(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

// =============================================================================================
// Per-row machinery shared by the single-image kernels (one CTA = one tile) and the persistent
// batched kernels (one CTA = many tiles).
//
// Stage protocol: the full barrier of a stage takes one arrival (the producer's lane 0, with the
// TMA transaction count when the stage is filled by TMA); the empty barrier takes one arrival
// per consumer warp.
// =============================================================================================

// Plain-load producer for planes TMA cannot address (pitch or base not 16-byte aligned).  Only
// the caller's own image takes this path (every scratch plane is TMA-eligible), so nothing the
// running kernel writes is read here.
//   transform (mirrored rows): each row is copied as the 16-byte-aligned chunks that hold its
//     elements xs .. xs + kSRow - 1 -- in one bulk copy per row issued by lane 0 (kBulk), or as
//     16-byte cp.async chunks spread over the lanes -- so the row lands shifted by the
//     misalignment m (0 .. 16 / sizeof(TI) - 1 elements) of element xs: element c sits at stage
//     index c - xs + m.  The copied chunks are those holding at least one element of the row: a
//     chunk that straddles an end of the row reads at most 15 bytes beyond it, inside the same
//     16-byte block (so inside mapped memory); those stage entries are never read (the
//     consumers read mirrored columns at the plane's edges).  Like a TMA load, a bulk copy
//     completes on the stage's full barrier with its byte count; cp.async chunks arrive on it
//     when they land.  The shifts go to *shift_slot (row 0 in bits 0-3, row 1 in bits 4-7).
//   adjoint (zeros outside the plane): 4-byte zero-filling cp.async copies (16-bit elements, below
//     cp.async's minimum, are loaded before the first shared-memory store), no shift.
// Either way the stage's full barrier completes when the copies have landed, so every stage of
// the ring can be in flight, as with TMA.  kUnroll: 1 in the single-image kernels (their TMA path
// keeps its instruction footprint), full in the persistent kernels.
template <typename TI, int kUnroll, bool kBulk>
__device__ __forceinline__ void fwd_produce_plain(const FwdArgs& a, bool adj, int r0, int r1,
                                                  int xs, TI* dst, uint64_t* full, int lane, int z,
                                                  volatile int* shift_slot) {
    const bool ok0 = r0 >= 0 && r0 < a.H, ok1 = r1 >= 0 && r1 < a.H;
    const char* base = static_cast<const char*>(a.in) + int64_t(z) * a.in_bstride;
    const TI* row0 = reinterpret_cast<const TI*>(base + int64_t(ok0 ? r0 : 0) * a.in_pitch);
    const TI* row1 = reinterpret_cast<const TI*>(base + int64_t(ok1 ? r1 : 0) * a.in_pitch);
    constexpr int kPer = kSRow / 32;
    if (!adj && !kBulk) {
        constexpr int kEpc = 16 / int(sizeof(TI));  // elements per chunk
        constexpr int kChunks = kSRow / kEpc;
        int sh = 0;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const TI* row = r ? row1 : row0;
            const uintptr_t first =
                reinterpret_cast<uintptr_t>(row) + intptr_t(xs) * intptr_t(sizeof(TI));
            const int m = int((first & 15u) / sizeof(TI));
            const int e0 = xs - m;  // element at the first chunk's (aligned) address
#pragma unroll kUnroll
            for (int k = lane; k < kChunks; k += 32) {
                const int c0 = e0 + k * kEpc;
                if (c0 + kEpc > 0 && c0 < a.W) cp_async_16(dst + r * kSRow + k * kEpc, row + c0);
            }
            sh |= m << (4 * r);
        }
        cp_async_arrive(full);
        if (lane == 0) *shift_slot = sh;
    } else if (!adj) {
        if (lane == 0) {
            constexpr int kEpc = 16 / int(sizeof(TI));  // elements per chunk
            constexpr int kChunks = kSRow / kEpc;
            const char* src[2];
            uint32_t bytes[2], dofs[2];
            int sh = 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const TI* row = r ? row1 : row0;
                const uintptr_t first =
                    reinterpret_cast<uintptr_t>(row) + intptr_t(xs) * intptr_t(sizeof(TI));
                const int m = int((first & 15u) / sizeof(TI));
                const int e0 = xs - m;  // element at the first chunk's (aligned) address
                // chunks k of the stage row hold elements e0 + k kEpc ..; those with an element
                // of the row are k_lo .. k_hi - 1
                const int k_lo = e0 >= 0 ? 0 : (-e0) / kEpc;
                const int k_hi = min(kChunks, (a.W - e0 + kEpc - 1) / kEpc);
                bytes[r] = k_hi > k_lo ? uint32_t(16 * (k_hi - k_lo)) : 0u;
                src[r] = reinterpret_cast<const char*>(first & ~uintptr_t(15)) + 16 * k_lo;
                dofs[r] = uint32_t(r * kSRow * int(sizeof(TI)) + 16 * k_lo);
                sh |= m << (4 * r);
            }
            *shift_slot = sh;
            mbar_arrive_expect_tx(full, bytes[0] + bytes[1]);
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (bytes[r]) bulk_copy_g2s(reinterpret_cast<char*>(dst) + dofs[r], src[r], bytes[r], full);
        }
        return;
    } else if constexpr (sizeof(TI) == 4) {
#pragma unroll kUnroll
        for (int j = 0; j < kPer; ++j) {
            const int k = lane + 32 * j, c = xs + k;
            const bool in = c >= 0 && c < a.W;
            cp_async_4(dst + k, row0 + (in ? c : 0), in && ok0);
            cp_async_4(dst + kSRow + k, row1 + (in ? c : 0), in && ok1);
        }
        cp_async_arrive(full);
        if (lane == 0) *shift_slot = 0;
    } else {
        TI v0[kPer], v1[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int c = xs + lane + 32 * j;
            const bool in = c >= 0 && c < a.W;
            v0[j] = (in && ok0) ? ldcg(row0 + c) : zero_of<TI>();
            v1[j] = (in && ok1) ? ldcg(row1 + c) : zero_of<TI>();
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            dst[lane + 32 * j] = v0[j];
            dst[kSRow + lane + 32 * j] = v1[j];
        }
        if (lane == 0) *shift_slot = 0;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(full);
}

// Which loader a kernel instantiation contains: decided per launch from a.tma (persistent
// kernels, whose units mix aligned and unaligned planes), or fixed at compile time (single-image
// kernels: the launcher picks the TMA or the plain-load instantiation, so the TMA kernels carry no
// plain-load code).
enum Loader { LOAD_RUNTIME = 0, LOAD_TMA = 1, LOAD_PLAIN = 2 };

// Forward data flow: loads of extended quad row q (pixel rows 2q, 2q + 1) of the input plane.
// Mirrored (whole-sample symmetric) rows for the transform; plain rows, zeros outside, for the
// adjoint of the inverse.
template <typename TI, int kUnrollPlain = 1, int kLoader = LOAD_RUNTIME, bool kBulk = true>
__device__ __forceinline__ void fwd_produce_row(const FwdArgs& a, const CUtensorMap* tm, bool adj,
                                                int q, int xs, TI* dst, uint64_t* full, int lane,
                                                int z, volatile int* shift_slot,
                                                const uint64_t* l2_pol = nullptr) {
    const int r0 = adj ? 2 * q : refl(2 * q, a.H);
    const int r1 = adj ? 2 * q + 1 : refl(2 * q + 1, a.H);
    const bool use_tma = kLoader == LOAD_TMA || (kLoader == LOAD_RUNTIME && a.tma);
    if (kLoader != LOAD_PLAIN && use_tma) {
        if (lane == 0) {
            mbar_arrive_expect_tx(full, 2 * kSRow * sizeof(TI));
#pragma unroll
            for (int b = 0; b < kBoxes; ++b) {
                if (l2_pol) {
                    tma_load_3d_hint(dst + b * kBoxW, tm, full, xs + b * kBoxW, r0, z, *l2_pol);
                    tma_load_3d_hint(dst + kSRow + b * kBoxW, tm, full, xs + b * kBoxW, r1, z,
                                     *l2_pol);
                } else {
                    tma_load_3d(dst + b * kBoxW, tm, full, xs + b * kBoxW, r0, z);
                    tma_load_3d(dst + kSRow + b * kBoxW, tm, full, xs + b * kBoxW, r1, z);
                }
            }
        }
    } else if constexpr (kLoader != LOAD_TMA) {
        fwd_produce_plain<TI, kUnrollPlain, kBulk>(a, adj, r0, r1, xs, dst, full, lane, z,
                                                   shift_slot);
    }
}

// Stage offsets of a lane's 2*kQ pixel columns: consecutive (col0 - xs ...) inside the plane;
// at the left / right edge each column's whole-sample-symmetric source, clamped to the stage.
// Computed once per tile (the reflection needs a modulo).
struct FwdCols {
    bool edge;
    int base;          // col0 - xs (fast path)
    int ec[2 * kQ];    // edge path
    __device__ __forceinline__ void init(int col0, int xs, int W, bool mirror, bool at_edge) {
        edge = mirror && at_edge;
        base = col0 - xs;
#pragma unroll
        for (int k = 0; k < 2 * kQ; ++k)
            ec[k] = edge ? min(max(refl(col0 + k, W) - xs, 0), kSRow - 1) : base + k;
    }
};

// A lane's kQ quads of one stage (pixel rows 2q, 2q + 1).
template <typename TI, typename C>
__device__ __forceinline__ void fwd_lane_row(const TI* stage, const FwdCols& cols, QRow<C>& row) {
    const TI* r0 = stage;
    const TI* r1 = stage + kSRow;
    C v0[2 * kQ], v1[2 * kQ];
    if (!cols.edge) {
        ldN<2 * kQ>(r0 + cols.base, v0);
        ldN<2 * kQ>(r1 + cols.base, v1);
    } else {
#pragma unroll
        for (int k = 0; k < 2 * kQ; ++k) {
            v0[k] = to_c(r0[cols.ec[k]]);
            v1[k] = to_c(r1[cols.ec[k]]);
        }
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        row.a[q] = v0[2 * q];
        row.b[q] = v0[2 * q + 1];
        row.c[q] = v1[2 * q];
        row.e[q] = v1[2 * q + 1];
    }
}

// Four consecutive 4-byte elements starting sh (0..3) past the 16-byte-aligned p: two aligned
// vector loads and a selection (sh is the same across the warp).
template <typename TI, typename C>
__device__ __forceinline__ void ld4_shifted(const TI* p, int sh, C (&v)[4]) {
    C x[4], y[4];
    ld4(p, x);
    ld4(p + 4, y);
    switch (sh) {
    case 0: v[0] = x[0]; v[1] = x[1]; v[2] = x[2]; v[3] = x[3]; break;
    case 1: v[0] = x[1]; v[1] = x[2]; v[2] = x[3]; v[3] = y[0]; break;
    case 2: v[0] = x[2]; v[1] = x[3]; v[2] = y[0]; v[3] = y[1]; break;
    default: v[0] = x[3]; v[1] = y[0]; v[2] = y[1]; v[3] = y[2]; break;
    }
}

// The same from a stage filled by the plain-load path: row r of the stage is shifted by
// (shifts >> 4r) & 15 elements.  Lanes inside the plane read 4-byte elements with aligned vector
// loads; lanes at an edge (and 16-bit elements) read elementwise, kept inside the stage.
template <typename TI, typename C, bool kVec = true>
__device__ __forceinline__ void fwd_lane_row_shifted(const TI* stage, const FwdCols& cols,
                                                     QRow<C>& row, int shifts) {
    const int s0 = shifts & 15, s1 = (shifts >> 4) & 15;
    C v0[2 * kQ], v1[2 * kQ];
    if (kVec && sizeof(TI) == 4 && 2 * kQ == 4 && !cols.edge) {
        ld4_shifted(stage + cols.base, s0, v0);
        ld4_shifted(stage + kSRow + cols.base, s1, v1);
    } else {
#pragma unroll
        for (int k = 0; k < 2 * kQ; ++k) {
            const int i = cols.edge ? cols.ec[k] : cols.base + k;
            v0[k] = to_c(stage[min(i + s0, kSRow - 1)]);
            v1[k] = to_c(stage[kSRow + min(i + s1, kSRow - 1)]);
        }
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        row.a[q] = v0[2 * q];
        row.b[q] = v0[2 * q + 1];
        row.c[q] = v1[2 * q];
        row.e[q] = v1[2 * q + 1];
    }
}

// Separable convolution (Eq. 4): stage offsets of the 11 pixel columns 2 m0 - 4 .. 2 m0 + 6 a
// lane's two quads filter over; at the plane's edges each column's whole-sample-symmetric
// source.  Computed once per tile.
struct ConvCols {
    static constexpr int kN = 11;
    bool edge;
    int base;
    int idx[kN];
    __device__ __forceinline__ void init(int col0, int xs, int W, bool at_edge) {
        edge = at_edge;
        base = col0 - 4 - xs;
#pragma unroll
        for (int j = 0; j < kN; ++j)
            idx[j] = edge ? min(max(refl(col0 - 4 + j, W) - xs, 0), kSRow - 1) : base + j;
    }
};

// N^H on one stage: the low / high analysis filters along both pixel rows, at the lane's two
// quads (row r shifted by (shifts >> 4r) & 15 elements, as the plain-load path fills it).
template <int WV, typename TI>
__device__ __forceinline__ void conv_lane_row(const TI* stage, const ConvCols& cols, int shifts,
                                              QRow<float>& row) {
    constexpr ConvTaps<WV> T = conv_taps<WV>();
    constexpr int kL = ConvTaps<WV>::kL, kH = ConvTaps<WV>::kH;
    const int s0 = shifts & 15, s1 = (shifts >> 4) & 15;
    float x0[ConvCols::kN], x1[ConvCols::kN];
#pragma unroll
    for (int j = 0; j < ConvCols::kN; ++j) {
        x0[j] = to_c(stage[min(cols.idx[j] + s0, kSRow - 1)]);
        x1[j] = to_c(stage[kSRow + min(cols.idx[j] + s1, kSRow - 1)]);
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int c = 4 + 2 * q;  // the quad's even column in x0 / x1
        float l0 = 0.f, l1 = 0.f, h0 = 0.f, h1 = 0.f;
#pragma unroll
        for (int t = -kL; t <= kL; ++t) {
            l0 = fmaf(T.lo[t + kL], x0[c + t], l0);
            l1 = fmaf(T.lo[t + kL], x1[c + t], l1);
        }
#pragma unroll
        for (int t = -kH; t <= kH; ++t) {
            h0 = fmaf(T.hi[t + kH], x0[c + 1 + t], h0);
            h1 = fmaf(T.hi[t + kH], x1[c + 1 + t], h1);
        }
        row.a[q] = l0;
        row.b[q] = h0;
        row.c[q] = l1;
        row.e[q] = h1;
    }
}

// The row pass of the two-pass comparator (MODE_ROWS): stores quad row qo as two interleaved
// pixel rows (the band-plane modes store through fwd_store_bands).
template <typename TL, typename C>
__device__ __forceinline__ void fwd_store_interleaved(const FwdArgs& a, const QRow<C>& row, int qo,
                                                      int m0, int z) {
    const int col0 = 2 * m0;
    C va[2 * kQ], vc[2 * kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        va[2 * q] = row.a[q];
        va[2 * q + 1] = row.b[q];
        vc[2 * q] = row.c[q];
        vc[2 * q + 1] = row.e[q];
    }
    putN<2 * kQ>(row_ptr<TL>(a.ll, 2 * qo, z) + col0, va, col0, a.W, true);
    if (2 * qo + 1 < a.H) putN<2 * kQ>(row_ptr<TL>(a.ll, 2 * qo + 1, z) + col0, vc, col0, a.W, true);
}

// A lane's output positions (column m0) in the four band planes, at one quad row; advanced a
// row at a time, so the per-row addresses cost one add per band instead of a multiply.
struct BandRows {
    char* p[4];  // LL, HL, LH, HH
    template <typename TB, typename TL>
    __device__ __forceinline__ void init(const FwdArgs& a, int q, int m0, int z) {
        p[0] = reinterpret_cast<char*>(row_ptr<TL>(a.ll, q, z) + m0);
        p[1] = reinterpret_cast<char*>(row_ptr<TB>(a.hl, q, z) + m0);
        p[2] = reinterpret_cast<char*>(row_ptr<TB>(a.lh, q, z) + m0);
        p[3] = reinterpret_cast<char*>(row_ptr<TB>(a.hh, q, z) + m0);
    }
    __device__ __forceinline__ void next(const FwdArgs& a) {
        p[0] += a.ll.pitch;
        p[1] += a.hl.pitch;
        p[2] += a.lh.pitch;
        p[3] += a.hh.pitch;
    }
};

// The four band rows of finished quad row qo at the positions br holds.
template <typename TB, typename TL, typename C>
__device__ __forceinline__ void fwd_store_bands(const FwdArgs& a, const BandRows& br,
                                                const QRow<C>& row, int qo, int m0) {
    putN<kQ>(reinterpret_cast<TL*>(br.p[0]), row.a, m0, a.nec, true);
    putN<kQ>(reinterpret_cast<TB*>(br.p[1]), row.b, m0, a.ndc, true);
    if (qo < a.ndr) {
        putN<kQ>(reinterpret_cast<TB*>(br.p[2]), row.c, m0, a.nec, true);
        putN<kQ>(reinterpret_cast<TB*>(br.p[3]), row.e, m0, a.ndc, true);
    }
}

// fwd_store_bands with the LL row stored under the L2 policy ll_pol (evict_last when the next
// level reads LL back from L2, else evict_normal).
template <typename TB, typename TL, typename C>
__device__ __forceinline__ void fwd_store_bands_ll(const FwdArgs& a, const BandRows& br,
                                                   const QRow<C>& row, int qo, int m0,
                                                   uint64_t ll_pol) {
    putN_hint<kQ>(reinterpret_cast<TL*>(br.p[0]), row.a, m0, a.nec, true, ll_pol);
    putN<kQ>(reinterpret_cast<TB*>(br.p[1]), row.b, m0, a.ndc, true);
    if (qo < a.ndr) {
        putN<kQ>(reinterpret_cast<TB*>(br.p[2]), row.c, m0, a.nec, true);
        putN<kQ>(reinterpret_cast<TB*>(br.p[3]), row.e, m0, a.ndc, true);
    }
}

// Inverse data flow: band rows of extended quad row q.  Even pixel row 2q -> LL / HL row, odd
// pixel row 2q + 1 -> LH / HH row (mirrored; plain rows with zeros outside for the adjoint).
// tm[k] points to the tensor map of band k (LL, HL, LH, HH) in parameter or global memory.
template <typename TL, typename TB>
__device__ __forceinline__ void inv_produce_row(const InvArgs& a, const CUtensorMap* const* tm,
                                                bool adj, int q, int xb, uint8_t* stage,
                                                uint64_t* full, int lane, int z,
                                                const uint64_t* ll_pol = nullptr) {
    constexpr size_t kStageBytes = size_t(kBRow) * (sizeof(TL) + 3 * sizeof(TB));
    TL* sll = reinterpret_cast<TL*>(stage);
    TB* sb = reinterpret_cast<TB*>(stage + kBRow * sizeof(TL));
    const int re = adj ? q : refl(2 * q, a.H) >> 1;
    const int ro = adj ? q : (a.H > 1 ? (refl(2 * q + 1, a.H) - 1) >> 1 : -1);
    if (a.tma) {
        if (lane == 0) {
            mbar_arrive_expect_tx(full, uint32_t(kStageBytes));
#pragma unroll
            for (int b = 0; b < kBBoxes; ++b) {
                const int x = xb + b * kBoxW;
                if (ll_pol) tma_load_3d_hint(sll + b * kBoxW, tm[0], full, x, re, z, *ll_pol);
                else tma_load_3d(sll + b * kBoxW, tm[0], full, x, re, z);
                tma_load_3d(sb + b * kBoxW, tm[1], full, x, re, z);
                tma_load_3d(sb + kBRow + b * kBoxW, tm[2], full, x, ro, z);
                tma_load_3d(sb + 2 * kBRow + b * kBoxW, tm[3], full, x, ro, z);
            }
        }
    } else {
        // Plain loads (planes too small or too unaligned for TMA; in a persistent kernel they may
        // have been written by other SMs, hence .cg).  All loads of the stage are issued before
        // the first shared-memory store: one memory latency per stage.
        const int rows[4] = {re, re, ro, ro};
        const int widths[4] = {a.nec, a.ndc, a.nec, a.ndc};
        const int heights[4] = {a.ner, a.ner, a.ndr, a.ndr};
        constexpr int kPer = kBRow / 32;
        const char* src[4];
        bool row_ok[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            row_ok[b] = rows[b] >= 0 && rows[b] < heights[b];
            src[b] = static_cast<const char*>(a.band[b]) + int64_t(z) * a.band_bstride[b] +
                     int64_t(row_ok[b] ? rows[b] : 0) * a.band_pitch[b];
        }
        TL vl[kPer];
        TB vb[3][kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int c = xb + lane + 32 * j;
            vl[j] = (row_ok[0] && c >= 0 && c < widths[0])
                        ? ldcg(reinterpret_cast<const TL*>(src[0]) + c) : zero_of<TL>();
#pragma unroll
            for (int b = 1; b < 4; ++b)
                vb[b - 1][j] = (row_ok[b] && c >= 0 && c < widths[b])
                                   ? ldcg(reinterpret_cast<const TB*>(src[b]) + c) : zero_of<TB>();
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            sll[lane + 32 * j] = vl[j];
#pragma unroll
            for (int b = 0; b < 3; ++b) sb[b * kBRow + lane + 32 * j] = vb[b][j];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(full);
    }
}

// Stage offsets of a lane's kQ quads in the band rows: the quad itself inside the plane; at the
// edges the band column of each pixel column's symmetric source (even pixel column 2m -> LL / LH,
// odd 2m + 1 -> HL / HH; no odd columns in a 1-column plane).  Computed once per tile.
struct InvCols {
    bool edge, odd_zero;
    int base;
    int ie[kQ], io[kQ];
    __device__ __forceinline__ void init(int m0, int xb, int W, bool mirror, bool at_edge) {
        edge = mirror && at_edge;
        odd_zero = W <= 1;
        base = m0 - xb;
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            const int m = m0 + j;
            ie[j] = edge ? min(max((refl(2 * m, W) >> 1) - xb, 0), kBRow - 1) : base + j;
            io[j] = (edge && !odd_zero)
                        ? min(max(((refl(2 * m + 1, W) - 1) >> 1) - xb, 0), kBRow - 1)
                        : base + j;
        }
    }
};

// A lane's kQ quads of the four band rows of one stage.
template <typename TL, typename TB, typename C>
__device__ __forceinline__ void inv_lane_row(const uint8_t* stage, const InvCols& cols,
                                             QRow<C>& row) {
    const TL* sll = reinterpret_cast<const TL*>(stage);
    const TB* shl = reinterpret_cast<const TB*>(stage + kBRow * sizeof(TL));
    const TB* slh = shl + kBRow;
    const TB* shh = shl + 2 * kBRow;
    if (!cols.edge) {
        ldN<kQ>(sll + cols.base, row.a);
        ldN<kQ>(shl + cols.base, row.b);
        ldN<kQ>(slh + cols.base, row.c);
        ldN<kQ>(shh + cols.base, row.e);
    } else {
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            row.a[j] = to_c(sll[cols.ie[j]]);
            row.c[j] = to_c(slh[cols.ie[j]]);
            row.b[j] = cols.odd_zero ? C(0) : C(to_c(shl[cols.io[j]]));
            row.e[j] = cols.odd_zero ? C(0) : C(to_c(shh[cols.io[j]]));
        }
    }
}

// Stores a reconstructed quad row qo as pixel rows 2qo and 2qo + 1 of the output plane; p is the
// lane's position in it (pixel row 2 qo, column 2 m0), kept by the caller and advanced by two
// rows per quad row.
template <typename TO, typename C>
__device__ __forceinline__ void inv_store_rows_at(const InvArgs& a, const QRow<C>& row, int qo,
                                                  int m0, char* p) {
    const int c0 = 2 * m0;
    C va[2 * kQ], vc[2 * kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        va[2 * q] = row.a[q];
        va[2 * q + 1] = row.b[q];
        vc[2 * q] = row.c[q];
        vc[2 * q + 1] = row.e[q];
    }
    putN<2 * kQ>(reinterpret_cast<TO*>(p), va, c0, a.W, a.out_vec != 0);
    if (2 * qo + 1 < a.H)
        putN<2 * kQ>(reinterpret_cast<TO*>(p + a.out.pitch), vc, c0, a.W, a.out_vec != 0);
}

// inv_store_rows_at with the vector stores under the L2 policy pol.
template <typename TO, typename C>
__device__ __forceinline__ void inv_store_rows_at_hint(const InvArgs& a, const QRow<C>& row,
                                                       int qo, int m0, char* p, uint64_t pol) {
    const int c0 = 2 * m0;
    C va[2 * kQ], vc[2 * kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        va[2 * q] = row.a[q];
        va[2 * q + 1] = row.b[q];
        vc[2 * q] = row.c[q];
        vc[2 * q + 1] = row.e[q];
    }
    putN_hint<2 * kQ>(reinterpret_cast<TO*>(p), va, c0, a.W, a.out_vec != 0, pol);
    if (2 * qo + 1 < a.H)
        putN_hint<2 * kQ>(reinterpret_cast<TO*>(p + a.out.pitch), vc, c0, a.W, a.out_vec != 0,
                          pol);
}

// Shared-memory ring: NS stages, then the full / empty barriers, the abort flag and the
// per-stage tile ids (persistent kernels).
template <int NS>
struct Ring {
    static constexpr int kN = NS;
    uint8_t* stage0;
    size_t stage_bytes;
    uint64_t* full;
    uint64_t* empty;
    volatile int* abort;
    volatile int* meta;   // per stage: the ticket of its tile (persistent kernels)
    volatile int* shift;  // per stage: element shifts of its two rows (plain-load path)
    __device__ __forceinline__ uint8_t* stage(int s) const { return stage0 + size_t(s) * stage_bytes; }
};

// A position in a ring of NS stages: the stage and the parity of its current phase, advanced one
// row at a time (no division by the ring depth per row).
template <int NS>
struct RingPos {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next() {
        if (++s == NS) {
            s = 0;
            ph ^= 1u;
        }
    }
};

template <int NS>
__device__ __forceinline__ Ring<NS> make_ring(uint8_t* smem_raw, size_t stage_bytes) {
    Ring<NS> r;
    r.stage0 = align128(smem_raw);
    r.stage_bytes = stage_bytes;
    r.full = reinterpret_cast<uint64_t*>(r.stage0 + NS * stage_bytes);
    r.empty = r.full + NS;
    r.abort = reinterpret_cast<volatile int*>(r.empty + NS);
    r.meta = r.abort + 1;
    r.shift = r.meta + NS;
    return r;
}

// Thread 0 initialises the barriers (the empty barriers take one arrival per consumer warp);
// every thread must call __syncthreads() afterwards.
template <int NW, int NS>
__device__ __forceinline__ void init_ring(const Ring<NS>& r) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&r.full[s], 1);
            mbar_init(&r.empty[s], NW);
        }
        *r.abort = 0;
        fence_barrier_init();
    }
}

// Lets the last TMA copies of a producer land before its CTA exits (bounded).
template <int NS>
__device__ __forceinline__ void drain_ring(const Ring<NS>& r, int issued, int* status) {
    volatile int no_abort = 0;
    for (int i = max(0, issued - NS); i < issued; ++i)
        if (!mbar_wait(&r.full[i % NS], (i / NS) & 1, &no_abort, status)) break;
}

// Wavelets whose streaming levels keep the next level's LL in L2 (evict_last stores, read back
// with evict_normal).  Measured on GB300, 8192^2, 5 levels, same box: the integer 5/3 forward
// 131.5 -> 126.0 us and its inverse 132.7 -> 126.0 us (level 1 and 2 both faster); the 9/7
// forward 140.3 -> 141.3 us and inverse 139.5 -> 145.1 us, and its 192 x 1024^2 batch 10%
// slower: the 9/7 kernels are bound by instruction issue, and the hinted stores cost them more
// than the L2 reads save.  The 9/7 kernels therefore keep plain stores and loads.
__host__ __device__ constexpr bool keeps_ll_in_l2(int wv) {
    return wv == WV_CDF53_INT || wv == WV_CDF53;
}

// Forward levels that take the DC level shift: float lifting (every scheme but the convolution,
// whose only intermediates are the filter outputs) and not the adjoint (a linear map of
// gradients, with no DC to remove).
template <typename C, int MODE>
constexpr bool kShiftable =
    std::is_same<C, float>::value && MODE != MODE_CONV && MODE != MODE_ADJ_INV;

// =============================================================================================
// Single-image kernels: one CTA = one tile (cta_q<NW>() quad columns x rpc quad rows + halo) of one
// level.  MODE_ROWS writes the interleaved plane (the row pass of the two-pass separable
// comparator); MODE_ADJ_INV is the transpose of the inverse level; every other mode is the
// forward level.
// =============================================================================================
template <int WV, int MODE, typename TI, typename TB, typename TL, bool kPlain, bool kShift,
          int NW>
__global__ void __launch_bounds__(cta_threads<NW>(), min_ctas<WV, NW>())
    k_forward(const __grid_constant__ CUtensorMap tmap, const FwdArgs args) {
    constexpr int kNW = NW;
    constexpr int kCtaQ = cta_q<NW, WV>();
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    static_assert(fwd_tma_x_aligned<NW, TI, WV>(), "TMA x coordinates of this CTA width misaligned");
    constexpr bool kAdj = MODE == MODE_ADJ_INV;
    using Pipe = std::conditional_t<kAdj, AdjInvPipe<WV>, FwdPipe<WV, kAdj ? MODE_NONSEP : MODE>>;
    using C = typename Pipe::C;
    constexpr int kVH = vhalo<Pipe, kAdj>();  // 0 for the row pass (MODE_ROWS)
    constexpr int kS = fwd_stages<WV>();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const Ring<kS> ring = make_ring<kS>(smem_raw, size_t(2) * kSRow * sizeof(TI));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.z;  // image of a batch
    const int qx0 = blockIdx.x * kCtaQ;
    const int n0 = blockIdx.y * args.rpc;
    const int n1 = min(n0 + args.rpc, args.ner);
    const int nrows = n1 - n0 + 2 * kVH;
    const int qfirst = n0 - kVH;
    const int xs = 2 * qx0 - kXL;

    init_ring<kNW>(ring);
    if (!kPlain && warp == kNW && lane == 0) prefetch_tensormap(&tmap);
    __syncthreads();
    // Everything above overlaps the previous level's tail; nothing below may touch global memory
    // before that level has finished writing this level's input (and reading what we overwrite).
    grid_dependency_wait();
    allow_dependent_launch();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        const uint64_t in_pol = keeps_ll_in_l2(WV) ? l2_evict_normal() : 0;
        const uint64_t* in_hint = keeps_ll_in_l2(WV) && args.in_kept ? &in_pol : nullptr;
        int issued = 0;
        RingPos<kS> rp;
        for (int i = 0; i < nrows; ++i) {
            const int s = rp.s;
            const uint32_t par = rp.ph;
            rp.next();
            if (i >= kS) {
                bool ok = mbar_wait(&ring.empty[s], par ^ 1u, ring.abort, args.status);
                if (!__all_sync(kFull, ok)) break;
            }
            fwd_produce_row<TI, 1, kPlain ? LOAD_PLAIN : LOAD_TMA>(
                args, &tmap, kAdj, qfirst + i, xs, reinterpret_cast<TI*>(ring.stage(s)),
                &ring.full[s], lane, z, &ring.shift[s], in_hint);
            issued = i + 1;
        }
        if (lane == 0) drain_ring(ring, issued, args.status);
        cp_async_wait_all();  // no-op unless this lane issued cp.async copies
        return;
    }

    // ------------------------------------------------------------------------- consumers
    const int wq = qx0 - kHaloQ + warp * warp_out<WV>();  // first quad of the warp window
    const int m0 = wq + kQ * lane;                         // first quad of this lane
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    FwdCols cols;
    cols.init(2 * m0, xs, args.W, !kAdj, (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W));
    ConvCols ccols;
    if constexpr (MODE == MODE_CONV)
        ccols.init(2 * m0, xs, args.W, (2 * wq - 4 < 0) || (2 * wq + 2 * kWarpQ + 4 > args.W));
    // a warp whose output quads all lie beyond the plane only cycles the barriers
    const bool idle = wq + kHaloQ >= args.nec;
    LaneW hw;
    if constexpr (kAdj) hw.init(m0, AxisLen{args.nec, args.ndc});
    const AxisLen rows{args.ner, args.ndr};

    BandRows bands;
    if constexpr (MODE != MODE_ROWS) bands.init<TB, TL>(args, n0, m0, z);
    uint64_t ll_pol = 0;
    if constexpr (keeps_ll_in_l2(WV))
        ll_pol = args.ll_keep ? l2_evict_last() : l2_evict_normal();
    static_assert(!kShift || kShiftable<C, MODE>, "a level shift on a level that takes none");
    LevelShift sh{-0.f, -0.f};
    if constexpr (kShift) sh.init(args.shift, z);
    Pipe pipe;
    if constexpr (kShift) pipe.init(sh.out_add);
    else pipe.init();
    RingPos<kS> rp;
#pragma unroll row_unroll<WV>()
    for (int i = 0; i < nrows; ++i) {
        const int s = rp.s;
        const uint32_t par = rp.ph;
        rp.next();
        bool ok = mbar_wait(&ring.full[s], par, ring.abort, args.status);
        if (!__all_sync(kFull, ok)) break;
        if (idle) {
            if (lane == 0) mbar_arrive(&ring.empty[s]);
            continue;
        }
        QRow<C> row;
        if constexpr (MODE == MODE_CONV)
            conv_lane_row<WV, TI>(reinterpret_cast<const TI*>(ring.stage(s)), ccols,
                                  kPlain ? int(ring.shift[s]) : 0, row);
        else if constexpr (kPlain)
            fwd_lane_row_shifted<TI, C>(reinterpret_cast<const TI*>(ring.stage(s)), cols, row,
                                        ring.shift[s]);
        else
            fwd_lane_row<TI, C>(reinterpret_cast<const TI*>(ring.stage(s)), cols, row);
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring.empty[s]);
        if constexpr (kShift) add_row(row, sh.in_add);
        if constexpr (kAdj)
            pipe.push(row, qfirst + i, hw, rows, args.scale);
        else
            pipe.push(row);
        const int qo = qfirst + i - Pipe::kLag;
        if constexpr (MODE == MODE_ROWS) {
            if (qo >= n0 && qo < n1 && store_lane) fwd_store_interleaved<TL>(args, row, qo, m0, z);
        } else if (qo >= n0 && qo < n1) {
            if (store_lane) {
                if constexpr (keeps_ll_in_l2(WV))
                    fwd_store_bands_ll<TB, TL>(args, bands, row, qo, m0, ll_pol);
                else
                    fwd_store_bands<TB, TL>(args, bands, row, qo, m0);
            }
            bands.next(args);
        }
    }
}

// =============================================================================================
// Direct forward level for small planes (a few MB, in L2 after the previous level wrote them).
// The streaming kernel's fixed costs -- a producer warp, the stage ring and its barriers, the TMA
// latency of the first rows and the pipeline fill -- dominate there, and every level costs a
// few microseconds whatever its size.  Here each warp is one window (60 output quads, 56 for the
// Deslauriers-Dubuc wavelets) of kDirectRows output quad rows: it loads the kDirectRows + 2 kLag
// input quad rows it needs straight from global memory (L2) into registers, all at once, then
// pushes them through the same FwdPipe and stores through the same band rows as the streaming
// kernel, so the results are the same bits.  The halo rows are loaded and computed again by the
// windows above and below.
// =============================================================================================
constexpr int kDirectRows = 2;     // output quad rows per warp
constexpr int kDirectWarps = 4;    // warps (windows) per CTA
// Largest input (bytes, all images of a launch) a level takes the direct kernel for.
constexpr int64_t kDirectMaxBytes = int64_t(4) << 20;
// Whether a non-separable forward level over n planes of h x w elements of es bytes (an inverse
// level: n output planes of h x w LL elements) takes the direct kernel.
inline bool takes_direct(int h, int w, size_t es, int n) {
    return int64_t(h) * w * int64_t(es) * std::max(1, n) <= kDirectMaxBytes;
}

// refl for the direct kernels, whose rows and columns are mostly inside the plane already.
__device__ __forceinline__ int refl_in(int i, int n) {
    return unsigned(i) < unsigned(n) ? i : refl(i, n);
}

// A lane's 2 kQ pixels of pixel row r of the plane: aligned vector loads where the window lies
// inside the plane, else elementwise from the columns col (mirrored at the edges).
template <typename TI, typename C>
__device__ __forceinline__ void direct_load_row(const char* base, int64_t pitch, int r,
                                                const int (&col)[2 * kQ], bool vec,
                                                C (&v)[2 * kQ]) {
    const TI* row = reinterpret_cast<const TI*>(base + int64_t(r) * pitch);
    if (vec) {
        ldN<2 * kQ>(row + col[0], v);
    } else {
#pragma unroll
        for (int k = 0; k < 2 * kQ; ++k) v[k] = to_c(ldcg(row + col[k]));
    }
}

template <int WV, typename TI, typename TB, typename TL, bool kShift>
__global__ void __launch_bounds__(32 * kDirectWarps) k_forward_direct(const FwdArgs args) {
    using Pipe = FwdPipe<WV, MODE_NONSEP>;
    using C = typename Pipe::C;
    constexpr int kLag = Pipe::kLag;
    constexpr int kRows = kDirectRows + 2 * kLag;  // input quad rows per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.z;
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    // grid x runs over row blocks (a tall plane may have more than 65535 of them), y over strips
    const int wq = (blockIdx.y * kDirectWarps + warp) * warp_out<WV>() - kHaloQ;  // window start
    const int m0 = wq + kQ * lane;
    const int n0 = blockIdx.x * kDirectRows;
    const int n1 = min(n0 + kDirectRows, args.ner);
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    grid_dependency_wait();  // the input plane is the previous level's output
    allow_dependent_launch();
    if (wq + kHaloQ >= args.nec) return;  // a window wholly beyond the plane: no work

    const char* base = static_cast<const char*>(args.in) + int64_t(z) * args.in_bstride;
    const bool edge = (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W);
    const bool vec = !edge && (reinterpret_cast<uintptr_t>(base) % (4 * sizeof(TI))) == 0 &&
                     args.in_pitch % int64_t(4 * sizeof(TI)) == 0;
    int col[2 * kQ];
#pragma unroll
    for (int k = 0; k < 2 * kQ; ++k) col[k] = refl_in(2 * m0 + k, args.W);
    QRow<C> rows[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int q = n0 - kLag + i;
        C v0[2 * kQ], v1[2 * kQ];
        direct_load_row<TI, C>(base, args.in_pitch, refl_in(2 * q, args.H), col, vec, v0);
        direct_load_row<TI, C>(base, args.in_pitch, refl_in(2 * q + 1, args.H), col, vec, v1);
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
            rows[i].a[k] = v0[2 * k];
            rows[i].b[k] = v0[2 * k + 1];
            rows[i].c[k] = v1[2 * k];
            rows[i].e[k] = v1[2 * k + 1];
        }
    }
    LevelShift sh{-0.f, -0.f};
    if constexpr (kShift) sh.init(args.shift, z);
    Pipe pipe;
    if constexpr (kShift) pipe.init(sh.out_add);
    else pipe.init();
    BandRows bands;
    bands.init<TB, TL>(args, n0, m0, z);
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        QRow<C> row = rows[i];
        if constexpr (kShift) add_row(row, sh.in_add);
        pipe.push(row);
        const int qo = n0 - kLag + i - kLag;
        if (i >= 2 * kLag && qo < n1) {
            if (store_lane) fwd_store_bands<TB, TL>(args, bands, row, qo, m0);
            bands.next(args);
        }
    }
}

// Inverse level (ADJ = false) or the transpose of the forward level (ADJ = true): four band
// planes in, the interleaved plane out.
template <int WV, typename TB, typename TL, typename TO, bool ADJ, bool kShift, int NW>
__global__ void __launch_bounds__(cta_threads<NW>(), min_ctas<WV, NW>())
    k_inverse(const __grid_constant__ CUtensorMap tm_ll, const __grid_constant__ CUtensorMap tm_hl,
              const __grid_constant__ CUtensorMap tm_lh, const __grid_constant__ CUtensorMap tm_hh,
              const InvArgs args) {
    constexpr int kNW = NW;
    constexpr int kCtaQ = cta_q<NW, WV>();
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    static_assert(inv_tma_x_aligned<NW, TB, WV>() && inv_tma_x_aligned<NW, TL, WV>(),
                  "TMA x coordinates of this CTA width misaligned");
    using Pipe = std::conditional_t<ADJ, AdjFwdPipe<WV>, typename InvPipeOf<WV, TB>::type>;
    using C = typename Pipe::C;
    constexpr size_t kStageBytes = size_t(kBRow) * (sizeof(TL) + 3 * sizeof(TB));
    constexpr int kS = inv_stages<WV>();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const Ring<kS> ring = make_ring<kS>(smem_raw, kStageBytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.z;  // image of a batch
    const int qx0 = blockIdx.x * kCtaQ;
    const int n0 = blockIdx.y * args.rpc;
    const int n1 = min(n0 + args.rpc, args.ner);
    constexpr int kVH = vhalo<Pipe, ADJ>();
    const int nrows = n1 - n0 + 2 * kVH;
    const int qfirst = n0 - kVH;
    const int xb = qx0 - kXLB;

    init_ring<kNW>(ring);
    if (args.tma && warp == kNW && lane == 0) {
        prefetch_tensormap(&tm_ll);
        prefetch_tensormap(&tm_hl);
        prefetch_tensormap(&tm_lh);
        prefetch_tensormap(&tm_hh);
    }
    __syncthreads();
    grid_dependency_wait();
    allow_dependent_launch();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        // pointers to the __grid_constant__ parameters (TMA reads the maps where they live)
        const CUtensorMap* maps[4] = {&tm_ll, &tm_hl, &tm_lh, &tm_hh};
        const uint64_t ll_pol = keeps_ll_in_l2(WV) ? l2_evict_normal() : 0;
        const uint64_t* ll_hint = keeps_ll_in_l2(WV) && args.ll_kept ? &ll_pol : nullptr;
        int issued = 0;
        RingPos<kS> rp;
        for (int i = 0; i < nrows; ++i) {
            const int s = rp.s;
            const uint32_t par = rp.ph;
            rp.next();
            if (i >= kS) {
                bool ok = mbar_wait(&ring.empty[s], par ^ 1u, ring.abort, args.status);
                if (!__all_sync(kFull, ok)) break;
            }
            inv_produce_row<TL, TB>(args, maps, ADJ, qfirst + i, xb, ring.stage(s), &ring.full[s],
                                    lane, z, ll_hint);
            issued = i + 1;
        }
        if (args.tma && lane == 0) drain_ring(ring, issued, args.status);
        cp_async_wait_all();  // no-op unless this lane issued cp.async copies
        return;
    }

    // ------------------------------------------------------------------------- consumers
    const int wq = qx0 - kHaloQ + warp * warp_out<WV>();
    const int m0 = wq + kQ * lane;
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    InvCols cols;
    cols.init(m0, xb, args.W, !ADJ, (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W));
    const bool idle = wq + kHaloQ >= args.nec;
    LaneW hw;
    if constexpr (ADJ) hw.init(m0, AxisLen{args.nec, args.ndc});
    const AxisLen rows{args.ner, args.ndr};

    char* out_p = reinterpret_cast<char*>(row_ptr<TO>(args.out, 2 * n0, z) + 2 * m0);
    uint64_t out_pol = 0;
    if constexpr (keeps_ll_in_l2(WV))
        out_pol = args.out_keep ? l2_evict_last() : l2_evict_normal();
    static_assert(!kShift || (!ADJ && std::is_same<C, float>::value), "no shift on this level");
    LevelShift sh{-0.f, -0.f};
    if constexpr (kShift) sh.init(args.shift, z);
    Pipe pipe;
    pipe.init();
    RingPos<kS> rp;
#pragma unroll row_unroll<WV>()
    for (int i = 0; i < nrows; ++i) {
        const int s = rp.s;
        const uint32_t par = rp.ph;
        rp.next();
        bool ok = mbar_wait(&ring.full[s], par, ring.abort, args.status);
        if (!__all_sync(kFull, ok)) break;
        if (idle) {
            if (lane == 0) mbar_arrive(&ring.empty[s]);
            continue;
        }
        QRow<C> row;
        inv_lane_row<TL, TB, C>(ring.stage(s), cols, row);
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring.empty[s]);
        if constexpr (kShift) add_ll(row, sh.in_add);
        if constexpr (ADJ)
            pipe.push(row, qfirst + i, hw, rows, args.scale);
        else
            pipe.push(row);
        const int qo = qfirst + i - Pipe::kLag;
        if (qo >= n0 && qo < n1) {
            if constexpr (kShift) add_row(row, sh.out_add);
            if (store_lane) {
                if constexpr (keeps_ll_in_l2(WV))
                    inv_store_rows_at_hint<TO>(args, row, qo, m0, out_p, out_pol);
                else
                    inv_store_rows_at<TO>(args, row, qo, m0, out_p);
            }
            out_p += 2 * args.out.pitch;
        }
    }
}

// =============================================================================================
// Direct inverse level for small planes: the inverse counterpart of k_forward_direct.  Each warp
// loads the band rows of kDirectRows + 2 kLag extended quad rows (mirrored rows and columns,
// as the streaming kernel's stages hold them) straight from global memory into registers and
// pushes them through the same InvPipe.
// =============================================================================================
// A lane's kQ values of band row r (false ok: a row outside the band, zeros); columns m0 + j,
// or the mirrored columns col[j] at the plane's edges.
template <typename T, typename C>
__device__ __forceinline__ void direct_load_band(const char* row, bool ok, int m0, bool vec,
                                                 bool edge, const int (&col)[kQ], bool zero,
                                                 C (&v)[kQ]) {
    const T* p = reinterpret_cast<const T*>(row);
    if (!ok || zero) {
#pragma unroll
        for (int j = 0; j < kQ; ++j) v[j] = C(0);
    } else if (vec) {
        ldN<kQ>(p + m0, v);
    } else {
#pragma unroll
        for (int j = 0; j < kQ; ++j) v[j] = to_c(ldcg(p + (edge ? col[j] : m0 + j)));
    }
}

template <int WV, typename TB, typename TL, typename TO, bool kShift>
__global__ void __launch_bounds__(32 * kDirectWarps) k_inverse_direct(const InvArgs args) {
    using Pipe = InvPipe<WV>;
    using C = typename Pipe::C;
    constexpr int kLag = Pipe::kLag;
    constexpr int kRows = kDirectRows + 2 * kLag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.z;
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    const int wq = (blockIdx.y * kDirectWarps + warp) * warp_out<WV>() - kHaloQ;
    const int m0 = wq + kQ * lane;
    const int n0 = blockIdx.x * kDirectRows;
    const int n1 = min(n0 + kDirectRows, args.ner);
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    grid_dependency_wait();
    allow_dependent_launch();
    if (wq + kHaloQ >= args.nec) return;

    // columns: LL / LH hold the even pixel columns 2m, HL / HH the odd ones 2m + 1
    const bool edge = (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W);
    const bool odd_zero = args.W <= 1;
    int ce[kQ], co[kQ];
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
        ce[j] = refl_in(2 * (m0 + j), args.W) >> 1;
        co[j] = odd_zero ? 0 : (refl_in(2 * (m0 + j) + 1, args.W) - 1) >> 1;
    }
    const char* base[4];
    bool vec = !edge;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        base[b] = static_cast<const char*>(args.band[b]) + int64_t(z) * args.band_bstride[b];
        const int64_t esz = b == 0 ? sizeof(TL) : sizeof(TB);
        vec = vec && (reinterpret_cast<uintptr_t>(base[b]) % (kQ * esz)) == 0 &&
              args.band_pitch[b] % (kQ * esz) == 0;
    }
    QRow<C> rows[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int q = n0 - kLag + i;
        const int re = refl_in(2 * q, args.H) >> 1;                              // LL / HL row
        const int ro = args.H > 1 ? (refl_in(2 * q + 1, args.H) - 1) >> 1 : -1;  // LH / HH row
        const bool ok_o = ro >= 0;
        const int roc = ok_o ? ro : 0;
        direct_load_band<TL, C>(base[0] + int64_t(re) * args.band_pitch[0], true, m0, vec, edge,
                                ce, false, rows[i].a);
        direct_load_band<TB, C>(base[1] + int64_t(re) * args.band_pitch[1], true, m0, vec, edge,
                                co, odd_zero, rows[i].b);
        direct_load_band<TB, C>(base[2] + int64_t(roc) * args.band_pitch[2], ok_o, m0, vec, edge,
                                ce, false, rows[i].c);
        direct_load_band<TB, C>(base[3] + int64_t(roc) * args.band_pitch[3], ok_o, m0, vec, edge,
                                co, odd_zero, rows[i].e);
    }
    LevelShift sh{-0.f, -0.f};
    if constexpr (kShift) sh.init(args.shift, z);
    char* out_p = reinterpret_cast<char*>(row_ptr<TO>(args.out, 2 * n0, z) + 2 * m0);
    Pipe pipe;
    pipe.init();
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        QRow<C> row = rows[i];
        if constexpr (kShift) add_ll(row, sh.in_add);
        pipe.push(row);
        const int qo = n0 - 2 * kLag + i;
        if (i >= 2 * kLag && qo < n1) {
            if constexpr (kShift) add_row(row, sh.out_add);
            if (store_lane) inv_store_rows_at<TO>(args, row, qo, m0, out_p);
            out_p += 2 * args.out.pitch;
        }
    }
}

// =============================================================================================
// Host-side launch helpers (templated; instantiated per wavelet in the launcher files).
// =============================================================================================
struct LaunchGeom {
    dim3 grid;
    int rpc;
};

// Rows per CTA.  A CTA streams its rows one after another, so a launch lasts about
// waves x (rows per CTA + a fixed cost of halo rows and pipeline fill), waves being the CTA count
// over the resident slots (SM count x CTAs per SM).  The row-block count that minimises that
// estimate is taken: for one large plane, one wave of CTAs; for a batch of many planes, whole
// waves with no small last wave; for small planes, as many CTAs as fit.  Rows per CTA stay at
// least 16 for large data (the halo is then a small overhead on HBM reads) and at least 4 for
// data of a few MB (served from L2 after the previous level wrote it), where the per-row latency
// of a CTA, not bytes, sets the time.
inline LaunchGeom pick_geometry(int ner, int nec, int64_t plane_bytes, int sms, int ctas_per_sm,
                                int nbatch, int cta_quads) {
    constexpr int64_t kRowCost = 8;  // halo rows + pipeline fill, in rows
    const int n = std::max(1, nbatch);
    const int strips = (nec + cta_quads - 1) / cta_quads;
    const int64_t slots = int64_t(std::max(1, sms)) * std::max(1, ctas_per_sm);
    const int min_rows = plane_bytes * n < (int64_t(24) << 20) ? 2 : 16;
    const int rb_max = std::max(1, (ner + min_rows - 1) / min_rows);
    int best_rb = 1;
    int64_t best = -1;
    for (int rb = 1; rb <= rb_max; ++rb) {
        const int rpc = (ner + rb - 1) / rb;
        const int used = (ner + rpc - 1) / rpc;  // row blocks that are not empty
        if (used != rb) continue;
        const int64_t ctas = int64_t(strips) * used * n;
        const int64_t waves = (ctas + slots - 1) / slots;
        const int64_t cost = waves * (rpc + kRowCost);
        if (best < 0 || cost < best) {
            best = cost;
            best_rb = rb;
        }
    }
    LaunchGeom g;
    g.rpc = (ner + best_rb - 1) / best_rb;
    g.grid = dim3(strips, (ner + g.rpc - 1) / g.rpc, n);
    return g;
}

// Launch with programmatic stream serialization (the kernels wait for their predecessor with
// griddepcontrol.wait before touching global memory).
template <typename K, typename... Args>
cudaError_t launch_pdl(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int device_sm_count();

// Sets the kernel's dynamic shared memory limit and asks for the largest shared-memory carveout
// (the kernels need no L1 beyond the default; without this the driver may pick a smaller carveout
// and fit fewer CTAs per SM), then returns the resident CTAs per SM.
template <typename K>
int configure(K kernel, int threads, size_t smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess)
        n = 1;
    return n;
}

// Consumer warps per CTA for a launch over planes of nec quad columns and `bytes` of input in all:
// the narrow CTA where its strips keep at least 10 points more of the warp windows busy than the
// wide CTA's, on launches of 24 MB or more.  Smaller launches are latency-bound, and the wide CTA
// was faster there (levels 4 and 5 of an 8192^2 forward: 0.1412 against 0.1423 ms in all).
inline int pick_nw(int nec, int64_t bytes) {
    if (bytes < (int64_t(24) << 20)) return 4;
    auto busy = [nec](int q) {
        const int strips = (nec + q - 1) / q;
        return double(nec) / double(int64_t(strips) * q);
    };
    return busy(cta_q<3>()) >= busy(cta_q<4>()) + 0.1 ? 3 : 4;
}

template <int WV, int MODE, typename TI, typename TB, typename TL, bool kPlain, bool kShift,
          int NW>
cudaError_t launch_forward_k(const CUtensorMap& tm, FwdArgs a, cudaStream_t st) {
    auto k = k_forward<WV, MODE, TI, TB, TL, kPlain, kShift, NW>;
    constexpr size_t smem = fwd_smem_bytes<TI, fwd_stages<WV>()>();
    static const int occ = configure(k, cta_threads<NW>(), smem);
    const LaunchGeom g = pick_geometry(a.ner, a.nec, int64_t(a.H) * a.W * int64_t(sizeof(TI)),
                                       device_sm_count(), occ, a.nbatch, cta_q<NW, WV>());
    a.rpc = g.rpc;
    return launch_pdl(k, g.grid, cta_threads<NW>(), smem, st, tm, a);
}

// TMA-loading or plain-loading instantiation, by whether the input plane has a tensor map,
// and the instantiation with the DC level shift only for the levels that take it (the first and
// the last), so the others run exactly the code they would without it.
template <int WV, int MODE, typename TI, typename TB, typename TL, int NW>
cudaError_t launch_forward_nw(const CUtensorMap& tm, FwdArgs a, cudaStream_t st) {
    using C = std::conditional_t<WV == WV_CDF53_INT, int32_t, float>;
    if constexpr (kShiftable<C, MODE>) {
        if (a.shift.mode != 0)
            return a.tma ? launch_forward_k<WV, MODE, TI, TB, TL, false, true, NW>(tm, a, st)
                         : launch_forward_k<WV, MODE, TI, TB, TL, true, true, NW>(tm, a, st);
    }
    return a.tma ? launch_forward_k<WV, MODE, TI, TB, TL, false, false, NW>(tm, a, st)
                 : launch_forward_k<WV, MODE, TI, TB, TL, true, false, NW>(tm, a, st);
}

template <int WV, typename TI, typename TB, typename TL, bool kShift>
cudaError_t launch_forward_direct(FwdArgs a, cudaStream_t st) {
    auto k = k_forward_direct<WV, TI, TB, TL, kShift>;
    const int windows = (a.nec + warp_out<WV>() - 1) / warp_out<WV>();
    const dim3 grid((a.ner + kDirectRows - 1) / kDirectRows,
                    (windows + kDirectWarps - 1) / kDirectWarps, std::max(1, a.nbatch));
    a.rpc = kDirectRows;
    return launch_pdl(k, grid, 32 * kDirectWarps, 0, st, a);
}

// ... and the CTA width by the plane's width (the separable comparators keep the wide CTA).
// Small planes of the non-separable forward take the direct kernel.
template <int WV, int MODE, typename TI, typename TB, typename TL>
cudaError_t launch_forward_t(const CUtensorMap& tm, FwdArgs a, cudaStream_t st) {
    if constexpr (MODE == MODE_NONSEP) {
        if (takes_direct(a.H, a.W, sizeof(TI), a.nbatch)) {
            using C = std::conditional_t<WV == WV_CDF53_INT, int32_t, float>;
            if constexpr (kShiftable<C, MODE>) {
                if (a.shift.mode != 0) return launch_forward_direct<WV, TI, TB, TL, true>(a, st);
            }
            return launch_forward_direct<WV, TI, TB, TL, false>(a, st);
        }
    }
    if constexpr ((MODE == MODE_NONSEP || MODE == MODE_ADJ_INV) && !is_dd(WV)) {
        if (pick_nw(a.nec, int64_t(a.H) * a.W * int64_t(sizeof(TI)) * a.nbatch) == 3)
            return launch_forward_nw<WV, MODE, TI, TB, TL, 3>(tm, a, st);
    }
    return launch_forward_nw<WV, MODE, TI, TB, TL, kMaxNW>(tm, a, st);
}

template <int WV, typename TB, typename TL, typename TO, bool ADJ, bool kShift, int NW>
cudaError_t launch_inverse_k(const CUtensorMap* tm, InvArgs a, cudaStream_t st) {
    auto k = k_inverse<WV, TB, TL, TO, ADJ, kShift, NW>;
    constexpr size_t smem = inv_smem_bytes<TL, TB, inv_stages<WV>()>();
    static const int occ = configure(k, cta_threads<NW>(), smem);
    const LaunchGeom g = pick_geometry(a.ner, a.nec, int64_t(a.H) * a.W * int64_t(sizeof(TL)),
                                       device_sm_count(), occ, a.nbatch, cta_q<NW, WV>());
    a.rpc = g.rpc;
    return launch_pdl(k, g.grid, cta_threads<NW>(), smem, st, tm[0], tm[1], tm[2], tm[3], a);
}

template <int WV, typename TB, typename TL, typename TO, bool ADJ, bool kShift>
cudaError_t launch_inverse_s(const CUtensorMap* tm, InvArgs a, cudaStream_t st) {
    if constexpr (inv_narrow_nw<TB, TL>() == 3 && !is_dd(WV)) {
        const int64_t bytes = int64_t(a.H) * a.W * int64_t(sizeof(TL)) * a.nbatch;
        if (pick_nw(a.nec, bytes) == 3)
            return launch_inverse_k<WV, TB, TL, TO, ADJ, kShift, 3>(tm, a, st);
    }
    return launch_inverse_k<WV, TB, TL, TO, ADJ, kShift, kMaxNW>(tm, a, st);
}

// The inverse level with the DC level shift for the levels that take it (the last inverse level,
// which takes the shift off LL_J, and the first, which puts it back).
template <int WV, typename TB, typename TL, typename TO, bool kShift>
cudaError_t launch_inverse_direct(InvArgs a, cudaStream_t st) {
    auto k = k_inverse_direct<WV, TB, TL, TO, kShift>;
    const int windows = (a.nec + warp_out<WV>() - 1) / warp_out<WV>();
    const dim3 grid((a.ner + kDirectRows - 1) / kDirectRows,
                    (windows + kDirectWarps - 1) / kDirectWarps, std::max(1, a.nbatch));
    a.rpc = kDirectRows;
    return launch_pdl(k, grid, 32 * kDirectWarps, 0, st, a);
}

// Small output planes of the inverse take the direct kernel.
template <int WV, typename TB, typename TL, typename TO, bool ADJ = false>
cudaError_t launch_inverse_t(const CUtensorMap* tm, InvArgs a, cudaStream_t st) {
    if constexpr (!ADJ) {
        if (takes_direct(a.H, a.W, sizeof(TL), a.nbatch)) {
            if constexpr (WV != WV_CDF53_INT) {
                if (a.shift.mode != 0) return launch_inverse_direct<WV, TB, TL, TO, true>(a, st);
            }
            return launch_inverse_direct<WV, TB, TL, TO, false>(a, st);
        }
    }
    if constexpr (!ADJ && WV != WV_CDF53_INT) {
        if (a.shift.mode != 0) return launch_inverse_s<WV, TB, TL, TO, false, true>(tm, a, st);
    }
    return launch_inverse_s<WV, TB, TL, TO, ADJ, false>(tm, a, st);
}

}  // namespace dwt2
