// dwt2_stream.cuh -- the per-level kernels: a producer warp streams quad rows of the input into
// a ring of shared-memory stages (TMA 2-D tiles, or plain loads for unaligned inputs); four
// consumer warps run the lifting pipeline of dwt2_lifting.cuh in registers and write the
// results with vector stores.  One HBM read of the input and one write of the output per level.
//
// Geometry (all in polyphase quads; a quad is 2 x 2 pixels):
//   CTA   = a strip of kCtaQ = 240 output quad columns x rpc output quad rows;
//   warp  = a window of 64 quad columns (32 lanes x 2 quads) whose 2 outer quads on each side are
//           halo (lanes 0 and 31 compute but never store), i.e. 60 output quads per warp;
//   rows  = the CTA streams its rpc rows plus 2 halo quad rows above and below.
// Boundaries: the producer maps every (extended) row to its whole-sample-symmetric source row;
// warps whose window crosses the left or right image edge read each column from its mirrored
// source column.  The lifting then runs on the symmetric extension with no boundary rule.
#pragma once

#include "dwt2_lifting.cuh"

namespace dwt2 {

constexpr int kNW = 4;                   // consumer warps per CTA
constexpr int kHQ = 2;                   // halo quads on each side of a warp window
constexpr int kWarpQ = 64;               // quads in a warp window
constexpr int kWarpOut = kWarpQ - 2 * kHQ;  // 60 output quads per warp
constexpr int kCtaQ = kNW * kWarpOut;    // 240 output quads per CTA strip
constexpr int kThreads = 32 * (kNW + 1);
constexpr int kStages = 8;               // quad rows in flight per CTA
constexpr int kVHalo = 2;                // halo quad rows above and below a CTA's rows

// Forward: a stage holds 2 pixel rows of the strip's pixel columns [2*qx0 - kXL, +kSRow), loaded
// as two 256-wide boxes per row (every TMA destination starts on a 128-byte boundary).
constexpr int kXL = 8;
constexpr int kBoxW = 256;
constexpr int kSRow = 2 * kBoxW;  // 512 >= kXL + 2*kCtaQ + 2*kHQ
// Inverse: a stage holds one row of each band, quad columns [qx0 - kXLB, +kBRow).
constexpr int kXLB = 8;
constexpr int kBRow = 256;  // >= kXLB + kCtaQ + kHQ, one TMA box

struct PlaneOut {
    void* ptr;
    int64_t pitch;  // bytes
};

struct FwdArgs {
    const void* in;     // input plane (used by the plain-load path)
    int64_t in_pitch;   // bytes
    int H, W;           // input plane size in pixels
    int ner, ndr, nec, ndc;  // even/odd row and column counts = band sizes
    PlaneOut ll, hl, lh, hh;  // band planes (ll is the interleaved output plane in MODE_ROWS)
    int rpc;            // output quad rows per CTA
    int* status;        // workspace status word
};

struct InvArgs {
    const void* band[4];  // LL, HL, LH, HH (used by the plain-load path)
    int64_t band_pitch[4];
    int H, W;             // output plane size in pixels
    int ner, ndr, nec, ndc;
    PlaneOut out;         // output plane
    int out_vec;          // output rows may use 4-element vector stores
    int rpc;
    int* status;
};

template <typename T>
__device__ __forceinline__ T* row_ptr(const PlaneOut& p, int r) {
    return reinterpret_cast<T*>(static_cast<char*>(p.ptr) + static_cast<int64_t>(r) * p.pitch);
}

// Stores two adjacent quads' values of one band row (aligned pair, clipped at the band width).
template <typename T, typename C>
__device__ __forceinline__ void put2(T* p, C v0, C v1, int m0, int width) {
    if (m0 + 1 < width) st2(p, v0, v1);
    else if (m0 < width) *p = from_c<T>(v0);
}

// Bytes of dynamic shared memory of the kernels (+128 to align the base to 128 bytes).
template <typename TI>
constexpr size_t fwd_smem_bytes() {
    return size_t(kStages) * 2 * kSRow * sizeof(TI) + 2 * kStages * sizeof(uint64_t) + 16 + 128;
}
template <typename TL, typename TB>
constexpr size_t inv_smem_bytes() {
    return size_t(kStages) * kBRow * (sizeof(TL) + 3 * sizeof(TB)) +
           2 * kStages * sizeof(uint64_t) + 16 + 128;
}

__device__ __forceinline__ uint8_t* align128(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

// =============================================================================================
// Forward level.  MODE_ROWS writes the interleaved plane (the row pass of the two-pass
// separable comparator); every other mode writes the four band planes.
// =============================================================================================
template <int WV, int MODE, typename TI, typename TB, typename TL, bool TMA>
__global__ void __launch_bounds__(kThreads)
    k_forward(const __grid_constant__ CUtensorMap tmap, const FwdArgs args) {
    using Pipe = FwdPipe<WV, MODE>;
    using C = typename Pipe::C;
    constexpr int kVH = MODE == MODE_ROWS ? 0 : kVHalo;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = align128(smem_raw);
    TI* stages = reinterpret_cast<TI*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(kStages) * 2 * kSRow * sizeof(TI));
    uint64_t* empty = full + kStages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx0 = blockIdx.x * kCtaQ;
    const int n0 = blockIdx.y * args.rpc;
    const int n1 = min(n0 + args.rpc, args.ner);
    const int nrows = n1 - n0 + 2 * kVH;
    const int qfirst = n0 - kVH;
    const int xs = 2 * qx0 - kXL;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], TMA ? 1 : 32);
            mbar_init(&empty[s], kNW);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (TMA && warp == kNW && lane == 0) prefetch_tensormap(&tmap);
    __syncthreads();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        int issued = 0;
        for (int i = 0; i < nrows; ++i) {
            const int s = i % kStages;
            if (i >= kStages) {
                bool ok = mbar_wait(&empty[s], ((i / kStages) - 1) & 1, abort_flag, args.status);
                if (!__all_sync(kFull, ok)) break;
            }
            const int q = qfirst + i;
            const int r0 = refl(2 * q, args.H), r1 = refl(2 * q + 1, args.H);
            TI* dst = stages + size_t(s) * 2 * kSRow;
            if constexpr (TMA) {
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], 2 * kSRow * sizeof(TI));
                    tma_load_2d(dst, &tmap, &full[s], xs, r0);
                    tma_load_2d(dst + kBoxW, &tmap, &full[s], xs + kBoxW, r0);
                    tma_load_2d(dst + kSRow, &tmap, &full[s], xs, r1);
                    tma_load_2d(dst + kSRow + kBoxW, &tmap, &full[s], xs + kBoxW, r1);
                }
            } else {
                const TI* row0 = reinterpret_cast<const TI*>(static_cast<const char*>(args.in) +
                                                             int64_t(r0) * args.in_pitch);
                const TI* row1 = reinterpret_cast<const TI*>(static_cast<const char*>(args.in) +
                                                             int64_t(r1) * args.in_pitch);
                for (int k = lane; k < kSRow; k += 32) {
                    const int c = xs + k;
                    const bool in = c >= 0 && c < args.W;
                    dst[k] = in ? row0[c] : zero_of<TI>();
                    dst[kSRow + k] = in ? row1[c] : zero_of<TI>();
                }
                mbar_arrive(&full[s]);
            }
            issued = i + 1;
        }
        if (TMA && lane == 0) {  // let the last copies land before the CTA can exit
            volatile int no_abort = 0;
            for (int i = max(0, issued - kStages); i < issued; ++i)
                if (!mbar_wait(&full[i % kStages], (i / kStages) & 1, &no_abort, args.status))
                    break;
        }
        return;
    }

    // ------------------------------------------------------------------------- consumers
    const int wq = qx0 - kHQ + warp * kWarpOut;  // first quad of the warp window
    const int col0 = 2 * wq + 4 * lane;          // first pixel column of this lane
    const bool edge = (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W);
    const int sc = col0 - xs;
    int ec[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ec[k] = min(max(refl(col0 + k, args.W) - xs, 0), kSRow - 1);
    const int m0 = wq + 2 * lane;
    const bool store_lane = lane >= 1 && lane <= 30;

    Pipe pipe;
    pipe.init();
    for (int i = 0; i < nrows; ++i) {
        const int s = i % kStages;
        bool ok = mbar_wait(&full[s], (i / kStages) & 1, abort_flag, args.status);
        if (!__all_sync(kFull, ok)) break;
        const TI* r0 = stages + size_t(s) * 2 * kSRow;
        const TI* r1 = r0 + kSRow;
        C v0[4], v1[4];
        if (!edge) {
            ld4(r0 + sc, v0);
            ld4(r1 + sc, v1);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v0[k] = to_c(r0[ec[k]]);
                v1[k] = to_c(r1[ec[k]]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        QRow<C> row;
        row.a[0] = v0[0]; row.b[0] = v0[1]; row.a[1] = v0[2]; row.b[1] = v0[3];
        row.c[0] = v1[0]; row.e[0] = v1[1]; row.c[1] = v1[2]; row.e[1] = v1[3];
        pipe.push(row);

        const int qo = qfirst + i - Pipe::kLag;
        if (qo < n0 || qo >= n1 || !store_lane) continue;
        if constexpr (MODE == MODE_ROWS) {
            // interleaved output plane: pixel rows 2qo (a b a b) and 2qo + 1 (c e c e)
            const int c0 = 2 * m0;
            TL* o0 = row_ptr<TL>(args.ll, 2 * qo) + c0;
            if (c0 + 3 < args.W) {
                st4(o0, row.a[0], row.b[0], row.a[1], row.b[1]);
                if (2 * qo + 1 < args.H) {
                    TL* o1 = row_ptr<TL>(args.ll, 2 * qo + 1) + c0;
                    st4(o1, row.c[0], row.e[0], row.c[1], row.e[1]);
                }
            } else {
                const C va[4] = {row.a[0], row.b[0], row.a[1], row.b[1]};
                const C vc[4] = {row.c[0], row.e[0], row.c[1], row.e[1]};
                for (int k = 0; k < 4; ++k)
                    if (c0 + k < args.W) {
                        o0[k] = from_c<TL>(va[k]);
                        if (2 * qo + 1 < args.H) row_ptr<TL>(args.ll, 2 * qo + 1)[c0 + k] = from_c<TL>(vc[k]);
                    }
            }
        } else {
            put2(row_ptr<TL>(args.ll, qo) + m0, row.a[0], row.a[1], m0, args.nec);
            put2(row_ptr<TB>(args.hl, qo) + m0, row.b[0], row.b[1], m0, args.ndc);
            if (qo < args.ndr) {
                put2(row_ptr<TB>(args.lh, qo) + m0, row.c[0], row.c[1], m0, args.nec);
                put2(row_ptr<TB>(args.hh, qo) + m0, row.e[0], row.e[1], m0, args.ndc);
            }
        }
    }
}

// =============================================================================================
// Inverse level: four band planes in, the interleaved plane out.
// =============================================================================================
template <int WV, typename TB, typename TL, typename TO, bool TMA>
__global__ void __launch_bounds__(kThreads)
    k_inverse(const __grid_constant__ CUtensorMap tm_ll, const __grid_constant__ CUtensorMap tm_hl,
              const __grid_constant__ CUtensorMap tm_lh, const __grid_constant__ CUtensorMap tm_hh,
              const InvArgs args) {
    using Pipe = InvPipe<WV>;
    using C = typename Pipe::C;
    constexpr size_t kStageBytes = size_t(kBRow) * (sizeof(TL) + 3 * sizeof(TB));
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = align128(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx0 = blockIdx.x * kCtaQ;
    const int n0 = blockIdx.y * args.rpc;
    const int n1 = min(n0 + args.rpc, args.ner);
    const int nrows = n1 - n0 + 2 * kVHalo;
    const int qfirst = n0 - kVHalo;
    const int xb = qx0 - kXLB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], TMA ? 1 : 32);
            mbar_init(&empty[s], kNW);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (TMA && warp == kNW && lane == 0) {
        prefetch_tensormap(&tm_ll);
        prefetch_tensormap(&tm_hl);
        prefetch_tensormap(&tm_lh);
        prefetch_tensormap(&tm_hh);
    }
    __syncthreads();

    auto stage_ll = [&](int s) { return reinterpret_cast<TL*>(smem + s * kStageBytes); };
    auto stage_b = [&](int s, int k) {  // k = 0 HL, 1 LH, 2 HH
        return reinterpret_cast<TB*>(smem + s * kStageBytes + kBRow * sizeof(TL) +
                                     size_t(k) * kBRow * sizeof(TB));
    };

    if (warp == kNW) {  // ------------------------------------------------------ producer
        int issued = 0;
        for (int i = 0; i < nrows; ++i) {
            const int s = i % kStages;
            if (i >= kStages) {
                bool ok = mbar_wait(&empty[s], ((i / kStages) - 1) & 1, abort_flag, args.status);
                if (!__all_sync(kFull, ok)) break;
            }
            const int q = qfirst + i;
            // even pixel row 2q -> LL / HL row; odd pixel row 2q + 1 -> LH / HH row
            const int re = refl(2 * q, args.H) >> 1;
            const int ro = args.H > 1 ? (refl(2 * q + 1, args.H) - 1) >> 1 : -1;
            if constexpr (TMA) {
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], uint32_t(kStageBytes));
                    tma_load_2d(stage_ll(s), &tm_ll, &full[s], xb, re);
                    tma_load_2d(stage_b(s, 0), &tm_hl, &full[s], xb, re);
                    tma_load_2d(stage_b(s, 1), &tm_lh, &full[s], xb, ro);
                    tma_load_2d(stage_b(s, 2), &tm_hh, &full[s], xb, ro);
                }
            } else {
                const int rows[4] = {re, re, ro, ro};
                const int widths[4] = {args.nec, args.ndc, args.nec, args.ndc};
                const int heights[4] = {args.ner, args.ner, args.ndr, args.ndr};
                for (int b = 0; b < 4; ++b) {
                    const bool row_ok = rows[b] >= 0 && rows[b] < heights[b];
                    const char* src = static_cast<const char*>(args.band[b]) +
                                      int64_t(row_ok ? rows[b] : 0) * args.band_pitch[b];
                    for (int k = lane; k < kBRow; k += 32) {
                        const int c = xb + k;
                        const bool in = row_ok && c >= 0 && c < widths[b];
                        if (b == 0)
                            stage_ll(s)[k] = in ? reinterpret_cast<const TL*>(src)[c] : zero_of<TL>();
                        else
                            stage_b(s, b - 1)[k] =
                                in ? reinterpret_cast<const TB*>(src)[c] : zero_of<TB>();
                    }
                }
                mbar_arrive(&full[s]);
            }
            issued = i + 1;
        }
        if (TMA && lane == 0) {
            volatile int no_abort = 0;
            for (int i = max(0, issued - kStages); i < issued; ++i)
                if (!mbar_wait(&full[i % kStages], (i / kStages) & 1, &no_abort, args.status))
                    break;
        }
        return;
    }

    // ------------------------------------------------------------------------- consumers
    const int wq = qx0 - kHQ + warp * kWarpOut;
    const int m0 = wq + 2 * lane;
    const bool edge = (2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W);
    const int sidx = m0 - xb;  // smem index of the lane's first quad (fast path)
    int ie[2], io[2];          // edge path: smem indices of the even / odd source columns
    bool odd_zero = args.W <= 1;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int m = m0 + j;
        ie[j] = min(max((refl(2 * m, args.W) >> 1) - xb, 0), kBRow - 1);
        io[j] = odd_zero ? 0 : min(max(((refl(2 * m + 1, args.W) - 1) >> 1) - xb, 0), kBRow - 1);
    }
    const bool store_lane = lane >= 1 && lane <= 30;

    Pipe pipe;
    pipe.init();
    for (int i = 0; i < nrows; ++i) {
        const int s = i % kStages;
        bool ok = mbar_wait(&full[s], (i / kStages) & 1, abort_flag, args.status);
        if (!__all_sync(kFull, ok)) break;
        QRow<C> row;
        const TL* sll = stage_ll(s);
        const TB* shl = stage_b(s, 0);
        const TB* slh = stage_b(s, 1);
        const TB* shh = stage_b(s, 2);
        if (!edge) {
            ld2(sll + sidx, row.a);
            ld2(shl + sidx, row.b);
            ld2(slh + sidx, row.c);
            ld2(shh + sidx, row.e);
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                row.a[j] = to_c(sll[ie[j]]);
                row.c[j] = to_c(slh[ie[j]]);
                row.b[j] = odd_zero ? C(0) : C(to_c(shl[io[j]]));
                row.e[j] = odd_zero ? C(0) : C(to_c(shh[io[j]]));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        pipe.push(row);
        const int qo = qfirst + i - Pipe::kLag;
        if (qo < n0 || qo >= n1 || !store_lane) continue;
        const int c0 = 2 * m0;
        const bool has_odd_row = 2 * qo + 1 < args.H;
        TO* o0 = row_ptr<TO>(args.out, 2 * qo) + c0;
        TO* o1 = row_ptr<TO>(args.out, 2 * qo + 1) + c0;
        if (args.out_vec && c0 + 3 < args.W) {
            st4(o0, row.a[0], row.b[0], row.a[1], row.b[1]);
            if (has_odd_row) st4(o1, row.c[0], row.e[0], row.c[1], row.e[1]);
        } else {
            const C va[4] = {row.a[0], row.b[0], row.a[1], row.b[1]};
            const C vc[4] = {row.c[0], row.e[0], row.c[1], row.e[1]};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c0 + k >= 0 && c0 + k < args.W) {
                    o0[k] = from_c<TO>(va[k]);
                    if (has_odd_row) o1[k] = from_c<TO>(vc[k]);
                }
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

// Picks rows per CTA so that the grid fills the GPU about once (a multiple of the SM count
// times the resident CTAs per SM) without making a CTA's 4 halo rows a large overhead.
inline LaunchGeom pick_geometry(int ner, int nec, int sms, int ctas_per_sm) {
    const int strips = (nec + kCtaQ - 1) / kCtaQ;
    const int target = sms * (ctas_per_sm > 0 ? ctas_per_sm : 1);
    const int min_rows = 16;
    const int rb_max = (ner + min_rows - 1) / min_rows;
    int rb = target / strips;
    if (rb < 1) rb = 1;
    if (rb > rb_max) rb = rb_max;
    int rpc = (ner + rb - 1) / rb;
    if (rpc < 1) rpc = 1;
    rb = (ner + rpc - 1) / rpc;
    LaunchGeom g;
    g.grid = dim3(strips, rb, 1);
    g.rpc = rpc;
    return g;
}

int device_sm_count();

template <typename K>
int occupancy_of(K kernel, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, smem) != cudaSuccess)
        n = 1;
    return n;
}

template <int WV, int MODE, typename TI, typename TB, typename TL, bool TMA>
cudaError_t launch_forward_t(const CUtensorMap& tm, FwdArgs a, cudaStream_t st) {
    auto k = k_forward<WV, MODE, TI, TB, TL, TMA>;
    constexpr size_t smem = fwd_smem_bytes<TI>();
    static const int occ = [&] {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        return occupancy_of(k, smem);
    }();
    const LaunchGeom g = pick_geometry(a.ner, a.nec, device_sm_count(), occ);
    a.rpc = g.rpc;
    k<<<g.grid, kThreads, smem, st>>>(tm, a);
    return cudaGetLastError();
}

template <int WV, typename TB, typename TL, typename TO, bool TMA>
cudaError_t launch_inverse_t(const CUtensorMap* tm, InvArgs a, cudaStream_t st) {
    auto k = k_inverse<WV, TB, TL, TO, TMA>;
    constexpr size_t smem = inv_smem_bytes<TL, TB>();
    static const int occ = [&] {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        return occupancy_of(k, smem);
    }();
    const LaunchGeom g = pick_geometry(a.ner, a.nec, device_sm_count(), occ);
    a.rpc = g.rpc;
    k<<<g.grid, kThreads, smem, st>>>(tm[0], tm[1], tm[2], tm[3], a);
    return cudaGetLastError();
}

}  // namespace dwt2
