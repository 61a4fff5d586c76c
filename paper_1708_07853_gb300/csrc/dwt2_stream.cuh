// dwt2_stream.cuh -- the per-level kernels: a producer warp streams quad rows of the input into
// a ring of shared-memory stages (TMA 2-D tiles, or plain loads for unaligned inputs); four
// consumer warps run the lifting pipeline of dwt2_lifting.cuh in registers and write the
// results with vector stores.  One HBM read of the input and one write of the output per level.
//
// Geometry (all in polyphase quads; a quad is 2 x 2 pixels):
//   CTA   = a strip of kCtaQ output quad columns (4 warps x 30 lanes x kQ) x rpc quad rows;
//   warp  = a window of 32 x kQ quad columns (kQ adjacent quads per lane); lanes 0 and 31 are halo
//           (they compute but never store: the lifting reaches 2 quads to each side);
//   rows  = the CTA streams its rpc rows plus 2 halo quad rows above and below.
// Boundaries: the producer maps every (extended) row to its whole-sample-symmetric source row;
// warps whose window crosses the left or right image edge read each column from its mirrored
// source column.  The lifting then runs on the symmetric extension with no boundary rule.
#pragma once

#include "dwt2_lifting.cuh"

namespace dwt2 {

constexpr int kNW = 4;                   // consumer warps per CTA
constexpr int kHQ = kQ;                  // halo quads on each side of a warp window (one lane)
constexpr int kWarpQ = 32 * kQ;          // quads in a warp window
constexpr int kWarpOut = kWarpQ - 2 * kHQ;  // output quads per warp (30 lanes)
constexpr int kCtaQ = kNW * kWarpOut;    // output quads per CTA strip
constexpr int kThreads = 32 * (kNW + 1);
constexpr int kStages = 8;               // quad rows in flight per CTA
constexpr int kVHalo = 2;                // halo quad rows above and below a CTA's rows

// Forward: a stage holds 2 pixel rows of the strip's pixel columns [2*qx0 - kXL, +kSRow), loaded
// as 256-wide boxes (every TMA destination starts on a 128-byte boundary).
constexpr int kXL = 8;
constexpr int kBoxW = 256;
constexpr int kBoxes = (kXL + 2 * kCtaQ + 2 * kHQ + kBoxW - 1) / kBoxW;
constexpr int kSRow = kBoxes * kBoxW;
// Inverse: a stage holds one row of each band, quad columns [qx0 - kXLB, +kBRow).
constexpr int kXLB = 8;
constexpr int kBBoxes = (kXLB + kCtaQ + kHQ + kBoxW - 1) / kBoxW;
constexpr int kBRow = kBBoxes * kBoxW;
static_assert(kSRow >= kXL + 2 * kCtaQ + 2 * kHQ, "forward stage row too short");
static_assert(kBRow >= kXLB + kCtaQ + kHQ, "inverse stage row too short");

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
    Scale4 scale;       // MODE_ADJ_INV: the reciprocal band scales applied last
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
    Scale4 scale;         // adjoint: the band scales applied first
};

template <typename T>
__device__ __forceinline__ T* row_ptr(const PlaneOut& p, int r) {
    return reinterpret_cast<T*>(static_cast<char*>(p.ptr) + static_cast<int64_t>(r) * p.pitch);
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
    // MODE_ADJ_INV runs the transpose of the inverse level (gradient of an inverse transform):
    // same data flow, no mirroring (zeros outside the plane), boundary weights in the steps.
    constexpr bool kAdj = MODE == MODE_ADJ_INV;
    using Pipe = std::conditional_t<kAdj, AdjInvPipe<WV>, FwdPipe<WV, kAdj ? MODE_NONSEP : MODE>>;
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
    // Everything above overlaps the previous level's tail; nothing below may touch global memory
    // before that level has finished writing this level's input (and reading what we overwrite).
    grid_dependency_wait();
    allow_dependent_launch();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        int issued = 0;
        for (int i = 0; i < nrows; ++i) {
            const int s = i % kStages;
            if (i >= kStages) {
                bool ok = mbar_wait(&empty[s], ((i / kStages) - 1) & 1, abort_flag, args.status);
                if (!__all_sync(kFull, ok)) break;
            }
            const int q = qfirst + i;
            const int r0 = kAdj ? 2 * q : refl(2 * q, args.H);
            const int r1 = kAdj ? 2 * q + 1 : refl(2 * q + 1, args.H);
            TI* dst = stages + size_t(s) * 2 * kSRow;
            if constexpr (TMA) {
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], 2 * kSRow * sizeof(TI));
#pragma unroll
                    for (int b = 0; b < kBoxes; ++b) {
                        tma_load_2d(dst + b * kBoxW, &tmap, &full[s], xs + b * kBoxW, r0);
                        tma_load_2d(dst + kSRow + b * kBoxW, &tmap, &full[s], xs + b * kBoxW, r1);
                    }
                }
            } else {
                const bool ok0 = r0 >= 0 && r0 < args.H, ok1 = r1 >= 0 && r1 < args.H;
                const TI* row0 = reinterpret_cast<const TI*>(static_cast<const char*>(args.in) +
                                                             int64_t(ok0 ? r0 : 0) * args.in_pitch);
                const TI* row1 = reinterpret_cast<const TI*>(static_cast<const char*>(args.in) +
                                                             int64_t(ok1 ? r1 : 0) * args.in_pitch);
                for (int k = lane; k < kSRow; k += 32) {
                    const int c = xs + k;
                    const bool in = c >= 0 && c < args.W;
                    dst[k] = (in && ok0) ? row0[c] : zero_of<TI>();
                    dst[kSRow + k] = (in && ok1) ? row1[c] : zero_of<TI>();
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
    const int m0 = wq + kQ * lane;               // first quad of this lane
    const int col0 = 2 * m0;                     // first pixel column of this lane
    const bool edge = !kAdj && ((2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W));
    const int sc = col0 - xs;
    const bool store_lane = lane >= 1 && lane <= 30;
    LaneW hw;
    if constexpr (kAdj) hw.init(m0, AxisLen{args.nec, args.ndc});
    const AxisLen rows{args.ner, args.ndr};

    Pipe pipe;
    pipe.init();
    for (int i = 0; i < nrows; ++i) {
        const int s = i % kStages;
        bool ok = mbar_wait(&full[s], (i / kStages) & 1, abort_flag, args.status);
        if (!__all_sync(kFull, ok)) break;
        const TI* r0 = stages + size_t(s) * 2 * kSRow;
        const TI* r1 = r0 + kSRow;
        C v0[2 * kQ], v1[2 * kQ];
        if (!edge) {
            ldN<2 * kQ>(r0 + sc, v0);
            ldN<2 * kQ>(r1 + sc, v1);
        } else {
#pragma unroll
            for (int k = 0; k < 2 * kQ; ++k) {
                const int c = min(max(refl(col0 + k, args.W) - xs, 0), kSRow - 1);
                v0[k] = to_c(r0[c]);
                v1[k] = to_c(r1[c]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        QRow<C> row;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            row.a[q] = v0[2 * q];
            row.b[q] = v0[2 * q + 1];
            row.c[q] = v1[2 * q];
            row.e[q] = v1[2 * q + 1];
        }
        if constexpr (kAdj)
            pipe.push(row, qfirst + i, hw, rows, args.scale);
        else
            pipe.push(row);

        const int qo = qfirst + i - Pipe::kLag;
        if (qo < n0 || qo >= n1 || !store_lane) continue;
        if constexpr (MODE == MODE_ROWS) {
            // interleaved output plane: pixel rows 2qo (a b a b ...) and 2qo + 1 (c e c e ...)
            C va[2 * kQ], vc[2 * kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                va[2 * q] = row.a[q];
                va[2 * q + 1] = row.b[q];
                vc[2 * q] = row.c[q];
                vc[2 * q + 1] = row.e[q];
            }
            putN<2 * kQ>(row_ptr<TL>(args.ll, 2 * qo) + col0, va, col0, args.W, true);
            if (2 * qo + 1 < args.H)
                putN<2 * kQ>(row_ptr<TL>(args.ll, 2 * qo + 1) + col0, vc, col0, args.W, true);
        } else {
            putN<kQ>(row_ptr<TL>(args.ll, qo) + m0, row.a, m0, args.nec, true);
            putN<kQ>(row_ptr<TB>(args.hl, qo) + m0, row.b, m0, args.ndc, true);
            if (qo < args.ndr) {
                putN<kQ>(row_ptr<TB>(args.lh, qo) + m0, row.c, m0, args.nec, true);
                putN<kQ>(row_ptr<TB>(args.hh, qo) + m0, row.e, m0, args.ndc, true);
            }
        }
    }
}

// =============================================================================================
// Inverse level: four band planes in, the interleaved plane out.
// =============================================================================================
template <int WV, typename TB, typename TL, typename TO, bool TMA, bool ADJ>
__global__ void __launch_bounds__(kThreads)
    k_inverse(const __grid_constant__ CUtensorMap tm_ll, const __grid_constant__ CUtensorMap tm_hl,
              const __grid_constant__ CUtensorMap tm_lh, const __grid_constant__ CUtensorMap tm_hh,
              const InvArgs args) {
    // ADJ runs the transpose of the forward level (gradient of a forward transform): same data
    // flow, no mirroring (zeros outside the bands), boundary weights in the steps.
    using Pipe = std::conditional_t<ADJ, AdjFwdPipe<WV>, InvPipe<WV>>;
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
    grid_dependency_wait();
    allow_dependent_launch();

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
            const int re = ADJ ? q : refl(2 * q, args.H) >> 1;
            const int ro = ADJ ? q : (args.H > 1 ? (refl(2 * q + 1, args.H) - 1) >> 1 : -1);
            if constexpr (TMA) {
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], uint32_t(kStageBytes));
#pragma unroll
                    for (int b = 0; b < kBBoxes; ++b) {
                        const int x = xb + b * kBoxW;
                        tma_load_2d(stage_ll(s) + b * kBoxW, &tm_ll, &full[s], x, re);
                        tma_load_2d(stage_b(s, 0) + b * kBoxW, &tm_hl, &full[s], x, re);
                        tma_load_2d(stage_b(s, 1) + b * kBoxW, &tm_lh, &full[s], x, ro);
                        tma_load_2d(stage_b(s, 2) + b * kBoxW, &tm_hh, &full[s], x, ro);
                    }
                }
            } else {
                const int rows[4] = {re, re, ro, ro};
                const int widths[4] = {args.nec, args.ndc, args.nec, args.ndc};
                const int heights[4] = {args.ner, args.ner, args.ndr, args.ndr};
#pragma unroll
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
    const int m0 = wq + kQ * lane;
    const bool edge = !ADJ && ((2 * wq < 0) || (2 * wq + 2 * kWarpQ > args.W));
    const int sidx = m0 - xb;  // smem index of the lane's first quad (fast path)
    const bool odd_zero = args.W <= 1;
    const bool store_lane = lane >= 1 && lane <= 30;
    LaneW hw;
    if constexpr (ADJ) hw.init(m0, AxisLen{args.nec, args.ndc});
    const AxisLen rows{args.ner, args.ndr};

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
            ldN<kQ>(sll + sidx, row.a);
            ldN<kQ>(shl + sidx, row.b);
            ldN<kQ>(slh + sidx, row.c);
            ldN<kQ>(shh + sidx, row.e);
        } else {
            // even pixel column 2m -> LL / LH column; odd 2m + 1 -> HL / HH column (reflected)
#pragma unroll
            for (int j = 0; j < kQ; ++j) {
                const int m = m0 + j;
                const int ie = min(max((refl(2 * m, args.W) >> 1) - xb, 0), kBRow - 1);
                const int io =
                    odd_zero ? 0 : min(max(((refl(2 * m + 1, args.W) - 1) >> 1) - xb, 0), kBRow - 1);
                row.a[j] = to_c(sll[ie]);
                row.c[j] = to_c(slh[ie]);
                row.b[j] = odd_zero ? C(0) : C(to_c(shl[io]));
                row.e[j] = odd_zero ? C(0) : C(to_c(shh[io]));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        if constexpr (ADJ)
            pipe.push(row, qfirst + i, hw, rows, args.scale);
        else
            pipe.push(row);
        const int qo = qfirst + i - Pipe::kLag;
        if (qo < n0 || qo >= n1 || !store_lane) continue;
        const int c0 = 2 * m0;
        C va[2 * kQ], vc[2 * kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            va[2 * q] = row.a[q];
            va[2 * q + 1] = row.b[q];
            vc[2 * q] = row.c[q];
            vc[2 * q + 1] = row.e[q];
        }
        putN<2 * kQ>(row_ptr<TO>(args.out, 2 * qo) + c0, va, c0, args.W, args.out_vec != 0);
        if (2 * qo + 1 < args.H)
            putN<2 * kQ>(row_ptr<TO>(args.out, 2 * qo + 1) + c0, vc, c0, args.W, args.out_vec != 0);
    }
}

// =============================================================================================
// Host-side launch helpers (templated; instantiated per wavelet in the launcher files).
// =============================================================================================
struct LaunchGeom {
    dim3 grid;
    int rpc;
};

// Rows per CTA.  Large planes: about one wave of CTAs (SM count x resident CTAs per SM) with at
// least 16 quad rows each, so the 4 halo rows of a CTA stay a small overhead on HBM reads.
// Small planes (a few MB, served from L2 after the previous level wrote them): as many CTAs as
// fit, down to 4 rows each, because there the per-row latency of a CTA, not bytes, sets the time.
inline LaunchGeom pick_geometry(int ner, int nec, int64_t plane_bytes, int sms, int ctas_per_sm) {
    const int strips = (nec + kCtaQ - 1) / kCtaQ;
    const int target = sms * (ctas_per_sm > 0 ? ctas_per_sm : 1);
    const int min_rows = plane_bytes < (int64_t(24) << 20) ? 4 : 16;
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

// Launch with programmatic stream serialization (the kernels wait for their predecessor with
// griddepcontrol.wait before touching global memory).
template <typename K, typename... Args>
cudaError_t launch_pdl(K kernel, dim3 grid, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads, 1, 1);
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
    const LaunchGeom g = pick_geometry(a.ner, a.nec, int64_t(a.H) * a.W * int64_t(sizeof(TI)),
                                       device_sm_count(), occ);
    a.rpc = g.rpc;
    return launch_pdl(k, g.grid, smem, st, tm, a);
}

template <int WV, typename TB, typename TL, typename TO, bool TMA, bool ADJ = false>
cudaError_t launch_inverse_t(const CUtensorMap* tm, InvArgs a, cudaStream_t st) {
    auto k = k_inverse<WV, TB, TL, TO, TMA, ADJ>;
    constexpr size_t smem = inv_smem_bytes<TL, TB>();
    static const int occ = [&] {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        return occupancy_of(k, smem);
    }();
    const LaunchGeom g = pick_geometry(a.ner, a.nec, int64_t(a.H) * a.W * int64_t(sizeof(TL)),
                                       device_sm_count(), occ);
    a.rpc = g.rpc;
    return launch_pdl(k, g.grid, smem, st, tm[0], tm[1], tm[2], tm[3], a);
}

}  // namespace dwt2
