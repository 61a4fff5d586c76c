// dwt2_persist.cuh -- persistent kernels for batches: one launch runs every level of every image.
//
// Work list: tiles (image, level, strip, row block) in level-major ticket order (forward: level 1
// of all images, then level 2, ...; inverse: the coarsest level first).  Each CTA of a grid sized
// to the resident capacity claims tickets with an atomic counter.  Its producer warp resolves a
// ticket to its unit (one image at one level), waits until the unit it depends on (the same
// image's previous level) has completed, and streams the tile's rows into the stage ring, tagging
// each stage with the ticket; the consumer warps follow the tags, re-initialise their pipeline at
// each new tile and count completion per warp.
//
// Deadlock freedom: a tile waits only for tiles with smaller tickets, which were claimed by CTAs
// that are running (claims happen only in running CTAs) and never wait for larger tickets.
// Every wait is bounded in time; a wait that gives up records DWT2_ETIMEOUT and the CTA winds down.
#pragma once

#include "dwt2_stream.cuh"

namespace dwt2 {

// One image at one level of a batched plan (aligned like its tensor maps, which TMA reads here).
struct FwdUnit {
    CUtensorMap tm;  // input plane (when a.tma)
    FwdArgs a;
    int item_begin;  // first ticket of the unit
    int n_items;     // tiles: strips x row blocks
    int strips;
    int dep;         // unit that must complete first (-1: none)
};

struct InvUnit {
    CUtensorMap tm[4];  // LL, HL, LH, HH (when a.tma)
    InvArgs a;
    int item_begin;
    int n_items;
    int strips;
    int dep;
};

template <typename Unit>
struct PersistArgs {
    const Unit* units;
    const int* item_unit;  // ticket -> unit
    int n_items;
    int* ticket;           // claimed tickets (zero before the launch)
    int* done;             // per unit: consumer warps that finished one of its tiles (zeroed)
    int* status;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Makes data that other CTAs wrote with ordinary stores (and published with a release) visible
// to this thread's subsequent TMA (async proxy) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Waits (bounded) until *counter >= need.  On timeout raises the CTA abort flag and records
// DWT2_ETIMEOUT.
__device__ __forceinline__ bool wait_count(const int* counter, int need, volatile int* abort_flag,
                                           int* status) {
    if (ld_acquire_gpu(counter) >= need) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        __nanosleep(256);
        if (ld_acquire_gpu(counter) >= need) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitTimeoutNs) {
            *abort_flag = 1;
            if (status) atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}

// Marks one consumer warp's share of a tile done: every lane's stores are made visible at GPU
// scope before lane 0 counts the warp.
__device__ __forceinline__ void warp_done(int* counter, int lane) {
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(counter, 1);
}

// Consumer warps per CTA of the persistent kernels: the narrow CTA (180-quad tiles).  The plans'
// uneven images leave many tiles partly filled, and with it the 512-image batch ran faster on
// GB300: int 5/3 0.983 against 1.036 ms, 9/7 1.164 against 1.181 ms.  The inverse data flow
// with 16-bit bands keeps the wide CTA, whose band loads stay 16-byte aligned (see
// inv_tma_x_aligned).
constexpr int kPersistFwdNW = 3;
template <typename TB, typename TL>
constexpr int persist_inv_nw() {
    return inv_narrow_nw<TB, TL>();
}

// Geometry of one tile.
struct Tile {
    int qx0, n0, n1, nrows, qfirst;
};

template <int kVH, int NW, int WV, typename Args>
__device__ __forceinline__ Tile tile_of(const Args& a, int local, int strips) {
    Tile t;
    const int rb = local / strips, strip = local - rb * strips;
    t.qx0 = strip * cta_q<NW, WV>();
    t.n0 = rb * a.rpc;
    t.n1 = min(t.n0 + a.rpc, a.ner);
    t.nrows = t.n1 - t.n0 + 2 * kVH;
    t.qfirst = t.n0 - kVH;
    return t;
}

// Starts fetching a unit's tensor maps into the TMA unit's descriptor cache.
__device__ __forceinline__ void prefetch_unit_maps(const FwdUnit& u) {
    if (u.a.tma) prefetch_tensormap(&u.tm);
}
__device__ __forceinline__ void prefetch_unit_maps(const InvUnit& u) {
    if (u.a.tma)
        for (int k = 0; k < 4; ++k) prefetch_tensormap(&u.tm[k]);
}

// Resident CTAs per SM of the persistent kernels: the per-tile arguments they hold in registers
// do not fit the single-image kernels' 64-register budget of the 5/3 wavelets without spilling.
template <int WV>
constexpr int persist_min_ctas() {
    return (WV == WV_CDF97 || is_dd(WV)) ? 1 : 4;
}

// Plain-load path of the persistent kernels, per wavelet.  The integer 5/3 takes the single-image
// kernels' loader, one bulk copy per row and vector reads of the shifted stages: the 512-image
// batch measured 0.965 against 0.982 ms on GB300.  The 9/7 keeps 16-byte cp.async chunks and
// elementwise reads, with which it measured 1.165 against 1.179 ms.
template <int WV>
constexpr bool persist_bulk() {
    return WV == WV_CDF53_INT;
}
template <int WV>
constexpr bool persist_vec() {
    return WV == WV_CDF53_INT;
}

// Ring depth of the persistent kernels: 8 stages (the single-image depths, 6 for the 9/7 forward
// and 12 for the 5/3, made the 512-image batch 1.4% and 0.4% slower), 10 for the 9/7 forward
// data flow.  Same box, 512-image batch, default tile rows: 9/7 1.1669 -> 1.1615 ms with 10
// stages (its 5 CTAs per SM are set by registers); the int 5/3 1.0018 -> 1.0368 ms, as 10 stages
// of shared memory leave it 5 CTAs per SM instead of 6.
constexpr int kPersistStages = 8;
template <int WV>
constexpr int persist_fwd_stages() {
    return WV == WV_CDF97 ? 10 : kPersistStages;
}

// Per-tile arguments.  Each warp copies its tile's unit arguments into a local variable once per
// tile; every helper that reads them is inlined, so the compiler keeps the fields the per-row
// code uses in registers.  A copy in global or shared memory would be reloaded after every row's
// band stores and barrier operations (their memory clobbers), doubling the instructions per row.

// Producer side shared by both kernel shapes: claim the next ticket; returns -1 when the work is
// exhausted.  Waits for the ticket's dependency.
template <int NW, typename Unit>
__device__ __forceinline__ int claim(const PersistArgs<Unit>& p, volatile int* abort_flag,
                                     int lane, bool& ok) {
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(kFull, t, 0);
    ok = true;
    if (t >= p.n_items) return -1;
    const int u = __ldg(&p.item_unit[t]);
    if (lane == 0) prefetch_unit_maps(p.units[u]);  // overlaps the dependency wait
    const int dep = p.units[u].dep;
    if (dep >= 0) {
        int good = 1;
        if (lane == 0) good = wait_count(&p.done[dep], NW * p.units[dep].n_items, abort_flag, p.status);
        good = __shfl_sync(kFull, good, 0);
        if (!good) {
            ok = false;
            return -1;
        }
        fence_proxy_async_global();
    }
    return t;
}

// Producer: after the last tile (or on abort) a sentinel stage tells the consumers to stop.
template <int NS>
__device__ __forceinline__ void post_sentinel(const Ring<NS>& ring, int g, int lane, int* status) {
    const int s = g % NS;
    if (g >= NS) {
        bool ok = mbar_wait(&ring.empty[s], ((g / NS) - 1) & 1, ring.abort, status);
        if (!__all_sync(kFull, ok)) return;  // consumers are aborting anyway
    }
    if (lane == 0) {
        ring.meta[s] = -1;
        mbar_arrive(&ring.full[s]);
    }
}

template <int WV, int MODE, typename TI, typename TB, typename TL>
__global__ void __launch_bounds__(cta_threads<kPersistFwdNW>(), persist_min_ctas<WV>())
    k_forward_persistent(const PersistArgs<FwdUnit> p) {
    constexpr int kNW = kPersistFwdNW;
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    static_assert(fwd_tma_x_aligned<kNW, TI, WV>(),
                  "TMA x coordinates of this CTA width misaligned");
    constexpr bool kAdj = MODE == MODE_ADJ_INV;
    using Pipe = std::conditional_t<kAdj, AdjInvPipe<WV>, FwdPipe<WV, MODE_NONSEP>>;
    using C = typename Pipe::C;
    constexpr int kVH = vhalo<Pipe, kAdj>();
    constexpr int kS = persist_fwd_stages<WV>();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const Ring<kS> ring = make_ring<kS>(smem_raw, size_t(2) * kSRow * sizeof(TI));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    init_ring<kNW>(ring);
    __syncthreads();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        FwdArgs pargs;  // the current tile's unit arguments, held in registers (see below)
        int g = 0;
        bool bulk_used = false;  // TMA or bulk copies (async, tracked by the stage barriers)
        for (;;) {
            bool ok;
            const int t = claim<kNW>(p, ring.abort, lane, ok);
            if (t < 0) {
                if (ok) post_sentinel(ring, g, lane, p.status);
                break;
            }
            const FwdUnit& U = p.units[__ldg(&p.item_unit[t])];
            pargs = U.a;
            const Tile tl = tile_of<kVH, kNW, WV>(pargs, t - __ldg(&U.item_begin), __ldg(&U.strips));
            const int xs = 2 * tl.qx0 - kXL;
            bulk_used |= pargs.tma != 0 || (persist_bulk<WV>() && !kAdj);
            bool alive = true;
            for (int i = 0; i < tl.nrows; ++i, ++g) {
                const int s = g % kS;
                if (g >= kS) {
                    bool w = mbar_wait(&ring.empty[s], ((g / kS) - 1) & 1, ring.abort, p.status);
                    if (!__all_sync(kFull, w)) {
                        alive = false;
                        break;
                    }
                }
                if (lane == 0) ring.meta[s] = t;
                fwd_produce_row<TI, kSRow / 32, LOAD_RUNTIME, persist_bulk<WV>()>(
                                                pargs, &U.tm, kAdj, tl.qfirst + i, xs,
                                                reinterpret_cast<TI*>(ring.stage(s)),
                                                &ring.full[s], lane, 0, &ring.shift[s]);
            }
            if (!alive) break;
        }
        // Normally the consumers take every stage (the sentinel last) before the CTA can exit, so
        // all copies have landed.  After an abort, let the copies still in flight land first.  (No
        // drain otherwise: the sentinel's stage has moved one phase past its last copy.)
        if (bulk_used && lane == 0 && *ring.abort) drain_ring(ring, g, p.status);
        cp_async_wait_all();  // no-op unless this lane issued cp.async copies
        return;
    }

    // ------------------------------------------------------------------------- consumers
    FwdArgs A;  // the current tile's unit arguments, held in registers (see below)
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    int cur = -1, i = 0, unit = 0;
    Tile tl{};
    FwdCols cols;
    LaneW hw;
    bool idle = false;
    int m0 = 0;
    BandRows bands;
    Pipe pipe;
    constexpr bool kShift = kShiftable<C, MODE>;
    LevelShift sh{-0.f, -0.f};
    for (int g = 0;; ++g) {
        const int s = g % kS;
        bool ok = mbar_wait(&ring.full[s], (g / kS) & 1, ring.abort, p.status);
        if (!__all_sync(kFull, ok)) break;
        const int t = ring.meta[s];
        if (t < 0) break;
        if (t != cur) {  // first row of a new tile
            cur = t;
            unit = __ldg(&p.item_unit[t]);
            const FwdUnit* U = &p.units[unit];
            A = U->a;
            tl = tile_of<kVH, kNW, WV>(A, t - __ldg(&U->item_begin), __ldg(&U->strips));
            const int wq = tl.qx0 - kHaloQ + warp * warp_out<WV>();
            m0 = wq + kQ * lane;
            const int xs = 2 * tl.qx0 - kXL;
            cols.init(2 * m0, xs, A.W, !kAdj, (2 * wq < 0) || (2 * wq + 2 * kWarpQ > A.W));
            idle = wq + kHaloQ >= A.nec;
            if constexpr (kAdj) hw.init(m0, AxisLen{A.nec, A.ndc});
            bands.init<TB, TL>(A, tl.n0, m0, 0);
            if constexpr (kShift) {
                sh.init(A.shift, 0);
                pipe.init(sh.out_add);
            } else {
                pipe.init();
            }
            i = 0;
        }
        if (!idle) {
            QRow<C> row;
            if (A.tma)
                fwd_lane_row<TI, C>(reinterpret_cast<const TI*>(ring.stage(s)), cols, row);
            else
                fwd_lane_row_shifted<TI, C, persist_vec<WV>()>(reinterpret_cast<const TI*>(ring.stage(s)),
                                                         cols, row, ring.shift[s]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring.empty[s]);
            if constexpr (kShift) add_row(row, sh.in_add);
            if constexpr (kAdj)
                pipe.push(row, tl.qfirst + i, hw, AxisLen{A.ner, A.ndr}, A.scale);
            else
                pipe.push(row);
            const int qo = tl.qfirst + i - Pipe::kLag;
            if (qo >= tl.n0 && qo < tl.n1) {
                if (store_lane) fwd_store_bands<TB, TL>(A, bands, row, qo, m0);
                bands.next(A);
            }
        } else if (lane == 0) {
            mbar_arrive(&ring.empty[s]);
        }
        if (++i == tl.nrows) warp_done(&p.done[unit], lane);
    }
}

template <int WV, typename TB, typename TL, typename TO, bool ADJ>
__global__ void __launch_bounds__(cta_threads<persist_inv_nw<TB, TL>()>(), persist_min_ctas<WV>())
    k_inverse_persistent(const PersistArgs<InvUnit> p) {
    constexpr int kNW = persist_inv_nw<TB, TL>();
    constexpr int kHaloQ = halo_q<WV>();
    constexpr int kHaloLanes = kHaloQ / kQ;
    static_assert(inv_tma_x_aligned<kNW, TB, WV>() && inv_tma_x_aligned<kNW, TL, WV>(),
                  "TMA x coordinates of this CTA width misaligned");
    using Pipe = std::conditional_t<ADJ, AdjFwdPipe<WV>, InvPipe<WV>>;
    using C = typename Pipe::C;
    constexpr int kVH = vhalo<Pipe, ADJ>();
    constexpr size_t kStageBytes = size_t(kBRow) * (sizeof(TL) + 3 * sizeof(TB));
    constexpr int kS = kPersistStages;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const Ring<kS> ring = make_ring<kS>(smem_raw, kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    init_ring<kNW>(ring);
    __syncthreads();

    if (warp == kNW) {  // ------------------------------------------------------ producer
        InvArgs pargs;  // the current tile's unit arguments, held in registers (see below)
        int g = 0;
        bool tma_used = false;
        for (;;) {
            bool ok;
            const int t = claim<kNW>(p, ring.abort, lane, ok);
            if (t < 0) {
                if (ok) post_sentinel(ring, g, lane, p.status);
                break;
            }
            const InvUnit& U = p.units[__ldg(&p.item_unit[t])];
            pargs = U.a;
            const Tile tl = tile_of<kVH, kNW, WV>(pargs, t - __ldg(&U.item_begin), __ldg(&U.strips));
            const int xb = tl.qx0 - kXLB;
            const CUtensorMap* maps[4] = {&U.tm[0], &U.tm[1], &U.tm[2], &U.tm[3]};
            tma_used |= pargs.tma != 0;
            bool alive = true;
            for (int i = 0; i < tl.nrows; ++i, ++g) {
                const int s = g % kS;
                if (g >= kS) {
                    bool w = mbar_wait(&ring.empty[s], ((g / kS) - 1) & 1, ring.abort, p.status);
                    if (!__all_sync(kFull, w)) {
                        alive = false;
                        break;
                    }
                }
                if (lane == 0) ring.meta[s] = t;
                inv_produce_row<TL, TB>(pargs, maps, ADJ, tl.qfirst + i, xb, ring.stage(s),
                                        &ring.full[s], lane, 0);
            }
            if (!alive) break;
        }
        // Normally the consumers take every stage (the sentinel last) before the CTA can exit, so
        // all copies have landed.  After an abort, let the copies still in flight land first.  (No
        // drain otherwise: the sentinel's stage has moved one phase past its last copy.)
        if (tma_used && lane == 0 && *ring.abort) drain_ring(ring, g, p.status);
        cp_async_wait_all();  // no-op unless this lane issued cp.async copies
        return;
    }

    // ------------------------------------------------------------------------- consumers
    InvArgs A;  // the current tile's unit arguments, held in registers (see below)
    const bool store_lane = lane >= kHaloLanes && lane < 32 - kHaloLanes;
    int cur = -1, i = 0, unit = 0;
    Tile tl{};
    InvCols cols;
    LaneW hw;
    bool idle = false;
    int m0 = 0;
    char* out_p = nullptr;  // the lane's position in the output plane at the tile's next row
    Pipe pipe;
    constexpr bool kShift = !ADJ && std::is_same<C, float>::value;
    LevelShift sh{-0.f, -0.f};
    for (int g = 0;; ++g) {
        const int s = g % kS;
        bool ok = mbar_wait(&ring.full[s], (g / kS) & 1, ring.abort, p.status);
        if (!__all_sync(kFull, ok)) break;
        const int t = ring.meta[s];
        if (t < 0) break;
        if (t != cur) {  // first row of a new tile
            cur = t;
            unit = __ldg(&p.item_unit[t]);
            const InvUnit* U = &p.units[unit];
            A = U->a;
            tl = tile_of<kVH, kNW, WV>(A, t - __ldg(&U->item_begin), __ldg(&U->strips));
            const int wq = tl.qx0 - kHaloQ + warp * warp_out<WV>();
            m0 = wq + kQ * lane;
            cols.init(m0, tl.qx0 - kXLB, A.W, !ADJ, (2 * wq < 0) || (2 * wq + 2 * kWarpQ > A.W));
            idle = wq + kHaloQ >= A.nec;
            if constexpr (ADJ) hw.init(m0, AxisLen{A.nec, A.ndc});
            out_p = reinterpret_cast<char*>(row_ptr<TO>(A.out, 2 * tl.n0, 0) + 2 * m0);
            if constexpr (kShift) sh.init(A.shift, 0);
            pipe.init();
            i = 0;
        }
        if (!idle) {
            QRow<C> row;
            inv_lane_row<TL, TB, C>(ring.stage(s), cols, row);
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring.empty[s]);
            if constexpr (kShift) add_ll(row, sh.in_add);
            if constexpr (ADJ)
                pipe.push(row, tl.qfirst + i, hw, AxisLen{A.ner, A.ndr}, A.scale);
            else
                pipe.push(row);
            const int qo = tl.qfirst + i - Pipe::kLag;
            if (qo >= tl.n0 && qo < tl.n1) {
                if constexpr (kShift) add_row(row, sh.out_add);
                if (store_lane) inv_store_rows_at<TO>(A, row, qo, m0, out_p);
                out_p += 2 * A.out.pitch;
            }
        } else if (lane == 0) {
            mbar_arrive(&ring.empty[s]);
        }
        if (++i == tl.nrows) warp_done(&p.done[unit], lane);
    }
}

}  // namespace dwt2
