// gs_sort.cu -- tile binning: key emission and a hand-written onesweep LSD radix sort.
//
// Pipeline (all stream-ordered, no host synchronisation, K read from device memory):
//   0. one memset clears the look-back words, the digit histograms and the tile ranges;
//   1. k_scan_emit single-pass inclusive scan of tiles_touched with decoupled look-back; as soon
//                  as a partition of pairs has its prefix, the CTA emits the partition's keys
//                  (global tile << 32 | float bits of depth, one per touched tile, tiles in
//                  row-major order, value = flattened (view, Gaussian) index), a thread per key,
//                  and counts the digits of every 8-bit pass (a shared histogram per CTA, added
//                  to the global one at the end); the last partition writes K and flags
//                  K > capacity;
//   2. (each onesweep CTA turns its pass's histogram into digit start offsets itself);
//   3. k_onesweep  one launch per pass: each CTA claims the next partition of 4096 keys, ranks them
//                  stably (warp match_any + per-warp digit counters), publishes its digit counts,
//                  places the partition in digit order in shared memory, looks back over its
//                  predecessors' counts (bounded spins) and writes each digit run contiguously;
//   4. k_ranges    [start, end) of every global tile in the sorted keys, and every entry's record
//                  copied into list order (so a tile's list is one contiguous block for TMA);
//                  As it finds each tile's list length it appends the tile to the list of its
//                  claim class (half-octave length classes: the compositing kernels claim the
//                  longest lists first).
// Depth is positive (z > near > 0), so its float bit pattern orders like its value, and the sort is
// stable, so equal keys keep the emission order (ascending flattened index).
//
// Tile-bucket binning (sort_mode GS_SORT_TILE_BUCKET) reaches the same lists without a global sort:
//   1. gs_project counted the keys of every global tile; k_scan turns the G counts into
//      inclusive slice ends and K;
//   2. k_emit_bucket drops each key, as the 64-bit word (depth bits << 32 | pair index), into its
//      tile's slice by taking slots from the slice end (an atomic decrement), which leaves every
//      count at its slice start;
//   3. k_tile_sort: one warp per tile sorts the slice ascending (bitonic network in registers or in
//      the warp's shared-memory segment; the pair index makes every word distinct, so the order is
//      exactly (depth bits, index)); slices above kWarpSortMax words go to k_tile_sort_long, one
//      CTA per tile, with slices above kTileSortMax words as sorted runs merged pairwise in global
//      memory.  Both write the tile's range, the sorted keys and values and the records in list
//      order, and append each tile to its claim class.
#include <algorithm>
#include <cstddef>

#include "gs_kernels.cuh"

namespace gs {

constexpr unsigned long long kFlagAgg64 = 1ull << 62, kFlagInc64 = 2ull << 62, kVal64 = (1ull << 62) - 1;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kVal = (1u << 30) - 1;

// ------------------------------------------------------------------------------------------
// 1. inclusive scan with decoupled look-back
// ------------------------------------------------------------------------------------------
template <int THREADS>
struct ScanShared {
    unsigned long long wsum[THREADS / 32];
    unsigned long long prefix;
};

// Global exclusive prefix of this thread's first count in partition `part`, given tsum, the sum of
// the thread's counts (threads in order).  Block scan of the per-thread sums; warp 0 publishes the
// partition total, looks back over the predecessors (a warp reads 32 at a time, the nearest
// inclusive word ends it; bounded spins) and publishes the inclusive prefix; the last partition
// writes K and checks the capacity.  Every thread runs `overlap` (work that needs no prefix) before
// the closing barrier, warp 0 after its look-back.  sh.prefix holds the partition's prefix on
// return.
template <int THREADS, class Overlap>
__device__ unsigned long long scan_partition(const BinArgs &a, ScanShared<THREADS> &sh, long long part,
                                             long long nparts, unsigned long long tsum, Overlap &&overlap) {
    static_assert(THREADS / 32 <= 32, "warp 0 scans the warp sums");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh.wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < THREADS / 32 ? sh.wsum[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) sh.wsum[lane] = wi - w;   // exclusive warp offsets
        const unsigned long long total = __shfl_sync(0xffffffffu, wi, THREADS / 32 - 1);
        const bool silent = (part == a.fault_scan_part);
        unsigned long long prefix = 0;
        if (part == 0) {
            if (lane == 0 && !silent) st_relaxed_u64(a.scan_state, kFlagInc64 | total);
        } else {
            if (lane == 0 && !silent) st_relaxed_u64(a.scan_state + part, kFlagAgg64 | total);
            // warp look-back: lane i reads predecessor j - i; the nearest inclusive word ends it
            long long j = part - 1;
            unsigned long long spins = 0;
            bool timed_out = false;
            for (;;) {
                const long long jj = j - lane;
                const unsigned long long w2 = jj >= 0 ? ld_relaxed_u64(a.scan_state + jj) : kFlagInc64;
                const unsigned long long fl = w2 & ~kVal64;
                const unsigned ready = __ballot_sync(0xffffffffu, fl != 0);
                const unsigned inc = __ballot_sync(0xffffffffu, fl == kFlagInc64);
                const int first = inc ? __ffs(inc) - 1 : 32;               // nearest inclusive lane
                const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                if ((ready & need) == need) {
                    unsigned long long v = (lane <= first) ? (w2 & kVal64) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    prefix += v;
                    if (inc) break;
                    j -= 32;
                    continue;
                }
                if (++spins > a.spin_limit) { timed_out = true; break; }
                __nanosleep(100);
            }
            if (lane == 0) {
                if (timed_out) record_error(a.st, GS_ERR_TIMEOUT, 1);
                if (!silent) st_relaxed_u64(a.scan_state + part, kFlagInc64 | ((prefix + total) & kVal64));
            }
        }
        if (lane == 0) {
            sh.prefix = prefix;
            if (part == nparts - 1) {
                const unsigned long long K = prefix + total;
                a.st->num_keys = K;
                if (K > (unsigned long long)a.cap) {
                    a.st->required_keys = K;
                    record_error(a.st, GS_ERR_CAPACITY, 2);
                }
            }
        }
    }
    overlap();   // work that needs no prefix: warps 1.. while warp 0 looks back, warp 0 after it
    __syncthreads();
    return sh.prefix + sh.wsum[warp] + (incl - tsum);
}

__device__ __forceinline__ uint32_t sat32(unsigned long long x) { return x > 0xffffffffull ? 0xffffffffu : (uint32_t)x; }

// The IPT counts of this thread (consecutive pairs from base).
template <int IPT>
__device__ __forceinline__ void scan_load(const BinArgs &a, long long base, uint32_t (&x)[IPT]) {
    if (base + IPT <= a.P) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.touched + base);
#pragma unroll
        for (int q = 0; q < IPT / 4; ++q) {
            uint4 u = src[q];
            x[4 * q] = u.x; x[4 * q + 1] = u.y; x[4 * q + 2] = u.z; x[4 * q + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < IPT; ++k) x[k] = (base + k < a.P) ? a.touched[base + k] : 0u;
    }
}

// Inclusive sums y of this thread's counts back into tiles_touched.
template <int IPT>
__device__ __forceinline__ void scan_store(const BinArgs &a, long long base, const uint32_t (&y)[IPT]) {
    if (base + IPT <= a.P) {
        uint4 *dst = reinterpret_cast<uint4 *>(a.touched + base);
#pragma unroll
        for (int q = 0; q < IPT / 4; ++q) dst[q] = make_uint4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < IPT; ++k)
            if (base + k < a.P) a.touched[base + k] = y[k];
    }
}

// Next partition of a scan or onesweep CTA (thread 0), in claim order.  A CTA whose grid covers
// every partition claims once; otherwise every CTA ends with one claim past the partitions.  The
// launch's last claim returns the counter to zero for the next launch, so the counters need no
// clearing between launches (gs_workspace_init leaves them zero).
__device__ __forceinline__ uint32_t claim_part(uint32_t *ctr, long long nparts) {
    const uint32_t c = atomicAdd(ctr, 1u);
    const long long last = nparts <= (long long)gridDim.x ? (long long)gridDim.x - 1 : nparts + gridDim.x - 1;
    if ((long long)c == last) *ctr = 0u;
    return c;
}

// Scan alone: counts -> inclusive sums in place (tile-bucket binning and the bounded-wait test).
__global__ void __launch_bounds__(kScanThreads) k_scan(BinArgs a) {
    __shared__ uint32_t s_part;
    __shared__ ScanShared<kScanThreads> sh;
    const long long nparts = (a.P + kScanTile - 1) / kScanTile;
    for (;;) {
        if (threadIdx.x == 0) s_part = claim_part(&a.st->ctr[kCtrScan], nparts);
        __syncthreads();
        const long long part = s_part;
        if (part >= nparts) break;
        const long long base = part * kScanTile + (long long)threadIdx.x * kScanIPT;
        uint32_t x[kScanIPT];
        scan_load<kScanIPT>(a, base, x);
        unsigned long long tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanIPT; ++k) tsum += x[k];
        unsigned long long run = scan_partition<kScanThreads>(a, sh, part, nparts, tsum, [] {});
        uint32_t y[kScanIPT];
#pragma unroll
        for (int k = 0; k < kScanIPT; ++k) {
            run += x[k];
            y[k] = sat32(run);
        }
        scan_store<kScanIPT>(a, base, y);
        __syncthreads();
        if (nparts <= (long long)gridDim.x) break;   // every partition was taken by a first claim
    }
}

// View of flattened pair f: the last view whose pair offset is <= f (views with no Gaussians share
// their successor's offset, so the last such view is the non-empty one holding f).
__device__ __forceinline__ int view_of_pair(const ViewEntry *views, int V, long long f) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].pair_off <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Shared memory of k_scan_emit: per pair of the partition its inclusive key end, the global tile
// of its rectangle's top-left corner, the rectangle's width and the depth bits.
struct EmitSmem {
    uint32_t inc[kScanTile];
    uint32_t g0[kScanTile];
    uint32_t wr[kScanTile];
    uint32_t z[kScanTile];
};
constexpr size_t kEmitDynSmem = sizeof(EmitSmem);

// Scan of tiles_touched with the key emission and the digit histograms of every pass.  Per
// partition of kScanTile pairs: (1) the scan; (2) a thread per pair (kEmitThreads apart, so the
// record reads coalesce) puts the pair's rectangle and depth bits in shared memory and clears its
// backward accumulator; (3) a thread per key: consecutive threads write consecutive keys, each
// finding its pair by binary search over the inclusive ends, and the digits of every pass are
// counted per warp (match_any) into the CTA's histogram.  Every loop bound is the same for the
// whole CTA.
constexpr int kEmitThreads = 1024;                 // a partition of kScanTile pairs per CTA,
constexpr int kEmitIPT = kScanTile / kEmitThreads;  // kEmitIPT consecutive counts per thread in the scan
__global__ void __launch_bounds__(kEmitThreads) k_scan_emit(BinArgs a) {
    static_assert(kEmitIPT % 4 == 0, "counts load as uint4");
    extern __shared__ __align__(16) unsigned char em_smem[];
    EmitSmem &es = *reinterpret_cast<EmitSmem *>(em_smem);
    __shared__ uint32_t s_part;
    __shared__ ScanShared<kEmitThreads> sh;
    __shared__ uint32_t s_hist[kMaxPasses][256];
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0u;
    const long long nparts = (a.P + kScanTile - 1) / kScanTile;
    const unsigned long long cap = (unsigned long long)a.cap;
    const int lane = threadIdx.x & 31;
    // the claim classes of this binning start empty (k_ranges fills them; the compositing launches
    // of the previous binning, which read them, are complete)
    if (blockIdx.x == 0 && threadIdx.x < kClaimClasses) a.st->claim_cnt[threadIdx.x] = 0u;
    for (;;) {
        if (threadIdx.x == 0) s_part = claim_part(&a.st->ctr[kCtrScan], nparts);
        __syncthreads();
        const long long part = s_part;
        if (part >= nparts) break;
        const long long pbase = part * kScanTile;
        const long long base = pbase + (long long)threadIdx.x * kEmitIPT;
        const int np = (int)min((long long)kScanTile, a.P - pbase);   // pairs in this partition
        // (1) scan; the counts also go to shared memory for (2)
        uint32_t x[kEmitIPT];
        scan_load<kEmitIPT>(a, base, x);
        unsigned long long tsum = 0;
#pragma unroll
        for (int k = 0; k < kEmitIPT; ++k) {
            tsum += x[k];
            es.inc[threadIdx.x * kEmitIPT + k] = x[k];
        }
        // (2) per pair with keys, its rectangle and depth bits: needs no prefix, so it runs while
        // warp 0 looks back over the predecessor partitions
        auto rects = [&] {
#pragma unroll
            for (int j = 0; j < kEmitIPT; ++j) {
                const int li = j * kEmitThreads + threadIdx.x;
                if (li >= np) break;
                const uint32_t cnt = es.inc[li];
                if (cnt == 0) continue;
                const long long f = pbase + li;
                const uint32_t sl = a.slot[f];      // a pair with keys is visible and holds a slot
                if (sl >= (unsigned long long)a.vcap) {   // only after an earlier recorded failure
                    record_error(a.st, GS_ERR_DEVICE_FAULT, 7);
                    continue;
                }
                const float4 r0 = a.proj[3 * (size_t)sl], r1 = a.proj[3 * (size_t)sl + 1];
                int x0, x1, y0, y1;
                spec_rect(r0.x, r0.y, r1.w, a.itw, a.ith, (float)a.Tx, (float)a.Ty, x0, x1, y0, y1);
                const int v = view_of_pair(a.views, a.V, f);
                if ((uint32_t)((x1 - x0) * (y1 - y0)) != cnt || x1 <= x0) record_error(a.st, GS_ERR_DEVICE_FAULT, 3);
                es.g0[li] = (uint32_t)((unsigned long long)v * a.Tx * a.Ty + (unsigned long long)(y0 * a.Tx + x0));
                es.wr[li] = (uint32_t)max(x1 - x0, 1);
                es.z[li] = __float_as_uint(r1.z);
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                a.g2d[3 * (size_t)sl] = z4;
                a.g2d[3 * (size_t)sl + 1] = z4;
                a.g2d[3 * (size_t)sl + 2] = z4;
            }
        };
        unsigned long long run = scan_partition<kEmitThreads>(a, sh, part, nparts, tsum, rects);
        // the counts in shared memory become inclusive sums (every read of them in (2) is done)
        uint32_t y[kEmitIPT];
#pragma unroll
        for (int k = 0; k < kEmitIPT; ++k) {
            run += x[k];
            y[k] = sat32(run);
            es.inc[threadIdx.x * kEmitIPT + k] = y[k];
        }
        scan_store<kEmitIPT>(a, base, y);
        const uint32_t pstart = sat32(sh.prefix);
        __syncthreads();
        const uint32_t pend = es.inc[np - 1];
        // (3) per key, up to the capacity (< 2^30, so the counter cannot wrap even when the sums
        // saturated); keys at or beyond it are neither written nor counted
        const uint32_t kend = (uint32_t)min((unsigned long long)pend, cap);
        for (uint32_t k0 = pstart; k0 < kend; k0 += kEmitThreads) {
            const uint32_t kk = k0 + threadIdx.x;
            const bool valid = kk < kend;
            unsigned long long key = 0;
            if (valid) {
                // the pair: smallest li with inc[li] > kk (pairs without keys repeat their end)
                int lo = 0, hi = np - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (es.inc[mid] > kk) hi = mid;
                    else lo = mid + 1;
                }
                const uint32_t m = kk - (lo ? es.inc[lo - 1] : pstart);
                const uint32_t w = es.wr[lo];
                const uint32_t row = m / w;
                const unsigned long long g = (unsigned long long)es.g0[lo] + (unsigned long long)row * a.Tx + (m - row * w);
                key = (g << 32) | es.z[lo];
                a.keys[0][kk] = key;
                a.vals[0][kk] = (uint32_t)(pbase + lo);
            }
            for (int p = 0; p < a.passes; ++p) {
                const uint32_t dg = valid ? (uint32_t)((key >> (8 * p)) & 255u) : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, dg);
                if (dg < 256u && lane == __ffs(peers) - 1) atomicAdd(&s_hist[p][dg], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        if (nparts <= (long long)gridDim.x) break;   // every partition was taken by a first claim
    }
    for (int i = threadIdx.x; i < a.passes * 256; i += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(a.hist + i, c);
    }
}

// ------------------------------------------------------------------------------------------
// 3. onesweep pass
// ------------------------------------------------------------------------------------------
struct SweepArgs {
    const uint64_t *kin;
    const uint32_t *vin;
    uint64_t *kout;
    uint32_t *vout;
    const uint32_t *hist;        // [256] digit counts of this pass over all keys
    uint32_t *state;             // [parts][256]
    uint32_t *ctr;
    DevStatus *st;
    long long cap;
    int shift;
    unsigned long long spin_limit;
};

constexpr int kSweepWarps = kSortThreads / 32;
template <int IPT>
constexpr size_t sweep_dyn_smem() { return (size_t)kSortThreads * IPT * (sizeof(uint64_t) + sizeof(uint32_t)); }

// Predecessors whose digit words one look-back round loads together.  A partition's keys, values
// and ranks already sit in shared memory when it looks back, so the window costs registers only
// while it is consumed; a window this wide lets a partition of a small sort (tens of partitions,
// all running at once) add up every predecessor's published count in one or two rounds.
constexpr int kLookback = 32;

template <int IPT>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(SweepArgs a) {
    constexpr int kSortIPT = IPT;
    constexpr int kSortTile = kSortThreads * IPT;
    extern __shared__ __align__(16) unsigned char sw_smem[];
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(sw_smem);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kSortTile);
    __shared__ uint32_t s_wcnt[kSweepWarps][256];
    __shared__ uint32_t s_tstart[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_wsum[kSweepWarps];
    __shared__ uint32_t s_part;
    __shared__ int s_bad;
    __shared__ uint32_t s_goff[256];      // exclusive global start of each digit in this pass
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the first partition is claimed while the pass histogram is read and scanned
    if (threadIdx.x == 0) {
        s_part = atomicAdd(a.ctr, 1u);
        s_bad = 0;
    }
#pragma unroll
    for (int w = 0; w < kSweepWarps; ++w) s_wcnt[w][threadIdx.x] = 0;
    {
        // exclusive scan of the pass's 256 digit counts, once per CTA
        const uint32_t c = a.hist[threadIdx.x];
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t off = 0;
        for (int w = 0; w < warp; ++w) off += s_wsum[w];
        s_goff[threadIdx.x] = off + incl - c;
        __syncthreads();
    }
    const unsigned long long Kll = min(a.st->num_keys, (unsigned long long)a.cap);
    const uint32_t K = (uint32_t)Kll;
    const uint32_t nparts = (K + kSortTile - 1) / kSortTile;
    const unsigned lt_mask = lanemask_lt();
    {   // the first claim, made before nparts was known, may be the launch's last one (claim_part)
        const long long last =
            (long long)nparts <= (long long)gridDim.x ? (long long)gridDim.x - 1 : (long long)nparts + gridDim.x - 1;
        if (threadIdx.x == 0 && (long long)s_part == last) *a.ctr = 0u;
    }
    for (;;) {
        const uint32_t part = s_part;
        if (part >= nparts) break;
        const uint32_t base = part * kSortTile;
        const uint32_t tile_n = min((uint32_t)kSortTile, K - base);
        const int d = threadIdx.x;            // thread d owns digit d from the digit totals on
        uint32_t total = 0, tstart = 0;
        {
            uint64_t k[kSortIPT];
            uint32_t val[kSortIPT];
            uint32_t rk[kSortIPT];
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = warp * (kSortIPT * 32) + r * 32 + lane;
                const bool valid = li < tile_n;
                k[r] = valid ? a.kin[base + li] : 0ull;
                val[r] = valid ? a.vin[base + li] : 0u;
            }
            // stable rank inside the warp: match_any groups equal digits, per-warp digit counters
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = warp * (kSortIPT * 32) + r * 32 + lane;
                const uint32_t dg = li < tile_n ? (uint32_t)((k[r] >> a.shift) & 255u) : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, dg);
                const uint32_t c = dg < 256u ? s_wcnt[warp][dg] : 0u;
                __syncwarp();
                if (dg < 256u && lane == __ffs(peers) - 1) s_wcnt[warp][dg] = c + __popc(peers);
                __syncwarp();
                rk[r] = c + __popc(peers & lt_mask);
            }
            __syncthreads();
#pragma unroll
            for (int w = 0; w < kSweepWarps; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = total;
                total += c;
            }
            // publish this partition's digit count before anything else, for the successors
            st_relaxed_u32(a.state + (size_t)part * 256 + d, (part == 0 ? kFlagInc : kFlagAgg) | total);
            // exclusive scan of the digit totals inside the partition
            uint32_t incl = total;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            uint32_t woff = 0;
            for (int w = 0; w < warp; ++w) woff += s_wsum[w];
            tstart = woff + incl - total;
            s_tstart[d] = tstart;
            __syncthreads();
            // local scatter: the partition in digit order in shared memory (needs no global offset)
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = warp * (kSortIPT * 32) + r * 32 + lane;
                if (li < tile_n) {
                    const uint32_t dd = (uint32_t)((k[r] >> a.shift) & 255u);
                    const uint32_t lp = s_tstart[dd] + s_wcnt[warp][dd] + rk[r];
                    s_keys[lp] = k[r];
                    s_vals[lp] = val[r];
                }
            }
        }
        // look back over the predecessors' counts of digit d: a window of kLookback words loaded
        // together, consumed nearest first until an inclusive word (done) or a not-yet-published
        // one (wait, then reload from there); every wait is bounded
        uint32_t excl = 0;
        if (part > 0) {
            int j = (int)part - 1;
            unsigned long long spins = 0;
            bool timed_out = false;
            for (;;) {
                uint32_t w[kLookback];
#pragma unroll
                for (int q = 0; q < kLookback; ++q)
                    w[q] = (j - q >= 0) ? ld_relaxed_u32(a.state + (size_t)(j - q) * 256 + d) : kFlagInc;
                bool found = false, stop = false;
                int adv = 0;
#pragma unroll
                for (int q = 0; q < kLookback; ++q) {
                    if (!stop) {
                        const uint32_t fl = w[q] & ~kVal;
                        if (fl == 0u) {
                            stop = true;
                        } else {
                            excl += w[q] & kVal;
                            ++adv;
                            if (fl == kFlagInc) found = stop = true;
                        }
                    }
                }
                if (found) break;
                j -= adv;
                if (stop) {
                    if (++spins > a.spin_limit) { timed_out = true; break; }
                    __nanosleep(64);
                }
            }
            st_relaxed_u32(a.state + (size_t)part * 256 + d, kFlagInc | ((excl + total) & kVal));
            if (timed_out) {
                s_bad = 1;
                record_error(a.st, GS_ERR_TIMEOUT, 4);
            }
        }
        s_gbase[d] = s_goff[d] + excl - tstart;
        __syncthreads();
        if (!s_bad) {
            for (uint32_t i = threadIdx.x; i < tile_n; i += kSortThreads) {
                const uint64_t key = s_keys[i];
                const uint32_t dd = (uint32_t)((key >> a.shift) & 255u);
                const uint32_t gp = s_gbase[dd] + i;
                if (gp < K) {
                    a.kout[gp] = key;
                    a.vout[gp] = s_vals[i];
                }
            }
        }
        // a grid that covers every partition claimed them all with its first claims: leave without
        // another claim round trip
        if (nparts <= gridDim.x) break;
        __syncthreads();
        // next partition; the per-warp digit counters start from zero again
        if (threadIdx.x == 0) {
            s_part = claim_part(a.ctr, (long long)nparts);
            s_bad = 0;
        }
#pragma unroll
        for (int w = 0; w < kSweepWarps; ++w) s_wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// 4. claim classes of the compositing kernels' work items
// ------------------------------------------------------------------------------------------
// The persistent compositing kernels claim (view, tile) items from a counter.  Claimed in tile
// order, a long list taken near the end keeps its CTA running after the others have finished;
// claimed longest first, the last items are the short ones.  So every item is appended, once its
// list length is known, to the list of its claim class (half-octave length classes, class 0 the
// longest), and the kernels claim class by class.  The position inside a class is arbitrary: the
// order moves no result, only when each tile is composited.
__device__ __forceinline__ int claim_class(uint32_t n) {
    const int e = 31 - __clz(n | 1u);
    if (e > 15) return 0;
    const int half = e >= 1 ? (int)((n >> (e - 1)) & 1u) : 0;
    return kClaimClasses - 1 - (2 * e + half);
}

// items first .. first + count - 1 into class c's list (one atomic for the run)
__device__ __forceinline__ void claim_append(DevStatus *st, uint32_t *clist, long long G, int c, long long first,
                                             long long count) {
    const unsigned long long pos = atomicAdd(&st->claim_cnt[c], (uint32_t)count);
    if ((long long)pos + count > G) {   // only after an earlier failure (an item listed twice)
        record_error(st, GS_ERR_DEVICE_FAULT, 12);
        return;
    }
    uint32_t *dst = clist + (size_t)c * G + pos;
    for (long long j = 0; j < count; ++j) dst[j] = (uint32_t)(first + j);
}

// ------------------------------------------------------------------------------------------
// 5. tile ranges
// ------------------------------------------------------------------------------------------
constexpr int kRangesThreads = 256;
__global__ void __launch_bounds__(kRangesThreads) k_ranges(const uint64_t *keys, const uint32_t *vals,
                                                           const float4 *proj, const uint32_t *slot, long long vcap,
                                                           float4 *srec, DevStatus *st, long long cap, long long G,
                                                           long long P, uint32_t *ranges, unsigned long long *tword,
                                                           uint32_t *clist) {
    const unsigned long long K = min(st->num_keys, (unsigned long long)cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // the compositing launches on this binning count anew
        st->fwd_pairs = 0ull;
        st->bwd_pairs = 0ull;
    }
    if (K == 0) {   // every tile empty: all in the last claim class, in tile order
        for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x)
            clist[(size_t)(kClaimClasses - 1) * G + g] = (uint32_t)g;
        if (blockIdx.x == 0 && threadIdx.x == 0) st->claim_cnt[kClaimClasses - 1] = (uint32_t)G;
        return;
    }
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long g = keys[i] >> 32;
        uint32_t f = vals[i];
        if (g >= (unsigned long long)G || f >= (uint32_t)P) {   // only after an earlier recorded failure
            record_error(st, GS_ERR_DEVICE_FAULT, 5);
            continue;
        }
        const bool first = i == 0 || (keys[i - 1] >> 32) != g;
        const unsigned long long gn = i == K - 1 ? (unsigned long long)G : keys[i + 1] >> 32;
        const bool last = gn != g;
        if (first) ranges[2 * g] = (uint32_t)i;
        if (last) ranges[2 * g + 1] = (uint32_t)(i + 1);
        // claim class of the tile: the thread at its first entry and the one at its last add
        // (1 << 56) + 2^33 - start and (1 << 56) + end to the tile's word; the second one to add
        // sees one arrival in the top bits and takes n = end - start from the sum
        if (first && last) {
            claim_append(st, clist, G, claim_class(1u), (long long)g, 1);
        } else if (first || last) {
            const unsigned long long mine = (1ull << 56) + (first ? (1ull << 33) - i : i + 1);
            const unsigned long long old = atomicAdd(&tword[g], mine);
            if ((old >> 56) == 1ull) {
                const unsigned long long n = ((old + mine) & ((1ull << 56) - 1)) - (1ull << 33);
                claim_append(st, clist, G, claim_class((uint32_t)min(n, 0xffffffffull)), (long long)g, 1);
            }
        }
        // empty tiles: those between this tile and the next key's (or the end), and before the first key
        if (last && gn > g + 1)
            claim_append(st, clist, G, kClaimClasses - 1, (long long)g + 1, (long long)(gn - g - 1));
        if (i == 0 && g > 0) claim_append(st, clist, G, kClaimClasses - 1, 0, (long long)g);
        // the entry's record in list order, so a tile's batch is one contiguous block;
        // the radius field (used only by key emission) carries the pair's slot instead
        const uint32_t sl = slot[f];
        if (sl >= (unsigned long long)vcap) {   // only after an earlier recorded failure
            record_error(st, GS_ERR_DEVICE_FAULT, 8);
            continue;
        }
        float4 r1 = proj[3 * (size_t)sl + 1];
        r1.w = __uint_as_float(sl);
        srec[3 * i] = proj[3 * (size_t)sl];
        srec[3 * i + 1] = r1;
        srec[3 * i + 2] = proj[3 * (size_t)sl + 2];
    }
}

// ------------------------------------------------------------------------------------------
// tile-bucket binning
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kChunk) k_emit_bucket(BinArgs a) {
    const int v = blockIdx.y;
    __shared__ ViewEntry s_ve;
    if (threadIdx.x == 0) s_ve = a.views[v];
    __syncthreads();
    if ((long long)blockIdx.x * kChunk >= s_ve.count) return;   // whole block past the view
    const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
    const long long f = s_ve.pair_off + (i < s_ve.count ? i : 0);
    const uint32_t sl = i < s_ve.count ? a.slot[f] : kNoSlot;
    const bool vis = i < s_ve.count && a.touched[f] != 0u && sl < (unsigned long long)a.vcap;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    unsigned long long word = 0;
    if (vis) {
        const float4 r0 = a.proj[3 * (size_t)sl], r1 = a.proj[3 * (size_t)sl + 1];
        spec_rect(r0.x, r0.y, r1.w, a.itw, a.ith, (float)a.Tx, (float)a.Ty, x0, x1, y0, y1);
        word = ((unsigned long long)__float_as_uint(r1.z) << 32) | (unsigned long long)(uint32_t)f;
    }
    uint64_t *keys = a.keys[0];
    const long long cap = a.cap;
    // slots from the end of each touched tile's slice; the atomics of up to kEmitBatch tiles are in
    // flight together before their stores
    constexpr int kEmitBatch = 4;
    uint32_t *row = a.tile_cnt + (size_t)v * a.Tx * a.Ty;
    const int n = vis ? (x1 - x0) * (y1 - y0) : 0;
    int tx = x0, ty = y0;
    for (int t0 = 0; t0 < n; t0 += kEmitBatch) {
        uint32_t slot[kEmitBatch];
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u) {
            slot[u] = 0xffffffffu;
            if (t0 + u < n) {
                slot[u] = atomicSub(row + ty * a.Tx + tx, 1u) - 1u;
                if (++tx == x1) {
                    tx = x0;
                    ++ty;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kEmitBatch; ++u)
            if (t0 + u < n && (long long)slot[u] < cap) keys[slot[u]] = word;
    }
    if (vis) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        a.g2d[3 * (size_t)sl] = z4;
        a.g2d[3 * (size_t)sl + 1] = z4;
        a.g2d[3 * (size_t)sl + 2] = z4;
    }
}

constexpr int kTileSortThreads = 256;
constexpr int kTileSortMax = 4096;      // words sorted in shared memory by one CTA (32 KB)
constexpr int kWarpSortMax = 128;       // words sorted in shared memory by one warp (1 KB)

// Ascending bitonic sort of b[0, m), m a power of two, by the whole block.
__device__ __forceinline__ void block_bitonic(unsigned long long *b, int m) {
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));   // i has bit j clear
                const int l = i | j;
                const unsigned long long x = b[i], y = b[l];
                const bool up = (i & k) == 0;
                if ((x > y) == up) {
                    b[i] = y;
                    b[l] = x;
                }
            }
            __syncthreads();
        }
}

// The same network run by one warp on its own segment (m <= kWarpSortMax).
__device__ __forceinline__ void warp_bitonic(unsigned long long *b, int m, int lane) {
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (m >> 1); t += 32) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const int l = i | j;
                const unsigned long long x = b[i], y = b[l];
                const bool up = (i & k) == 0;
                if ((x > y) == up) {
                    b[i] = y;
                    b[l] = x;
                }
            }
            __syncwarp();
        }
}

// 32 words, one per lane, sorted ascending across the warp in registers.
__device__ __forceinline__ unsigned long long warp_bitonic32(unsigned long long x, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
            const bool lower = (lane & j) == 0, up = (lane & k) == 0;
            x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
        }
    return x;
}

// Number of entries of the ascending run r[0, n) that are smaller than x.
__device__ __forceinline__ long long count_below(const unsigned long long *r, long long n, unsigned long long x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (r[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The slice [s, e) of tile g (clamped to the capacity) and its published range.
__device__ __forceinline__ void tile_slice(const BinArgs &a, long long g, long long &s, long long &n) {
    const unsigned long long K = a.st->num_keys;
    const unsigned long long cap = (unsigned long long)a.cap;
    const unsigned long long s0 = a.tile_cnt[g];
    const unsigned long long e0 = g + 1 < a.G ? a.tile_cnt[g + 1] : K;
    s = (long long)min(s0, cap);
    n = (long long)max((unsigned long long)s, min(e0, cap)) - s;
}

// Outputs of one sorted entry: key (tile << 32 | depth bits), value, record in list order.
__device__ __forceinline__ void tile_emit(const BinArgs &a, uint64_t *kout, uint32_t *vout, long long g, long long pos,
                                          unsigned long long w) {
    const uint32_t f = (uint32_t)w;
    if ((long long)f >= a.P) {   // only after an earlier recorded failure
        record_error(a.st, GS_ERR_DEVICE_FAULT, 6);
        return;
    }
    kout[pos] = ((unsigned long long)g << 32) | (w >> 32);
    vout[pos] = f;
    const uint32_t sl = a.slot[f];
    if (sl >= (unsigned long long)a.vcap) {   // only after an earlier recorded failure
        record_error(a.st, GS_ERR_DEVICE_FAULT, 9);
        return;
    }
    float4 r1 = a.proj[3 * (size_t)sl + 1];
    r1.w = __uint_as_float(sl);
    a.srec[3 * pos] = a.proj[3 * (size_t)sl];
    a.srec[3 * pos + 1] = r1;
    a.srec[3 * pos + 2] = a.proj[3 * (size_t)sl + 2];
}

// One warp per tile: every warp claims tiles from a counter, publishes the tile's range and sorts
// slices of up to kWarpSortMax words itself (registers for 32 or fewer, its shared-memory segment
// otherwise); longer slices are appended to the list of long tiles for k_tile_sort_long.
__global__ void __launch_bounds__(kTileSortThreads) k_tile_sort(BinArgs a) {
    __shared__ unsigned long long seg[kTileSortThreads / 32][kWarpSortMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *b = seg[warp];
    uint64_t *kout = a.keys[a.passes & 1];
    uint32_t *vout = a.vals[a.passes & 1];
    const unsigned long long *words = reinterpret_cast<const unsigned long long *>(a.keys[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // the compositing launches on this binning count anew
        a.st->fwd_pairs = 0ull;
        a.st->bwd_pairs = 0ull;
    }
    for (;;) {
        long long g = 0;
        if (lane == 0) g = (long long)atomicAdd(&a.st->ctr[kCtrTileSort], 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= a.G) break;
        long long s, n;
        tile_slice(a, g, s, n);
        if (lane == 0) {   // an empty tile reads [0, 0), as the onesweep path leaves it
            a.ranges[2 * g] = n > 0 ? (uint32_t)s : 0u;
            a.ranges[2 * g + 1] = n > 0 ? (uint32_t)(s + n) : 0u;
            claim_append(a.st, a.clist, a.G, claim_class((uint32_t)n), g, 1);
        }
        if (n == 0) continue;
        if (n > kWarpSortMax) {
            if (lane == 0) a.tile_list[atomicAdd(&a.st->ctr[kCtrTileList], 1u)] = (uint32_t)g;
            continue;
        }
        if (n <= 32) {
            const unsigned long long x = warp_bitonic32(lane < n ? words[s + lane] : ~0ull, lane);
            if (lane < n) tile_emit(a, kout, vout, g, s + lane, x);
            continue;
        }
        int m = 64;
        while (m < n) m <<= 1;
        for (int i = lane; i < m; i += 32) b[i] = i < n ? words[s + i] : ~0ull;
        __syncwarp();
        warp_bitonic(b, m, lane);
        for (int i = lane; i < n; i += 32) tile_emit(a, kout, vout, g, s + i, b[i]);
        __syncwarp();
    }
}

// One CTA per long tile (more than kWarpSortMax words) from the list built by k_tile_sort: a
// shared-memory bitonic sort up to kTileSortMax words, beyond that sorted runs merged pairwise
// between this tile's slices of the two key buffers.
__global__ void __launch_bounds__(kTileSortThreads) k_tile_sort_long(BinArgs a) {
    __shared__ unsigned long long b[kTileSortMax];
    __shared__ long long s_item;
    uint64_t *kout = a.keys[a.passes & 1];
    uint32_t *vout = a.vals[a.passes & 1];
    const long long count = a.st->ctr[kCtrTileList];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&a.st->ctr[kCtrTileLong], 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= count) break;
        const long long g = a.tile_list[item];
        long long s, n;
        tile_slice(a, g, s, n);
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.keys[0] + s);
        if (n > kTileSortMax) {
            // sorted runs of kTileSortMax words, in place
            for (long long r0 = 0; r0 < n; r0 += kTileSortMax) {
                const int len = (int)min((long long)kTileSortMax, n - r0);
                for (int i = threadIdx.x; i < kTileSortMax; i += blockDim.x) b[i] = i < len ? src[r0 + i] : ~0ull;
                __syncthreads();
                block_bitonic(b, kTileSortMax);
                for (int i = threadIdx.x; i < len; i += blockDim.x) a.keys[0][s + r0 + i] = b[i];
                __syncthreads();
            }
            // pairwise merges between the two key buffers (this tile's slice of each)
            unsigned long long *in = reinterpret_cast<unsigned long long *>(a.keys[0] + s);
            unsigned long long *out = reinterpret_cast<unsigned long long *>(a.keys[1] + s);
            for (long long w = kTileSortMax; w < n; w <<= 1) {
                for (long long i = threadIdx.x; i < n; i += blockDim.x) {
                    const long long base = (i / (2 * w)) * (2 * w);
                    const long long aend = min(base + w, n), bend = min(base + 2 * w, n);
                    const unsigned long long x = in[i];
                    const long long pos = i < aend ? (i - base) + count_below(in + aend, bend - aend, x)
                                                   : (i - aend) + count_below(in + base, aend - base, x);
                    out[base + pos] = x;
                }
                __syncthreads();
                unsigned long long *t = in;
                in = out;
                out = t;
            }
            src = in;
        } else {
            int m = 1;
            while (m < n) m <<= 1;
            for (int i = threadIdx.x; i < m; i += blockDim.x) b[i] = i < n ? src[i] : ~0ull;
            __syncthreads();
            block_bitonic(b, m);
            src = b;
        }
        for (long long i = threadIdx.x; i < n; i += blockDim.x) tile_emit(a, kout, vout, g, s + i, src[i]);
        __syncthreads();
    }
}

static int occupancy(const void *fn, int threads, size_t dyn);
static int run_scan(const BinArgs &a, cudaStream_t s, bool counter_cleared);

static int run_bucket(const BinArgs &a, cudaStream_t s) {
    // counters of the scan and of the per-tile sort, and the claim-class counts
    static_assert(offsetof(DevStatus, claim_cnt) == offsetof(DevStatus, ctr) + sizeof(uint32_t) * kNumCounters,
                  "the claim-class counts follow the counters");
    if (cudaMemsetAsync(&a.st->ctr[kCtrScan], 0, sizeof(uint32_t) * (kNumCounters + kClaimClasses), s) != cudaSuccess)
        return GS_ERR_CUDA;
    // inclusive scan of the G tile counts (K and the capacity check come with it)
    BinArgs sa = a;
    sa.touched = a.tile_cnt;
    sa.P = a.G;
    int rc = run_scan(sa, s, true);   // run_bin_sort cleared the scan counter
    if (rc) return rc;
    if (a.P > 0) {
        dim3 grid((unsigned)a.max_chunks, (unsigned)a.V);
        k_emit_bucket<<<grid, kChunk, 0, s>>>(a);
        count_launches(1);
    }
    static int occ = occupancy((const void *)k_tile_sort, kTileSortThreads, 0);
    const long long tiles_per_block = kTileSortThreads / 32;
    const long long grid = std::max<long long>(
        1, std::min<long long>((a.G + tiles_per_block - 1) / tiles_per_block, (long long)device_sm_count() * occ));
    k_tile_sort<<<(unsigned)grid, kTileSortThreads, 0, s>>>(a);
    static int occ_long = occupancy((const void *)k_tile_sort_long, kTileSortThreads, 0);
    k_tile_sort_long<<<(unsigned)std::max(1, device_sm_count() * occ_long), kTileSortThreads, 0, s>>>(a);
    count_launches(2);
    return check_launch();
}

// ------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------
static int occupancy(const void *fn, int threads, size_t dyn) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, dyn) != cudaSuccess || b < 1) b = 1;
    return b;
}

static int run_scan(const BinArgs &a, cudaStream_t s, bool counter_cleared) {
    if (!counter_cleared && cudaMemsetAsync(&a.st->ctr[kCtrScan], 0, sizeof(uint32_t), s) != cudaSuccess)
        return GS_ERR_CUDA;
    const long long parts = (a.P + kScanTile - 1) / kScanTile;
    if (parts > 0) {
        if (cudaMemsetAsync(a.scan_state, 0, sizeof(unsigned long long) * parts, s) != cudaSuccess) return GS_ERR_CUDA;
        static int occ = occupancy((const void *)k_scan, kScanThreads, 0);
        long long grid = std::min<long long>(parts, (long long)device_sm_count() * occ);
        k_scan<<<(unsigned)grid, kScanThreads, 0, s>>>(a);
        count_launches(1);
    } else {
        // no pairs: K = 0
        if (cudaMemsetAsync(&a.st->num_keys, 0, sizeof(unsigned long long), s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return check_launch();
}

int run_scan_only(const BinArgs &a, cudaStream_t s) { return run_scan(a, s, false); }

template <int IPT>
static int sweep_passes(const BinArgs &a, cudaStream_t s) {
    static bool attr = [] {
        return cudaFuncSetAttribute((const void *)k_onesweep<IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep_dyn_smem<IPT>()) == cudaSuccess;
    }();
    if (!attr) return GS_ERR_CUDA;
    static int occ = occupancy((const void *)k_onesweep<IPT>, kSortThreads, sweep_dyn_smem<IPT>());
    const int sms = device_sm_count();
    const long long grid = std::max<long long>(1, std::min<long long>(a.sort_parts, (long long)sms * occ));
    for (int p = 0; p < a.passes; ++p) {
        SweepArgs sa;
        sa.kin = a.keys[p & 1];
        sa.vin = a.vals[p & 1];
        sa.kout = a.keys[(p + 1) & 1];
        sa.vout = a.vals[(p + 1) & 1];
        sa.hist = a.hist + 256 * p;
        sa.state = a.sort_state + (size_t)256 * a.sort_parts * p;
        sa.ctr = &a.st->ctr[kCtrSort0 + p];
        sa.st = a.st;
        sa.cap = a.cap;
        sa.shift = 8 * p;
        sa.spin_limit = a.spin_limit;
        k_onesweep<IPT><<<(unsigned)grid, kSortThreads, sweep_dyn_smem<IPT>(), s>>>(sa);
        count_launches(1);
    }
    return GS_OK;
}

int run_bin_sort(const BinArgs &a, cudaStream_t s) {
    // (the onesweep path's claim counters return to zero at the end of every launch and k_scan_emit
    // clears the claim-class counts: no memset for them)
    if (a.sort_mode == GS_SORT_TILE_BUCKET) return run_bucket(a, s);
    // look-back words of the scan and of every pass, digit histograms and tile ranges
    if (cudaMemsetAsync(a.clear_begin, 0, a.clear_bytes, s) != cudaSuccess) return GS_ERR_CUDA;
    const int sms = device_sm_count();
    const long long parts = (a.P + kScanTile - 1) / kScanTile;
    if (parts > 0) {
        static bool attr = cudaFuncSetAttribute((const void *)k_scan_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)kEmitDynSmem) == cudaSuccess;
        if (!attr) return GS_ERR_CUDA;
        static int occ = occupancy((const void *)k_scan_emit, kEmitThreads, kEmitDynSmem);
        const long long grid = std::min<long long>(parts, (long long)sms * occ);
        k_scan_emit<<<(unsigned)grid, kEmitThreads, kEmitDynSmem, s>>>(a);
        count_launches(1);
    } else {   // no pairs: K = 0, and the claim classes start empty (k_scan_emit clears them otherwise)
        if (cudaMemsetAsync(&a.st->num_keys, 0, sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemsetAsync(a.st->claim_cnt, 0, sizeof(uint32_t) * kClaimClasses, s) != cudaSuccess)
            return GS_ERR_CUDA;
    }
    const int rc2 = sweep_passes<kSortIPT>(a, s);
    if (rc2) return rc2;
    k_ranges<<<sms * 8, kRangesThreads, 0, s>>>(a.keys[a.passes & 1], a.vals[a.passes & 1], a.proj, a.slot, a.vcap,
                                                 a.srec, a.st, a.cap, a.G, a.P, a.ranges, a.tword, a.clist);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
