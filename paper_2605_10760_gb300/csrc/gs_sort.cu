// gs_sort.cu -- tile binning: key emission and a hand-written onesweep LSD radix sort.
//
// Pipeline (all stream-ordered, no host synchronisation, K read from device memory):
//   1. k_scan      single-pass inclusive scan of tiles_touched with decoupled look-back;
//                  the last partition writes K and flags K > capacity;
//   2. k_emit      one key (global tile << 32 | float bits of depth) per touched tile, tiles in
//                  row-major order, value = flattened (view, Gaussian) index; also clears that
//                  pair's backward accumulator;
//   3. k_hist      digit histograms of every 8-bit pass in one read of the keys (the scan kernel
//                  cleared the histograms, look-back words and ranges beforehand);
//   4. (each onesweep CTA turns its pass's histogram into digit start offsets itself);
//   5. k_onesweep  one launch per pass: each CTA claims the next partition of 4096 keys, ranks them
//                  stably (warp match_any + per-warp digit counters), publishes its digit counts,
//                  looks back over its predecessors' counts (bounded spins) and scatters through
//                  shared memory so that each digit run is written contiguously;
//   6. k_ranges    [start, end) of every global tile in the sorted keys, and every entry's record
//                  copied into list order (so a tile's list is one contiguous block for TMA).
// Depth is positive (z > near > 0), so its float bit pattern orders like its value, and the sort is
// stable, so equal keys keep the emission order (ascending flattened index).
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr unsigned long long kFlagAgg64 = 1ull << 62, kFlagInc64 = 2ull << 62, kVal64 = (1ull << 62) - 1;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kVal = (1u << 30) - 1;

// ------------------------------------------------------------------------------------------
// 1. inclusive scan with decoupled look-back
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan(BinArgs a) {
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_wsum[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    const long long nparts = (a.P + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.zero_for_sort) {
        // clear what the later binning kernels accumulate into (they run after this kernel)
        const long long stride = (long long)gridDim.x * blockDim.x;
        const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (long long i = t0; i < (long long)kMaxPasses * 256; i += stride) a.hist[i] = 0u;
        const long long ns = 256LL * a.sort_parts * a.passes / 4;
        uint4 *ss = reinterpret_cast<uint4 *>(a.sort_state);
        for (long long i = t0; i < ns; i += stride) ss[i] = make_uint4(0u, 0u, 0u, 0u);
        for (long long i = t0; i < 2 * a.G; i += stride) a.ranges[i] = 0u;
    }
    for (;;) {
        if (threadIdx.x == 0) s_part = atomicAdd(&a.st->ctr[kCtrScan], 1u);
        __syncthreads();
        const long long part = s_part;
        if (part >= nparts) break;
        const long long base = part * kScanTile + (long long)threadIdx.x * kScanIPT;
        uint32_t x[kScanIPT];
        if (base + kScanIPT <= a.P) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.touched + base);
#pragma unroll
            for (int q = 0; q < kScanIPT / 4; ++q) {
                uint4 u = src[q];
                x[4 * q] = u.x; x[4 * q + 1] = u.y; x[4 * q + 2] = u.z; x[4 * q + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanIPT; ++k) x[k] = (base + k < a.P) ? a.touched[base + k] : 0u;
        }
        unsigned long long tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanIPT; ++k) tsum += x[k];
        // block exclusive scan of the per-thread sums
        unsigned long long incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < kScanThreads / 32 ? s_wsum[lane] : 0ull;
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < kScanThreads / 32) s_wsum[lane] = wi - w;   // exclusive warp offsets
            const unsigned long long total = __shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
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
                s_prefix = prefix;
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
        __syncthreads();
        unsigned long long run = s_prefix + s_wsum[warp] + (incl - tsum);
        uint32_t y[kScanIPT];
#pragma unroll
        for (int k = 0; k < kScanIPT; ++k) {
            run += x[k];
            y[k] = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
        }
        if (base + kScanIPT <= a.P) {
            uint4 *dst = reinterpret_cast<uint4 *>(a.touched + base);
#pragma unroll
            for (int q = 0; q < kScanIPT / 4; ++q) dst[q] = make_uint4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < kScanIPT; ++k)
                if (base + k < a.P) a.touched[base + k] = y[k];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// 2. key emission
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kChunk) k_emit(BinArgs a) {
    const int v = blockIdx.y;
    __shared__ ViewEntry s_ve;
    if (threadIdx.x == 0) s_ve = a.views[v];
    __syncthreads();
    const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (i >= s_ve.count) return;
    const long long f = s_ve.pair_off + i;
    const uint32_t end = a.touched[f];
    const uint32_t start = f > 0 ? a.touched[f - 1] : 0u;
    if (end == start) return;
    const float4 r0 = a.proj[3 * f], r1 = a.proj[3 * f + 1];
    int x0, x1, y0, y1;
    spec_rect(r0.x, r0.y, r1.w, a.tw, a.th, (float)a.Tx, (float)a.Ty, x0, x1, y0, y1);
    const unsigned long long zbits = __float_as_uint(r1.z);
    const unsigned long long gbase = (unsigned long long)v * a.Tx * a.Ty;
    unsigned long long k = start;
    uint64_t *keys = a.keys[0];
    uint32_t *vals = a.vals[0];
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
            if (k < (unsigned long long)a.cap) {
                keys[k] = ((gbase + (unsigned long long)(ty * a.Tx + tx)) << 32) | zbits;
                vals[k] = (uint32_t)f;
            }
            ++k;
        }
    if (k != end) record_error(a.st, GS_ERR_DEVICE_FAULT, 3);
    float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    a.g2d[3 * f] = z4;
    a.g2d[3 * f + 1] = z4;
    a.g2d[3 * f + 2] = z4;
}

// ------------------------------------------------------------------------------------------
// 3./4. digit histograms
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_hist(BinArgs a) {
    __shared__ uint32_t sh[kMaxPasses][256];
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += 256) (&sh[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long K = min(a.st->num_keys, (unsigned long long)a.cap);
    const uint64_t *keys = a.keys[0];
    const int lane = threadIdx.x & 31;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * 256; i0 < K; i0 += (unsigned long long)gridDim.x * 256) {
        const unsigned long long i = i0 + threadIdx.x;
        const bool valid = i < K;
        const uint64_t key = valid ? keys[i] : 0ull;
        for (int p = 0; p < a.passes; ++p) {
            const uint32_t d = valid ? (uint32_t)((key >> (8 * p)) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&sh[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.passes * 256; i += 256) {
        uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(a.hist + i, c);
    }
}

// ------------------------------------------------------------------------------------------
// 5. onesweep pass
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
    {
        // exclusive scan of the pass's 256 digit counts, once per CTA
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const uint32_t c = a.hist[threadIdx.x];
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_tstart[warp] = incl;   // scratch: per-warp totals
        __syncthreads();
        uint32_t off = 0;
        for (int w = 0; w < warp; ++w) off += s_tstart[w];
        s_goff[threadIdx.x] = off + incl - c;
        __syncthreads();
    }
    const unsigned long long Kll = min(a.st->num_keys, (unsigned long long)a.cap);
    const uint32_t K = (uint32_t)Kll;
    const uint32_t nparts = (K + kSortTile - 1) / kSortTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = lanemask_lt();
    for (;;) {
        if (threadIdx.x == 0) {
            s_part = atomicAdd(a.ctr, 1u);
            s_bad = 0;
        }
#pragma unroll
        for (int w = 0; w < kSweepWarps; ++w) s_wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= nparts) break;
        const uint32_t base = part * kSortTile;
        const uint32_t tile_n = min((uint32_t)kSortTile, K - base);
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
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const uint32_t li = warp * (kSortIPT * 32) + r * 32 + lane;
            const uint32_t d = li < tile_n ? (uint32_t)((k[r] >> a.shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t c = d < 256u ? s_wcnt[warp][d] : 0u;
            __syncwarp();
            if (d < 256u && lane == __ffs(peers) - 1) s_wcnt[warp][d] = c + __popc(peers);
            __syncwarp();
            rk[r] = c + __popc(peers & lt_mask);
        }
        __syncthreads();
        // thread d owns digit d
        const int d = threadIdx.x;
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kSweepWarps; ++w) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = total;
            total += c;
        }
        uint32_t *my_state = a.state + (size_t)part * 256 + d;
        if (part == 0) st_relaxed_u32(my_state, kFlagInc | total);
        else st_relaxed_u32(my_state, kFlagAgg | total);
        // exclusive scan of the digit totals inside the tile
        uint32_t incl = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        // look back over the predecessors' counts of digit d
        uint32_t excl = 0;
        if (part > 0) {
            // window of kLookback predecessors loaded together, consumed nearest first until an
            // inclusive word (done) or a not-yet-published one (wait, then reload from there)
            constexpr int kLookback = 8;
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
            st_relaxed_u32(my_state, kFlagInc | ((excl + total) & kVal));
            if (timed_out) {
                s_bad = 1;
                record_error(a.st, GS_ERR_TIMEOUT, 4);
            }
        }
        __syncthreads();
        uint32_t woff = 0;
        for (int w = 0; w < warp; ++w) woff += s_wsum[w];
        const uint32_t tstart = woff + incl - total;
        s_tstart[d] = tstart;
        s_gbase[d] = s_goff[d] + excl - tstart;
        __syncthreads();
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
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// 6. tile ranges
// ------------------------------------------------------------------------------------------
__global__ void k_ranges(const uint64_t *keys, const uint32_t *vals, const float4 *proj, float4 *srec, DevStatus *st,
                         long long cap, long long G, long long P, uint32_t *ranges) {
    const unsigned long long K = min(st->num_keys, (unsigned long long)cap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long g = keys[i] >> 32;
        uint32_t f = vals[i];
        if (g >= (unsigned long long)G || f >= (uint32_t)P) {   // only after an earlier recorded failure
            record_error(st, GS_ERR_DEVICE_FAULT, 5);
            continue;
        }
        if (i == 0 || (keys[i - 1] >> 32) != g) ranges[2 * g] = (uint32_t)i;
        if (i == K - 1 || (keys[i + 1] >> 32) != g) ranges[2 * g + 1] = (uint32_t)(i + 1);
        // the entry's record in list order, so a tile's batch is one contiguous block;
        // the radius slot (used only by key emission) carries the pair index instead
        float4 r1 = proj[3 * (size_t)f + 1];
        r1.w = __uint_as_float(f);
        srec[3 * i] = proj[3 * (size_t)f];
        srec[3 * i + 1] = r1;
        srec[3 * i + 2] = proj[3 * (size_t)f + 2];
    }
}

// ------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------
static int occupancy(const void *fn, int threads, size_t dyn) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, dyn) != cudaSuccess || b < 1) b = 1;
    return b;
}

int run_scan_only(const BinArgs &a, cudaStream_t s) {
    if (cudaMemsetAsync(&a.st->ctr[kCtrScan], 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
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
    // counters of the scan and of every sort pass
    if (cudaMemsetAsync(&a.st->ctr[kCtrScan], 0, sizeof(uint32_t) * (1 + kMaxPasses), s) != cudaSuccess)
        return GS_ERR_CUDA;
    BinArgs sa = a;
    sa.zero_for_sort = 1;                 // the scan also clears hist, look-back state and ranges
    if (a.P == 0) {
        if (cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * kMaxPasses * 256, s) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaMemsetAsync(a.ranges, 0, sizeof(uint32_t) * 2 * (size_t)a.G, s) != cudaSuccess) return GS_ERR_CUDA;
    }
    int rc = run_scan_only(sa, s);
    if (rc) return rc;
    if (a.P > 0) {
        dim3 grid((unsigned)a.max_chunks, (unsigned)a.V);
        k_emit<<<grid, kChunk, 0, s>>>(a);
        count_launches(1);
    }
    const int sms = device_sm_count();
    const int hist_grid = (int)std::min<long long>(sms * 4, std::max<long long>(sms, (a.cap + 2047) / 2048));
    k_hist<<<hist_grid, 256, 0, s>>>(a);
    count_launches(1);
    const int rc2 = a.sort_ipt == kSortIPTSmall ? sweep_passes<kSortIPTSmall>(a, s) : sweep_passes<kSortIPTLarge>(a, s);
    if (rc2) return rc2;
    k_ranges<<<sms * 8, 256, 0, s>>>(a.keys[a.passes & 1], a.vals[a.passes & 1], a.proj, a.srec, a.st, a.cap, a.G,
                                      a.P, a.ranges);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
