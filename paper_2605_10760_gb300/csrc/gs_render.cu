// gs_render.cu -- per-tile compositing (forward) and its adjoint (backward).
//
// One CTA = one tile of TW x TH pixels, two vertically adjacent pixels per thread; a warp covers a
// square 8 x 8 block of the tile (lanes 8 wide, 4 tall, 2 pixels each), the shape whose bounding
// box a footprint overlaps least, which keeps the per-warp region masks selective.  Both kernels are persistent: a grid of (#SM x resident
// CTAs) claims (view, tile) work items from a device counter, so one launch covers every tile of
// every view of every scene, whatever the per-tile list lengths.
//
// Staging: a tile's list is a contiguous block of records (gs_bin_sort writes them in list order),
// so each batch of TW*TH records is one TMA bulk copy (cp.async.bulk) issued by one thread into one
// of two shared-memory buffers and completed on that buffer's mbarrier; the next batch is copied
// while the current one is processed.  All mbarrier waits are bounded (error + drain + return).
//
// Forward: each thread walks the staged records front to back for its two pixels taking the FP32
// decisions of the decision chain (sigma < 0 skip, alpha < alpha_min skip, stop before blending
// when T (1 - alpha) < t_min).  The CTA leaves the list once every pixel has stopped.  Each record
// carries a cut-off sigma_cut = ln(o / alpha_min) + 1e-3: for sigma > sigma_cut the exponential is
// not evaluated because alpha < alpha_min is certain (the decision-chain exp is within 2 ulp of
// e^x), so every decision is exactly the one the full test takes.
//
// Backward: from final_T and last_idx of each pixel the CTA walks the list back to front,
// recovering T_j = T_{j+1} / (1 - alpha_j) and one running scalar Q (the upstream-weighted colour
// and depth accumulated behind each entry, with the background and alpha-output terms), so no
// per-pixel list is stored.  Each thread sums the 10 per-Gaussian gradient components of its two
// pixels, then the warp reduces them with a transposed butterfly (12 shuffles instead of 50) after
// which 20 lanes issue one atomic add each (two halves per component): a (Gaussian, warp) pair
// costs one warp-wide atomic instruction; warps whose 64 pixels all skip the entry issue nothing, and entries past the
// warp's last blended position are not visited at all.
//
// In both kernels each warp drops the entries whose region bit is clear 32 at a time (a ballot
// over the mask bytes) and visits only the rest.  A thread's two pixels are the two components of
// packed FP32x2 arithmetic (one instruction for both pixels, each component rounded exactly as
// the scalar operation, so the decision chain is unchanged bit for bit); the decisions
// themselves are scalar compares and selects.  The forward can also evaluate the L1 terms of
// the mapping loss and their gradient in its per-pixel epilogue (gs_render_fwd_l1).
#include "gs_kernels.cuh"

namespace gs {

constexpr int kPPT = 2;   // pixels per thread
constexpr int kWX = 8;    // warp block: kWX columns x (32 / kWX) * kPPT rows
constexpr int kWY = 32 / kWX * kPPT;

// Pixel of a thread inside its tile: warp w takes block (w mod (TW / kWX), w div (TW / kWX)).
template <int TW>
__device__ __forceinline__ void thread_pixel(int tid, int &lx, int &ly) {
    const int w = tid >> 5, lane = tid & 31;
    lx = (w % (TW / kWX)) * kWX + lane % kWX;
    ly = (w / (TW / kWX)) * kWY + (lane / kWX) * kPPT;
}

// sigma(d) = 1/2 (A dx^2 + C dy^2) + B dx dy in the decision chain's operation order (spec_sigma),
// used for the box minimum below so that its rounding error has the same bound
__device__ __forceinline__ float sigma_rn(float A, float B, float C, float dx, float dy) {
    const float q = fp::fma(fp::mul(A, dx), dx, fp::mul(fp::mul(C, dy), dy));
    return fp::fma(fp::mul(B, dx), dy, fp::mul(0.5f, q));
}

// True when the decision chain's sigma exceeds `cut` at every pixel centre of the box
// [xa, xb] x [ya, yb] (pixel centres; the mean (mx, my) and the conic (A, B, C) as recorded), so
// that every pixel of the box skips the entry.
//
// The box minimum of the convex quadratic sigma is 0 when the mean is inside the box, else it is
// attained on an edge at the 1-D minimiser clamped to that edge; s is that minimum evaluated in
// FP32.  Error bound, with u = 2^-24 and M = 1/2 (A Dx^2 + C Dy^2) + |B| Dx Dy (Dx, Dy the largest
// |offset| of the box from the mean along each axis, so M bounds the sum of the magnitudes of the
// three terms of sigma anywhere in the box):
//  * the decision chain at a pixel rounds dx and dy once (at most 2u M on sigma), forms the
//    non-negative A dx^2 + C dy^2 with three roundings (3u M) and adds B dx dy with one fused
//    rounding (u M): it is within 6u M of the exact sigma of that pixel;
//  * s rounds each candidate's edge offset once and evaluates sigma with the same sequence
//    (6u M); its minimiser, computed with an approximate reciprocal, is off by a relative
//    O(u), which raises sigma only by O(u^2) M (sigma is quadratic about the minimiser);
// so s - 12u M (up to O(u^2) M) is below the chain's sigma at every pixel of the box.  The box
// is skipped when s > cut + 0.01 + 1e-3 |cut| + 32u M: the 32u term covers the 12u bound with
// room for the rounding of M itself, and for thin footprints (conic entries of 1e4 and more,
// where B dx dy cancels most of the other two terms) it is what keeps the skip exact.  Non-finite
// or non-positive-definite input never skips.
__device__ __forceinline__ bool box_skips(float A, float B, float C, float mx, float my, float xa, float xb,
                                          float ya, float yb, float cut) {
    if (!(A > 0.f && C > 0.f && A < 1e30f && C < 1e30f && fabsf(B) < 1e30f && fabsf(mx) < 1e30f &&
          fabsf(my) < 1e30f && fabsf(cut) < 1e30f))
        return false;
    const float dxa = xa - mx, dxb = xb - mx, dya = ya - my, dyb = yb - my;
    if (dxa <= 0.f && dxb >= 0.f && dya <= 0.f && dyb >= 0.f) return false;
    const float iA = __fdividef(1.f, A), iC = __fdividef(1.f, C);
    float best = 3.0e38f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = e ? dxb : dxa;
        const float dy = fminf(fmaxf(-B * dx * iC, dya), dyb);
        best = fminf(best, sigma_rn(A, B, C, dx, dy));
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dy = e ? dyb : dya;
        const float dx = fminf(fmaxf(-B * dy * iA, dxa), dxb);
        best = fminf(best, sigma_rn(A, B, C, dx, dy));
    }
    const float Dx = fmaxf(fabsf(dxa), fabsf(dxb)), Dy = fmaxf(fabsf(dya), fabsf(dyb));
    const float M = 0.5f * (A * Dx * Dx + C * Dy * Dy) + fabsf(B) * Dx * Dy;
    const float thr = cut + 0.01f + 1e-3f * fabsf(cut) + 0x1p-19f * M;
    return best > thr;   // false for a NaN or infinite threshold
}

// Bit w set <=> warp w's block of pixels (kWX x kWY, see thread_pixel) may blend the entry.  A
// cleared bit means the decision chain's sigma exceeds the cut at every pixel of that block
// (box_skips): every pixel there skips the entry, so the warp may skip it without evaluating it.
template <int TW, int TH>
__device__ __forceinline__ uint32_t warp_region_mask(const float4 &r0, const float4 &r1, float cut, int tile_x0,
                                                     int tile_y0) {
    constexpr int NW = TW * TH / (kPPT * 32);
    static_assert(TW % kWX == 0 && TH % kWY == 0, "tile must hold whole warp blocks");
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const float xa = (float)(tile_x0 + (w % (TW / kWX)) * kWX) + 0.5f;
        const float ya = (float)(tile_y0 + (w / (TW / kWX)) * kWY) + 0.5f;
        if (!box_skips(r0.z, r0.w, r1.x, r0.x, r0.y, xa, xa + (float)(kWX - 1), ya, ya + (float)(kWY - 1), cut))
            m |= 1u << w;
    }
    return m;
}

constexpr unsigned long long kTmaWaitLimit = 1ull << 22;   // polls of a batch's mbarrier before giving up

// Claim order: the binning lists every (view, tile) item under its claim class (class 0 the
// longest lists); coff[k] is the number of items in classes below k (coff[kClaimClasses] = all),
// so the counter's value c falls in the class k with coff[k] <= c < coff[k + 1].
__device__ __forceinline__ void claim_offsets(const DevStatus *st, uint32_t *coff) {
    if (threadIdx.x < 32) {
        static_assert(kClaimClasses == 32, "one class per lane");
        const uint32_t x = st->claim_cnt[threadIdx.x];
        uint32_t y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
            if ((int)threadIdx.x >= o) y += t;
        }
        coff[threadIdx.x] = y - x;
        if (threadIdx.x == 31) coff[32] = y;
    }
}

// Next work item of a persistent compositing CTA (thread 0), -1 when all are taken.  Every CTA
// makes exactly one claim past the last item; the CTA that draws the last of those (every other
// claim of the launch is made by then) returns the counter to zero for the next launch.  Class
// lists inconsistent with G (only after an earlier binning failure) record a device fault; the
// claim then falls back to the counter's own value.
__device__ __forceinline__ long long claim_item(DevStatus *st, uint32_t *ctr, const uint32_t *coff,
                                                const uint32_t *clist, long long G) {
    const long long c = (long long)atomicAdd(ctr, 1u);
    const long long total = min((long long)coff[kClaimClasses], G);
    if (c >= total) {
        if (c == total + (long long)gridDim.x - 1) *ctr = 0u;
        return -1;
    }
    int k = 0;   // the largest k with coff[k] <= c (coff[0] = 0)
#pragma unroll
    for (int step = kClaimClasses / 2; step > 0; step >>= 1)
        if ((long long)coff[k + step] <= c) k += step;
    const long long r = c - (long long)coff[k];
    const uint32_t g = r < G ? clist[(size_t)k * G + r] : 0xffffffffu;
    if ((long long)g >= G) {
        record_error(st, GS_ERR_DEVICE_FAULT, 10);
        return c;
    }
    return (long long)g;
}

// A CTA leaving early (after a failed wait, an error already recorded) claims until it draws a
// value past the items, skipping the items it draws, so that every CTA still makes exactly one
// claim past them and the launch's last claim returns the counter to zero.
__device__ __forceinline__ void claim_exit(uint32_t *ctr, const uint32_t *coff, long long G) {
    if (threadIdx.x == 0) {
        const long long total = min((long long)coff[kClaimClasses], G);
        long long c;
        do {
            c = (long long)atomicAdd(ctr, 1u);
        } while (c < total);
        if (c == total + (long long)gridDim.x - 1) *ctr = 0u;
    }
}

// Shared memory of one render CTA: two batches of records (double buffer filled by TMA), the
// per-entry warp-region masks of each batch, one mbarrier per buffer.
// NB records per staged batch: 64, 128 or 256, at most one per pixel of the tile (two buffers of
// 256 records take 24 KB)
template <int NB>
struct __align__(128) RenderSmem {
    float4 rec[2][3 * NB];
    uint8_t mask[2][NB];
    uint64_t bar[2];
    long long item;
    int maxlast;
    uint32_t coff[kClaimClasses + 1];   // claim-class offsets (claim_offsets)
};

// Waits for both buffers' outstanding copies (bounded) after a failed wait, so that the CTA never
// leaves with a copy still targeting its shared memory unless that copy is itself stuck.
template <int NB>
__device__ __forceinline__ void drain_after_timeout(RenderSmem<NB> &sm, const uint32_t (&parity)[2],
                                                    const bool (&pending)[2], DevStatus *st) {
    if (threadIdx.x == 0) {
        record_error(st, GS_ERR_TIMEOUT, 8);
        for (int bb = 0; bb < 2; ++bb)
            if (pending[bb]) mbar_wait_bounded(&sm.bar[bb], parity[bb], kTmaWaitLimit);
    }
    __syncthreads();
}

template <int TW, int TH, int NB>
__global__ void __launch_bounds__(TW *TH / kPPT) k_render_fwd(FwdArgs a) {
    static_assert(NB <= TW * TH, "at most one staged record per pixel of the tile");
    constexpr int NT = TW * TH / kPPT;            // threads
    __shared__ RenderSmem<NB> sm;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t wbit = 1u << (tid >> 5);
    const long long tpv = (long long)a.Tx * a.Ty;
    const long long HW = (long long)a.W * a.H;
    int lx, ly;
    thread_pixel<TW>(tid, lx, ly);
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_proxy_async_smem();
    }
    claim_offsets(a.st, sm.coff);
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    unsigned long long pairs = 0;
    float l1_rgb = 0.f, l1_d = 0.f;      // per-thread sums of |rendered - target| (L1 epilogue)
    for (;;) {
        if (tid == 0) sm.item = claim_item(a.st, &a.st->fwd_items, sm.coff, a.clist, a.G);
        __syncthreads();
        const long long g = sm.item;
        if (g < 0) break;
        const int v = (int)(g / tpv);
        const int tl = (int)(g - (long long)v * tpv);
        const int ty = tl / a.Tx, tx = tl - ty * a.Tx;
        const int x = tx * TW + lx, y0 = ty * TH + ly;
        const uint32_t start = a.ranges[2 * g], end = a.ranges[2 * g + 1];
        // the tile's list must lie inside the records (its batches are copied by TMA)
        const int n = gs_guard(a.st, end >= start && (long long)end <= a.cap, 10) ? (int)(end - start) : 0;
        // per-pixel state of the thread's two pixels, packed (component p = pixel p)
        static_assert(kPPT == 2, "two pixels per thread, one per packed component");
        bool done[kPPT];
        int last[kPPT], visited[kPPT];
        float2 T = fp2::splat(1.0f), C0 = fp2::splat(0.f), C1 = fp2::splat(0.f), C2 = fp2::splat(0.f),
               D = fp2::splat(0.f);
        const float2 py = make_float2((float)y0 + 0.5f, (float)(y0 + 1) + 0.5f);
#pragma unroll
        for (int p = 0; p < kPPT; ++p) {
            done[p] = !(x < a.W && y0 + p < a.H);
            last[p] = 0;
            visited[p] = done[p] ? 0 : n;      // entries visited, up to and including the stopping one
        }
        const float px = (float)x + 0.5f;
        const int nb = (n + NB - 1) / NB;
        auto issue = [&](int bi, int bb) {     // thread 0: batch bi of this tile into buffer bb
            const int b = bi * NB;
            fence_proxy_async_smem();
            tma_load_1d(&sm.rec[bb][0], a.srec + 3 * (size_t)(start + b), (uint32_t)min(NB, n - b) * 48u,
                        &sm.bar[bb]);
        };
        if (tid == 0 && nb > 0) issue(0, 0);
        int buf = 0;
        for (int bi = 0; bi < nb; ++bi) {
            const int b = bi * NB, cnt = min(NB, n - b);
            if (tid == 0 && bi + 1 < nb) issue(bi + 1, buf ^ 1);
            const bool ok = mbar_wait_bounded(&sm.bar[buf], parity[buf], kTmaWaitLimit);
            if (__syncthreads_or(!ok)) {
                const bool pending[2] = {buf == 0 || bi + 1 < nb, buf == 1 || bi + 1 < nb};
                drain_after_timeout<NB>(sm, parity, pending, a.st);
                claim_exit(&a.st->fwd_items, sm.coff, a.G);
                return;
            }
            parity[buf] ^= 1u;
            const float4 *rec = sm.rec[buf];
#pragma unroll
            for (int q = 0; q < kPPT; ++q) {
                const int e = tid + q * NT;
                if (e < cnt)
                    sm.mask[buf][e] = (uint8_t)warp_region_mask<TW, TH>(rec[3 * e], rec[3 * e + 1], rec[3 * e + 2].w,
                                                                        tx * TW, ty * TH);
            }
            __syncthreads();
            const uint8_t *msk = sm.mask[buf];
            // entries whose region bit is clear for this warp are dropped 32 at a time: a ballot over
            // the mask bytes gives the entries to visit, walked front to back
            for (int k0 = 0; k0 < cnt; k0 += 32) {
              const int kk = k0 + lane;
              uint32_t bits = __ballot_sync(0xffffffffu, kk < cnt && (msk[kk] & wbit));
              if (done[0] && done[1]) continue;   // after the ballot, which every lane takes part in
              while (bits) {
                const int k = k0 + __ffs(bits) - 1;
                bits &= bits - 1u;
                const float4 r0 = rec[3 * k];
                const float4 r1 = rec[3 * k + 1];
                const float cut = rec[3 * k + 2].w;
                const float dx = fp::sub(px, r0.x);
                const float2 sg = spec_sigma2(r0.z, r0.w, r1.x, dx, fp2::add(py, fp2::splat(-r0.y)));
                const bool ev0 = !done[0] && !(sg.x < 0.0f) && !(sg.x > cut);
                const bool ev1 = !done[1] && !(sg.y < 0.0f) && !(sg.y > cut);
                if (!(ev0 || ev1)) continue;
                const float2 ar = fp2::mul(fp2::splat(r1.y), spec_expf2(fp2::neg(sg)));
                const float2 al = make_float2(fminf(a.amax, ar.x), fminf(a.amax, ar.y));
                const float4 r2 = rec[3 * k + 2];
                // both pixels without branches: the same FP32 decisions (skip, stop before
                // blending), taken as selects
                const float2 Tn = fp2::mul(T, fp2::add(fp2::splat(1.0f), fp2::neg(al)));
                const float2 w = fp2::mul(al, T);
                const bool bl0 = ev0 && !(al.x < a.amin), bl1 = ev1 && !(al.y < a.amin);
                const bool stop0 = bl0 && Tn.x < a.tmin, stop1 = bl1 && Tn.y < a.tmin;
                const bool acc0 = bl0 && !stop0, acc1 = bl1 && !stop1;
                done[0] = done[0] || stop0;
                done[1] = done[1] || stop1;
                visited[0] = stop0 ? b + k + 1 : visited[0];
                visited[1] = stop1 ? b + k + 1 : visited[1];
                const float2 wgt = make_float2(acc0 ? w.x : 0.f, acc1 ? w.y : 0.f);
                C0 = fp2::fma(fp2::splat(r2.x), wgt, C0);
                C1 = fp2::fma(fp2::splat(r2.y), wgt, C1);
                C2 = fp2::fma(fp2::splat(r2.z), wgt, C2);
                D = fp2::fma(fp2::splat(r1.z), wgt, D);
                T = make_float2(acc0 ? Tn.x : T.x, acc1 ? Tn.y : T.y);
                last[0] = acc0 ? b + k + 1 : last[0];
                last[1] = acc1 ? b + k + 1 : last[1];
                if (done[0] && done[1]) break;
              }
            }
            const bool all_done = __syncthreads_and(done[0] && done[1]);   // also: buffer reads finished
            if (all_done) {
                if (bi + 1 < nb) {   // the prefetched batch must land before its buffer is reused
                    const bool ok2 = mbar_wait_bounded(&sm.bar[buf ^ 1], parity[buf ^ 1], kTmaWaitLimit);
                    if (__syncthreads_or(!ok2)) {
                        const bool pending[2] = {buf == 1, buf == 0};
                        drain_after_timeout<NB>(sm, parity, pending, a.st);
                        claim_exit(&a.st->fwd_items, sm.coff, a.G);
                        return;
                    }
                    parity[buf ^ 1] ^= 1u;
                }
                break;
            }
            buf ^= 1;
        }
#pragma unroll
        for (int p = 0; p < kPPT; ++p) {
            pairs += (unsigned long long)visited[p];
            if (x < a.W && y0 + p < a.H) {
                const long long pix = (long long)(y0 + p) * a.W + x;
                const float Tp = p ? T.y : T.x, Dp = p ? D.y : D.x;
                const float c[3] = {(p ? C0.y : C0.x) + Tp * a.bg0, (p ? C1.y : C1.x) + Tp * a.bg1,
                                    (p ? C2.y : C2.x) + Tp * a.bg2};
                if (a.rgb) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) a.rgb[(3 * (long long)v + ch) * HW + pix] = c[ch];
                }
                if (a.depth) a.depth[(long long)v * HW + pix] = Dp;
                if (a.alpha) a.alpha[(long long)v * HW + pix] = 1.0f - Tp;
                a.finalT[(long long)v * HW + pix] = Tp;
                a.last[(long long)v * HW + pix] = last[p];
                if (a.rgb_t) {   // L1 terms and their gradient, as gs_loss_l1 computes them
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const long long idx = (3 * (long long)v + ch) * HW + pix;
                        const float d = c[ch] - a.rgb_t[idx];
                        l1_rgb += fabsf(d);
                        a.d_rgb[idx] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * a.sc_rgb;
                    }
                    if (a.depth_t) {
                        const long long idx = (long long)v * HW + pix;
                        const float d = Dp - a.depth_t[idx];
                        l1_d += fabsf(d);
                        a.d_depth[idx] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * a.sc_d;
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if ((tid & 31) == 0 && pairs) atomicAdd(&a.st->fwd_pairs, pairs);
    if (a.rgb_t) {   // one double atomic per warp for the loss
        double l = (double)l1_rgb * a.sc_rgb + (double)l1_d * a.sc_d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((tid & 31) == 0 && l != 0.0) atomicAdd(a.loss, l);
    }
}

// Transposed butterfly over 16 slots: after the call lanes 2s and 2s + 1 hold, in v[0], two
// halves of the warp sum of slot s(l) = 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of l); both add
// theirs to the gradient (the last butterfly stage is left to the atomic unit).  The 10 gradient
// components live in slots 0..4 and 8..12 (kSlot); slots 5..7 and 13..15 are zero in every lane,
// so the first stage skips their three all-zero pairs: 12 shuffles in total.
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane) {
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float send = up ? v[i] : v[i + 8];
            const float keep = up ? v[i + 8] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        v[5] = v[6] = v[7] = 0.f;
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float send = up ? v[i] : v[i + 4];
            const float keep = up ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool up = lane & 4;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = up ? v[i] : v[i + 2];
            const float keep = up ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
}

// slot of each gradient component (mean_x, mean_y, A, B, C, opacity, depth, r, g, b)
enum : int { kSMx = 0, kSMy = 1, kSA = 2, kSB = 3, kSC = 4, kSO = 8, kSZ = 9, kSR = 10, kSG = 11, kSBl = 12 };

template <int TW, int TH, int NB>
__global__ void __launch_bounds__(TW *TH / kPPT) k_render_bwd(BwdArgs a) {
    static_assert(NB <= TW * TH, "at most one staged record per pixel of the tile");
    constexpr int NT = TW * TH / kPPT;
    __shared__ RenderSmem<NB> sm;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t wbit = 1u << (tid >> 5);
    const int slot = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    const int comp = slot < 5 ? slot : slot - 3;           // component index in the grad2d record
    const bool issuer = slot < 5 || (slot >= 8 && slot < 13);   // 20 lanes, two per component
    const long long tpv = (long long)a.Tx * a.Ty;
    const long long HW = (long long)a.W * a.H;
    int lx, ly;
    thread_pixel<TW>(tid, lx, ly);
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_proxy_async_smem();
    }
    claim_offsets(a.st, sm.coff);
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    unsigned long long pairs = 0;
    for (;;) {
        if (tid == 0) {
            sm.item = claim_item(a.st, &a.st->bwd_items, sm.coff, a.clist, a.G);
            sm.maxlast = 0;
        }
        __syncthreads();
        const long long g = sm.item;
        if (g < 0) break;
        const int v = (int)(g / tpv);
        const int tl = (int)(g - (long long)v * tpv);
        const int ty = tl / a.Tx, tx = tl - ty * a.Tx;
        const int x = tx * TW + lx, y0 = ty * TH + ly;
        const uint32_t start = a.ranges[2 * g], end = a.ranges[2 * g + 1];
        const int n = gs_guard(a.st, end >= start && (long long)end <= a.cap, 11) ? (int)(end - start) : 0;
        const float px = (float)x + 0.5f;
        // per-pixel state of the thread's two pixels, packed (component p = pixel p)
        static_assert(kPPT == 2, "two pixels per thread, one per packed component");
        int lst[kPPT];
        float tT[kPPT], tQ[kPPT], tC0[kPPT], tC1[kPPT], tC2[kPPT], tD[kPPT];
        int tmax = 0;
#pragma unroll
        for (int p = 0; p < kPPT; ++p) {
            lst[p] = 0;
            tT[p] = 1.0f;
            tC0[p] = tC1[p] = tC2[p] = tD[p] = 0.f;
            float gA = 0.f;
            if (x < a.W && y0 + p < a.H) {
                const long long pix = (long long)(y0 + p) * a.W + x;
                lst[p] = min(max(a.last[(long long)v * HW + pix], 0), n);   // never past the list
                tT[p] = a.finalT[(long long)v * HW + pix];
                if (a.d_rgb) {
                    tC0[p] = a.d_rgb[(3 * (long long)v + 0) * HW + pix];
                    tC1[p] = a.d_rgb[(3 * (long long)v + 1) * HW + pix];
                    tC2[p] = a.d_rgb[(3 * (long long)v + 2) * HW + pix];
                }
                if (a.d_depth) tD[p] = a.d_depth[(long long)v * HW + pix];
                if (a.d_alpha) gA = a.d_alpha[(long long)v * HW + pix];
            }
            // rgb = sum c alpha T + T_final bg, alpha_out = 1 - T_final
            tQ[p] = tT[p] * (tC0[p] * a.bg0 + tC1[p] * a.bg1 + tC2[p] * a.bg2 - gA);
            pairs += (unsigned long long)lst[p];
            tmax = max(tmax, lst[p]);
        }
        // Q = sum over blended entries behind the current one of (gC . c + gD z) alpha T, plus the
        // background and alpha-output terms: dL/dalpha_j = T_j (gC . c_j + gD z_j) - Q / (1 - alpha_j)
        float2 T = make_float2(tT[0], tT[1]), Q = make_float2(tQ[0], tQ[1]);
        const float2 gC0 = make_float2(tC0[0], tC0[1]), gC1 = make_float2(tC1[0], tC1[1]),
                     gC2 = make_float2(tC2[0], tC2[1]), gD = make_float2(tD[0], tD[1]);
        const float2 py = make_float2((float)y0 + 0.5f, (float)(y0 + 1) + 0.5f);
        const int wmax = __reduce_max_sync(0xffffffffu, tmax);
        if (lane == 0) atomicMax(&sm.maxlast, wmax);
        __syncthreads();
        const int maxl = sm.maxlast;
        const int nb = (maxl + NB - 1) / NB;   // batches, back to front: [max(0, maxl-(bi+1)NB), maxl-bi NB)
        auto issue = [&](int bi, int bb) {
            const int hi = maxl - bi * NB, lo = max(0, hi - NB);
            fence_proxy_async_smem();
            tma_load_1d(&sm.rec[bb][0], a.srec + 3 * (size_t)(start + lo), (uint32_t)(hi - lo) * 48u, &sm.bar[bb]);
        };
        if (tid == 0 && nb > 0) issue(0, 0);
        int buf = 0;
        for (int bi = 0; bi < nb; ++bi) {
            const int hi = maxl - bi * NB, lo = max(0, hi - NB), cnt = hi - lo;
            if (tid == 0 && bi + 1 < nb) issue(bi + 1, buf ^ 1);
            const bool ok = mbar_wait_bounded(&sm.bar[buf], parity[buf], kTmaWaitLimit);
            if (__syncthreads_or(!ok)) {
                const bool pending[2] = {buf == 0 || bi + 1 < nb, buf == 1 || bi + 1 < nb};
                drain_after_timeout<NB>(sm, parity, pending, a.st);
                claim_exit(&a.st->bwd_items, sm.coff, a.G);
                return;
            }
            parity[buf] ^= 1u;
            const float4 *rec = sm.rec[buf];
#pragma unroll
            for (int q = 0; q < kPPT; ++q) {
                const int e = tid + q * NT;
                if (e < cnt)
                    sm.mask[buf][e] = (uint8_t)warp_region_mask<TW, TH>(rec[3 * e], rec[3 * e + 1], rec[3 * e + 2].w,
                                                                        tx * TW, ty * TH);
            }
            __syncthreads();
            const uint8_t *msk = sm.mask[buf];
            // entries at or beyond the warp's largest last_idx contribute nothing to this warp; entries
            // whose region bit is clear are dropped 32 at a time (a ballot over the mask bytes), and
            // the rest walked back to front
            const int kend = min(hi, wmax) - lo;
            for (int k0 = ((kend - 1) >> 5) << 5; k0 >= 0 && kend > 0; k0 -= 32) {
              const int kk = k0 + lane;
              uint32_t bits = __ballot_sync(0xffffffffu, kk < kend && (msk[kk] & wbit));
              while (bits) {
                const int k = k0 + 31 - __clz(bits);
                bits &= ~(1u << (k - k0));
                const int pos = lo + k;
                const float4 r0 = rec[3 * k];
                const float4 r1 = rec[3 * k + 1];
                const float cut = rec[3 * k + 2].w;
                const float dx = fp::sub(px, r0.x);
                const float2 dy = fp2::add(py, fp2::splat(-r0.y));
                const float2 sg = spec_sigma2(r0.z, r0.w, r1.x, dx, dy);
                const bool ev0 = pos < lst[0] && !(sg.x < 0.0f) && !(sg.x > cut);
                const bool ev1 = pos < lst[1] && !(sg.y < 0.0f) && !(sg.y > cut);
                float gv[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) gv[c] = 0.f;
                bool contrib = false;
                if (ev0 || ev1) {
                    const float2 e = spec_expf2(fp2::neg(sg));
                    const float2 araw = fp2::mul(fp2::splat(r1.y), e);
                    const float2 al = make_float2(fminf(a.amax, araw.x), fminf(a.amax, araw.y));
                    const float4 r2 = rec[3 * k + 2];
                    // both pixels evaluated without branches; a pixel that does not blend the
                    // entry contributes zero (selects, not products, so an infinite e or a
                    // meaningless alpha of a skipped pixel never reaches a sum)
                    const bool bl0 = ev0 && !(al.x < a.amin), bl1 = ev1 && !(al.y < a.amin);
                    const bool un0 = bl0 && araw.x <= a.amax, un1 = bl1 && araw.y <= a.amax;
                    contrib = bl0 || bl1;
                    const float2 oma = fp2::add(fp2::splat(1.0f), fp2::neg(al));
                    const float2 ioma = make_float2(__fdividef(1.0f, oma.x), __fdividef(1.0f, oma.y));
                    const float2 Tj = fp2::mul(T, ioma);
                    const float2 wr = fp2::mul(al, Tj);
                    const float2 w = make_float2(bl0 ? wr.x : 0.f, bl1 ? wr.y : 0.f);
                    const float2 Pj = fp2::fma(gD, fp2::splat(r1.z),
                                               fp2::fma(gC2, fp2::splat(r2.z),
                                                        fp2::fma(gC1, fp2::splat(r2.y), fp2::mul(gC0, fp2::splat(r2.x)))));
                    const float2 dLda = fp2::fma(Tj, Pj, fp2::neg(fp2::mul(Q, ioma)));
                    Q = fp2::fma(Pj, w, Q);
                    T = make_float2(bl0 ? Tj.x : T.x, bl1 ? Tj.y : T.y);
                    const float2 cR = fp2::mul(gC0, w), cG = fp2::mul(gC1, w), cB = fp2::mul(gC2, w),
                                 cZ = fp2::mul(gD, w);
                    gv[kSR] = cR.x + cR.y;
                    gv[kSG] = cG.x + cG.y;
                    gv[kSBl] = cB.x + cB.y;
                    gv[kSZ] = cZ.x + cZ.y;
                    const float2 oe = fp2::mul(dLda, e);
                    gv[kSO] = (un0 ? oe.x : 0.f) + (un1 ? oe.y : 0.f);
                    // dL/dsigma per pixel; the conic and mean gradients are sums over the two
                    // pixels of dL/dsigma times 1/2 dx^2, dx dy, 1/2 dy^2 and -(A dx + B dy),
                    // -(B dx + C dy): dx is the pair's, so only s0 = sum dL/dsigma,
                    // s1 = sum dL/dsigma dy and s2 = sum dL/dsigma dy^2 need both pixels
                    const float2 ds = fp2::mul(dLda, al);
                    const float2 dLds = make_float2(un0 ? -ds.x : 0.f, un1 ? -ds.y : 0.f);
                    const float2 t1 = fp2::mul(dLds, dy);
                    const float2 t2 = fp2::mul(t1, dy);
                    const float s0 = dLds.x + dLds.y, s1 = t1.x + t1.y, s2 = t2.x + t2.y;
                    const float s0dx = s0 * dx;
                    gv[kSA] = 0.5f * s0dx * dx;
                    gv[kSB] = s1 * dx;
                    gv[kSC] = 0.5f * s2;
                    gv[kSMx] = -(r0.z * s0dx + r0.w * s1);
                    gv[kSMy] = -(r0.w * s0dx + r1.x * s1);
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    warp_transpose_reduce16(gv, lane);
                    const uint32_t sl = __float_as_uint(r1.w);   // the record's slot in g2d
                    if (issuer && gs_guard(a.st, (long long)sl < a.P, 12)) atomicAdd(a.g2d + 12 * (size_t)sl + comp, gv[0]);
                }
              }
            }
            __syncthreads();                          // buffer reads finished before its refill
            buf ^= 1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if (lane == 0 && pairs) atomicAdd(&a.st->bwd_pairs, pairs);
}

template <class F>
static int persistent_grid(F fn, int threads) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, 0) != cudaSuccess || b < 1) b = 1;
    return b * device_sm_count();
}

template <int TW, int TH, int NB>
static int fwd_t(const FwdArgs &a, cudaStream_t s) {
    constexpr int NT = TW * TH / kPPT;
    static int grid = persistent_grid(k_render_fwd<TW, TH, NB>, NT);
    if (a.rgb_t && cudaMemsetAsync(a.loss, 0, sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    const long long g = std::min<long long>(grid, std::max<long long>(1, a.G));
    k_render_fwd<TW, TH, NB><<<(unsigned)g, NT, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

template <int TW, int TH, int NB>
static int bwd_t(const BwdArgs &a, cudaStream_t s) {
    constexpr int NT = TW * TH / kPPT;
    static int grid = persistent_grid(k_render_bwd<TW, TH, NB>, NT);
    const long long g = std::min<long long>(grid, std::max<long long>(1, a.G));
    k_render_bwd<TW, TH, NB><<<(unsigned)g, NT, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

// (tile, records per batch) pairs with a compiled kernel; the API layer validates the values
int launch_render_fwd(int tw, int th, int nb, const FwdArgs &a, cudaStream_t s) {
    if (tw == 16 && th == 16)
        return nb == 64 ? fwd_t<16, 16, 64>(a, s) : nb == 128 ? fwd_t<16, 16, 128>(a, s) : fwd_t<16, 16, 256>(a, s);
    if (tw == 16 && th == 8) return nb == 64 ? fwd_t<16, 8, 64>(a, s) : fwd_t<16, 8, 128>(a, s);
    if (tw == 32 && th == 16)
        return nb == 64 ? fwd_t<32, 16, 64>(a, s) : nb == 128 ? fwd_t<32, 16, 128>(a, s) : fwd_t<32, 16, 256>(a, s);
    return GS_ERR_INVALID_ARG;
}

int launch_render_bwd(int tw, int th, int nb, const BwdArgs &a, cudaStream_t s) {
    if (tw == 16 && th == 16)
        return nb == 64 ? bwd_t<16, 16, 64>(a, s) : nb == 128 ? bwd_t<16, 16, 128>(a, s) : bwd_t<16, 16, 256>(a, s);
    if (tw == 16 && th == 8) return nb == 64 ? bwd_t<16, 8, 64>(a, s) : bwd_t<16, 8, 128>(a, s);
    if (tw == 32 && th == 16)
        return nb == 64 ? bwd_t<32, 16, 64>(a, s) : nb == 128 ? bwd_t<32, 16, 128>(a, s) : bwd_t<32, 16, 256>(a, s);
    return GS_ERR_INVALID_ARG;
}

}  // namespace gs
