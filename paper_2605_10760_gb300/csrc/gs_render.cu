// gs_render.cu -- per-tile compositing (forward) and its adjoint (backward).
//
// One CTA = one tile of TW x TH pixels (one thread per pixel).  Both kernels are persistent: a
// grid of (#SM x resident CTAs) claims (view, tile) work items from a device counter, so one launch
// covers every tile of every view of every scene, whatever the per-tile list lengths.
//
// Forward: the tile's list (a contiguous range of the sorted values) is staged into shared memory in
// batches of TW*TH records; each thread walks it front to back taking the FP32 decisions of the
// decision chain (sigma < 0 skip, alpha < alpha_min skip, stop before blending when
// T (1 - alpha) < t_min).  The CTA leaves the list once every pixel has stopped.
//
// Backward: from final_T and last_idx of each pixel the CTA walks the list back to front,
// recovering T_j = T_{j+1} / (1 - alpha_j) and the colour / depth accumulated behind each entry, so
// no per-pixel list is stored.  Each warp reduces the 10 per-Gaussian gradient components of its
// 32 pixels with a transposed butterfly (16 shuffles instead of 50) after which 10 lanes issue one
// atomic add each, so a (Gaussian, warp) pair costs one warp-wide atomic instruction; warps whose
// pixels all skipped the entry issue nothing.
#include "gs_kernels.cuh"

namespace gs {

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_render_fwd(FwdArgs a) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_r0[NT], s_r1[NT], s_r2[NT];
    __shared__ long long s_item;
    const int tid = threadIdx.x;
    const long long tpv = (long long)a.Tx * a.Ty;
    const long long HW = (long long)a.W * a.H;
    unsigned long long pairs = 0;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&a.st->ctr[kCtrFwd], 1u);
        __syncthreads();
        const long long g = s_item;
        if (g >= a.G) break;
        const int v = (int)(g / tpv);
        const int tl = (int)(g - (long long)v * tpv);
        const int ty = tl / a.Tx, tx = tl - ty * a.Tx;
        const int x = tx * TW + (tid % TW), y = ty * TH + (tid / TW);
        const bool inside = x < a.W && y < a.H;
        const uint32_t start = a.ranges[2 * g], end = a.ranges[2 * g + 1];
        const int n = (int)(end - start);
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
        int last = 0;
        bool done = !inside;
        for (int b = 0; b < n; b += NT) {
            if (__syncthreads_and(done)) break;
            const int j = b + tid;
            if (j < n) {
                uint32_t f = a.vals[start + j];
                if (f >= (uint32_t)a.P) {                 // only after an earlier recorded failure
                    record_error(a.st, GS_ERR_DEVICE_FAULT, 6);
                    f = 0;
                }
                s_r0[tid] = a.proj[3 * (size_t)f];
                s_r1[tid] = a.proj[3 * (size_t)f + 1];
                s_r2[tid] = a.proj[3 * (size_t)f + 2];
            }
            __syncthreads();
            const int cnt = min(NT, n - b);
            if (!done) {
                for (int k = 0; k < cnt; ++k) {
                    const float4 r0 = s_r0[k];
                    const float4 r1 = s_r1[k];
                    ++pairs;
                    const float dx = fp::sub(px, r0.x), dy = fp::sub(py, r0.y);
                    const float sg = spec_sigma(r0.z, r0.w, r1.x, dx, dy);
                    if (sg < 0.0f) continue;
                    const float al = fminf(a.amax, fp::mul(r1.y, spec_expf(-sg)));
                    if (al < a.amin) continue;
                    const float Tn = fp::mul(T, fp::sub(1.0f, al));
                    if (Tn < a.tmin) {
                        done = true;
                        break;
                    }
                    const float4 r2 = s_r2[k];
                    const float wgt = al * T;
                    C0 += r2.x * wgt;
                    C1 += r2.y * wgt;
                    C2 += r2.z * wgt;
                    D += r1.z * wgt;
                    T = Tn;
                    last = b + k + 1;
                }
            }
        }
        if (inside) {
            const long long pix = (long long)y * a.W + x;
            if (a.rgb) {
                a.rgb[(3 * (long long)v + 0) * HW + pix] = C0 + T * a.bg0;
                a.rgb[(3 * (long long)v + 1) * HW + pix] = C1 + T * a.bg1;
                a.rgb[(3 * (long long)v + 2) * HW + pix] = C2 + T * a.bg2;
            }
            if (a.depth) a.depth[(long long)v * HW + pix] = D;
            if (a.alpha) a.alpha[(long long)v * HW + pix] = 1.0f - T;
            a.finalT[(long long)v * HW + pix] = T;
            a.last[(long long)v * HW + pix] = last;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if ((tid & 31) == 0 && pairs) atomicAdd(&a.st->fwd_pairs, pairs);
}

// Transposed butterfly: after the call lane l holds the warp sum of component
// c(l) = 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of l) in v[0].
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane) {
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float send = up ? v[i] : v[i + 8];
            const float keep = up ? v[i + 8] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
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
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_render_bwd(BwdArgs a) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_r0[NT], s_r1[NT], s_r2[NT];
    __shared__ uint32_t s_f[NT];
    __shared__ long long s_item;
    __shared__ int s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31;
    const int comp = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    const bool issuer = ((lane & 1) == 0) && comp < 10;
    const long long tpv = (long long)a.Tx * a.Ty;
    const long long HW = (long long)a.W * a.H;
    unsigned long long pairs = 0;
    for (;;) {
        if (tid == 0) {
            s_item = (long long)atomicAdd(&a.st->ctr[kCtrBwd], 1u);
            s_maxlast = 0;
        }
        __syncthreads();
        const long long g = s_item;
        if (g >= a.G) break;
        const int v = (int)(g / tpv);
        const int tl = (int)(g - (long long)v * tpv);
        const int ty = tl / a.Tx, tx = tl - ty * a.Tx;
        const int x = tx * TW + (tid % TW), y = ty * TH + (tid / TW);
        const bool inside = x < a.W && y < a.H;
        const uint32_t start = a.ranges[2 * g];
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        int lst = 0;
        float T = 1.0f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f;
        if (inside) {
            const long long pix = (long long)y * a.W + x;
            lst = a.last[(long long)v * HW + pix];
            T = a.finalT[(long long)v * HW + pix];
            if (a.d_rgb) {
                gC0 = a.d_rgb[(3 * (long long)v + 0) * HW + pix];
                gC1 = a.d_rgb[(3 * (long long)v + 1) * HW + pix];
                gC2 = a.d_rgb[(3 * (long long)v + 2) * HW + pix];
            }
            if (a.d_depth) gD = a.d_depth[(long long)v * HW + pix];
            if (a.d_alpha) gA = a.d_alpha[(long long)v * HW + pix];
        }
        pairs += (unsigned long long)lst;
        const float Tfin = T;
        float SC0 = Tfin * a.bg0, SC1 = Tfin * a.bg1, SC2 = Tfin * a.bg2, SD = 0.f;
        const int wmax = __reduce_max_sync(0xffffffffu, lst);
        if (lane == 0) atomicMax(&s_maxlast, wmax);
        __syncthreads();
        const int maxl = s_maxlast;
        for (int hi = maxl; hi > 0; hi -= NT) {
            const int lo = max(0, hi - NT);
            __syncthreads();
            const int j = lo + tid;
            if (j < hi) {
                uint32_t f = a.vals[start + j];
                if (f >= (uint32_t)a.P) {                 // only after an earlier recorded failure
                    record_error(a.st, GS_ERR_DEVICE_FAULT, 7);
                    f = 0;
                }
                s_f[tid] = f;
                s_r0[tid] = a.proj[3 * (size_t)f];
                s_r1[tid] = a.proj[3 * (size_t)f + 1];
                s_r2[tid] = a.proj[3 * (size_t)f + 2];
            }
            __syncthreads();
            for (int k = hi - lo - 1; k >= 0; --k) {
                float gv[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) gv[c] = 0.f;
                bool contrib = false;
                if (lo + k < lst) {
                    const float4 r0 = s_r0[k];
                    const float4 r1 = s_r1[k];
                    const float dx = fp::sub(px, r0.x), dy = fp::sub(py, r0.y);
                    const float sg = spec_sigma(r0.z, r0.w, r1.x, dx, dy);
                    if (sg >= 0.0f) {
                        const float e = spec_expf(-sg);
                        const float araw = fp::mul(r1.y, e);
                        const float al = fminf(a.amax, araw);
                        if (al >= a.amin) {
                            contrib = true;
                            const float4 r2 = s_r2[k];
                            const float oma = 1.0f - al;
                            const float ioma = 1.0f / oma;
                            const float Tj = T * ioma;
                            const float w = al * Tj;
                            gv[7] = gC0 * w;
                            gv[8] = gC1 * w;
                            gv[9] = gC2 * w;
                            gv[6] = gD * w;
                            const float dLda = gA * Tfin * ioma + gC0 * (r2.x * Tj - SC0 * ioma) +
                                               gC1 * (r2.y * Tj - SC1 * ioma) + gC2 * (r2.z * Tj - SC2 * ioma) +
                                               gD * (r1.z * Tj - SD * ioma);
                            SC0 += r2.x * w;
                            SC1 += r2.y * w;
                            SC2 += r2.z * w;
                            SD += r1.z * w;
                            T = Tj;
                            if (araw <= a.amax) {
                                gv[5] = dLda * e;
                                const float dLds = -dLda * al;
                                gv[2] = 0.5f * dLds * dx * dx;
                                gv[3] = dLds * dx * dy;
                                gv[4] = 0.5f * dLds * dy * dy;
                                gv[0] = -dLds * (r0.z * dx + r0.w * dy);
                                gv[1] = -dLds * (r0.w * dx + r1.x * dy);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    warp_transpose_reduce16(gv, lane);
                    if (issuer) atomicAdd(a.g2d + 12 * (size_t)s_f[k] + comp, gv[0]);
                }
            }
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

template <int TW, int TH>
static int fwd_t(const FwdArgs &a, cudaStream_t s) {
    static int grid = persistent_grid(k_render_fwd<TW, TH>, TW * TH);
    if (cudaMemsetAsync(&a.st->ctr[kCtrFwd], 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(&a.st->fwd_pairs, 0, sizeof(unsigned long long), s) != cudaSuccess) return GS_ERR_CUDA;
    const long long g = std::min<long long>(grid, std::max<long long>(1, a.G));
    k_render_fwd<TW, TH><<<(unsigned)g, TW * TH, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

template <int TW, int TH>
static int bwd_t(const BwdArgs &a, cudaStream_t s) {
    static int grid = persistent_grid(k_render_bwd<TW, TH>, TW * TH);
    if (cudaMemsetAsync(&a.st->ctr[kCtrBwd], 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(&a.st->bwd_pairs, 0, sizeof(unsigned long long), s) != cudaSuccess) return GS_ERR_CUDA;
    const long long g = std::min<long long>(grid, std::max<long long>(1, a.G));
    k_render_bwd<TW, TH><<<(unsigned)g, TW * TH, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

int launch_render_fwd(int tw, int th, const FwdArgs &a, cudaStream_t s) {
    if (tw == 16 && th == 16) return fwd_t<16, 16>(a, s);
    if (tw == 16 && th == 8) return fwd_t<16, 8>(a, s);
    if (tw == 32 && th == 16) return fwd_t<32, 16>(a, s);
    return GS_ERR_INVALID_ARG;
}

int launch_render_bwd(int tw, int th, const BwdArgs &a, cudaStream_t s) {
    if (tw == 16 && th == 16) return bwd_t<16, 16>(a, s);
    if (tw == 16 && th == 8) return bwd_t<16, 8>(a, s);
    if (tw == 32 && th == 16) return bwd_t<32, 16>(a, s);
    return GS_ERR_INVALID_ARG;
}

}  // namespace gs
