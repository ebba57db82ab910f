// gs_loss.cu -- loss terms of the mapping / refinement objectives and the Adam step.
//
// L1 (Eq. 4's photometric and depth terms): one pass per pixel producing the loss and its
// gradient.  SSIM (Eq. 23's structural term): two tiled passes with an 11-tap separable Gaussian
// (sigma 1.5, zero padding) in shared memory:
//   pass 1 blurs x, y, x^2, y^2, xy and writes the per-pixel derivatives of the SSIM map with
//          respect to mu_x, E[x^2] and E[xy];
//   pass 2 blurs those three maps (the adjoint of a zero-padded symmetric blur is the same blur)
//          and combines dSSIM/dx = blur(dS/dmu_x) + 2 x blur(dS/dE[x^2]) + y blur(dS/dE[xy]),
//          fused with the L1 gradient.
// Adam: one thread per Gaussian, 14 parameters, bias-corrected, opacity through its logit.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "gs_kernels.cuh"

namespace gs {

__device__ __forceinline__ float sgnf(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ void block_add_double(double v, double *out) {
    __shared__ double s_part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < (int)(blockDim.x >> 5) ? s_part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0 && w != 0.0) atomicAdd(out, w);
    }
}

// grid (blocks, V): view v = blockIdx.y; pixels of the view strided over the x-blocks, four at a
// time (16-byte loads and stores) when the plane size and the pointers allow it.
template <bool kVec>
__global__ void k_l1(long long HWn, const float *rgb, const float *rgb_t, const float *depth, const float *depth_t,
                     float sc_rgb, float sc_d, float *d_rgb, float *d_depth, double *loss) {
    float acc_rgb = 0.f, acc_d = 0.f;      // per-thread sums of |d| (a few dozen terms each)
    const long long v = blockIdx.y;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (kVec) {
        const long long n4 = HWn >> 2;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long off = (3 * v + c) * n4 + q;
                const float4 x = reinterpret_cast<const float4 *>(rgb)[off];
                const float4 y = reinterpret_cast<const float4 *>(rgb_t)[off];
                const float4 d = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
                acc_rgb += (fabsf(d.x) + fabsf(d.y)) + (fabsf(d.z) + fabsf(d.w));
                reinterpret_cast<float4 *>(d_rgb)[off] =
                    make_float4(sgnf(d.x) * sc_rgb, sgnf(d.y) * sc_rgb, sgnf(d.z) * sc_rgb, sgnf(d.w) * sc_rgb);
            }
            if (depth) {
                const long long off = v * n4 + q;
                const float4 x = reinterpret_cast<const float4 *>(depth)[off];
                const float4 y = reinterpret_cast<const float4 *>(depth_t)[off];
                const float4 d = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
                acc_d += (fabsf(d.x) + fabsf(d.y)) + (fabsf(d.z) + fabsf(d.w));
                reinterpret_cast<float4 *>(d_depth)[off] =
                    make_float4(sgnf(d.x) * sc_d, sgnf(d.y) * sc_d, sgnf(d.z) * sc_d, sgnf(d.w) * sc_d);
            }
        }
    } else {
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < HWn; p += stride) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long idx = (3 * v + c) * HWn + p;
                const float d = rgb[idx] - rgb_t[idx];
                acc_rgb += fabsf(d);
                d_rgb[idx] = sgnf(d) * sc_rgb;
            }
            if (depth) {
                const long long idx = v * HWn + p;
                const float d = depth[idx] - depth_t[idx];
                acc_d += fabsf(d);
                d_depth[idx] = sgnf(d) * sc_d;
            }
        }
    }
    block_add_double((double)acc_rgb * sc_rgb + (double)acc_d * sc_d, loss);
}

static bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

int launch_loss_l1(int V, int W, int H, const float *rgb, const float *rgb_t, const float *depth,
                   const float *depth_t, float w_rgb, float w_depth, float *d_rgb, float *d_depth, double *loss,
                   cudaStream_t s) {
    const long long HWn = (long long)W * H;
    const float sc_rgb = (float)((double)w_rgb / (3.0 * V * HWn));
    const float sc_d = (float)((double)w_depth / ((double)V * HWn));
    const bool use_d = depth && depth_t && d_depth && w_depth != 0.f;
    const bool vec = (HWn % 4 == 0) && aligned16(rgb) && aligned16(rgb_t) && aligned16(d_rgb) &&
                     (!use_d || (aligned16(depth) && aligned16(depth_t) && aligned16(d_depth)));
    const long long units = vec ? HWn / 4 : HWn;
    // about four resident blocks of 256 threads per SM in total, spread over the views
    const long long want = std::max<long long>(1, ((long long)device_sm_count() * 4 + V - 1) / V);
    const int gx = (int)std::max<long long>(1, std::min<long long>((units + 255) / 256, want));
    if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    const dim3 grid(gx, V);
    if (vec)
        k_l1<true><<<grid, 256, 0, s>>>(HWn, rgb, rgb_t, use_d ? depth : nullptr, depth_t, sc_rgb, sc_d, d_rgb,
                                        use_d ? d_depth : nullptr, loss);
    else
        k_l1<false><<<grid, 256, 0, s>>>(HWn, rgb, rgb_t, use_d ? depth : nullptr, depth_t, sc_rgb, sc_d, d_rgb,
                                         use_d ? d_depth : nullptr, loss);
    count_launches(1);
    return check_launch();
}

// ------------------------------------------------------------------------------------------
// SSIM
// ------------------------------------------------------------------------------------------
constexpr int kSB = 32;            // output tile
constexpr int kR = 5;              // window radius
constexpr int kSI = kSB + 2 * kR;  // input tile with halo
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;

struct SsimTaps {
    float w[11];
};

static SsimTaps make_taps() {
    SsimTaps t;
    double g[11], sum = 0.0;
    for (int k = 0; k < 11; ++k) {
        const double d = k - 5;
        g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[k];
    }
    for (int k = 0; k < 11; ++k) t.w[k] = (float)(g[k] / sum);
    return t;
}

// Both passes map the 256 threads of a CTA as 32 columns x 8 rows: loads and the horizontal
// filter walk rows ty, ty + 8, ... of column tx; the vertical filter gives each thread kVRows
// consecutive output rows of its column and slides over the kVRows + 10 filtered rows they need,
// so every filtered value is read from shared memory once per thread instead of once per tap.
constexpr int kVRows = kSB / 8;

struct Ssim1Smem {
    float sx[kSI][kSI], sy[kSI][kSI];
    float h[5][kSI][kSB];
};
struct Ssim2Smem {
    float s[3][kSI][kSI];
    float h[3][kSI][kSB];
};

template <int M>
__device__ __forceinline__ void ssim_vpass(const float (&h)[M][kSI][kSB], const SsimTaps &tp, int tx, int ty,
                                           float (&out)[M][kVRows]) {
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < kVRows; ++q) out[m][q] = 0.f;
#pragma unroll
    for (int j = 0; j < kVRows + 2 * kR; ++j) {
        float hv[M];
#pragma unroll
        for (int m = 0; m < M; ++m) hv[m] = h[m][ty * kVRows + j][tx];
#pragma unroll
        for (int q = 0; q < kVRows; ++q) {
            const int k = j - q;
            if (k >= 0 && k <= 2 * kR) {
#pragma unroll
                for (int m = 0; m < M; ++m) out[m][q] += tp.w[k] * hv[m];
            }
        }
    }
}

// Pass 1 of one tile of one plane: x, y (x optionally as fl(fl(ea x) + eb)), zero padding; the
// five blurred moments, the SSIM map summed into the return value and the three per-pixel
// derivatives dS/dmu_x, dS/dE[x^2], dS/dE[xy] (scaled by inv_n) written for pass 2.
__device__ __forceinline__ double ssim_pass1_tile(Ssim1Smem &sm, int W, int H, const float *xp, const float *yp,
                                                  bool expo, float ea, float eb, const SsimTaps &tp, float inv_n,
                                                  float *dmu, float *dexx, float *dexy) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x0 = blockIdx.x * kSB - kR, y0 = blockIdx.y * kSB - kR;
    for (int r = ty; r < kSI; r += 8)
        for (int c = tx; c < kSI; c += 32) {
            const int gx = x0 + c, gy = y0 + r;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const long long o = (long long)gy * W + gx;
            const float xv = in ? xp[o] : 0.f;
            sm.sx[r][c] = in ? (expo ? fp::add(fp::mul(ea, xv), eb) : xv) : 0.f;   // zero padding
            sm.sy[r][c] = in ? yp[o] : 0.f;
        }
    __syncthreads();
    for (int r = ty; r < kSI; r += 8) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float xv = sm.sx[r][tx + k], yv = sm.sy[r][tx + k], w = tp.w[k];
            a0 += w * xv;
            a1 += w * yv;
            a2 += w * xv * xv;
            a3 += w * yv * yv;
            a4 += w * xv * yv;
        }
        sm.h[0][r][tx] = a0; sm.h[1][r][tx] = a1; sm.h[2][r][tx] = a2; sm.h[3][r][tx] = a3; sm.h[4][r][tx] = a4;
    }
    __syncthreads();
    float v5[5][kVRows];
    ssim_vpass<5>(sm.h, tp, tx, ty, v5);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < kVRows; ++q) {
        const int gx = blockIdx.x * kSB + tx, gy = blockIdx.y * kSB + ty * kVRows + q;
        if (gx >= W || gy >= H) continue;
        const float mx = v5[0][q], my = v5[1][q], exx = v5[2][q], eyy = v5[3][q], exy = v5[4][q];
        const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float iB = 1.f / (B1 * B2);
        const float S = A1 * A2 * iB;
        acc += (double)S;
        const long long o = (long long)gy * W + gx;
        dmu[o] = inv_n * ((2.f * my * A2 - 2.f * my * A1) * iB - S * (2.f * mx / B1 - 2.f * mx / B2));
        dexx[o] = inv_n * (-S / B2);
        dexy[o] = inv_n * (2.f * A1 * iB);
    }
    return acc;
}

// Pass 2 of one tile: the three derivative maps blurred (the adjoint of a zero-padded symmetric
// blur is the same blur); out[0..2] = blur(dS/dmu_x), blur(dS/dE[x^2]), blur(dS/dE[xy]) for the
// thread's kVRows outputs.
__device__ __forceinline__ void ssim_pass2_tile(Ssim2Smem &sm, int W, int H, const float *dmu, const float *dexx,
                                                const float *dexy, const SsimTaps &tp, float (&out)[3][kVRows]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x0 = blockIdx.x * kSB - kR, y0 = blockIdx.y * kSB - kR;
    for (int r = ty; r < kSI; r += 8)
        for (int c = tx; c < kSI; c += 32) {
            const int gx = x0 + c, gy = y0 + r;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const long long o = (long long)gy * W + gx;
            sm.s[0][r][c] = in ? dmu[o] : 0.f;
            sm.s[1][r][c] = in ? dexx[o] : 0.f;
            sm.s[2][r][c] = in ? dexy[o] : 0.f;
        }
    __syncthreads();
    for (int r = ty; r < kSI; r += 8) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float w = tp.w[k];
            a0 += w * sm.s[0][r][tx + k];
            a1 += w * sm.s[1][r][tx + k];
            a2 += w * sm.s[2][r][tx + k];
        }
        sm.h[0][r][tx] = a0; sm.h[1][r][tx] = a1; sm.h[2][r][tx] = a2;
    }
    __syncthreads();
    ssim_vpass<3>(sm.h, tp, tx, ty, out);
}

// pass 1: per image plane (view * 3 + channel) = blockIdx.z, tile (bx, by)
__global__ void __launch_bounds__(256) k_ssim1(int W, int H, const float *x, const float *y, SsimTaps tp,
                                               float inv_n, float *dmu, float *dexx, float *dexy, double *ssim_sum) {
    __shared__ Ssim1Smem sm;
    const long long off = (long long)blockIdx.z * W * H;
    const double acc = ssim_pass1_tile(sm, W, H, x + off, y + off, false, 1.f, 0.f, tp, inv_n, dmu + off, dexx + off,
                                       dexy + off);
    block_add_double(acc, ssim_sum);
}

// pass 2: blur the three derivative maps and combine with the L1 gradient
__global__ void __launch_bounds__(256) k_ssim2(int W, int H, const float *x, const float *y, SsimTaps tp,
                                               const float *dmu, const float *dexx, const float *dexy, float l1_scale,
                                               float w_ssim, float *d_rgb) {
    __shared__ Ssim2Smem sm;
    const long long off = (long long)blockIdx.z * W * H;
    float b[3][kVRows];
    ssim_pass2_tile(sm, W, H, dmu + off, dexx + off, dexy + off, tp, b);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kVRows; ++q) {
        const int gx = blockIdx.x * kSB + tx, gy = blockIdx.y * kSB + ty * kVRows + q;
        if (gx >= W || gy >= H) continue;
        const long long o = off + (long long)gy * W + gx;
        const float xv = x[o], yv = y[o];
        const float gs = b[0][q] + 2.f * xv * b[1][q] + yv * b[2][q];
        d_rgb[o] = l1_scale * sgnf(xv - yv) - w_ssim * gs;
    }
}

__global__ void k_l1_sum(long long n, const float *x, const float *y, double *out) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)fabsf(x[i] - y[i]);
    block_add_double(acc, out);
}

__global__ void k_ssim_finish(double *scratch_sums, float w_l1, float w_ssim, double inv_n, double *loss) {
    // scratch_sums[0] = sum |x - y|, scratch_sums[1] = sum of the SSIM map
    *loss = w_l1 * scratch_sums[0] * inv_n + w_ssim * (1.0 - scratch_sums[1] * inv_n);
}

size_t ssim_scratch_bytes(int V, int W, int H) {
    return 256 + 3 * sizeof(float) * (size_t)V * 3 * W * H;
}

int launch_loss_l1_ssim(int V, int W, int H, const float *rgb, const float *rgb_t, float w_l1, float w_ssim,
                        float *d_rgb, double *loss, void *scratch, cudaStream_t s) {
    static const SsimTaps taps = make_taps();
    const long long plane = (long long)W * H, n = 3LL * V * plane;
    double *sums = reinterpret_cast<double *>(scratch);
    float *dmu = reinterpret_cast<float *>(static_cast<char *>(scratch) + 256);
    float *dexx = dmu + n, *dexy = dexx + n;
    if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    dim3 grid((W + kSB - 1) / kSB, (H + kSB - 1) / kSB, 3 * V);
    const float inv_n = (float)(1.0 / (double)n);
    k_l1_sum<<<device_sm_count() * 4, 256, 0, s>>>(n, rgb, rgb_t, sums);
    k_ssim1<<<grid, 256, 0, s>>>(W, H, rgb, rgb_t, taps, inv_n, dmu, dexx, dexy, sums + 1);
    k_ssim2<<<grid, 256, 0, s>>>(W, H, rgb, rgb_t, taps, dmu, dexx, dexy, w_l1 * inv_n, w_ssim, d_rgb);
    k_ssim_finish<<<1, 1, 0, s>>>(sums, w_l1, w_ssim, 1.0 / (double)n, loss);
    count_launches(4);
    return check_launch();
}

// ------------------------------------------------------------------------------------------
// The loss above without a caller-provided scratch buffer (for callers that cannot allocate).
// Its scratch is this file's static device array: two running sums (256 bytes) followed by the
// three derivative maps of ONE image plane; planes are processed one after another on the
// caller's stream, each reusing the maps.
// ------------------------------------------------------------------------------------------
constexpr long long kNoallocMaxPlane = GS_SSIM_NOALLOC_MAX_PLANE;
constexpr size_t kNoallocBytes = 256 + 3 * sizeof(float) * (size_t)kNoallocMaxPlane;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

// Device address of g_noalloc_scratch on the current device.  (On the host the symbol names a
// host-side stand-in, never the device memory itself.)  Outside stream capture every call looks
// the address up again, which is cheap and stays right after a device reset has reloaded the
// module; while `s` is being captured the address cached by the last call outside capture is
// used, and without one the lookup is attempted once more.
static int noalloc_scratch(cudaStream_t s, void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GS_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return GS_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return GS_OK;
}

int launch_loss_l1_ssim_noalloc(int V, int W, int H, const float *rgb, const float *rgb_t, float w_l1,
                                float w_ssim, float *d_rgb, double *loss, cudaStream_t s) {
    const long long plane = (long long)W * H, n = 3LL * V * plane;
    if (plane > kNoallocMaxPlane) return GS_ERR_TOO_LARGE;
    static const SsimTaps taps = make_taps();
    void *base = nullptr;
    int rc = noalloc_scratch(s, &base);
    if (rc) return rc;
    double *sums = reinterpret_cast<double *>(base);
    float *dmu = reinterpret_cast<float *>(static_cast<char *>(base) + 256);
    float *dexx = dmu + plane, *dexy = dexx + plane;
    if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    const float inv_n = (float)(1.0 / (double)n);
    k_l1_sum<<<device_sm_count() * 4, 256, 0, s>>>(n, rgb, rgb_t, sums);
    dim3 grid((W + kSB - 1) / kSB, (H + kSB - 1) / kSB, 1);
    for (long long p = 0; p < 3LL * V; ++p) {
        const long long off = p * plane;
        k_ssim1<<<grid, 256, 0, s>>>(W, H, rgb + off, rgb_t + off, taps, inv_n, dmu, dexx, dexy, sums + 1);
        k_ssim2<<<grid, 256, 0, s>>>(W, H, rgb + off, rgb_t + off, taps, dmu, dexx, dexy, w_l1 * inv_n, w_ssim,
                                     d_rgb + off);
    }
    k_ssim_finish<<<1, 1, 0, s>>>(sums, w_l1, w_ssim, 1.0 / (double)n, loss);
    count_launches((int)(2 + 6LL * V));
    return check_launch();
}

// ------------------------------------------------------------------------------------------
// Adam
// ------------------------------------------------------------------------------------------
struct AdamArgs {
    long long n;
    float *p[5];            // means, log_scales, quats, opacity_logits, colors
    float *opac;            // activated opacity (rewritten)
    float *g[5];            // grads: means, log_scales, quats, opacities (w.r.t. o), colors
    float *m, *v;
    const int32_t *step;
    float lr[5];
    int zero;
    float iso_weight;       // lambda_s of the isotropy regulariser (0: none)
    double *iso_loss;       // optional: receives lambda_s L_iso (overwritten)
};

// One thread per Gaussian.  Moments are stored group-major, in the same layout as the parameters
// ([N,3] means | [N,3] log-scales | [N,4] quats | [N] logits | [N,3] colours), so a warp's moment
// accesses are as contiguous as its parameter accesses.
__global__ void __launch_bounds__(256) k_adam(AdamArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < a.n;
    const int t = *a.step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-15f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    const int dims[5] = {3, 3, 4, 1, 3};
    const long long goff[5] = {0, 3 * a.n, 6 * a.n, 10 * a.n, 11 * a.n};   // group offsets in m, v
    // isotropy regulariser (Eq. 4): lambda_s sum_axes |s - mean(s)|, s = exp(log-scale); its
    // gradient with respect to log-scale b is lambda_s (sg_b - mean(sg)) s_b, sg = sign(s - mean)
    float giso[3] = {0.f, 0.f, 0.f};
    float lsum = 0.f;
    if (a.iso_weight != 0.f && in) {
        float sc[3], sg[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) sc[k] = expf(a.p[1][3 * i + k]);
        const float sbar = (sc[0] + sc[1] + sc[2]) * (1.f / 3.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float d = sc[k] - sbar;
            sg[k] = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            lsum += fabsf(d);
        }
        const float sgm = (sg[0] + sg[1] + sg[2]) * (1.f / 3.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) giso[k] = a.iso_weight * (sg[k] - sgm) * sc[k];
    }
    if (a.iso_loss && a.iso_weight != 0.f) {   // one double atomic per warp
        double l = (double)(a.iso_weight * lsum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(a.iso_loss, l);
    }
    if (!in) return;
#pragma unroll
    for (int grp = 0; grp < 5; ++grp) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (d >= dims[grp]) break;
            const long long idx = i * dims[grp] + d;
            float gr = a.g[grp][idx];
            if (grp == 1) gr += giso[d];
            if (grp == 3) {
                const float o = a.opac[i];
                gr *= o * (1.f - o);
            }
            float *mp = a.m + goff[grp] + idx, *vp = a.v + goff[grp] + idx;
            const float mm = b1 * *mp + (1.f - b1) * gr;
            const float vv = b2 * *vp + (1.f - b2) * gr * gr;
            *mp = mm;
            *vp = vv;
            const float upd = a.lr[grp] * (mm / c1) / (sqrtf(vv / c2) + eps);
            const float np = a.p[grp][idx] - upd;
            a.p[grp][idx] = np;
            if (grp == 3) a.opac[i] = 1.f / (1.f + __expf(-np));
            if (a.zero) a.g[grp][idx] = 0.f;
        }
    }
}

__global__ void k_step_inc(int32_t *step) { *step += 1; }

int launch_adam(long long n, const gs_adam_state &st, const gs_grads &g, const float lr[5], int zero_grads,
                cudaStream_t s, float iso_weight, double *iso_loss) {
    AdamArgs a;
    a.iso_weight = iso_weight;
    a.iso_loss = iso_loss;
    if (iso_loss && cudaMemsetAsync(iso_loss, 0, sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    a.n = n;
    a.p[0] = st.means; a.p[1] = st.log_scales; a.p[2] = st.quats; a.p[3] = st.opacity_logits; a.p[4] = st.colors;
    a.opac = st.opacities;
    a.g[0] = g.means; a.g[1] = g.log_scales; a.g[2] = g.quats; a.g[3] = g.opacities; a.g[4] = g.colors;
    a.m = st.m;
    a.v = st.v;
    a.step = st.step;
    for (int k = 0; k < 5; ++k) a.lr[k] = lr[k];
    a.zero = zero_grads;
    if (n > 0) {
        k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
        count_launches(1);
    }
    k_step_inc<<<1, 1, 0, s>>>(st.step);
    count_launches(1);
    return check_launch();
}

}  // namespace gs

namespace gs {

// ------------------------------------------------------------------------------------------
// Joint refinement (Sec. III-C, Eq. 23): loss on the exposure-compensated render
// I~_v = exp(a_v) I^_v + b_v, its gradients with respect to I^, D^ and (a_v, b_v); pruning of
// Gaussians with opacity below a threshold; Adam on per-view pose deltas and exposures.
// ------------------------------------------------------------------------------------------
// I~ is formed as fl(fl(e^a I^) + b) with the decision-chain exponential, so the sign of the L1 term
// (an FP32 decision) is reproducible by any implementation that follows the same two roundings.
struct RefineArgs {
    int V, W, H;
    const float *rgb, *rgb_t, *depth, *depth_t, *expo;
    float w_l1, w_ssim, w_depth;
    float *d_rgb, *d_depth, *d_expo;
    double *loss;
    double *sums;          // [0] sum |I~ - I|, [1] sum SSIM map, [2] sum |D^ - D-|, then g_a[V], g_b[V]
    float *dmu, *dexx, *dexy;
};

__global__ void k_refine_l1(RefineArgs a) {
    const long long HWn = (long long)a.W * a.H, total = (long long)a.V * HWn;
    float acc_rgb = 0.f, acc_d = 0.f;
    const float sc_d = (float)((double)a.w_depth / (double)total);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / HWn, p = i - v * HWn;
        const float ea = spec_expf(a.expo[2 * v]), eb = a.expo[2 * v + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long idx = (3 * v + c) * HWn + p;
            acc_rgb += fabsf(fp::add(fp::mul(ea, a.rgb[idx]), eb) - a.rgb_t[idx]);
        }
        if (a.depth && a.d_depth) {
            const float d = a.depth[i] - a.depth_t[i];
            acc_d += fabsf(d);
            a.d_depth[i] = sgnf(d) * sc_d;
        }
    }
    block_add_double((double)acc_rgb, a.sums);
    block_add_double((double)acc_d, a.sums + 2);
}

__global__ void __launch_bounds__(256) k_refine_ssim1(RefineArgs a, SsimTaps tp, float inv_n) {
    __shared__ Ssim1Smem sm;
    const long long plane = blockIdx.z;
    const int v = (int)(plane / 3);
    const float ea = spec_expf(a.expo[2 * v]), eb = a.expo[2 * v + 1];
    const long long off = plane * (long long)a.W * a.H;
    const double acc = ssim_pass1_tile(sm, a.W, a.H, a.rgb + off, a.rgb_t + off, true, ea, eb, tp, inv_n,
                                       a.dmu + off, a.dexx + off, a.dexy + off);
    block_add_double(acc, a.sums + 1);
}

__global__ void __launch_bounds__(256) k_refine_ssim2(RefineArgs a, SsimTaps tp, float l1_scale) {
    __shared__ Ssim2Smem sm;
    const int W = a.W, H = a.H;
    const long long plane = blockIdx.z;
    const int v = (int)(plane / 3);
    const float ea = spec_expf(a.expo[2 * v]), eb = a.expo[2 * v + 1];
    const long long off = plane * (long long)W * H;
    float b[3][kVRows];
    ssim_pass2_tile(sm, W, H, a.dmu + off, a.dexx + off, a.dexy + off, tp, b);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float ga = 0.f, gb = 0.f;
#pragma unroll
    for (int q = 0; q < kVRows; ++q) {
        const int gx = blockIdx.x * kSB + tx, gy = blockIdx.y * kSB + ty * kVRows + q;
        if (gx >= W || gy >= H) continue;
        const long long o = off + (long long)gy * W + gx;
        const float xv = a.rgb[o], yv = a.rgb_t[o];
        const float xt = fp::add(fp::mul(ea, xv), eb);       // I~ exactly as the FP32 L1 sign decision takes it
        const float g = l1_scale * sgnf(xt - yv) - a.w_ssim * (b[0][q] + 2.f * xt * b[1][q] + yv * b[2][q]);
        a.d_rgb[o] = ea * g;                                 // dL/dI^ = e^a dL/dI~
        ga += g * ea * xv;
        gb += g;
    }
    block_add_double((double)ga, a.sums + 3 + v);
    block_add_double((double)gb, a.sums + 3 + a.V + v);
}

__global__ void k_refine_finish(RefineArgs a, double inv_n) {
    const int v = threadIdx.x;
    if (v == 0) {
        const double npx = (double)a.V * a.W * a.H;
        *a.loss = a.w_l1 * a.sums[0] * inv_n + a.w_ssim * (1.0 - a.sums[1] * inv_n) + a.w_depth * a.sums[2] / npx;
    }
    if (v < a.V && a.d_expo) {
        a.d_expo[2 * v] = (float)a.sums[3 + v];
        a.d_expo[2 * v + 1] = (float)a.sums[3 + a.V + v];
    }
}

size_t refine_scratch_bytes(int V, int W, int H) {
    const size_t head = ((size_t)(3 + 2 * V) * sizeof(double) + 255) & ~(size_t)255;
    return head + 3 * sizeof(float) * (size_t)V * 3 * W * H;
}

int launch_loss_refine(int V, int W, int H, const float *rgb, const float *rgb_t, const float *depth,
                       const float *depth_t, const float *expo, float w_l1, float w_ssim, float w_depth, float *d_rgb,
                       float *d_depth, float *d_expo, double *loss, void *scratch, cudaStream_t s) {
    static const SsimTaps taps = make_taps();
    const long long plane = (long long)W * H, n = 3LL * V * plane;
    const size_t head = ((size_t)(3 + 2 * V) * sizeof(double) + 255) & ~(size_t)255;
    RefineArgs a;
    a.V = V; a.W = W; a.H = H;
    a.rgb = rgb; a.rgb_t = rgb_t; a.depth = depth; a.depth_t = depth_t; a.expo = expo;
    a.w_l1 = w_l1; a.w_ssim = w_ssim; a.w_depth = (depth && depth_t && d_depth) ? w_depth : 0.f;
    a.d_rgb = d_rgb; a.d_depth = (depth && depth_t) ? d_depth : nullptr; a.d_expo = d_expo;
    a.loss = loss;
    a.sums = reinterpret_cast<double *>(scratch);
    a.dmu = reinterpret_cast<float *>(static_cast<char *>(scratch) + head);
    a.dexx = a.dmu + n;
    a.dexy = a.dexx + n;
    if (cudaMemsetAsync(a.sums, 0, (size_t)(3 + 2 * V) * sizeof(double), s) != cudaSuccess) return GS_ERR_CUDA;
    const float inv_n = (float)(1.0 / (double)n);
    const long long total = (long long)V * plane;
    const int g1 = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)device_sm_count() * 8));
    k_refine_l1<<<g1, 256, 0, s>>>(a);
    dim3 grid((W + kSB - 1) / kSB, (H + kSB - 1) / kSB, 3 * V);
    k_refine_ssim1<<<grid, 256, 0, s>>>(a, taps, inv_n);
    k_refine_ssim2<<<grid, 256, 0, s>>>(a, taps, w_l1 * inv_n);
    k_refine_finish<<<1, ((V + 31) / 32) * 32, 0, s>>>(a, 1.0 / (double)n);
    count_launches(4);
    return check_launch();
}

// ---- pruning: order-preserving compaction of the Gaussians with opacity >= threshold ----
__global__ void k_prune_flags(long long n, const float *op, float thr, uint32_t *flags) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        flags[i] = op[i] >= thr ? 1u : 0u;
}

__global__ void k_prune_scatter(long long n, gs_gaussians in, gs_gaussian_arrays out, const uint32_t *incl,
                                long long *kept) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t hi = incl[i], lo = i > 0 ? incl[i - 1] : 0u;
        if (i == n - 1) *kept = (long long)hi;
        if (hi == lo) continue;
        const long long j = hi - 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out.means[3 * j + k] = in.means[3 * i + k];
            out.log_scales[3 * j + k] = in.log_scales[3 * i + k];
            out.colors[3 * j + k] = in.colors[3 * i + k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) out.quats[4 * j + k] = in.quats[4 * i + k];
        out.opacities[j] = in.opacities[i];
    }
}

size_t prune_scratch_bytes(long long n) {
    const long long parts = (n + kScanTile - 1) / kScanTile;
    return 256 + (((size_t)n * 4 + 255) & ~(size_t)255) + (size_t)parts * 8;
}

int launch_prune(long long n, const gs_gaussians &in, float thr, const gs_gaussian_arrays &out, long long *kept,
                 void *scratch, cudaStream_t s) {
    BinArgs b;
    std::memset(&b, 0, sizeof(b));
    b.st = reinterpret_cast<DevStatus *>(scratch);
    b.touched = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + 256);
    b.scan_state = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 256 +
                                                          (((size_t)n * 4 + 255) & ~(size_t)255));
    b.P = n;
    b.cap = (1LL << 30) - 1;
    b.fault_scan_part = -1;
    b.spin_limit = kSpinLimit;
    if (cudaMemsetAsync(b.st, 0, sizeof(DevStatus), s) != cudaSuccess) return GS_ERR_CUDA;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 8));
    k_prune_flags<<<grid, 256, 0, s>>>(n, in.opacities, thr, b.touched);
    count_launches(1);
    int rc = run_scan_only(b, s);
    if (rc) return rc;
    k_prune_scatter<<<grid, 256, 0, s>>>(n, in, out, b.touched, kept);
    count_launches(1);
    return check_launch();
}

// ---- per-view Adam on the pose delta (applied as T <- Exp(delta) T) and the exposure ----
__global__ void k_view_adam(int V, gs_camera *cams, float *expo, float *m, float *vv, const int32_t *step,
                            const float *pose_grad, const float *expo_grad, float lr_pose, float lr_expo) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int t = *step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-15f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    float d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float g = k < 6 ? pose_grad[6 * v + k] : expo_grad[2 * v + (k - 6)];
        const float mm = b1 * m[8 * v + k] + (1.f - b1) * g;
        const float vk = b2 * vv[8 * v + k] + (1.f - b2) * g * g;
        m[8 * v + k] = mm;
        vv[8 * v + k] = vk;
        d[k] = -(k < 6 ? lr_pose : lr_expo) * (mm / c1) / (sqrtf(vk / c2) + eps);
    }
    expo[2 * v] += d[6];
    expo[2 * v + 1] += d[7];
    // Exp of the twist (rho = d[0..2], phi = d[3..5]): Rodrigues rotation and left Jacobian
    const float px = d[3], py = d[4], pz = d[5];
    const float th2 = px * px + py * py + pz * pz, th = sqrtf(th2);
    float A, B, Cc;   // Exp(phi) = I + A K + B K^2 ; Jl = I + B K + Cc K^2
    if (th < 1e-4f) {
        A = 1.f - th2 / 6.f;
        B = 0.5f - th2 / 24.f;
        Cc = 1.f / 6.f - th2 / 120.f;
    } else {
        A = sinf(th) / th;
        B = (1.f - cosf(th)) / th2;
        Cc = (th - sinf(th)) / (th2 * th);
    }
    const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
    float K2[9], Rx[9], Jl[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float I = (i % 4 == 0) ? 1.f : 0.f;
        Rx[i] = I + A * K[i] + B * K2[i];
        Jl[i] = I + B * K[i] + Cc * K2[i];
    }
    gs_camera c = cams[v];
    float R[9], tt[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) R[3 * i + j] = Rx[3 * i] * c.R[j] + Rx[3 * i + 1] * c.R[3 + j] + Rx[3 * i + 2] * c.R[6 + j];
        tt[i] = Rx[3 * i] * c.t[0] + Rx[3 * i + 1] * c.t[1] + Rx[3 * i + 2] * c.t[2] + Jl[3 * i] * d[0] +
                Jl[3 * i + 1] * d[1] + Jl[3 * i + 2] * d[2];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) c.R[i] = R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) c.t[i] = tt[i];
    cams[v] = c;
}

int launch_view_adam(int V, const gs_view_adam_state &st, const float *pose_grad, const float *expo_grad, float lr_pose,
                     float lr_expo, cudaStream_t s) {
    k_view_adam<<<(V + 127) / 128, 128, 0, s>>>(V, st.cameras, st.expo, st.m, st.v, st.step, pose_grad, expo_grad,
                                                 lr_pose, lr_expo);
    k_step_inc<<<1, 1, 0, s>>>(st.step);
    count_launches(2);
    return check_launch();
}

// ------------------------------------------------------------------------------------------
// zeroing of the five gradient arrays in one launch
// ------------------------------------------------------------------------------------------
struct ZeroArgs {
    float *p[5];
    long long len[5];     // floats per array
};

// grid (blocks, 5): row y clears array y, 16 bytes per store where the pointer allows it.
__global__ void k_zero_grads(ZeroArgs a) {
    float *p = a.p[blockIdx.y];
    const long long n = a.len[blockIdx.y];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long head = 0;
    if (((uintptr_t)p & 15u) == 0) {
        const long long n4 = n >> 2;
        float4 *q = reinterpret_cast<float4 *>(p);
        for (long long i = t0; i < n4; i += stride) q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        head = n4 << 2;
    }
    for (long long i = head + t0; i < n; i += stride) p[i] = 0.f;
}

int launch_grads_zero(long long n, const gs_grads &g, cudaStream_t s) {
    ZeroArgs a;
    float *ptr[5] = {g.means, g.log_scales, g.quats, g.opacities, g.colors};
    const long long per[5] = {3, 3, 4, 1, 3};
    for (int k = 0; k < 5; ++k) {
        a.p[k] = ptr[k];
        a.len[k] = per[k] * n;
    }
    const long long blocks = std::max<long long>(1, std::min<long long>((4 * n + 1023) / 1024,
                                                                        (long long)device_sm_count() * 2));
    k_zero_grads<<<dim3((unsigned)blocks, 5), 256, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
