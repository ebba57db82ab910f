// gs_normal.cu -- the normal term of the mapping loss (Eq. 4, lambda_n L_normal): the cosine loss
// |1 - N_hat . N_bar| between the normal induced by the rendered depth and a given normal prior,
// and its gradient with respect to the depth.
//
// One persistent kernel; a CTA takes (view, 32 x 8 tile) items in turn.  Per item the tile's depths
// with a 2-pixel halo and the prior over the tile plus a 1-pixel halo go to shared memory (loaded
// one item ahead into registers, so the next tile's loads overlap this tile's arithmetic); every
// pixel of the tile plus a 1-pixel halo computes, from P = D r with
// r = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1) its pixel ray (nm_ray), the central-difference
// tangents t_x = P(x+1, y) - P(x-1, y), t_y = P(x, y+1) - P(x, y-1), u = t_y x t_x and
// N_hat = u / |u| (facing the camera for a surface seen from the front), and the adjoints
// G_x = dL/dt_x, G_y = dL/dt_y into shared memory (zero where the pixel is invalid: on the image
// border, a depth of the pixel or of its four neighbours not positive and finite, or |u| = 0).
// The loss of the tile's own pixels goes to a per-thread FP64 sum (one atomic per CTA).  Then every
// pixel q of the tile adds r(q) . (G_x(q-x) - G_x(q+x) + G_y(q-y) - G_y(q+y)) to d_depth.  The halo
// pixels' adjoints are recomputed by each neighbouring tile instead of going through global
// memory, so a pixel costs its depth, its prior and a read-modify-write of d_depth.  Values in
// FP32.
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int kNormalThreads = 256;

__device__ __forceinline__ float3 nm_cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float nm_dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ bool nm_depth_ok(float d) { return d > 0.0f && d < __int_as_float(0x7f800000); }

// sum of v over the block, added to *out by one FP64 atomic
__device__ __forceinline__ void nm_block_add(double v, double *out) {
    __shared__ double s_part[kNormalThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < kNormalThreads / 32 ? s_part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0 && w != 0.0) atomicAdd(out, w);
    }
}

constexpr int kNTW = 32, kNTH = 8;                        // output tile
constexpr int kNDW = kNTW + 4, kNDH = kNTH + 4;            // depths: 2-pixel halo
constexpr int kNGW = kNTW + 2, kNGH = kNTH + 2;            // adjoints: 1-pixel halo
static_assert(kNTW * kNTH == kNormalThreads, "one output pixel per thread");

// the pixel ray of column x / row y (one expression for the normal and for its adjoint)
__device__ __forceinline__ float nm_ray(int x, float c, float inv_f) { return ((float)x + 0.5f - c) * inv_f; }

constexpr int kNDElems = kNDH * kNDW;                    // depths staged per tile
constexpr int kNPElems = 3 * kNGH * kNGW;                // prior components staged per tile
constexpr int kNDPer = (kNDElems + kNormalThreads - 1) / kNormalThreads;
constexpr int kNPPer = (kNPElems + kNormalThreads - 1) / kNormalThreads;

// Global inputs of one (view, tile) item, held in registers from the previous item on: the
// thread's share of the depth halo and of the prior over the adjoint region, and d_depth of its
// own output pixel.  Everything is loaded one item ahead, so a CTA's loads for the next tile are in
// flight while it computes the current one.
struct NormalStage {
    float d[kNDPer];
    float p[kNPPer];
    float dd;
};

__device__ __forceinline__ void nm_item(const NormalArgs &a, long long item, int tiles_x, int tiles_y, int &v,
                                        int &x0, int &y0) {
    v = (int)(item / ((long long)tiles_x * tiles_y));
    const int t = (int)(item - (long long)v * tiles_x * tiles_y);
    x0 = (t % tiles_x) * kNTW;
    y0 = (t / tiles_x) * kNTH;
}

__device__ __forceinline__ void nm_fetch(const NormalArgs &a, int v, int x0, int y0, NormalStage &st) {
    const long long HW = (long long)a.H * a.W;
    const float *D = a.depth + (long long)v * HW;
#pragma unroll
    for (int k = 0; k < kNDPer; ++k) {
        const int i = threadIdx.x + k * kNormalThreads;
        const int ly = i / kNDW, lx = i - ly * kNDW;
        const int x = x0 - 2 + lx, y = y0 - 2 + ly;
        st.d[k] = (i < kNDElems && x >= 0 && x < a.W && y >= 0 && y < a.H) ? D[(long long)y * a.W + x] : -1.0f;
    }
    const float *Pr = a.prior + (long long)v * 3 * HW;
#pragma unroll
    for (int k = 0; k < kNPPer; ++k) {
        const int i = threadIdx.x + k * kNormalThreads;
        const int ch = i / (kNGH * kNGW), r = i - ch * (kNGH * kNGW);
        const int gy_ = r / kNGW, gx_ = r - gy_ * kNGW;
        const int x = x0 - 1 + gx_, y = y0 - 1 + gy_;
        st.p[k] = (i < kNPElems && x >= 0 && x < a.W && y >= 0 && y < a.H)
                      ? Pr[(long long)ch * HW + (long long)y * a.W + x] : 0.0f;
    }
    const int x = x0 + threadIdx.x % kNTW, y = y0 + threadIdx.x / kNTW;
    st.dd = (x < a.W && y < a.H) ? a.d_depth[(long long)v * HW + (long long)y * a.W + x] : 0.0f;
}

__global__ void __launch_bounds__(kNormalThreads) k_normal(NormalArgs a) {
    __shared__ float s_d[kNDH][kNDW];
    __shared__ float s_p[3][kNGH][kNGW];
    __shared__ float s_g[6][kNGH][kNGW];
    const long long HW = (long long)a.H * a.W;
    const int tiles_x = (a.W + kNTW - 1) / kNTW, tiles_y = (a.H + kNTH - 1) / kNTH;
    const long long tiles = (long long)a.V * tiles_x * tiles_y;
    double acc = 0.0;      // the CTA's loss, summed per item in FP32 then once per item in FP64
    NormalStage st;
    long long item = blockIdx.x;
    int v = 0, x0 = 0, y0 = 0;
    if (item < tiles) {
        nm_item(a, item, tiles_x, tiles_y, v, x0, y0);
        nm_fetch(a, v, x0, y0, st);
    }
    // persistent over the (view, tile) items, so the loss needs one atomic per CTA, not per tile
    for (; item < tiles; item += gridDim.x) {
        __syncthreads();   // the previous item's reads of s_d, s_p and s_g are done
#pragma unroll
        for (int k = 0; k < kNDPer; ++k) {
            const int i = threadIdx.x + k * kNormalThreads;
            if (i < kNDElems) (&s_d[0][0])[i] = st.d[k];
        }
#pragma unroll
        for (int k = 0; k < kNPPer; ++k) {
            const int i = threadIdx.x + k * kNormalThreads;
            if (i < kNPElems) (&s_p[0][0][0])[i] = st.p[k];
        }
        const float dd_own = st.dd;
        const int cv = v, cx0 = x0, cy0 = y0;
        const long long next = item + gridDim.x;
        if (next < tiles) {   // the next item's inputs, in flight while this one is computed
            nm_item(a, next, tiles_x, tiles_y, v, x0, y0);
            nm_fetch(a, v, x0, y0, st);
        }
        const gs_camera &cam = a.cams[cv];
        const float ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy;
        __syncthreads();
        float acc_item = 0.f;
        for (int i = threadIdx.x; i < kNGH * kNGW; i += kNormalThreads) {
            const int gy_ = i / kNGW, gx_ = i - gy_ * kNGW;
            const int x = cx0 - 1 + gx_, y = cy0 - 1 + gy_;
            float3 gx = make_float3(0.f, 0.f, 0.f), gy = make_float3(0.f, 0.f, 0.f);
            if (x >= 1 && x <= a.W - 2 && y >= 1 && y <= a.H - 2) {
                const int cx = gx_ + 1, cy = gy_ + 1;            // position in s_d
                const float dc = s_d[cy][cx], dl = s_d[cy][cx - 1], dr = s_d[cy][cx + 1], du = s_d[cy - 1][cx],
                            dd = s_d[cy + 1][cx];
                if (nm_depth_ok(dc) && nm_depth_ok(dl) && nm_depth_ok(dr) && nm_depth_ok(du) && nm_depth_ok(dd)) {
                    const float rxc = nm_ray(x, cam.cx, ifx), rxl = nm_ray(x - 1, cam.cx, ifx),
                                rxr = nm_ray(x + 1, cam.cx, ifx);
                    const float ryc = nm_ray(y, cam.cy, ify), ryu = nm_ray(y - 1, cam.cy, ify),
                                ryd = nm_ray(y + 1, cam.cy, ify);
                    // neighbours in a row share the ray's y component, in a column its x component
                    const float3 tx = make_float3(dr * rxr - dl * rxl, (dr - dl) * ryc, dr - dl);
                    const float3 ty = make_float3((dd - du) * rxc, dd * ryd - du * ryu, dd - du);
                    const float3 u = nm_cross(ty, tx);
                    const float uu = nm_dot(u, u);
                    // 1/|u| by the hardware reciprocal square root (a value, not a decision: the
                    // validity test is on |u|^2 > 0, in FP32 like the oracle's |u| > 0)
                    if (uu > 0.0f) {
                        const float inu = rsqrtf(uu);
                        const float3 nh = make_float3(u.x * inu, u.y * inu, u.z * inu);
                        const float3 nb = make_float3(s_p[0][gy_][gx_], s_p[1][gy_][gx_], s_p[2][gy_][gx_]);
                        const float c = 1.0f - nm_dot(nh, nb);
                        if (gx_ >= 1 && gx_ <= kNTW && gy_ >= 1 && gy_ <= kNTH) acc_item += fabsf(c);   // own pixel
                        const float k = c > 0.f ? -a.scale : (c < 0.f ? a.scale : 0.f);   // -scale sign(c)
                        const float3 gn = make_float3(k * nb.x, k * nb.y, k * nb.z);
                        const float pn = nm_dot(nh, gn);
                        const float3 gu = make_float3((gn.x - nh.x * pn) * inu, (gn.y - nh.y * pn) * inu,
                                                      (gn.z - nh.z * pn) * inu);
                        gx = nm_cross(gu, ty);
                        gy = nm_cross(tx, gu);
                    }
                }
            }
            s_g[0][gy_][gx_] = gx.x; s_g[1][gy_][gx_] = gx.y; s_g[2][gy_][gx_] = gx.z;
            s_g[3][gy_][gx_] = gy.x; s_g[4][gy_][gx_] = gy.y; s_g[5][gy_][gx_] = gy.z;
        }
        acc += (double)acc_item;
        __syncthreads();
        const int tx_ = threadIdx.x % kNTW, ty_ = threadIdx.x / kNTW;
        const int x = cx0 + tx_, y = cy0 + ty_;
        if (x < a.W && y < a.H) {
            const int gx_ = tx_ + 1, gy_ = ty_ + 1;
            // + G_x of the left neighbour (t_x there = P(q) - P(q - 2)), - G_x of the right one,
            // + G_y of the pixel above, - G_y of the pixel below (zero outside the image)
            float3 dP;
            dP.x = s_g[0][gy_][gx_ - 1] - s_g[0][gy_][gx_ + 1] + s_g[3][gy_ - 1][gx_] - s_g[3][gy_ + 1][gx_];
            dP.y = s_g[1][gy_][gx_ - 1] - s_g[1][gy_][gx_ + 1] + s_g[4][gy_ - 1][gx_] - s_g[4][gy_ + 1][gx_];
            dP.z = s_g[2][gy_][gx_ - 1] - s_g[2][gy_][gx_ + 1] + s_g[5][gy_ - 1][gx_] - s_g[5][gy_ + 1][gx_];
            const float3 r = make_float3(nm_ray(x, cam.cx, ifx), nm_ray(y, cam.cy, ify), 1.0f);
            a.d_depth[(long long)cv * HW + (long long)y * a.W + x] = dd_own + nm_dot(r, dP);
        }
    }
    nm_block_add(acc * (double)a.scale, a.loss);
}

int launch_loss_normal(const NormalArgs &a, cudaStream_t s) {
    // persistent: as many CTAs as are resident at once (a second wave would only add a tail)
    static int occ = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_normal, kNormalThreads, 0) != cudaSuccess || b < 1) b = 1;
        return b;
    }();
    const long long tiles = (long long)a.V * ((a.W + kNTW - 1) / kNTW) * ((a.H + kNTH - 1) / kNTH);
    const long long grid = std::max<long long>(1, std::min<long long>(tiles, (long long)device_sm_count() * occ));
    k_normal<<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
