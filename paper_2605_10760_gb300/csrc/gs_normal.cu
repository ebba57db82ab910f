// gs_normal.cu -- the normal term of the mapping loss (Eq. 4, lambda_n L_normal): the cosine loss
// |1 - N_hat . N_bar| between the normal induced by the rendered depth and a given normal prior,
// and its gradient with respect to the depth.
//
// k_normal_terms: a thread per pixel.  P = D r with r = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy,
// 1) the pixel's ray; central-difference tangents t_x = P(x+1, y) - P(x-1, y),
// t_y = P(x, y+1) - P(x, y-1); u = t_y x t_x, N_hat = u / |u| (facing the camera for a surface
// seen from the front).  A pixel is valid when it is not on the image border, its depth and its
// four neighbours' depths are positive and finite, and |u| > 0.  The pixel's loss term goes to a
// per-thread FP64 sum (one atomic per block); the adjoints G_x = dL/dt_x and G_y = dL/dt_y go to a
// scratch plane (zero for invalid pixels).  k_normal_gather: a thread per pixel q adds
// r(q) . (G_x(q-x) - G_x(q+x) + G_y(q-y) - G_y(q+y)) to d_depth, every neighbour read inside the
// image.  Values in FP32.
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

__global__ void __launch_bounds__(kNormalThreads) k_normal_terms(NormalArgs a) {
    const long long HW = (long long)a.H * a.W, n = (long long)a.V * HW;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * kNormalThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kNormalThreads) {
        const int v = (int)(i / HW);
        const long long pix = i - (long long)v * HW;
        const int y = (int)(pix / a.W), x = (int)(pix - (long long)y * a.W);
        float3 gx = make_float3(0.f, 0.f, 0.f), gy = make_float3(0.f, 0.f, 0.f);
        if (x >= 1 && x <= a.W - 2 && y >= 1 && y <= a.H - 2) {
            const float *D = a.depth + (long long)v * HW;
            const float dc = D[pix], dl = D[pix - 1], dr = D[pix + 1], du = D[pix - a.W], dd = D[pix + a.W];
            if (nm_depth_ok(dc) && nm_depth_ok(dl) && nm_depth_ok(dr) && nm_depth_ok(du) && nm_depth_ok(dd)) {
                const gs_camera &cam = a.cams[v];
                const float ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy;
                const float rxc = ((float)x + 0.5f - cam.cx) * ifx;
                const float rxl = ((float)(x - 1) + 0.5f - cam.cx) * ifx, rxr = ((float)(x + 1) + 0.5f - cam.cx) * ifx;
                const float ryc = ((float)y + 0.5f - cam.cy) * ify;
                const float ryu = ((float)(y - 1) + 0.5f - cam.cy) * ify, ryd = ((float)(y + 1) + 0.5f - cam.cy) * ify;
                // neighbours in a row share the ray's y component, in a column its x component
                const float3 tx = make_float3(dr * rxr - dl * rxl, (dr - dl) * ryc, dr - dl);
                const float3 ty = make_float3((dd - du) * rxc, dd * ryd - du * ryu, dd - du);
                const float3 u = nm_cross(ty, tx);
                const float nu = sqrtf(nm_dot(u, u));
                if (nu > 0.0f) {
                    const float inu = 1.0f / nu;
                    const float3 nh = make_float3(u.x * inu, u.y * inu, u.z * inu);
                    const float *pr = a.prior + (long long)v * 3 * HW + pix;
                    const float3 nb = make_float3(pr[0], pr[HW], pr[2 * HW]);
                    const float c = 1.0f - nm_dot(nh, nb);
                    acc += (double)fabsf(c);
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
        float *G = a.scratch + (long long)v * 6 * HW + pix;
        G[0] = gx.x;
        G[HW] = gx.y;
        G[2 * HW] = gx.z;
        G[3 * HW] = gy.x;
        G[4 * HW] = gy.y;
        G[5 * HW] = gy.z;
    }
    nm_block_add(acc * (double)a.scale, a.loss);
}

__global__ void __launch_bounds__(kNormalThreads) k_normal_gather(NormalArgs a) {
    const long long HW = (long long)a.H * a.W, n = (long long)a.V * HW;
    for (long long i = (long long)blockIdx.x * kNormalThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kNormalThreads) {
        const int v = (int)(i / HW);
        const long long pix = i - (long long)v * HW;
        const int y = (int)(pix / a.W), x = (int)(pix - (long long)y * a.W);
        const float *G = a.scratch + (long long)v * 6 * HW;
        float3 dP = make_float3(0.f, 0.f, 0.f);
        if (x >= 1) {                   // + G_x of the left neighbour (t_x there = P(q) - P(q - 2))
            const long long q = pix - 1;
            dP.x += G[q]; dP.y += G[HW + q]; dP.z += G[2 * HW + q];
        }
        if (x + 1 < a.W) {              // - G_x of the right neighbour
            const long long q = pix + 1;
            dP.x -= G[q]; dP.y -= G[HW + q]; dP.z -= G[2 * HW + q];
        }
        if (y >= 1) {                   // + G_y of the pixel above
            const long long q = pix - a.W;
            dP.x += G[3 * HW + q]; dP.y += G[4 * HW + q]; dP.z += G[5 * HW + q];
        }
        if (y + 1 < a.H) {              // - G_y of the pixel below
            const long long q = pix + a.W;
            dP.x -= G[3 * HW + q]; dP.y -= G[4 * HW + q]; dP.z -= G[5 * HW + q];
        }
        const gs_camera &cam = a.cams[v];
        const float3 r = make_float3(((float)x + 0.5f - cam.cx) / cam.fx, ((float)y + 0.5f - cam.cy) / cam.fy, 1.0f);
        a.d_depth[i] += nm_dot(r, dP);
    }
}

size_t normal_scratch_bytes(int V, int W, int H) { return (size_t)6 * sizeof(float) * (size_t)V * W * H; }

int launch_loss_normal(const NormalArgs &a, cudaStream_t s) {
    const long long n = (long long)a.V * a.W * a.H;
    const long long grid = std::max<long long>(1, std::min<long long>((n + kNormalThreads - 1) / kNormalThreads,
                                                                      (long long)device_sm_count() * 8));
    k_normal_terms<<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    k_normal_gather<<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    count_launches(2);
    return check_launch();
}

}  // namespace gs
