// gs_normal.cu -- the normal term of the mapping loss (Eq. 4, lambda_n L_normal): the cosine loss
// |1 - N_hat . N_bar| between the normal induced by the rendered depth and a given normal prior,
// and its gradient with respect to the depth.
//
// Per pixel q: P = D r with r = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1) its pixel ray
// (nm_ray), the central-difference tangents t_x = P(x+1, y) - P(x-1, y),
// t_y = P(x, y+1) - P(x, y-1), u = t_y x t_x and N_hat = u / |u| (facing the camera for a surface
// seen from the front), and the adjoints G_x = dL/dt_x, G_y = dL/dt_y (zero where the pixel is
// invalid: on the image border, a depth of the pixel or of its four neighbours not positive and
// finite, or |u| = 0).  The depth gradient of q gathers r(q) . (G_x(q-x) - G_x(q+x) + G_y(q-y) -
// G_y(q+y)).
//
// One persistent kernel of independent warps (no CTA barrier until the final loss sum).  A warp
// takes (view, 16-row strip, 30-column block) items in turn: lane l holds column x0 - 1 + l (lanes
// 0 and 31 are the block's halo columns) and the warp walks down the strip's rows, one row per
// step, with the depths of the rows above and below in registers.  A step loads one depth and one
// prior row (lane 0 and lane 31 one more depth each: the columns beside the halo), computes the
// normal and the adjoints of its row, and finishes the depth gradient of the row above: the left
// and right neighbours' G_x come by warp shuffles, G_y of the rows above and below from
// registers.  Every normal is computed once per item (the two halo columns and the two rows
// beyond the strip are recomputed by the neighbouring items), and a pixel costs its depth, its
// prior and a read-modify-write of d_depth.  The next row's loads are issued before the current
// row's arithmetic.  Values in FP32; the loss in FP32 per item and FP64 per CTA.
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int kNormalThreads = 256;
constexpr int kNCols = 30;           // output columns of a warp's item (32 lanes less two halo lanes)
constexpr int kNRows = 16;           // output rows of an item

__device__ __forceinline__ bool nm_depth_ok(float d) { return d > 0.0f && d < __int_as_float(0x7f800000); }

// the pixel ray of column x / row y (one expression for the normal and for its adjoint)
__device__ __forceinline__ float nm_ray(int x, float c, float inv_f) { return ((float)x + 0.5f - c) * inv_f; }

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

// The global inputs of one row step: the lane's depth one row below the row being normalised, its
// extra depth (lane 0: the column left of the halo, lane 31: the one right of it, of the row
// itself), the prior of its pixel, and d_depth of its pixel one row above (whose gradient the step
// finishes).  Every load reads a clamped (in-image) address; out-of-image depths then read as -1
// (invalid), priors and d_depth as 0.
struct NormalRow {
    float d_below, d_ext, p0, p1, p2, dd;
};

// Per item and lane: the column pointers (clamped into the image) and which of them are real.
struct NormalCol {
    const float *d, *de, *p;
    float *dd;
    bool xin, xein;
};

__device__ __forceinline__ void nm_fetch_row(const NormalCol &c, int HW, int W, int H, int y, NormalRow &r) {
    const int yb = min(max(y + 1, 0), H - 1), yc = min(max(y, 0), H - 1), ya = min(max(y - 1, 0), H - 1);
    const float db = __ldg(c.d + yb * W), de = __ldg(c.de + yc * W);
    const float p0 = __ldg(c.p + yc * W), p1 = __ldg(c.p + HW + yc * W), p2 = __ldg(c.p + 2 * HW + yc * W);
    const float dd = c.dd[ya * W];
    const bool bin = (unsigned)(y + 1) < (unsigned)H, cin = (unsigned)y < (unsigned)H, ain = (unsigned)(y - 1) < (unsigned)H;
    r.d_below = c.xin && bin ? db : -1.0f;
    r.d_ext = c.xein && cin ? de : -1.0f;
    const bool pin = c.xin && cin;
    r.p0 = pin ? p0 : 0.0f;
    r.p1 = pin ? p1 : 0.0f;
    r.p2 = pin ? p2 : 0.0f;
    r.dd = c.xin && ain ? dd : 0.0f;
}

__global__ void __launch_bounds__(kNormalThreads, 3) k_normal(NormalArgs a) {
    const int lane = threadIdx.x & 31;
    const int W = a.W, H = a.H, HW = a.H * a.W;      // the launcher checks 3 H W < 2^31
    const int cblocks = (W + kNCols - 1) / kNCols, strips = (H + kNRows - 1) / kNRows;
    const int per_view = cblocks * strips;
    const long long items = (long long)a.V * per_view;
    const long long nwarps = (long long)gridDim.x * (kNormalThreads / 32);
    double acc = 0.0;
    for (long long item = (long long)blockIdx.x * (kNormalThreads / 32) + (threadIdx.x >> 5); item < items;
         item += nwarps) {
        const int v = (int)(item / per_view);
        const int t = (int)(item - (long long)v * per_view);
        const int sr = t / cblocks;
        const int y0 = sr * kNRows, x = (t - sr * cblocks) * kNCols - 1 + lane;
        // lane 0 also reads the column left of it, lane 31 the one right of it
        const int xe = lane == 0 ? x - 1 : (lane == 31 ? x + 1 : -1);
        const bool own_col = lane >= 1 && lane <= kNCols && x < W;
        const gs_camera &cam = a.cams[v];
        const float ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy, cy = cam.cy;
        const float rxl = nm_ray(x - 1, cam.cx, ifx), rxc = nm_ray(x, cam.cx, ifx), rxr = nm_ray(x + 1, cam.cx, ifx);
        const bool colok = x >= 1 && x <= W - 2;
        NormalCol c;
        const int xc = min(max(x, 0), W - 1), xec = min(max(xe, 0), W - 1);
        c.d = a.depth + (size_t)v * HW + xc;
        c.de = a.depth + (size_t)v * HW + xec;
        c.p = a.prior + (size_t)v * 3 * HW + xc;
        c.dd = a.d_depth + (size_t)v * HW + xc;
        c.xin = (unsigned)x < (unsigned)W;
        c.xein = (unsigned)xe < (unsigned)W;
        // rows y0 - 2 and y0 - 1 of the own column, then the first step's inputs (row y0 - 1)
        const float dm2 = __ldg(c.d + min(max(y0 - 2, 0), H - 1) * W), dm1 = __ldg(c.d + min(max(y0 - 1, 0), H - 1) * W);
        float d_up = c.xin && y0 >= 2 ? dm2 : -1.0f;
        float d_mid = c.xin && y0 >= 1 ? dm1 : -1.0f;
        bool ok_up = nm_depth_ok(d_up), ok_mid = nm_depth_ok(d_mid);
        float ry_up = nm_ray(y0 - 2, cy, ify), ry_mid = nm_ray(y0 - 1, cy, ify);
        const int yend = min(y0 + kNRows, H);                // the rows y0 .. yend - 1 are this item's
        NormalRow cur;
        nm_fetch_row(c, HW, W, H, y0 - 1, cur);
        float gxp0 = 0.f, gxp1 = 0.f, gxp2 = 0.f;            // G_x of the row above the current one
        float gyp0 = 0.f, gyp1 = 0.f, gyp2 = 0.f;            // G_y of the row above
        float gyq0 = 0.f, gyq1 = 0.f, gyq2 = 0.f;            // G_y two rows above
        float acc_item = 0.f;
        for (int y = y0 - 1; y <= yend; ++y) {
            NormalRow nxt;
            if (y < yend) nm_fetch_row(c, HW, W, H, y + 1, nxt);
            const float d_dn = cur.d_below;
            const bool ok_dn = nm_depth_ok(d_dn);
            const float ry_dn = nm_ray(y + 1, cy, ify);
            // the row's depths left and right of the lane (lanes 0 and 31 from their extra read)
            const float d_l0 = __shfl_up_sync(0xffffffffu, d_mid, 1), d_r0 = __shfl_down_sync(0xffffffffu, d_mid, 1);
            const float d_l = lane == 0 ? cur.d_ext : d_l0, d_r = lane == 31 ? cur.d_ext : d_r0;
            const bool ok = colok && y >= 1 && y <= H - 2 && ok_mid && ok_up && ok_dn && nm_depth_ok(d_l) &&
                            nm_depth_ok(d_r);
            float gx0 = 0.f, gx1 = 0.f, gx2 = 0.f, gy0 = 0.f, gy1 = 0.f, gy2 = 0.f;
            if (ok) {
                // neighbours in a row share the ray's y component, in a column its x component
                const float dx_ = d_r - d_l, dy_ = d_dn - d_up;
                const float tx0 = d_r * rxr - d_l * rxl, tx1 = dx_ * ry_mid, tx2 = dx_;
                const float ty0 = dy_ * rxc, ty1 = d_dn * ry_dn - d_up * ry_up, ty2 = dy_;
                // u = t_y x t_x
                const float u0 = ty1 * tx2 - ty2 * tx1, u1 = ty2 * tx0 - ty0 * tx2, u2 = ty0 * tx1 - ty1 * tx0;
                const float uu = u0 * u0 + u1 * u1 + u2 * u2;
                if (uu > 0.0f) {
                    // 1/|u| by the hardware reciprocal square root (a value, not a decision)
                    const float inu = rsqrtf(uu);
                    const float n0 = u0 * inu, n1 = u1 * inu, n2 = u2 * inu;
                    const float cc = 1.0f - (n0 * cur.p0 + n1 * cur.p1 + n2 * cur.p2);
                    if (own_col && y >= y0 && y < yend) acc_item += fabsf(cc);
                    // -scale sign(c) weights the adjoint (sign(0) = 0)
                    const float kk = cc > 0.f ? -a.scale : (cc < 0.f ? a.scale : 0.f);
                    const float gn0 = kk * cur.p0, gn1 = kk * cur.p1, gn2 = kk * cur.p2;
                    const float pn = n0 * gn0 + n1 * gn1 + n2 * gn2;
                    const float gu0 = (gn0 - n0 * pn) * inu, gu1 = (gn1 - n1 * pn) * inu, gu2 = (gn2 - n2 * pn) * inu;
                    // G_x = gu x t_y, G_y = t_x x gu
                    gx0 = gu1 * ty2 - gu2 * ty1; gx1 = gu2 * ty0 - gu0 * ty2; gx2 = gu0 * ty1 - gu1 * ty0;
                    gy0 = tx1 * gu2 - tx2 * gu1; gy1 = tx2 * gu0 - tx0 * gu2; gy2 = tx0 * gu1 - tx1 * gu0;
                }
            }
            // the row above (y - 1) is complete: + G_x of its left neighbour (t_x there =
            // P(q) - P(q - 2)), - G_x of its right one, + G_y of the pixel above it, - G_y of this row
            const float l0 = __shfl_up_sync(0xffffffffu, gxp0, 1), r0 = __shfl_down_sync(0xffffffffu, gxp0, 1);
            const float l1 = __shfl_up_sync(0xffffffffu, gxp1, 1), r1 = __shfl_down_sync(0xffffffffu, gxp1, 1);
            const float l2 = __shfl_up_sync(0xffffffffu, gxp2, 1), r2 = __shfl_down_sync(0xffffffffu, gxp2, 1);
            if (own_col && y > y0 && y <= yend) {
                const float dP0 = l0 - r0 + gyq0 - gy0, dP1 = l1 - r1 + gyq1 - gy1, dP2 = l2 - r2 + gyq2 - gy2;
                c.dd[(y - 1) * W] = cur.dd + (rxc * dP0 + ry_up * dP1 + dP2);
            }
            gyq0 = gyp0; gyq1 = gyp1; gyq2 = gyp2;
            gyp0 = gy0; gyp1 = gy1; gyp2 = gy2;
            gxp0 = gx0; gxp1 = gx1; gxp2 = gx2;
            d_up = d_mid; ok_up = ok_mid; ry_up = ry_mid;
            d_mid = d_dn; ok_mid = ok_dn; ry_mid = ry_dn;
            if (y < yend) cur = nxt;
        }
        acc += (double)acc_item;
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
    if (3LL * a.H * a.W >= (1LL << 31)) return GS_ERR_INVALID_ARG;   // 32-bit offsets inside a view
    const long long items = (long long)a.V * ((a.W + kNCols - 1) / kNCols) * ((a.H + kNRows - 1) / kNRows);
    const long long warps = kNormalThreads / 32;
    const long long grid = std::max<long long>(1, std::min<long long>((items + warps - 1) / warps,
                                                                      (long long)device_sm_count() * occ));
    k_normal<<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
