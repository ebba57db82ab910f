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

// item = (view, tile) in view-major, row-major tile order (32-bit: the launcher checks the count)
__device__ __forceinline__ void nm_item(int item, int tiles_x, int tiles_per_view, int &v, int &x0, int &y0) {
    v = item / tiles_per_view;
    const int t = item - v * tiles_per_view;
    const int ty = t / tiles_x;
    x0 = (t - ty * tiles_x) * kNTW;
    y0 = ty * kNTH;
}

__device__ __forceinline__ void nm_fetch(const NormalArgs &a, int v, int x0, int y0, NormalStage &st) {
    const size_t HW = (size_t)a.H * a.W;
    const float *D = a.depth + (size_t)v * HW;
#pragma unroll
    for (int k = 0; k < kNDPer; ++k) {
        const int i = threadIdx.x + k * kNormalThreads;
        const int ly = i / kNDW, lx = i - ly * kNDW;
        const int x = x0 - 2 + lx, y = y0 - 2 + ly;
        st.d[k] = (i < kNDElems && (unsigned)x < (unsigned)a.W && (unsigned)y < (unsigned)a.H)
                      ? D[(size_t)y * a.W + x] : -1.0f;
    }
    const float *Pr = a.prior + (size_t)v * 3 * HW;
#pragma unroll
    for (int k = 0; k < kNPPer; ++k) {
        const int i = threadIdx.x + k * kNormalThreads;
        const int ch = i / (kNGH * kNGW), r = i - ch * (kNGH * kNGW);
        const int gy_ = r / kNGW, gx_ = r - gy_ * kNGW;
        const int x = x0 - 1 + gx_, y = y0 - 1 + gy_;
        st.p[k] = (i < kNPElems && (unsigned)x < (unsigned)a.W && (unsigned)y < (unsigned)a.H)
                      ? Pr[(size_t)ch * HW + (size_t)y * a.W + x] : 0.0f;
    }
    const int x = x0 + threadIdx.x % kNTW, y = y0 + threadIdx.x / kNTW;
    st.dd = (x < a.W && y < a.H) ? a.d_depth[(size_t)v * HW + (size_t)y * a.W + x] : 0.0f;
}

__global__ void __launch_bounds__(kNormalThreads, 4) k_normal(NormalArgs a) {
    __shared__ float s_d[kNDH][kNDW];
    __shared__ float s_p[3][kNGH][kNGW];
    __shared__ float s_g[6][kNGH][kNGW];
    const long long HW = (long long)a.H * a.W;
    const int tiles_x = (a.W + kNTW - 1) / kNTW, tiles_y = (a.H + kNTH - 1) / kNTH;
    const int tpv = tiles_x * tiles_y, tiles = a.V * tpv;
    double acc = 0.0;      // the CTA's loss, summed per item in FP32 then once per item in FP64
    NormalStage st;
    int item = blockIdx.x;
    int v = 0, x0 = 0, y0 = 0;
    if (item < tiles) {
        nm_item(item, tiles_x, tpv, v, x0, y0);
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
        const int next = item + (int)gridDim.x;
        if (next < tiles) {   // the next item's inputs, in flight while this one is computed
            nm_item(next, tiles_x, tpv, v, x0, y0);
            nm_fetch(a, v, x0, y0, st);
        }
        const gs_camera &cam = a.cams[cv];
        const float ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy;
        __syncthreads();
        float acc_item = 0.f;
        // two horizontally adjacent pixels per thread, the two components of packed FP32x2
        // arithmetic (values only: every decision here is a validity test taken per component)
        static_assert(kNGW % 2 == 0 && kNGH * kNGW / 2 <= kNormalThreads, "one pixel pair per thread");
        if (threadIdx.x < kNGH * kNGW / 2) {
            const int gy_ = threadIdx.x / (kNGW / 2), gx0 = 2 * (threadIdx.x % (kNGW / 2));
            const int x = cx0 - 1 + gx0, y = cy0 - 1 + gy_;      // image coordinates of the first pixel
            const int cx = gx0 + 1, cy = gy_ + 1;                  // its position in s_d
            const float2 dc = make_float2(s_d[cy][cx], s_d[cy][cx + 1]);
            const float2 dl = make_float2(s_d[cy][cx - 1], s_d[cy][cx]);
            const float2 dr = make_float2(s_d[cy][cx + 1], s_d[cy][cx + 2]);
            const float2 du = make_float2(s_d[cy - 1][cx], s_d[cy - 1][cx + 1]);
            const float2 dd = make_float2(s_d[cy + 1][cx], s_d[cy + 1][cx + 1]);
            const bool rowok = y >= 1 && y <= a.H - 2;
            bool ok[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int xc = x + c;
                const float pc = c ? dc.y : dc.x, pl = c ? dl.y : dl.x, pr = c ? dr.y : dr.x, pu = c ? du.y : du.x,
                            pd = c ? dd.y : dd.x;
                ok[c] = rowok && xc >= 1 && xc <= a.W - 2 && nm_depth_ok(pc) && nm_depth_ok(pl) && nm_depth_ok(pr) &&
                        nm_depth_ok(pu) && nm_depth_ok(pd);
            }
            float3 gx2[2] = {make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 0.f)};
            float3 gy2[2] = {gx2[0], gx2[0]};
            if (ok[0] || ok[1]) {
                using namespace fp2;
                const float r0 = nm_ray(x, cam.cx, ifx);
                const float2 rxc = make_float2(r0, nm_ray(x + 1, cam.cx, ifx));
                const float2 rxl = make_float2(nm_ray(x - 1, cam.cx, ifx), r0);
                const float2 rxr = make_float2(rxc.y, nm_ray(x + 2, cam.cx, ifx));
                const float ryc = nm_ray(y, cam.cy, ify), ryu = nm_ray(y - 1, cam.cy, ify), ryd = nm_ray(y + 1, cam.cy, ify);
                // neighbours in a row share the ray's y component, in a column its x component
                const float2 dx_ = add(dr, neg(dl)), dy_ = add(dd, neg(du));
                const float2 tx0 = add(mul(dr, rxr), neg(mul(dl, rxl))), tx1 = mul(dx_, splat(ryc)), tx2 = dx_;
                const float2 ty0 = mul(dy_, rxc), ty1 = add(mul(dd, splat(ryd)), neg(mul(du, splat(ryu)))), ty2 = dy_;
                // u = t_y x t_x
                const float2 u0 = add(mul(ty1, tx2), neg(mul(ty2, tx1)));
                const float2 u1 = add(mul(ty2, tx0), neg(mul(ty0, tx2)));
                const float2 u2 = add(mul(ty0, tx1), neg(mul(ty1, tx0)));
                const float2 uu = fma(u0, u0, fma(u1, u1, mul(u2, u2)));
                const bool v0 = ok[0] && uu.x > 0.0f, v1 = ok[1] && uu.y > 0.0f;
                // 1/|u| by the hardware reciprocal square root (a value, not a decision)
                const float2 inu = make_float2(v0 ? rsqrtf(uu.x) : 0.f, v1 ? rsqrtf(uu.y) : 0.f);
                const float2 n0 = mul(u0, inu), n1 = mul(u1, inu), n2 = mul(u2, inu);
                const float2 b0 = make_float2(s_p[0][gy_][gx0], s_p[0][gy_][gx0 + 1]);
                const float2 b1 = make_float2(s_p[1][gy_][gx0], s_p[1][gy_][gx0 + 1]);
                const float2 b2 = make_float2(s_p[2][gy_][gx0], s_p[2][gy_][gx0 + 1]);
                const float2 cc = add(splat(1.0f), neg(fma(n0, b0, fma(n1, b1, mul(n2, b2)))));
                // own pixels of the tile add their loss; -scale sign(c) weights the adjoint
                const bool own0 = v0 && gx0 >= 1 && gx0 <= kNTW && gy_ >= 1 && gy_ <= kNTH;
                const bool own1 = v1 && gx0 + 1 >= 1 && gx0 + 1 <= kNTW && gy_ >= 1 && gy_ <= kNTH;
                acc_item += (own0 ? fabsf(cc.x) : 0.f) + (own1 ? fabsf(cc.y) : 0.f);   // selects: NaN-safe
                const float2 kk = make_float2(!v0 ? 0.f : (cc.x > 0.f ? -a.scale : (cc.x < 0.f ? a.scale : 0.f)),
                                              !v1 ? 0.f : (cc.y > 0.f ? -a.scale : (cc.y < 0.f ? a.scale : 0.f)));
                const float2 gn0 = mul(kk, b0), gn1 = mul(kk, b1), gn2 = mul(kk, b2);
                const float2 pn = fma(n0, gn0, fma(n1, gn1, mul(n2, gn2)));
                const float2 gu0 = mul(add(gn0, neg(mul(n0, pn))), inu);
                const float2 gu1 = mul(add(gn1, neg(mul(n1, pn))), inu);
                const float2 gu2 = mul(add(gn2, neg(mul(n2, pn))), inu);
                // G_x = gu x t_y, G_y = t_x x gu (zero where the pixel is invalid: kk = inu = 0)
                const float2 gxa = add(mul(gu1, ty2), neg(mul(gu2, ty1)));
                const float2 gxb = add(mul(gu2, ty0), neg(mul(gu0, ty2)));
                const float2 gxc = add(mul(gu0, ty1), neg(mul(gu1, ty0)));
                const float2 gya = add(mul(tx1, gu2), neg(mul(tx2, gu1)));
                const float2 gyb = add(mul(tx2, gu0), neg(mul(tx0, gu2)));
                const float2 gyc = add(mul(tx0, gu1), neg(mul(tx1, gu0)));
                // selects, not products with zero: an invalid pixel's tangents may hold NaN or inf
                if (v0) {
                    gx2[0] = make_float3(gxa.x, gxb.x, gxc.x);
                    gy2[0] = make_float3(gya.x, gyb.x, gyc.x);
                }
                if (v1) {
                    gx2[1] = make_float3(gxa.y, gxb.y, gxc.y);
                    gy2[1] = make_float3(gya.y, gyb.y, gyc.y);
                }
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                s_g[0][gy_][gx0 + c] = gx2[c].x; s_g[1][gy_][gx0 + c] = gx2[c].y; s_g[2][gy_][gx0 + c] = gx2[c].z;
                s_g[3][gy_][gx0 + c] = gy2[c].x; s_g[4][gy_][gx0 + c] = gy2[c].y; s_g[5][gy_][gx0 + c] = gy2[c].z;
            }
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
    if (tiles >= (1LL << 31)) return GS_ERR_INVALID_ARG;   // items are 32-bit
    const long long grid = std::max<long long>(1, std::min<long long>(tiles, (long long)device_sm_count() * occ));
    k_normal<<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
