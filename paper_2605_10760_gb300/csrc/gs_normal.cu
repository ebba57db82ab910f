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
// takes (view, 16-row strip, 60-column block) items in turn: lane l holds the two columns
// x0 - 2 + 2l and x0 - 1 + 2l as the two components of packed FP32x2 arithmetic (lanes 0 and 31
// are the block's halo), and the warp walks down the strip's rows, one row per step, with the
// depths of the rows above and below in registers.  A step loads one depth and one prior row
// (8-byte pairs when the width is even), computes the normals and the adjoints of its row, and
// finishes the depth gradient of the row above: the neighbouring columns' depths and G_x come from
// the lane's other component or by one warp shuffle, G_y of the rows above and below from
// registers.  Every normal is computed once per item (the halo columns and the two rows beyond the
// strip are recomputed by the neighbouring items), and a pixel costs its depth, its prior and a
// read-modify-write of d_depth.  A row's inputs are copied by cp.async into a per-warp ring of
// shared-memory rows kNRing - 1 steps before the row is needed (each lane copies and later reads
// only its own two columns), so every warp keeps several rows of loads in flight without holding
// them in registers.  An item away from the image border (every row and column it reads inside,
// every pixel it normalises off the border) runs a copy of the item loop without index clamps or
// out-of-image selects.  Each depth's validity is tested once, when its row arrives, and rolled
// down with it.  Values in FP32; the loss in FP32 per item and FP64 per CTA.
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int kNormalThreads = 256;
constexpr int kNCols = 60;           // output columns of a warp's item (32 lanes x 2, less two halo lanes)
constexpr int kNRows = 16;           // output rows of an item
constexpr int kNRing = 4;            // rows of inputs per warp in shared memory (kNRing - 1 in flight)
constexpr int kNPlanes = 5;          // per ring row: depth below, three prior components, d_depth above

__device__ __forceinline__ bool nm_depth_ok(float d) { return d > 0.0f && d < __int_as_float(0x7f800000); }
__device__ __forceinline__ uint32_t nm_ok2(float2 d) {
    return (nm_depth_ok(d.x) ? 1u : 0u) | (nm_depth_ok(d.y) ? 2u : 0u);
}

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

// Per item and lane: the column indices of its two pixels clamped into the image (consecutive when
// the width is even, so that a pair is one aligned 8-byte copy) and which of them are real.
struct NormalCols {
    int ia, ib;
    bool ina, inb;
};

template <bool EVEN>
__device__ __forceinline__ float2 nm_ld2(const float *row, const NormalCols &c) {
    if constexpr (EVEN) return __ldg(reinterpret_cast<const float2 *>(row + c.ia));
    else return make_float2(__ldg(row + c.ia), __ldg(row + c.ib));
}

__device__ __forceinline__ float2 nm_sel2(bool a, bool b, float2 v, float z) {
    return make_float2(a ? v.x : z, b ? v.y : z);
}

template <int BYTES>
__device__ __forceinline__ void nm_cp_async(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void nm_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void nm_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kNRing - 1) : "memory"); }

// Copies the inputs of the step that normalises row y into ring row `slot` (the lane's two
// columns of each plane): the depths of row y + 1, the prior of row y, d_depth of row y - 1, every
// row clamped into the image (the out-of-image values are replaced when the ring row is read).
// One commit group per step; a step past the item's last row commits an empty group, so that
// waiting for all but the kNRing - 1 newest groups always completes the step being consumed.
template <bool EVEN, bool INTERIOR>
__device__ __forceinline__ void nm_issue_row(float (*ring)[64], const float *D, const float *Pr, const float *DD,
                                             const NormalCols &c, int HW, int W, int H, int y, int lane) {
    // an interior item's rows y - 1 .. y + 1 are inside the image: no clamping
    const int yb = INTERIOR ? y + 1 : min(max(y + 1, 0), H - 1), yc = INTERIOR ? y : min(max(y, 0), H - 1),
              ya = INTERIOR ? y - 1 : min(max(y - 1, 0), H - 1);
    const float *src[kNPlanes] = {D + yb * W, Pr + yc * W, Pr + HW + yc * W, Pr + 2 * HW + yc * W, DD + ya * W};
#pragma unroll
    for (int k = 0; k < kNPlanes; ++k) {
        float *dst = ring[k] + 2 * lane;
        if constexpr (EVEN) {
            nm_cp_async<8>(dst, src[k] + c.ia);
        } else {
            nm_cp_async<4>(dst, src[k] + c.ia);
            nm_cp_async<4>(dst + 1, src[k] + c.ib);
        }
    }
}

// One (view, 16-row strip, 60-column block) item of a warp (lane's first column xa = x0 - 2 + 2 lane);
// returns the loss of its own pixels.  INTERIOR: every row the item reads (y0 - 2 .. y0 + kNRows +
// 1) and every column (x0 - 3 .. x0 + kNCols + 2) lies inside the image and every pixel it
// normalises off the border, so no index is clamped and no value replaced.
template <bool EVEN, bool INTERIOR>
__device__ __forceinline__ float nm_run_item(const NormalArgs &a, float (*ring)[kNPlanes][64], int lane, int v,
                                             int y0, int xa) {
    using namespace fp2;
    const int W = a.W, H = a.H, HW = a.H * a.W;
    const float2 z2 = splat(0.0f);
    const bool inner = lane >= 1 && lane <= kNCols / 2;
    const bool own_a = inner && (INTERIOR || xa < W), own_b = inner && (INTERIOR || xa + 1 < W);
    const gs_camera &cam = a.cams[v];
    const float ifx = 1.0f / cam.fx, ify = 1.0f / cam.fy, cy = cam.cy;
    const float r_m = nm_ray(xa - 1, cam.cx, ifx), r_a = nm_ray(xa, cam.cx, ifx), r_b = nm_ray(xa + 1, cam.cx, ifx),
                r_p = nm_ray(xa + 2, cam.cx, ifx);
    const float2 rxl = make_float2(r_m, r_a), rxc = make_float2(r_a, r_b), rxr = make_float2(r_b, r_p);
    const bool colok_a = INTERIOR || (xa >= 1 && xa <= W - 2), colok_b = INTERIOR || (xa + 1 >= 1 && xa + 1 <= W - 2);
    NormalCols c;
    c.ina = INTERIOR || (unsigned)xa < (unsigned)W;
    c.inb = INTERIOR || (unsigned)(xa + 1) < (unsigned)W;
    if (INTERIOR) {
        c.ia = xa;
        c.ib = xa + 1;
    } else if (EVEN) {   // xa is even: both columns or neither inside the image
        c.ia = min(max(xa, 0), W - 2);
        c.ib = c.ia + 1;
    } else {
        c.ia = min(max(xa, 0), W - 1);
        c.ib = min(max(xa + 1, 0), W - 1);
    }
    const float *D = a.depth + (size_t)v * HW;
    const float *Pr = a.prior + (size_t)v * 3 * HW;
    float *DD = a.d_depth + (size_t)v * HW;
    const int yend = min(y0 + kNRows, H);              // the rows y0 .. yend - 1 are this item's
    const int nsteps = yend - y0 + 2;                  // rows y0 - 1 .. yend are normalised
    // the first kNRing - 1 steps' inputs in flight, then rows y0 - 2 and y0 - 1 of the lane's
    // columns (plain loads)
#pragma unroll
    for (int q = 0; q < kNRing - 1; ++q) {
        if (q < nsteps) nm_issue_row<EVEN, INTERIOR>(ring[q], D, Pr, DD, c, HW, W, H, y0 - 1 + q, lane);
        nm_cp_commit();
    }
    const float2 dm2 = nm_ld2<EVEN>(D + (INTERIOR ? y0 - 2 : min(max(y0 - 2, 0), H - 1)) * W, c);
    const float2 dm1 = nm_ld2<EVEN>(D + (INTERIOR ? y0 - 1 : min(max(y0 - 1, 0), H - 1)) * W, c);
    float2 d_up = nm_sel2(c.ina && (INTERIOR || y0 >= 2), c.inb && (INTERIOR || y0 >= 2), dm2, -1.0f);
    float2 d_mid = nm_sel2(c.ina && (INTERIOR || y0 >= 1), c.inb && (INTERIOR || y0 >= 1), dm1, -1.0f);
    // which of the lane's two depths are usable (bit 0: first column, bit 1: second), per row,
    // rolled down with the depths
    uint32_t ok_up = nm_ok2(d_up), ok_mid = nm_ok2(d_mid);
    float ry_up = nm_ray(y0 - 2, cy, ify), ry_mid = nm_ray(y0 - 1, cy, ify);
    float2 gxp0 = z2, gxp1 = z2, gxp2 = z2;            // G_x of the row above the current one
    float2 gyp0 = z2, gyp1 = z2, gyp2 = z2;            // G_y of the row above
    float2 gyq0 = z2, gyq1 = z2, gyq2 = z2;            // G_y two rows above
    float acc_item = 0.f;
    for (int st = 0; st < nsteps; ++st) {
        const int y = y0 - 1 + st;
        // the inputs kNRing - 1 steps ahead go into the ring row the previous step read
        const int ahead = st + kNRing - 1;
        if (ahead < nsteps) nm_issue_row<EVEN, INTERIOR>(ring[ahead % kNRing], D, Pr, DD, c, HW, W, H, y0 - 1 + ahead, lane);
        nm_cp_commit();
        nm_cp_wait();                                  // this step's group has landed
        const float(*rr)[64] = ring[st % kNRing];
        const bool bin = INTERIOR || (unsigned)(y + 1) < (unsigned)H, cin = INTERIOR || (unsigned)y < (unsigned)H,
                   ain = INTERIOR || (unsigned)(y - 1) < (unsigned)H;
        const float2 d_dn = nm_sel2(c.ina && bin, c.inb && bin, *reinterpret_cast<const float2 *>(rr[0] + 2 * lane), -1.0f);
        const float2 p0 = nm_sel2(c.ina && cin, c.inb && cin, *reinterpret_cast<const float2 *>(rr[1] + 2 * lane), 0.0f);
        const float2 p1 = nm_sel2(c.ina && cin, c.inb && cin, *reinterpret_cast<const float2 *>(rr[2] + 2 * lane), 0.0f);
        const float2 p2 = nm_sel2(c.ina && cin, c.inb && cin, *reinterpret_cast<const float2 *>(rr[3] + 2 * lane), 0.0f);
        const float2 ddv = nm_sel2(c.ina && ain, c.inb && ain, *reinterpret_cast<const float2 *>(rr[4] + 2 * lane), 0.0f);
        const float ry_dn = nm_ray(y + 1, cy, ify);
        // the row's depths left and right of each column: the lane's other column, or the
        // neighbouring lane's by one shuffle
        const float2 d_l = make_float2(__shfl_up_sync(0xffffffffu, d_mid.y, 1), d_mid.x);
        const float2 d_r = make_float2(d_mid.y, __shfl_down_sync(0xffffffffu, d_mid.x, 1));
        const bool rowok = INTERIOR || (y >= 1 && y <= H - 2);
        // the flags of d_l and d_r: the lane's other column, or the neighbouring lane's flag (the
        // same shuffles as the depths, so each flag belongs to the depth it stands for)
        const uint32_t ok_dn = nm_ok2(d_dn);
        const uint32_t ok_l = ((__shfl_up_sync(0xffffffffu, ok_mid, 1) >> 1) & 1u) | ((ok_mid & 1u) << 1);
        const uint32_t ok_r = ((ok_mid >> 1) & 1u) | ((__shfl_down_sync(0xffffffffu, ok_mid, 1) & 1u) << 1);
        const uint32_t ok5 = ok_mid & ok_up & ok_dn & ok_l & ok_r;
        const bool ok_a = colok_a && rowok && (ok5 & 1u), ok_b = colok_b && rowok && (ok5 & 2u);
        float2 gx0 = z2, gx1 = z2, gx2 = z2, gy0 = z2, gy1 = z2, gy2 = z2;
        if (ok_a || ok_b) {
            // neighbours in a row share the ray's y component, in a column its x component
            const float2 dx_ = add(d_r, neg(d_l)), dy_ = add(d_dn, neg(d_up));
            const float2 tx0 = add(mul(d_r, rxr), neg(mul(d_l, rxl))), tx1 = mul(dx_, splat(ry_mid)), tx2 = dx_;
            const float2 ty0 = mul(dy_, rxc), ty1 = add(mul(d_dn, splat(ry_dn)), neg(mul(d_up, splat(ry_up)))),
                         ty2 = dy_;
            // u = t_y x t_x
            const float2 u0 = add(mul(ty1, tx2), neg(mul(ty2, tx1)));
            const float2 u1 = add(mul(ty2, tx0), neg(mul(ty0, tx2)));
            const float2 u2 = add(mul(ty0, tx1), neg(mul(ty1, tx0)));
            const float2 uu = fma(u0, u0, fma(u1, u1, mul(u2, u2)));
            const bool va = ok_a && uu.x > 0.0f, vb = ok_b && uu.y > 0.0f;
            // 1/|u| by the hardware reciprocal square root (a value, not a decision)
            const float2 inu = make_float2(va ? rsqrtf(uu.x) : 0.f, vb ? rsqrtf(uu.y) : 0.f);
            const float2 n0 = mul(u0, inu), n1 = mul(u1, inu), n2 = mul(u2, inu);
            const float2 cc = add(splat(1.0f), neg(fma(n0, p0, fma(n1, p1, mul(n2, p2)))));
            if (y >= y0 && y < yend)   // the own pixels of the item add their loss (selects: NaN-safe)
                acc_item += (own_a && va ? fabsf(cc.x) : 0.f) + (own_b && vb ? fabsf(cc.y) : 0.f);
            // -scale sign(c) weights the adjoint (sign(0) = 0)
            const float2 kk = make_float2(!va ? 0.f : (cc.x > 0.f ? -a.scale : (cc.x < 0.f ? a.scale : 0.f)),
                                          !vb ? 0.f : (cc.y > 0.f ? -a.scale : (cc.y < 0.f ? a.scale : 0.f)));
            const float2 gn0 = mul(kk, p0), gn1 = mul(kk, p1), gn2 = mul(kk, p2);
            const float2 pn = fma(n0, gn0, fma(n1, gn1, mul(n2, gn2)));
            const float2 gu0 = mul(add(gn0, neg(mul(n0, pn))), inu);
            const float2 gu1 = mul(add(gn1, neg(mul(n1, pn))), inu);
            const float2 gu2 = mul(add(gn2, neg(mul(n2, pn))), inu);
            // G_x = gu x t_y, G_y = t_x x gu; selects, not products with zero: an invalid
            // pixel's tangents may hold NaN or inf
            gx0 = nm_sel2(va, vb, add(mul(gu1, ty2), neg(mul(gu2, ty1))), 0.f);
            gx1 = nm_sel2(va, vb, add(mul(gu2, ty0), neg(mul(gu0, ty2))), 0.f);
            gx2 = nm_sel2(va, vb, add(mul(gu0, ty1), neg(mul(gu1, ty0))), 0.f);
            gy0 = nm_sel2(va, vb, add(mul(tx1, gu2), neg(mul(tx2, gu1))), 0.f);
            gy1 = nm_sel2(va, vb, add(mul(tx2, gu0), neg(mul(tx0, gu2))), 0.f);
            gy2 = nm_sel2(va, vb, add(mul(tx0, gu1), neg(mul(tx1, gu0))), 0.f);
        }
        // the row above (y - 1) is complete: + G_x of each pixel's left neighbour (t_x there =
        // P(q) - P(q - 2)), - G_x of its right one, + G_y of the pixel above it, - G_y of this row
        const float2 l0 = make_float2(__shfl_up_sync(0xffffffffu, gxp0.y, 1), gxp0.x);
        const float2 l1 = make_float2(__shfl_up_sync(0xffffffffu, gxp1.y, 1), gxp1.x);
        const float2 l2 = make_float2(__shfl_up_sync(0xffffffffu, gxp2.y, 1), gxp2.x);
        const float2 r0 = make_float2(gxp0.y, __shfl_down_sync(0xffffffffu, gxp0.x, 1));
        const float2 r1 = make_float2(gxp1.y, __shfl_down_sync(0xffffffffu, gxp1.x, 1));
        const float2 r2 = make_float2(gxp2.y, __shfl_down_sync(0xffffffffu, gxp2.x, 1));
        if ((own_a || own_b) && y > y0 && y <= yend) {
            const float2 dP0 = add(add(l0, neg(r0)), add(gyq0, neg(gy0)));
            const float2 dP1 = add(add(l1, neg(r1)), add(gyq1, neg(gy1)));
            const float2 dP2 = add(add(l2, neg(r2)), add(gyq2, neg(gy2)));
            const float2 nd = add(ddv, fma(rxc, dP0, fma(splat(ry_up), dP1, dP2)));
            float *row = DD + (y - 1) * W;
            if (EVEN) {   // xa even and inside: both pixels inside
                *reinterpret_cast<float2 *>(row + c.ia) = nd;
            } else {
                if (own_a) row[c.ia] = nd.x;
                if (own_b) row[c.ib] = nd.y;
            }
        }
        gyq0 = gyp0; gyq1 = gyp1; gyq2 = gyp2;
        gyp0 = gy0; gyp1 = gy1; gyp2 = gy2;
        gxp0 = gx0; gxp1 = gx1; gxp2 = gx2;
        d_up = d_mid;
        ok_up = ok_mid;
        ry_up = ry_mid;
        d_mid = d_dn;
        ok_mid = ok_dn;
        ry_mid = ry_dn;
    }
    return acc_item;
}

template <bool EVEN>
__global__ void __launch_bounds__(kNormalThreads, 2) k_normal(NormalArgs a) {
    __shared__ __align__(16) float s_ring[kNormalThreads / 32][kNRing][kNPlanes][64];
    const int lane = threadIdx.x & 31;
    float (*ring)[kNPlanes][64] = s_ring[threadIdx.x >> 5];
    const int W = a.W, H = a.H;                        // the launcher checks 3 H W < 2^31
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
        const int y0 = sr * kNRows, xa = (t - sr * cblocks) * kNCols - 2 + 2 * lane;   // the lane's first column
        const int x0 = xa + 2 - 2 * lane;
        const bool interior = x0 >= 3 && x0 + kNCols + 2 <= W - 1 && y0 >= 2 && y0 + kNRows + 1 <= H - 1;
        acc += (double)(interior ? nm_run_item<EVEN, true>(a, ring, lane, v, y0, xa)
                                 : nm_run_item<EVEN, false>(a, ring, lane, v, y0, xa));
    }
    nm_block_add(acc * (double)a.scale, a.loss);
}

int launch_loss_normal(const NormalArgs &a, cudaStream_t s) {
    if (a.W < 3 || a.H < 3) return check_launch();   // no pixel has four neighbours: L and d_depth unchanged
    if (3LL * a.H * a.W >= (1LL << 31)) return GS_ERR_INVALID_ARG;   // 32-bit offsets inside a view
    // an even width keeps every pixel pair 8-byte aligned (given 8-byte aligned planes)
    const bool even = (a.W % 2 == 0) && (((uintptr_t)a.depth | (uintptr_t)a.prior | (uintptr_t)a.d_depth) % 8 == 0);
    static int occ_e = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_normal<true>, kNormalThreads, 0) != cudaSuccess || b < 1)
            b = 1;
        return b;
    }();
    static int occ_o = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_normal<false>, kNormalThreads, 0) != cudaSuccess || b < 1)
            b = 1;
        return b;
    }();
    // persistent: as many CTAs as are resident at once (a second wave would only add a tail)
    const long long items = (long long)a.V * ((a.W + kNCols - 1) / kNCols) * ((a.H + kNRows - 1) / kNRows);
    const long long warps = kNormalThreads / 32;
    const long long grid = std::max<long long>(1, std::min<long long>((items + warps - 1) / warps,
                                                                      (long long)device_sm_count() * (even ? occ_e : occ_o)));
    if (even) k_normal<true><<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    else k_normal<false><<<(unsigned)grid, kNormalThreads, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

}  // namespace gs
