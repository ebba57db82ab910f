// gs_photometric.cu -- anchor-image photometric residuals of the submap pose graph (Sec. III-B,
// Eq. 12) with their Jacobians w.r.t. the two Sim(3) submap corrections, reduced on the device to
// the robust Gauss-Newton blocks of each edge.
//
// For every anchor pixel u of an edge's source keyframe (every stride-th row and column):
//   p = R_s^T (d K_s^-1 [u + 0.5, 1] - t_s),  w = C_src p,  q = C_tgt^-1 w,  c = R_a q + t_a,
//   r_ch = I_s,ch(u) - I_t,ch(pi(c) - 0.5) (bilinear), Huber weight omega_ch and cost rho_ch.
// Membership in U_e (0 < d < inf, c_z > near, both bilinear taps inside the target image) and the
// bilinear cell are integer decisions, taken by one fixed FP32 operation sequence with
// round-to-nearest intrinsics and no fused multiply-add; the Jacobian and the sums use FP32 values.
//
// Left Sim(3) twists xi = (rho, phi, sigma) of the global frame perturb C_src and C_tgt, so
// dq/dxi_tgt = -dq/dxi_src and the 14 x 14 normal matrix has the block form [[S, -S], [-S, S]].
// With A = d pi / d xi_src (2 x 7) and the image gradient n_ch = dI_t,ch / d(sx, sy), the source
// Jacobian row of channel ch is j_ch = -n_ch^T A, hence per pixel
//   S += A^T (sum_ch omega n n^T) A,   s_g += -A^T (sum_ch omega r n),   cost += sum_ch rho,
// i.e. 28 + 7 + 2 running sums per thread (the 2 x 2 moment matrix folds the three channels).
// k_pho_edge: grid (blocks per edge, edges); the edge's anchor rows are dealt to its blocks, the
// block's threads sweep a row, and each thread keeps its sums in registers; a warp butterfly and
// a per-block FP64 sum write one partial per block.  k_pho_finish: one block per edge sums the partials in FP64 in a fixed order (results
// are deterministic) and scales by w_e / |U_e|.
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int kPhoThreads = 256;
constexpr int kPhoPPT = 2;            // anchor pixels per thread per step
constexpr int kPhoSums = 37;          // S (28, upper triangle row-major), s_g (7), cost, count
constexpr int kPhoStride = 40;        // doubles per partial

// FP32 rotation of a (w, x, y, z) quaternion, normalised first; operation order fixed.
__device__ void pho_quat_matrix(const float *qin, float *M) {
    using namespace fp;
    float w = qin[0], x = qin[1], y = qin[2], z = qin[3];
    const float n = fp::sqrt(add(add(add(mul(w, w), mul(x, x)), mul(y, y)), mul(z, z)));
    w = div(w, n);
    x = div(x, n);
    y = div(y, n);
    z = div(z, n);
    M[0] = sub(1.0f, mul(2.0f, add(mul(y, y), mul(z, z))));
    M[1] = mul(2.0f, sub(mul(x, y), mul(w, z)));
    M[2] = mul(2.0f, add(mul(x, z), mul(w, y)));
    M[3] = mul(2.0f, add(mul(x, y), mul(w, z)));
    M[4] = sub(1.0f, mul(2.0f, add(mul(x, x), mul(z, z))));
    M[5] = mul(2.0f, sub(mul(y, z), mul(w, x)));
    M[6] = mul(2.0f, sub(mul(x, z), mul(w, y)));
    M[7] = mul(2.0f, add(mul(y, z), mul(w, x)));
    M[8] = sub(1.0f, mul(2.0f, add(mul(x, x), mul(y, y))));
}

// (M v)_i = (M_i0 v_0 + M_i1 v_1) + M_i2 v_2 and the transposed form, every operation rounded.
__device__ __forceinline__ float pho_row(const float *M, int i, float a, float b, float c) {
    return fp::add(fp::add(fp::mul(M[3 * i], a), fp::mul(M[3 * i + 1], b)), fp::mul(M[3 * i + 2], c));
}
__device__ __forceinline__ float pho_col(const float *M, int i, float a, float b, float c) {
    return fp::add(fp::add(fp::mul(M[i], a), fp::mul(M[3 + i], b)), fp::mul(M[6 + i], c));
}

struct PhoEdgeConst {
    float Rs[9], ts[3], Ks[4];        // source anchor camera (world-to-camera) and intrinsics
    float ifx, ify;                   // rounded 1 / f_x, 1 / f_y of the source camera
    float Q1[9], t1[3], s1;           // C_src
    float Q2[9], t2[3], is2;          // C_tgt (rotation, translation, rounded 1 / s)
    float Ra[9], ta[3], Ka[4];        // target anchor camera
    float M[9];                       // dc/dw = R_a Q2^T / s2 (values)
    const float *img_s, *dep_s, *img_t;
    int valid;
};

__device__ bool pho_load_edge(const PhoArgs &a, int e, PhoEdgeConst &k) {
    const gs_pho_edge ed = a.edges[e];
    if (ed.src_image < 0 || ed.src_image >= a.num_images || ed.tgt_image < 0 || ed.tgt_image >= a.num_images ||
        ed.src_corr < 0 || ed.src_corr >= a.num_corr || ed.tgt_corr < 0 || ed.tgt_corr >= a.num_corr)
        return false;
    const gs_camera cs = a.cams[ed.src_image], ct = a.cams[ed.tgt_image];
    for (int i = 0; i < 9; ++i) {
        k.Rs[i] = cs.R[i];
        k.Ra[i] = ct.R[i];
    }
    for (int i = 0; i < 3; ++i) {
        k.ts[i] = cs.t[i];
        k.ta[i] = ct.t[i];
    }
    k.Ks[0] = cs.fx; k.Ks[1] = cs.fy; k.Ks[2] = cs.cx; k.Ks[3] = cs.cy;
    k.Ka[0] = ct.fx; k.Ka[1] = ct.fy; k.Ka[2] = ct.cx; k.Ka[3] = ct.cy;
    const gs_sim3 c1 = a.corrs[ed.src_corr], c2 = a.corrs[ed.tgt_corr];
    pho_quat_matrix(c1.q, k.Q1);
    pho_quat_matrix(c2.q, k.Q2);
    for (int i = 0; i < 3; ++i) {
        k.t1[i] = c1.t[i];
        k.t2[i] = c2.t[i];
    }
    k.s1 = c1.s;
    k.is2 = fp::div(1.0f, c2.s);
    k.ifx = fp::div(1.0f, cs.fx);
    k.ify = fp::div(1.0f, cs.fy);
    const float inv = k.is2;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)   // (R_a Q2^T)_ij = sum_k Ra_ik Q2_jk
            k.M[3 * i + j] = (k.Ra[3 * i] * k.Q2[3 * j] + k.Ra[3 * i + 1] * k.Q2[3 * j + 1] +
                              k.Ra[3 * i + 2] * k.Q2[3 * j + 2]) * inv;
    const size_t plane = (size_t)a.width * a.height;
    k.img_s = a.images + (size_t)ed.src_image * 3 * plane;
    k.dep_s = a.depths + (size_t)ed.src_image * plane;
    k.img_t = a.images + (size_t)ed.tgt_image * 3 * plane;
    return true;
}

struct PhoSample {
    bool ok;                          // pixel in U_e
    int x0, y0;                       // bilinear cell
    float ax, ay;                     // weights inside the cell
    float w0, w1, w2, c0, c1, iz;     // global point, target camera x, y and 1 / z
};

// The FP32 decision chain of one anchor pixel (column px as a float, yn of its row, depth d).
__device__ __forceinline__ PhoSample pho_chain(const PhoEdgeConst &k, float px, float yn, float d, float near_plane,
                                               int W, int H) {
    using namespace fp;
    PhoSample o;
    o.ok = false;
    o.x0 = o.y0 = 0;
    o.ax = o.ay = o.w0 = o.w1 = o.w2 = o.c0 = o.c1 = o.iz = 0.0f;
    if (!(d > 0.0f) || !(d < __int_as_float(0x7f800000))) return o;
    const float xn = mul(sub(add(px, 0.5f), k.Ks[2]), k.ifx);
    const float pc0 = sub(mul(xn, d), k.ts[0]), pc1 = sub(mul(yn, d), k.ts[1]), pc2 = sub(d, k.ts[2]);
    const float p0 = pho_col(k.Rs, 0, pc0, pc1, pc2), p1 = pho_col(k.Rs, 1, pc0, pc1, pc2),
                p2 = pho_col(k.Rs, 2, pc0, pc1, pc2);
    const float w0 = add(mul(k.s1, pho_row(k.Q1, 0, p0, p1, p2)), k.t1[0]);
    const float w1 = add(mul(k.s1, pho_row(k.Q1, 1, p0, p1, p2)), k.t1[1]);
    const float w2 = add(mul(k.s1, pho_row(k.Q1, 2, p0, p1, p2)), k.t1[2]);
    const float d0 = sub(w0, k.t2[0]), d1 = sub(w1, k.t2[1]), d2 = sub(w2, k.t2[2]);
    const float q0 = mul(pho_col(k.Q2, 0, d0, d1, d2), k.is2), q1 = mul(pho_col(k.Q2, 1, d0, d1, d2), k.is2),
                q2 = mul(pho_col(k.Q2, 2, d0, d1, d2), k.is2);
    const float c0 = add(pho_row(k.Ra, 0, q0, q1, q2), k.ta[0]);
    const float c1 = add(pho_row(k.Ra, 1, q0, q1, q2), k.ta[1]);
    const float c2 = add(pho_row(k.Ra, 2, q0, q1, q2), k.ta[2]);
    if (!(c2 > near_plane)) return o;
    const float iz = div(1.0f, c2);
    const float sx = sub(add(mul(k.Ka[0], mul(c0, iz)), k.Ka[2]), 0.5f);
    const float sy = sub(add(mul(k.Ka[1], mul(c1, iz)), k.Ka[3]), 0.5f);
    if (!(sx >= 0.0f) || !(sx < (float)(W - 1)) || !(sy >= 0.0f) || !(sy < (float)(H - 1))) return o;
    const float fx0 = floorf(sx), fy0 = floorf(sy);
    o.ok = true;
    o.x0 = (int)fx0;
    o.y0 = (int)fy0;
    o.ax = sx - fx0;
    o.ay = sy - fy0;
    o.w0 = w0;
    o.w1 = w1;
    o.w2 = w2;
    o.c0 = c0;
    o.c1 = c1;
    o.iz = iz;
    return o;
}

__global__ void __launch_bounds__(kPhoThreads, 2) k_pho_edge(PhoArgs a) {
    using namespace fp;
    __shared__ PhoEdgeConst k;
    __shared__ float red[kPhoThreads / 32][kPhoSums];
    const int e = blockIdx.y;
    if (threadIdx.x == 0) k.valid = pho_load_edge(a, e, k) ? 1 : 0;
    __syncthreads();

    float S[28], sg[7], cost = 0.0f, cnt = 0.0f;
#pragma unroll
    for (int i = 0; i < 28; ++i) S[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 7; ++i) sg[i] = 0.0f;

    const int W = a.width, H = a.height, st = a.stride;
    const int nx = (W + st - 1) / st, ny = (H + st - 1) / st;
    const size_t plane = (size_t)W * H;
    // anchor rows are dealt to the edge's blocks round-robin; the block's threads sweep each row,
    // kPhoPPT pixels per thread per step: all loads of a step are issued before the arithmetic
    // that needs them (depth and source colour first, then the bilinear taps of every valid pixel)
    for (int ry = blockIdx.x; k.valid && ry < ny; ry += gridDim.x) {
        const int py = ry * st;
        const float yn = mul(sub(add((float)py, 0.5f), k.Ks[3]), k.ify);
        const float *dep_row = k.dep_s + (size_t)py * W;
        const size_t os_row = (size_t)py * W;
        for (int rx0 = threadIdx.x; rx0 < nx; rx0 += kPhoThreads * kPhoPPT) {
            float dd[kPhoPPT], src[kPhoPPT][3];
#pragma unroll
            for (int p = 0; p < kPhoPPT; ++p) {
                const int rx = rx0 + p * kPhoThreads;
                const bool in = rx < nx;
                const int px = in ? rx * st : 0;
                dd[p] = in ? __ldg(dep_row + px) : 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) src[p][ch] = in ? __ldg(k.img_s + ch * plane + os_row + px) : 0.0f;
            }
            PhoSample sm[kPhoPPT];
#pragma unroll
            for (int p = 0; p < kPhoPPT; ++p)
                sm[p] = pho_chain(k, (float)((rx0 + p * kPhoThreads) * st), yn, dd[p], a.near_plane, W, H);
            float tap[kPhoPPT][3][4];
#pragma unroll
            for (int p = 0; p < kPhoPPT; ++p) {
                const size_t o00 = sm[p].ok ? (size_t)sm[p].y0 * W + sm[p].x0 : 0;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float *It = k.img_t + ch * plane + o00;
                    tap[p][ch][0] = sm[p].ok ? __ldg(It) : 0.0f;
                    tap[p][ch][1] = sm[p].ok ? __ldg(It + 1) : 0.0f;
                    tap[p][ch][2] = sm[p].ok ? __ldg(It + W) : 0.0f;
                    tap[p][ch][3] = sm[p].ok ? __ldg(It + W + 1) : 0.0f;
                }
            }
#pragma unroll
            for (int p = 0; p < kPhoPPT; ++p) {
                if (!sm[p].ok) continue;
                const float ax = sm[p].ax, ay = sm[p].ay;
                // ---- bilinear samples, image gradient, Huber ----
                float G00 = 0.0f, G01 = 0.0f, G11 = 0.0f, h0 = 0.0f, h1 = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float i00 = tap[p][ch][0], i01 = tap[p][ch][1], i10 = tap[p][ch][2], i11 = tap[p][ch][3];
                    const float top = i00 + ax * (i01 - i00);
                    const float bot = i10 + ax * (i11 - i10);
                    const float val = top + ay * (bot - top);
                    const float gx = (i01 - i00) * (1.0f - ay) + (i11 - i10) * ay;
                    const float gy = bot - top;
                    const float r = src[p][ch] - val;
                    const float ar = fabsf(r);
                    float om, rho;
                    if (ar <= a.huber_delta) {
                        om = 1.0f;
                        rho = r * r;
                    } else {
                        om = a.huber_delta / ar;
                        rho = a.huber_delta * (2.0f * ar - a.huber_delta);
                    }
                    cost += rho;
                    G00 += om * gx * gx;
                    G01 += om * gx * gy;
                    G11 += om * gy * gy;
                    h0 += om * r * gx;
                    h1 += om * r * gy;
                }
                cnt += 1.0f;
                // ---- A = d(sx, sy)/d xi_src (2 x 7) ----
                const float iz = sm[p].iz, c0 = sm[p].c0, c1 = sm[p].c1;
                const float w0 = sm[p].w0, w1 = sm[p].w1, w2 = sm[p].w2;
                const float e00 = k.Ka[0] * iz, e02 = -k.Ka[0] * c0 * iz * iz;
                const float e11 = k.Ka[1] * iz, e12 = -k.Ka[1] * c1 * iz * iz;
                float A0[7], A1[7];
#pragma unroll
                for (int j = 0; j < 3; ++j) {   // P = dpi/dc . M
                    A0[j] = e00 * k.M[j] + e02 * k.M[6 + j];
                    A1[j] = e11 * k.M[3 + j] + e12 * k.M[6 + j];
                }
                // rotation columns: P (-[w]x); scale column: P w
                A0[3] = A0[2] * w1 - A0[1] * w2;
                A0[4] = A0[0] * w2 - A0[2] * w0;
                A0[5] = A0[1] * w0 - A0[0] * w1;
                A0[6] = A0[0] * w0 + A0[1] * w1 + A0[2] * w2;
                A1[3] = A1[2] * w1 - A1[1] * w2;
                A1[4] = A1[0] * w2 - A1[2] * w0;
                A1[5] = A1[1] * w0 - A1[0] * w1;
                A1[6] = A1[0] * w0 + A1[1] * w1 + A1[2] * w2;
                float B0[7], B1[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    B0[j] = G00 * A0[j] + G01 * A1[j];
                    B1[j] = G01 * A0[j] + G11 * A1[j];
                    sg[j] -= A0[j] * h0 + A1[j] * h1;
                }
                int idx = 0;
#pragma unroll
                for (int i = 0; i < 7; ++i)
#pragma unroll
                    for (int j = i; j < 7; ++j) S[idx++] += A0[i] * B0[j] + A1[i] * B1[j];
            }
        }
    }
    // ---- block reduction: warp butterfly, then FP64 over warps ----
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[kPhoSums];
#pragma unroll
    for (int i = 0; i < 28; ++i) v[i] = S[i];
#pragma unroll
    for (int i = 0; i < 7; ++i) v[28 + i] = sg[i];
    v[35] = cost;
    v[36] = cnt;
#pragma unroll
    for (int i = 0; i < kPhoSums; ++i) {
        float x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[i] = x;
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < kPhoSums; ++i) red[warp][i] = v[i];
    __syncthreads();
    if (threadIdx.x < kPhoSums) {
        double s = 0.0;
        for (int w = 0; w < kPhoThreads / 32; ++w) s += (double)red[w][threadIdx.x];
        a.partials[((size_t)e * gridDim.x + blockIdx.x) * kPhoStride + threadIdx.x] = s;
    }
}

__global__ void k_pho_finish(PhoArgs a, int bpe) {
    __shared__ double tot[kPhoSums];
    const int e = blockIdx.x;
    const gs_pho_edge ed = a.edges[e];
    const bool ok = !(ed.src_image < 0 || ed.src_image >= a.num_images || ed.tgt_image < 0 ||
                      ed.tgt_image >= a.num_images || ed.src_corr < 0 || ed.src_corr >= a.num_corr ||
                      ed.tgt_corr < 0 || ed.tgt_corr >= a.num_corr);
    if (threadIdx.x < kPhoSums) {
        double s = 0.0;
        for (int b = 0; b < bpe; ++b) s += a.partials[((size_t)e * bpe + b) * kPhoStride + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    const double n = tot[36];
    const double scale = (ok && n > 0.0) ? (double)ed.weight / n : 0.0;
    if (threadIdx.x == 0) {
        a.cost[e] = tot[35] * scale;
        a.count[e] = ok ? (int64_t)n : -1;
    }
    // H = scale [[S, -S], [-S, S]], g = scale [s_g, -s_g]
    for (int t = threadIdx.x; t < 196; t += blockDim.x) {
        const int r = t / 14, c = t % 14;
        const int i = r % 7, j = c % 7;
        const int lo = min(i, j), hi = max(i, j);
        const int idx = lo * 7 - lo * (lo - 1) / 2 + (hi - lo);
        const double sgn = ((r < 7) == (c < 7)) ? 1.0 : -1.0;
        a.H[(size_t)e * 196 + t] = sgn * scale * tot[idx];
    }
    if (threadIdx.x < 14) {
        const int i = threadIdx.x % 7;
        a.g[(size_t)e * 14 + threadIdx.x] = (threadIdx.x < 7 ? 1.0 : -1.0) * scale * tot[28 + i];
    }
}

size_t pho_scratch_bytes(int num_edges) {
    return (size_t)num_edges * kPhoMaxBlocksPerEdge * kPhoStride * sizeof(double);
}

int launch_pho(const PhoArgs &a, int num_edges, cudaStream_t s) {
    if (num_edges == 0) return GS_OK;
    // blocks per edge: enough to fill every SM at the kernel's occupancy, no more than the edge's
    // pixels need, at most kPhoMaxBlocksPerEdge (the scratch holds that many partials per edge)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pho_edge, kPhoThreads, 0) != cudaSuccess) per_sm = 1;
    const long long need = std::max<long long>(1, (a.height + a.stride - 1) / a.stride);   // anchor rows
    long long want = ((long long)device_sm_count() * std::max(per_sm, 1) + num_edges - 1) / num_edges;
    want = std::min<long long>(std::min<long long>(std::max<long long>(want, 1), need), kPhoMaxBlocksPerEdge);
    const int bpe = (int)want;
    k_pho_edge<<<dim3(bpe, num_edges), kPhoThreads, 0, s>>>(a);
    k_pho_finish<<<num_edges, 64, 0, s>>>(a, bpe);
    return GS_OK;
}

}  // namespace gs
