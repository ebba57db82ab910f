// gs_project.cu -- EWA projection of (view, Gaussian) pairs and its adjoint.
//
// Forward: the FP32 decision chain of gs_internal.cuh, grid (chunk, view), a pre-test per pair and
// the chain on the block's compacted candidates.
// Backward: per block, one thread per slot of the forward block's candidates (holes, the slots of
// candidates the chain found invisible, flagged and skipped); the chain rule through the same
// projection in FP32 value arithmetic, accumulating dL/d(mean, log-scale, quaternion, opacity,
// colour) with atomics (several views of one scene add into the same Gaussian; a reduction is
// issued without waiting for a result, which also makes it cheaper than a load and a store where
// no two views share a Gaussian) and the per-view SE(3) pose gradient as one partial sum per block.
#include "gs_kernels.cuh"

namespace gs {



// Pre-test of a pair before the decision chain: false only when the chain certainly finds the pair
// invisible.  The near-plane test and the mean are the chain's own operations; the radius is
// bounded from above: lambda_max(Sigma_2) <= trace = |U|_F^2 + 2 dilation with
// |U|_F <= |W|_F |M|_F, |M|_F^2 = s0^2 + s1^2 + s2^2 (unit quaternion) and
// |W|_F^2 <= (wx^2 + wy^2) / z^2 (wx = |fx| (|R_0| + |limx| |R_2|), wy likewise: the clamped
// Jacobian and the camera rows; `wb2` = wx^2 + wy^2 per view).  The bound is padded by 2 % in
// lambda, 1 % in the radius and one pixel, far above the FP32 error of either side, and the tile
// rectangle grows monotonically with the radius; a non-finite bound or a non-positive sigma
// multiplier never rejects.
__device__ __forceinline__ bool may_be_visible(const float *R, const float *t, float fx, float fy, float cx, float cy,
                                               float wb2, float itw, float ith, float Tx, float Ty, float near_plane,
                                               float dil, float sigmas, float m0, float m1, float m2,
                                               const float *ls) {
    using namespace fp;
    const float xc = fma(R[0], m0, fma(R[1], m1, fma(R[2], m2, t[0])));
    const float yc = fma(R[3], m0, fma(R[4], m1, fma(R[5], m2, t[1])));
    const float zc = fma(R[6], m0, fma(R[7], m1, fma(R[8], m2, t[2])));
    if (!(zc > near_plane)) return false;
    if (!(sigmas > 0.0f)) return true;
    const float iz = div(1.0f, zc);
    const float mx = fma(fx, mul(xc, iz), cx), my = fma(fy, mul(yc, iz), cy);
    const float ssum = __expf(2.0f * __ldg(ls)) + __expf(2.0f * __ldg(ls + 1)) + __expf(2.0f * __ldg(ls + 2));
    const float lam = (wb2 * iz * iz * ssum + 2.0f * fmaxf(dil, 0.0f)) * 1.02f;
    const float rb = sigmas * sqrtf(lam) * 1.01f + 1.0f;
    if (!(rb >= 0.0f && rb < 1e30f)) return true;
    int x0, x1, y0, y1;
    spec_rect(mx, my, rb, itw, ith, Tx, Ty, x0, x1, y0, y1);
    return x1 > x0 && y1 > y0;
}

// One block of kProjThreads threads = the 256 pairs (chunk) of one view, so that every chunk of a
// single-view problem is resident at once.  Phase 1: each thread pre-tests kProjPre pairs
// (may_be_visible); the candidates are compacted in pair order and take consecutive slots, reserved
// by one atomic per block on the slot counter, issued before the decision chain so that the
// chain's arithmetic hides its latency (the last block to reserve returns the counter to zero).  Phase 2: the candidates run the decision chain
// kProjThreads at a time; a visible one writes its record into its slot, an invisible one leaves
// its slot a hole.  The block records its first slot and candidate count (blk) and, per slot, the
// pair's position in the chunk, flagged kSlotHole for a hole (slane).  Slots beyond the capacity
// record GS_ERR_CAPACITY for a visible pair and drop it.
constexpr int kProjThreads = 64;
constexpr int kProjPre = kChunk / kProjThreads;   // pairs pre-tested per thread

__global__ void __launch_bounds__(kProjThreads) k_project(ProjArgs a) {
    const int v = blockIdx.y;
    __shared__ ViewEntry s_ve;
    __shared__ float s_cam[19];   // R, t, fx, fy, cx, cy, the clamp limits, then wb2
    __shared__ uint8_t s_cl[kChunk];
    __shared__ uint32_t s_wcnt[kProjPre][kProjThreads / 32];
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_ve = a.views[v];
    if (threadIdx.x < 16) s_cam[threadIdx.x] = reinterpret_cast<const float *>(a.cams + v)[threadIdx.x];
    if (threadIdx.x == 32) {      // once per view and block, the same operations as the per-pair chain
        const gs_camera &c = a.cams[v];
        const float limx = fp::div(fp::mul(0.65f, (float)a.W), c.fx);
        const float limy = fp::div(fp::mul(0.65f, (float)a.H), c.fy);
        s_cam[16] = limx;
        s_cam[17] = limy;
        const float n0 = sqrtf(c.R[0] * c.R[0] + c.R[1] * c.R[1] + c.R[2] * c.R[2]);
        const float n1 = sqrtf(c.R[3] * c.R[3] + c.R[4] * c.R[4] + c.R[5] * c.R[5]);
        const float n2 = sqrtf(c.R[6] * c.R[6] + c.R[7] * c.R[7] + c.R[8] * c.R[8]);
        const float wx = fabsf(c.fx) * (n0 + fabsf(limx) * n2), wy = fabsf(c.fy) * (n1 + fabsf(limy) * n2);
        s_cam[18] = wx * wx + wy * wy;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base_i = (long long)blockIdx.x * kChunk;
    // phase 1: pairs base_i + k kProjThreads + thread
    unsigned cmask[kProjPre];
#pragma unroll
    for (int k = 0; k < kProjPre; ++k) {
        const int li = k * kProjThreads + threadIdx.x;
        const long long i = base_i + li;
        const bool in = i < s_ve.count;
        const long long f = s_ve.pair_off + (in ? i : 0);
        const bool fok = gs_guard(a.st, !in || f < a.P, 1);   // the pair index comes from the views table
        bool cand = false;
        if (in && fok) {
            const long long gi = s_ve.gauss_begin + i;
            const float *mu = a.means + 3 * gi;
            cand = may_be_visible(s_cam, s_cam + 9, s_cam[12], s_cam[13], s_cam[14], s_cam[15], s_cam[18], a.itw,
                                  a.ith, a.Tx, a.Ty, a.near_plane, a.dil, a.sigmas, __ldg(mu), __ldg(mu + 1),
                                  __ldg(mu + 2), a.log_scales + 3 * gi);
            a.slot[f] = kNoSlot;   // a visible candidate overwrites it below
            if (!cand) a.touched[f] = 0u;
        }
        cmask[k] = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) s_wcnt[k][warp] = (uint32_t)__popc(cmask[k]);
    }
    __syncthreads();
    uint32_t ncand = 0;
#pragma unroll
    for (int k = 0; k < kProjPre; ++k) {
        uint32_t pre = ncand + (uint32_t)__popc(cmask[k] & lanemask_lt());
        for (int w = 0; w < warp; ++w) pre += s_wcnt[k][w];
        if ((cmask[k] >> lane) & 1u) s_cl[pre] = (uint8_t)(k * kProjThreads + threadIdx.x);
#pragma unroll
        for (int w = 0; w < kProjThreads / 32; ++w) ncand += s_wcnt[k][w];
    }
    __syncthreads();   // s_cl complete
    // the candidates' slots: one atomic, whose result is needed only after the first round's chain.
    // Every block takes part (also with no candidate) and counts itself in the high bits; the block
    // arriving last publishes the slot total and returns the counter to zero for the next launch
    unsigned long long base_reg = 0ull;
    if (threadIdx.x == 0) {
        const unsigned long long old = atomicAdd(&a.st->slot_ctr, (1ull << 40) + (unsigned long long)ncand);
        base_reg = old & ((1ull << 40) - 1ull);
        if ((old >> 40) == (unsigned long long)gridDim.x * gridDim.y - 1ull) {
            a.st->num_visible = base_reg + ncand;
            a.st->slot_ctr = 0ull;
        }
    }
    // phase 2: candidates r kProjThreads + thread through the decision chain
    const int rounds = (int)((ncand + kProjThreads - 1) / kProjThreads);
    for (int r = 0; r < rounds; ++r) {
        const int t = r * kProjThreads + threadIdx.x;
        const bool act = (uint32_t)t < ncand;
        const int li = act ? (int)s_cl[t] : 0;
        const long long i = base_i + li;
        const long long gi = s_ve.gauss_begin + i;
        const long long f = s_ve.pair_off + i;
        SpecProj o;
        o.visible = false;
        o.x0 = o.x1 = o.y0 = o.y1 = 0;
        float op = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
        if (act) {
            const float *mu = a.means + 3 * gi;
            const float *ls = a.log_scales + 3 * gi;
            const float4 q = __ldg(reinterpret_cast<const float4 *>(a.quats) + gi);
            // the record's other inputs, in flight during the chain
            op = __ldg(a.opacities + gi);
            c0 = __ldg(a.colors + 3 * gi);
            c1 = __ldg(a.colors + 3 * gi + 1);
            c2 = __ldg(a.colors + 3 * gi + 2);
            o = spec_project(s_cam, s_cam + 9, s_cam[12], s_cam[13], s_cam[14], s_cam[15], s_cam[16], s_cam[17],
                             a.itw, a.ith, a.Tx, a.Ty, a.near_plane, a.dil, a.sigmas, __ldg(mu), __ldg(mu + 1),
                             __ldg(mu + 2), __ldg(ls), __ldg(ls + 1), __ldg(ls + 2), q.x, q.y, q.z, q.w);
        }
        if (r == 0) {
            if (threadIdx.x == 0) s_base = base_reg;
            __syncthreads();
        }
        const unsigned long long slot = s_base + (unsigned long long)t;
        if (act) {
            if (slot < (unsigned long long)a.vcap) {
                a.slane[slot] = (uint16_t)(li | (o.visible ? 0 : kSlotHole));   // the adjoint skips holes
            } else if (o.visible) {
                record_error(a.st, GS_ERR_CAPACITY, 11);
                o.visible = false;
            }
            uint32_t cnt = 0;
            if (o.visible) {
                cnt = (uint32_t)((o.x1 - o.x0) * (o.y1 - o.y0));
                a.slot[f] = (uint32_t)slot;
                float4 *rec = a.proj + 3 * slot;
                // sigma beyond which alpha < alpha_min is certain (see gs_render.cu); +inf disables the cut
                float cut = __int_as_float(0x7f800000);
                if (a.alpha_min > 0.0f) {
                    if (op > 0.0f) cut = logf(op / a.alpha_min) + 1e-3f;
                    else if (op <= 0.0f) cut = -1.0f;
                }
                rec[0] = make_float4(o.mx, o.my, o.A, o.B);
                rec[1] = make_float4(o.C, op, o.z, o.rf);
                rec[2] = make_float4(c0, c1, c2, cut);
            }
            a.touched[f] = cnt;
        }
        if (a.tile_cnt && o.visible) {   // tile-bucket binning: one key per touched tile of this view
            uint32_t *row = a.tile_cnt + (size_t)v * a.Txi * a.Ty_i;
            for (int ty = o.y0; ty < o.y1; ++ty)
                for (int tx = o.x0; tx < o.x1; ++tx) atomicAdd(row + ty * a.Txi + tx, 1u);
        }
    }
    if (threadIdx.x == 0) {
        const long long ch = s_ve.chunk_off + blockIdx.x;
        if (base_i < s_ve.count && gs_guard(a.st, ch < a.chunks, 6))
            a.blk[ch] = make_uint4((uint32_t)min(base_reg, (unsigned long long)a.vcap), ncand, 0u, 0u);
    }
}

void launch_project(const Layout &L, const ProjArgs &a, cudaStream_t s) {
    dim3 grid((unsigned)L.max_chunks, (unsigned)L.V);
    k_project<<<grid, kProjThreads, 0, s>>>(a);
    count_launches(1);
}

// ------------------------------------------------------------------------------------------
// projection adjoint
// ------------------------------------------------------------------------------------------


__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One block of kProjBwdThreads threads per (chunk, view): the chunk's visible pairs, i.e. the
// slots of its one or two projection rounds, taken kProjBwdThreads at a time; each thread sums the
// pose terms of its pairs in order, then the block sums the threads (a fixed tree).
constexpr int kProjBwdThreads = 64;

// 16 CTAs per SM (64 registers, a small spill), so that a single view's 1954 chunks are resident
// at once: measured faster than 10 per SM at 92 registers without spills
__global__ void __launch_bounds__(kProjBwdThreads, 16) k_project_bwd(ProjBwdArgs a) {
    const int v = blockIdx.y;
    __shared__ ViewEntry s_ve;
    __shared__ float s_cam[18];
    __shared__ float s_red[kProjBwdThreads / 32][6];
    __shared__ uint4 s_blk;
    if (threadIdx.x == 0) s_ve = a.views[v];
    if (threadIdx.x < 16) s_cam[threadIdx.x] = reinterpret_cast<const float *>(a.cams + v)[threadIdx.x];
    if (threadIdx.x == 32) {      // the forward's clamp limits, the same operations
        const gs_camera &c = a.cams[v];
        s_cam[16] = fp::div(fp::mul(0.65f, (float)a.W), c.fx);
        s_cam[17] = fp::div(fp::mul(0.65f, (float)a.H), c.fy);
    }
    __syncthreads();
    if ((long long)blockIdx.x * kChunk >= s_ve.count) return;   // whole block idle: no partial slot
    const long long ch = s_ve.chunk_off + blockIdx.x;
    if (threadIdx.x == 0) s_blk = gs_guard(a.st, ch < a.chunks, 3) ? a.blk[ch] : make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // the chunk's candidates hold the slots [b0, b0 + n0) (beyond the capacity: dropped by the
    // projection); holes (candidates the decision chain culled) are flagged in their slot lane
    const unsigned long long vc = (unsigned long long)a.vcap;
    const unsigned long long b0 = s_blk.x;
    const unsigned long long n0 = b0 < vc ? min((unsigned long long)s_blk.y, vc - b0) : 0ull;
    float pose[6] = {0, 0, 0, 0, 0, 0};
    for (unsigned long long u = threadIdx.x; u < n0; u += kProjBwdThreads) {
        const uint32_t sl = (uint32_t)(b0 + u);
        const uint32_t lanev = a.slane[sl];
        if (lanev & kSlotHole) continue;
        const long long i = (long long)blockIdx.x * kChunk + (lanev & 0xffu);
        if (!gs_guard(a.st, i < s_ve.count && s_ve.pair_off + i < a.P && s_ve.gauss_begin + i < a.N, 2)) continue;
        {
            const long long gi = s_ve.gauss_begin + i;
            const float *R = s_cam, *t = s_cam + 9;
            const float fx = s_cam[12], fy = s_cam[13];
            const float4 g0 = a.g2d[3 * (size_t)sl], g1 = a.g2d[3 * (size_t)sl + 1], g2 = a.g2d[3 * (size_t)sl + 2];
            const float gmx = g0.x, gmy = g0.y, gA = g0.z, gB = g0.w, gC = g1.x, gop = g1.y, gz = g1.z;
            atomicAdd(a.g_op + gi, gop);
            atomicAdd(a.g_col + 3 * gi, g1.w);
            atomicAdd(a.g_col + 3 * gi + 1, g2.x);
            atomicAdd(a.g_col + 3 * gi + 2, g2.y);
            const float m0 = a.means[3 * gi], m1 = a.means[3 * gi + 1], m2 = a.means[3 * gi + 2];
            // camera-space centre exactly as in the forward decision chain
            const float xc = fp::fma(R[0], m0, fp::fma(R[1], m1, fp::fma(R[2], m2, t[0])));
            const float yc = fp::fma(R[3], m0, fp::fma(R[4], m1, fp::fma(R[5], m2, t[1])));
            const float zc = fp::fma(R[6], m0, fp::fma(R[7], m1, fp::fma(R[8], m2, t[2])));
            const float4 qr = reinterpret_cast<const float4 *>(a.quats)[gi];
            const float qn = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
            const float w = qr.x / qn, x = qr.y / qn, y = qr.z / qn, z = qr.w / qn;
            float Rq[9];
            Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z);       Rq[2] = 2.f * (x * z + w * y);
            Rq[3] = 2.f * (x * y + w * z);       Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
            Rq[6] = 2.f * (x * z - w * y);       Rq[7] = 2.f * (y * z + w * x);       Rq[8] = 1.f - 2.f * (x * x + y * y);
            float s[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) s[k] = spec_expf(a.log_scales[3 * gi + k]);
            float M[9];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) M[3 * j + k] = Rq[3 * j + k] * s[k];
            // clamp decisions as in the forward decision chain
            const float izs = fp::div(1.0f, zc);
            const float limx = s_cam[16], limy = s_cam[17];
            const float uxs = fp::mul(xc, izs), uys = fp::mul(yc, izs);
            const bool clx = (uxs < -limx) || (uxs > limx);
            const bool cly = (uys < -limy) || (uys > limy);
            const float iz = 1.0f / zc;
            const float ux = xc * iz, uy = yc * iz;
            const float tx = fminf(limx, fmaxf(-limx, ux)), ty = fminf(limy, fmaxf(-limy, uy));
            const float J00 = fx * iz, J11 = fy * iz, J02 = -fx * tx * iz, J12 = -fy * ty * iz;
            float Wm[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Wm[k] = J00 * R[k] + J02 * R[6 + k];
                Wm[3 + k] = J11 * R[3 + k] + J12 * R[6 + k];
            }
            float U[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    U[3 * r + k] = Wm[3 * r] * M[k] + Wm[3 * r + 1] * M[3 + k] + Wm[3 * r + 2] * M[6 + k];
            float gpc0 = gmx * fx * iz, gpc1 = gmy * fy * iz;
            float gpc2 = -(gmx * fx * xc + gmy * fy * yc) * iz * iz + gz;
            // conic adjoint
            const float a_ = U[0] * U[0] + U[1] * U[1] + U[2] * U[2] + a.dil;
            const float b_ = U[0] * U[3] + U[1] * U[4] + U[2] * U[5];
            const float c_ = U[3] * U[3] + U[4] * U[4] + U[5] * U[5] + a.dil;
            const float det = a_ * c_ - b_ * b_;
            const float id = 1.0f / det, id2 = id * id;
            const float ga = gA * (-c_ * c_ * id2) + gB * (b_ * c_ * id2) + gC * (id - a_ * c_ * id2);
            const float gb = gA * (2.f * b_ * c_ * id2) + gB * (-id - 2.f * b_ * b_ * id2) + gC * (2.f * a_ * b_ * id2);
            const float gc = gA * (id - a_ * c_ * id2) + gB * (a_ * b_ * id2) + gC * (-a_ * a_ * id2);
            float gU[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gU[k] = 2.f * ga * U[k] + gb * U[3 + k];
                gU[3 + k] = 2.f * gc * U[3 + k] + gb * U[k];
            }
            float gW[6], gM[9];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gW[j] = gU[0] * M[3 * j] + gU[1] * M[3 * j + 1] + gU[2] * M[3 * j + 2];
                gW[3 + j] = gU[3] * M[3 * j] + gU[4] * M[3 * j + 1] + gU[5] * M[3 * j + 2];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) gM[3 * j + k] = Wm[j] * gU[k] + Wm[3 + j] * gU[3 + k];
            float gRq[9], gs[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gRq[3 * j + k] = gM[3 * j + k] * s[k];
                    gs[k] += gM[3 * j + k] * Rq[3 * j + k];
                }
#pragma unroll
            for (int k = 0; k < 3; ++k) atomicAdd(a.g_ls + 3 * gi + k, gs[k] * s[k]);
            float gq[4];
            gq[0] = 2.f * (-z * gRq[1] + y * gRq[2] + z * gRq[3] - x * gRq[5] - y * gRq[6] + x * gRq[7]);
            gq[1] = 2.f * (y * gRq[1] + z * gRq[2] + y * gRq[3] - w * gRq[5] + z * gRq[6] + w * gRq[7]) -
                    4.f * x * (gRq[4] + gRq[8]);
            gq[2] = 2.f * (x * gRq[1] + w * gRq[2] + x * gRq[3] + z * gRq[5] - w * gRq[6] + z * gRq[7]) -
                    4.f * y * (gRq[0] + gRq[8]);
            gq[3] = 2.f * (-w * gRq[1] + x * gRq[2] + w * gRq[3] + y * gRq[5] + x * gRq[6] + y * gRq[7]) -
                    4.f * z * (gRq[0] + gRq[4]);
            const float dq = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
            const float qv[4] = {w, x, y, z};
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(a.g_quats + 4 * gi + k, (gq[k] - qv[k] * dq) / qn);
            float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f, gR[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gJ00 += gW[k] * R[k];
                gJ02 += gW[k] * R[6 + k];
                gJ11 += gW[3 + k] * R[3 + k];
                gJ12 += gW[3 + k] * R[6 + k];
                gR[k] = gW[k] * J00;
                gR[3 + k] = gW[3 + k] * J11;
                gR[6 + k] = gW[k] * J02 + gW[3 + k] * J12;
            }
            gpc2 += -(gJ00 * fx + gJ11 * fy) * iz * iz + (gJ02 * fx * tx + gJ12 * fy * ty) * iz * iz;
            const float gtx = -gJ02 * fx * iz, gty = -gJ12 * fy * iz;
            if (!clx) { gpc0 += gtx * iz; gpc2 -= gtx * xc * iz * iz; }
            if (!cly) { gpc1 += gty * iz; gpc2 -= gty * yc * iz * iz; }
#pragma unroll
            for (int k = 0; k < 3; ++k)
                atomicAdd(a.g_means + 3 * gi + k, R[k] * gpc0 + R[3 + k] * gpc1 + R[6 + k] * gpc2);
            // pose: d p_c = rho + phi x p_c, d R = [phi]x R
            float N[9];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int m = 0; m < 3; ++m) N[3 * j + m] = gR[3 * j] * R[3 * m] + gR[3 * j + 1] * R[3 * m + 1] +
                                                          gR[3 * j + 2] * R[3 * m + 2];
            pose[0] += gpc0; pose[1] += gpc1; pose[2] += gpc2;
            pose[3] += yc * gpc2 - zc * gpc1 + N[7] - N[5];
            pose[4] += zc * gpc0 - xc * gpc2 + N[2] - N[6];
            pose[5] += xc * gpc1 - yc * gpc0 + N[3] - N[1];
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float r = warp_sum(pose[k]);
        if (lane == 0) s_red[warp][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < 6 && ch < a.chunks) {
        float r = 0.f;
#pragma unroll
        for (int wi = 0; wi < kProjBwdThreads / 32; ++wi) r += s_red[wi][threadIdx.x];
        a.pose_part[(s_ve.chunk_off + blockIdx.x) * 8 + threadIdx.x] = r;
    }
}

void launch_project_bwd(const Layout &L, const ProjBwdArgs &a, cudaStream_t s) {
    dim3 grid((unsigned)L.max_chunks, (unsigned)L.V);
    k_project_bwd<<<grid, kProjBwdThreads, 0, s>>>(a);
    count_launches(1);
}

// deterministic per-view sum of the pose partials: one 256-thread block per view, each thread
// reading its chunks' 8-float partials as two 16-byte loads; fixed per-thread strides and a fixed
// reduction tree per component
__global__ void __launch_bounds__(256) k_pose_reduce(const ViewEntry *views, const float *pose_part, float *out,
                                                     long long total_chunks, DevStatus *st) {
    __shared__ float s_w[8][6];
    const int v = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const ViewEntry ve = views[v];
    const long long chunks = (ve.count + kChunk - 1) / kChunk;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float4 *part4 = reinterpret_cast<const float4 *>(pose_part);
    for (long long c = threadIdx.x; c < chunks; c += 256) {
        if (gs_guard(st, ve.chunk_off + c < total_chunks, 4)) {
            const float4 p0 = part4[2 * (ve.chunk_off + c)], p1 = part4[2 * (ve.chunk_off + c) + 1];
            acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w; acc[4] += p1.x; acc[5] += p1.y;
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float r = warp_sum(acc[k]);
        if (lane == 0) s_w[warp][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) r += s_w[w][threadIdx.x];
        out[6 * v + threadIdx.x] = r;
    }
}

void launch_pose_reduce(const Layout &L, const ViewEntry *views, const float *part, float *out, DevStatus *st,
                        cudaStream_t s) {
    k_pose_reduce<<<L.V, 256, 0, s>>>(views, part, out, std::max<long long>(L.chunks_total, 1), st);
    count_launches(1);
}

}  // namespace gs
