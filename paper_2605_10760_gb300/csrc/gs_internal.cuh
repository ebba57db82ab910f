// gs_internal.cuh -- shared device helpers of libgs (sm_103a).
//
// The FP32 decision chain (culling, tile rectangle, depth key, sigma, alpha, transmittance) is
// written with explicit round-to-nearest intrinsics (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn,
// __fdiv_rn, __fsqrt_rn): the compiler never contracts or reorders them, so every branch is taken
// exactly as the operation sequence below prescribes, whatever the -fmad setting of the
// translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kMaxPasses = 8;          // 8-bit digits of a 64-bit key
constexpr int kSortThreads = 256;
// keys per thread of a onesweep partition: 4096-key partitions (16 per thread).  Smaller
// partitions (4 or 8 keys per thread) make the per-digit look-back chains longer, larger ones
// (32 keys per thread, 255 registers) lengthen each CTA's ranking: both measured slower on GB300.
constexpr int kSortIPT = 16;
constexpr int kScanThreads = 256;
constexpr int kScanIPT = 16;
constexpr int kScanTile = kScanThreads * kScanIPT;
constexpr int kChunk = 256;            // (view, Gaussian) pairs per projection block
constexpr unsigned long long kSpinLimit = 1ull << 21;  // bounded waits (x ~100 ns sleep)

// counters inside the status block (zeroed by the call that uses them)
enum Counter {
    kCtrScan = 0, kCtrSort0 = 1, kCtrTileSort = 14, kCtrTileList = 15, kCtrTileLong = 16,
    kNumCounters = 32
};

struct DevStatus {
    int32_t code;                 // first recorded GS_ERR_* (0 = none)
    int32_t where;                // stage tag of that error
    unsigned long long required_keys;
    unsigned long long num_keys;  // K written by the scan
    // the compositing kernels' work-queue counters return to zero at the end of every launch (the
    // CTA drawing a launch's last claim resets it); their pair counts are cleared by each binning
    // and count the (pixel, entry) pairs of the launches since
    unsigned long long fwd_pairs;
    uint32_t fwd_items, fwd_pad;
    unsigned long long bwd_pairs;
    uint32_t bwd_items, bwd_pad;
    uint32_t ctr[kNumCounters];
    uint32_t claim_cnt[32];       // items in each claim class (cleared with ctr by gs_bin_sort)
    int32_t guard_bad;            // gs_check_guards: index of the first changed guard block
    int32_t guard_pad;
    unsigned long long num_visible;   // slots the last projection took (its visible pairs and holes)
    // the projection's slot counter: blocks that have reserved << 40 | slots reserved; the block
    // arriving last publishes num_visible and returns it to zero
    unsigned long long slot_ctr;
};

struct ViewEntry {                // per-view table in the workspace (32 bytes)
    long long gauss_begin;
    long long count;
    long long pair_off;
    long long chunk_off;
};

constexpr int kNumGuards = 15;

struct Layout {
    int V, W, H, tw, th, Tx, Ty, passes;
    long long G, P, N, cap, max_count, max_chunks;
    long long vcap;                    // slots of the projection records and 2-D gradients
    long long scan_parts, sort_parts, chunks_total;
    int sort_mode, nb;                 // binning mode; records per staged render batch
    size_t o_status, o_views, o_proj, o_touched, o_scan_state, o_keys[2], o_vals[2], o_hist,
        o_sort_state, o_ranges, o_tword, o_tcnt, o_tlist, o_srec, o_g2d, o_pose_part, o_slot, o_clist, o_slane,
        o_blk, total;
    size_t o_guard[kNumGuards];        // guard blocks after proj, touched, keys x2, vals x2, ranges,
                                       // the tile lists, srec, g2d, the pose partials, the slots,
                                       // the claim-class lists, the slot lanes, the block slot ranges
};
constexpr uint32_t kNoSlot = 0xffffffffu;   // pair_slot of a culled pair
constexpr uint16_t kSlotHole = 0x100;        // slot lane flag: a candidate the decision chain culled
// The compositing kernels claim (view, tile) items class by class: class k lists the items whose
// list length n has 2 min(floor(log2 n), 15) + (the bit below the leading one) = 31 - k, so class
// 0 holds the longest lists and class 31 the lists of 0 or 1 entries (k = 0 from 2^16 entries on).
constexpr int kClaimClasses = 32;
constexpr size_t kGuardBytes = 256;
constexpr int kGuardByte = 0x5A;       // every byte of an intact guard block

// ------------------------------------------------------------------------------------------
// bounds-checked build (-DGS_CHECKED=1, libgs_checked.so): every index that comes from data (a
// record's slot, a key's tile, a range, a scatter position, a hash or tap position) is
// compared with its buffer's length before the access; a violation records GS_ERR_DEVICE_FAULT
// with site 100 + `site` and the access is skipped.  In the release build gs_guard is `true`.
// ------------------------------------------------------------------------------------------
#ifndef GS_CHECKED
#define GS_CHECKED 0
#endif

// ------------------------------------------------------------------------------------------
// error recording (first error wins)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void record_error(DevStatus *st, int code, int where) {
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ bool gs_guard(DevStatus *st, bool ok, int site) {
#if GS_CHECKED
    if (!ok) record_error(st, GS_ERR_DEVICE_FAULT, 100 + site);
    return ok;
#else
    (void)st;
    (void)site;
    return ok || true;
#endif
}

// ------------------------------------------------------------------------------------------
// FP32 decision-chain arithmetic
// ------------------------------------------------------------------------------------------
namespace fp {
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
}  // namespace fp

// e^x in FP32: x = k ln2 + r with k = rint(x log2 e) and a two-part ln2 (hi has 16 significant
// bits so k*hi is exact for |k| < 256), e^r by the degree-7 Taylor polynomial in Horner form with
// fused multiply-adds, then 2^k through the exponent field.  x <= -87 gives 0, x > 88 gives +inf.
__device__ __forceinline__ float spec_expf(float x) {
    if (!(x > -87.0f)) return 0.0f;
    if (x > 88.0f) return __int_as_float(0x7f800000);
    const float kLog2e = 0x1.715476p+0f;
    const float kLn2Hi = 0x1.62e4p-1f;
    const float kLn2Lo = 0x1.7f7d1cp-20f;
    // round x log2(e) to the nearest integer, ties to even: adding and subtracting 1.5 * 2^23
    // rounds exactly that way for |t| < 2^22, and the low bits of the sum hold the integer itself
    const float kShift = 12582912.0f;
    const float t = fp::add(fp::mul(x, kLog2e), kShift);
    const float kf = fp::sub(t, kShift);
    const int k = __float_as_int(t) - 0x4B400000;
    float r = fp::fma(-kf, kLn2Hi, x);
    r = fp::fma(-kf, kLn2Lo, r);
    float p = 0x1.a01a02p-13f;              // 1/7!
    p = fp::fma(p, r, 0x1.6c16c2p-10f);     // 1/6!
    p = fp::fma(p, r, 0x1.111112p-7f);      // 1/5!
    p = fp::fma(p, r, 0x1.555556p-5f);      // 1/4!
    p = fp::fma(p, r, 0x1.555556p-3f);      // 1/3!
    p = fp::fma(p, r, 0.5f);
    p = fp::fma(p, r, 1.0f);
    p = fp::fma(p, r, 1.0f);
    return fp::mul(p, __int_as_float((k + 127) << 23));
}

struct SpecProj {
    float mx, my, A, B, C, z, rf;
    int x0, x1, y0, y1;
    bool visible;
};

// Tile rectangle of the bounding square [m - r, m + r] (x1, y1 exclusive), clamped to the grid.
// itw, ith are 1/tile_w and 1/tile_h: tile sizes are powers of two (16, 8, 32), so multiplying by
// the exact reciprocal rounds exactly like the division by the tile size.
__device__ __forceinline__ void spec_rect(float mx, float my, float rf, float itw, float ith, float Tx, float Ty,
                                          int &x0, int &x1, int &y0, int &y1) {
    float fx0 = fminf(fmaxf(floorf(fp::mul(fp::sub(mx, rf), itw)), 0.0f), Tx);
    float fx1 = fminf(fmaxf(fp::add(floorf(fp::mul(fp::add(mx, rf), itw)), 1.0f), 0.0f), Tx);
    float fy0 = fminf(fmaxf(floorf(fp::mul(fp::sub(my, rf), ith)), 0.0f), Ty);
    float fy1 = fminf(fmaxf(fp::add(floorf(fp::mul(fp::add(my, rf), ith)), 1.0f), 0.0f), Ty);
    x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
}

// EWA projection of one Gaussian into one view (the FP32 decision chain).
//   p_c = R mu + t; unit quaternion -> rotation Rq; M = Rq diag(exp(l));
//   J = [[fx/z, 0, -fx tx/z], [0, fy/z, -fy ty/z]] with tx, ty = x/z, y/z clamped to
//   +-limx, +-limy (limx = fl(fl(0.65 W) / fx), limy likewise: per-view constants the caller
//   computes once); U = (J R) M; Sigma_2 = U U^T + dilation I; conic = Sigma_2^-1;
//   mean2D = (fx x/z + cx, fy y/z + cy); radius = ceil(sigmas sqrt(lambda_max)).
__device__ __forceinline__ SpecProj spec_project(const float *R, const float *t, float fx, float fy, float cx,
                                                 float cy, float limx, float limy, float itw, float ith, float Tx,
                                                 float Ty, float near_plane, float dil, float sigmas, float m0,
                                                 float m1, float m2, float l0, float l1, float l2, float qw,
                                                 float qx, float qy, float qz) {
    using namespace fp;
    SpecProj o;
    o.visible = false;
    o.mx = o.my = o.A = o.B = o.C = o.rf = 0.0f;
    o.x0 = o.x1 = o.y0 = o.y1 = 0;
    float xc = fma(R[0], m0, fma(R[1], m1, fma(R[2], m2, t[0])));
    float yc = fma(R[3], m0, fma(R[4], m1, fma(R[5], m2, t[1])));
    float zc = fma(R[6], m0, fma(R[7], m1, fma(R[8], m2, t[2])));
    o.z = zc;
    if (!(zc > near_plane)) return o;
    float n2 = fma(qw, qw, fma(qx, qx, fma(qy, qy, mul(qz, qz))));
    if (!(n2 > 0.0f)) return o;
    float inv = div(1.0f, sqrt(n2));
    float w = mul(qw, inv), x = mul(qx, inv), y = mul(qy, inv), z = mul(qz, inv);
    float xx = mul(x, x), yy = mul(y, y), zz = mul(z, z);
    float xy = mul(x, y), xz = mul(x, z), yz = mul(y, z);
    float wx = mul(w, x), wy = mul(w, y), wz = mul(w, z);
    float Rq[9];
    Rq[0] = sub(1.0f, mul(2.0f, add(yy, zz)));
    Rq[1] = mul(2.0f, sub(xy, wz));
    Rq[2] = mul(2.0f, add(xz, wy));
    Rq[3] = mul(2.0f, add(xy, wz));
    Rq[4] = sub(1.0f, mul(2.0f, add(xx, zz)));
    Rq[5] = mul(2.0f, sub(yz, wx));
    Rq[6] = mul(2.0f, sub(xz, wy));
    Rq[7] = mul(2.0f, add(yz, wx));
    Rq[8] = sub(1.0f, mul(2.0f, add(xx, yy)));
    float s0 = spec_expf(l0), s1 = spec_expf(l1), s2 = spec_expf(l2);
    float M[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        M[3 * j + 0] = mul(Rq[3 * j + 0], s0);
        M[3 * j + 1] = mul(Rq[3 * j + 1], s1);
        M[3 * j + 2] = mul(Rq[3 * j + 2], s2);
    }
    float iz = div(1.0f, zc);
    float ux = mul(xc, iz), uy = mul(yc, iz);
    float tx = fminf(limx, fmaxf(-limx, ux));
    float ty = fminf(limy, fmaxf(-limy, uy));
    float J00 = mul(fx, iz), J11 = mul(fy, iz);
    float J02 = -mul(mul(fx, tx), iz), J12 = -mul(mul(fy, ty), iz);
    float Wm[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Wm[k] = fma(J00, R[k], mul(J02, R[6 + k]));
        Wm[3 + k] = fma(J11, R[3 + k], mul(J12, R[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            U[3 * r + k] = fma(Wm[3 * r], M[k], fma(Wm[3 * r + 1], M[3 + k], mul(Wm[3 * r + 2], M[6 + k])));
    float a = add(fma(U[0], U[0], fma(U[1], U[1], mul(U[2], U[2]))), dil);
    float b = fma(U[0], U[3], fma(U[1], U[4], mul(U[2], U[5])));
    float c = add(fma(U[3], U[3], fma(U[4], U[4], mul(U[5], U[5]))), dil);
    float det = fma(a, c, -mul(b, b));
    if (!(det > 0.0f)) return o;
    o.A = div(c, det);
    o.B = div(-b, det);
    o.C = div(a, det);
    o.mx = fma(fx, ux, cx);
    o.my = fma(fy, uy, cy);
    float mid = mul(0.5f, add(a, c));
    float disc = fma(mid, mid, -det);
    float lam = add(mid, sqrt(fmaxf(0.0f, disc)));
    o.rf = ceilf(mul(sigmas, sqrt(lam)));
    spec_rect(o.mx, o.my, o.rf, itw, ith, Tx, Ty, o.x0, o.x1, o.y0, o.y1);
    o.visible = (o.x1 > o.x0) && (o.y1 > o.y0);
    return o;
}

// sigma = 1/2 (A dx^2 + C dy^2) + B dx dy with d = pixel - mean2D (decision chain order).
__device__ __forceinline__ float spec_sigma(float A, float B, float C, float dx, float dy) {
    float q = fp::fma(fp::mul(A, dx), dx, fp::mul(fp::mul(C, dy), dy));
    return fp::fma(fp::mul(B, dx), dy, fp::mul(0.5f, q));
}

// ------------------------------------------------------------------------------------------
// the same chain on two arguments at once (two pixels of a thread): packed FP32x2 operations
// round each component exactly like the scalar operation, so every component equals the scalar
// chain's result bit for bit
// ------------------------------------------------------------------------------------------
namespace fp2 {
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
}  // namespace fp2

// spec_expf of both components (a - b is computed as a + (-b) and (-k) c as k (-c), both exact)
__device__ __forceinline__ float2 spec_expf2(float2 x) {
    const float kLog2e = 0x1.715476p+0f;
    const float kLn2Hi = 0x1.62e4p-1f;
    const float kLn2Lo = 0x1.7f7d1cp-20f;
    const float kShift = 12582912.0f;
    const float2 t = fp2::add(fp2::mul(x, fp2::splat(kLog2e)), fp2::splat(kShift));
    const float2 kf = fp2::add(t, fp2::splat(-kShift));
    float2 r = fp2::fma(kf, fp2::splat(-kLn2Hi), x);
    r = fp2::fma(kf, fp2::splat(-kLn2Lo), r);
    float2 p = fp2::fma(fp2::splat(0x1.a01a02p-13f), r, fp2::splat(0x1.6c16c2p-10f));
    p = fp2::fma(p, r, fp2::splat(0x1.111112p-7f));
    p = fp2::fma(p, r, fp2::splat(0x1.555556p-5f));
    p = fp2::fma(p, r, fp2::splat(0x1.555556p-3f));
    p = fp2::fma(p, r, fp2::splat(0.5f));
    p = fp2::fma(p, r, fp2::splat(1.0f));
    p = fp2::fma(p, r, fp2::splat(1.0f));
    const int kx = __float_as_int(t.x) - 0x4B400000, ky = __float_as_int(t.y) - 0x4B400000;
    float2 e = fp2::mul(p, make_float2(__int_as_float((kx + 127) << 23), __int_as_float((ky + 127) << 23)));
    const float inf = __int_as_float(0x7f800000);
    e.x = !(x.x > -87.0f) ? 0.0f : (x.x > 88.0f ? inf : e.x);
    e.y = !(x.y > -87.0f) ? 0.0f : (x.y > 88.0f ? inf : e.y);
    return e;
}

// spec_sigma at two pixels of one column (dy per pixel)
__device__ __forceinline__ float2 spec_sigma2(float A, float B, float C, float dx, float2 dy) {
    const float2 q = fp2::fma(fp2::splat(fp::mul(A, dx)), fp2::splat(dx), fp2::mul(fp2::mul(fp2::splat(C), dy), dy));
    return fp2::fma(fp2::splat(fp::mul(B, dx)), dy, fp2::mul(fp2::splat(0.5f), q));
}

// ------------------------------------------------------------------------------------------
// relaxed device-scope loads / stores for decoupled look-back
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}


// ------------------------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, 1-D) completing on shared-memory mbarriers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// orders this thread's earlier generic-proxy accesses of shared memory before later async-proxy
// (TMA) accesses, and makes initialised mbarriers visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces `bytes` of transaction count, then the bulk copy that completes
// them; dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit) {
    for (unsigned long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
int compute_layout(const gs_problem *pb, Layout *L);
// scans the guard blocks (synchronises the stream); *first_bad = index of the first changed block or -1
int run_check_guards(const unsigned char *const *guards, DevStatus *st, int32_t *first_bad, cudaStream_t s);
void count_launches(int n);
int device_sm_count();
int check_launch();

template <class T>
__host__ __device__ inline T *ws_ptr(void *ws, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

}  // namespace gs
