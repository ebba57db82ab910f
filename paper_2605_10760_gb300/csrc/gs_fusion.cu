// gs_fusion.cu -- occupancy-aware fusion of aligned submaps (Sec. III-C, Eqs. 19-22).
//
//  * k_sim3: the Sim(3) correction C = (s, R, t) acting on Gaussians (Eq. 19): mu' = s R mu + t,
//    rotation q' = q_R (x) q, log-scales + ln s; opacity and colour copied.
//  * Voxel sets: open-addressing hash sets of 64-bit keys (voxel index kappa(x) = floor(x / v) per
//    axis, 21 bits per axis with offset 2^20) with linear probing; insertion by compare-and-swap,
//    membership by probing to the first empty slot.  Probing is bounded by the capacity; a full
//    table records GS_ERR_CAPACITY in the set's status word instead of looping.
//  * k_add_boxes (Eq. 20): every voxel of [kappa(mu - k s), kappa(mu + k s)].
//  * k_add_rays (Eq. 21): one thread per (keyframe, strided pixel) walks the voxels crossed by the
//    segment from the camera centre to the back-projected depth point, t in [0, 1), with a 3-D
//    digital differential analyser (ties between axes go to the lowest axis).
//  * k_keep (Eq. 22): keep a borrowed Gaussian iff kappa(mu) is in neither set.
// Every voxel decision uses the same FP32 operation sequence as the fusion oracle (explicit
// round-to-nearest intrinsics, never contracted), so the voxel sets agree bit for bit.
#include <algorithm>
#include <cmath>

#include "gs_kernels.cuh"

namespace gs {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kKeyBits = 21;
constexpr long long kKeyOff = 1LL << 20;
constexpr int kMaxBoxExtent = 64;      // voxels per axis of one Gaussian's box before it is flagged

struct VoxSet {
    int32_t *status;                   // first error
    unsigned long long *keys;          // [capacity]
    unsigned long long mask;           // capacity - 1
};

__host__ __device__ __forceinline__ VoxSet voxset_of_host(void *mem, long long capacity) {
    VoxSet s;
    s.status = reinterpret_cast<int32_t *>(mem);
    s.keys = reinterpret_cast<unsigned long long *>(static_cast<char *>(mem) + 256);
    s.mask = (unsigned long long)capacity - 1ull;
    return s;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // splitmix64 finaliser (Vigna): a bijective 64-bit mix
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long pack_key(long long ix, long long iy, long long iz) {
    ix = min(max(ix, -kKeyOff), kKeyOff - 1) + kKeyOff;
    iy = min(max(iy, -kKeyOff), kKeyOff - 1) + kKeyOff;
    iz = min(max(iz, -kKeyOff), kKeyOff - 1) + kKeyOff;
    return ((unsigned long long)ix << (2 * kKeyBits)) | ((unsigned long long)iy << kKeyBits) |
           (unsigned long long)iz;
}

__device__ __forceinline__ bool voxset_insert(const VoxSet &s, unsigned long long key) {
    unsigned long long slot = mix64(key) & s.mask;
    for (unsigned long long probe = 0; probe <= s.mask; ++probe) {
        const unsigned long long cur = s.keys[slot];
        if (cur == key) return true;
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(&s.keys[slot], kEmptyKey, key);
            if (prev == kEmptyKey || prev == key) return true;
        }
        slot = (slot + 1) & s.mask;
    }
    atomicCAS(s.status, 0, GS_ERR_CAPACITY);
    return false;
}

__device__ __forceinline__ bool voxset_contains(const VoxSet &s, unsigned long long key) {
    unsigned long long slot = mix64(key) & s.mask;
    for (unsigned long long probe = 0; probe <= s.mask; ++probe) {
        const unsigned long long cur = s.keys[slot];
        if (cur == key) return true;
        if (cur == kEmptyKey) return false;
        slot = (slot + 1) & s.mask;
    }
    return false;
}

__device__ __forceinline__ long long vox_index(float x, float v) { return (long long)floorf(fp::div(x, v)); }

// ------------------------------------------------------------------------------------------
__global__ void k_voxset_clear(unsigned long long *keys, long long capacity, int32_t *status) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < capacity;
         i += (long long)gridDim.x * blockDim.x)
        keys[i] = kEmptyKey;
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

__global__ void k_add_boxes(VoxSet s, long long n, const float *means, const float *log_scales, float k, float v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long lo[3], hi[3];
        bool big = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float mu = means[3 * i + a];
            const float ks = fp::mul(k, spec_expf(log_scales[3 * i + a]));
            lo[a] = vox_index(fp::sub(mu, ks), v);
            hi[a] = vox_index(fp::add(mu, ks), v);
            big |= (hi[a] - lo[a] + 1) > kMaxBoxExtent;
        }
        if (big) {
            atomicCAS(s.status, 0, GS_ERR_INVALID_ARG);   // a box wider than kMaxBoxExtent voxels
            continue;
        }
        for (long long x = lo[0]; x <= hi[0]; ++x)
            for (long long y = lo[1]; y <= hi[1]; ++y)
                for (long long z = lo[2]; z <= hi[2]; ++z) voxset_insert(s, pack_key(x, y, z));
    }
}

struct RayArgs {
    VoxSet s;
    const gs_camera *cams;
    const float *depth;       // [V,H,W] camera depth (z) per pixel; <= 0 or non-finite: no ray
    int V, W, H, stride, sw, sh;
    float v;
    long long max_steps;
};

__global__ void k_add_rays(RayArgs a) {
    const long long total = (long long)a.V * a.sw * a.sh;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(r / ((long long)a.sw * a.sh));
        const long long rem = r - (long long)k * a.sw * a.sh;
        const int y = (int)(rem / a.sw) * a.stride, x = (int)(rem % a.sw) * a.stride;
        const float d = a.depth[((long long)k * a.H + y) * a.W + x];
        if (!(d > 0.f) || !isfinite(d)) continue;
        const gs_camera cam = a.cams[k];
        const float *R = cam.R, *t = cam.t;
        float c[3], p[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) c[q] = -fp::fma(R[q], t[0], fp::fma(R[3 + q], t[1], fp::mul(R[6 + q], t[2])));
        const float xn = fp::div(fp::sub(fp::add((float)x, 0.5f), cam.cx), cam.fx);
        const float yn = fp::div(fp::sub(fp::add((float)y, 0.5f), cam.cy), cam.fy);
        const float pc0 = fp::sub(fp::mul(xn, d), t[0]), pc1 = fp::sub(fp::mul(yn, d), t[1]), pc2 = fp::sub(d, t[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) p[q] = fp::fma(R[q], pc0, fp::fma(R[3 + q], pc1, fp::mul(R[6 + q], pc2)));
        // digital differential analyser over [c, p)
        long long cur[3];
        int step[3];
        float tmax[3], tdel[3];
        const float inf = __int_as_float(0x7f800000);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            cur[q] = vox_index(c[q], a.v);
            const float dq = fp::sub(p[q], c[q]);
            if (dq > 0.f) {
                step[q] = 1;
                tmax[q] = fp::div(fp::sub(fp::mul((float)(cur[q] + 1), a.v), c[q]), dq);
                tdel[q] = fp::div(a.v, dq);
            } else if (dq < 0.f) {
                step[q] = -1;
                tmax[q] = fp::div(fp::sub(fp::mul((float)cur[q], a.v), c[q]), dq);
                tdel[q] = fp::div(-a.v, dq);
            } else {
                step[q] = 0;
                tmax[q] = inf;
                tdel[q] = inf;
            }
        }
        voxset_insert(a.s, pack_key(cur[0], cur[1], cur[2]));
        long long n = 0;
        for (; n < a.max_steps; ++n) {
            int q = 0;
            if (tmax[1] < tmax[q]) q = 1;
            if (tmax[2] < tmax[q]) q = 2;
            if (!(tmax[q] < 1.0f)) break;
            cur[q] += step[q];
            tmax[q] = fp::add(tmax[q], tdel[q]);
            voxset_insert(a.s, pack_key(cur[0], cur[1], cur[2]));
        }
        if (n == a.max_steps) atomicCAS(a.s.status, 0, GS_ERR_INVALID_ARG);   // ray longer than allowed
    }
}

__global__ void k_keep(long long n, const float *means, VoxSet occ, VoxSet fre, bool has_free, float v,
                       uint8_t *keep) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key =
            pack_key(vox_index(means[3 * i], v), vox_index(means[3 * i + 1], v), vox_index(means[3 * i + 2], v));
        const bool drop = voxset_contains(occ, key) || (has_free && voxset_contains(fre, key));
        keep[i] = drop ? 0 : 1;
    }
}

__global__ void k_sim3(long long n, gs_gaussians in, gs_gaussian_arrays out, float s, float R00, float R01, float R02,
                       float R10, float R11, float R12, float R20, float R21, float R22, float t0, float t1, float t2,
                       float qw, float qx, float qy, float qz, float ln_s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float m0 = in.means[3 * i], m1 = in.means[3 * i + 1], m2 = in.means[3 * i + 2];
        out.means[3 * i] = s * (R00 * m0 + R01 * m1 + R02 * m2) + t0;
        out.means[3 * i + 1] = s * (R10 * m0 + R11 * m1 + R12 * m2) + t1;
        out.means[3 * i + 2] = s * (R20 * m0 + R21 * m1 + R22 * m2) + t2;
#pragma unroll
        for (int a = 0; a < 3; ++a) out.log_scales[3 * i + a] = in.log_scales[3 * i + a] + ln_s;
        const float bw = in.quats[4 * i], bx = in.quats[4 * i + 1], by = in.quats[4 * i + 2], bz = in.quats[4 * i + 3];
        out.quats[4 * i] = qw * bw - qx * bx - qy * by - qz * bz;
        out.quats[4 * i + 1] = qw * bx + qx * bw + qy * bz - qz * by;
        out.quats[4 * i + 2] = qw * by - qx * bz + qy * bw + qz * bx;
        out.quats[4 * i + 3] = qw * bz + qx * by - qy * bx + qz * bw;
        out.opacities[i] = in.opacities[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) out.colors[3 * i + a] = in.colors[3 * i + a];
    }
}

static int grid_for(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 16));
}

int launch_voxset_clear(void *mem, long long capacity, cudaStream_t s) {
    k_voxset_clear<<<grid_for(capacity), 256, 0, s>>>(
        reinterpret_cast<unsigned long long *>(static_cast<char *>(mem) + 256), capacity, reinterpret_cast<int32_t *>(mem));
    count_launches(1);
    return check_launch();
}

int launch_voxset_add_boxes(void *mem, long long capacity, long long n, const float *means, const float *log_scales,
                            float k, float v, cudaStream_t s) {
    if (n > 0) {
        k_add_boxes<<<grid_for(n), 256, 0, s>>>(voxset_of_host(mem, capacity), n, means, log_scales, k, v);
        count_launches(1);
    }
    return check_launch();
}

int launch_voxset_add_rays(void *mem, long long capacity, int V, int W, int H, const gs_camera *cams,
                           const float *depth, int stride, float v, cudaStream_t s) {
    RayArgs a;
    a.s = voxset_of_host(mem, capacity);
    a.cams = cams;
    a.depth = depth;
    a.V = V; a.W = W; a.H = H; a.stride = stride;
    a.sw = (W + stride - 1) / stride;
    a.sh = (H + stride - 1) / stride;
    a.v = v;
    a.max_steps = 1LL << 16;
    const long long total = (long long)V * a.sw * a.sh;
    k_add_rays<<<grid_for(total), 256, 0, s>>>(a);
    count_launches(1);
    return check_launch();
}

int launch_voxset_keep(long long n, const float *means, void *occ, long long occ_cap, void *fre, long long free_cap,
                       float v, uint8_t *keep, cudaStream_t s) {
    if (n > 0) {
        const VoxSet o = voxset_of_host(occ, occ_cap);
        const VoxSet f = fre ? voxset_of_host(fre, free_cap) : o;
        k_keep<<<grid_for(n), 256, 0, s>>>(n, means, o, f, fre != nullptr, v, keep);
        count_launches(1);
    }
    return check_launch();
}

int launch_sim3(long long n, const gs_gaussians &in, const float q[4], const float t[3], float sc,
                const gs_gaussian_arrays &out, cudaStream_t s) {
    // rotation matrix of the unit quaternion (normalised here, in double on the host)
    const double nq = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    const double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
    const float R[9] = {(float)(1 - 2 * (y * y + z * z)), (float)(2 * (x * y - w * z)), (float)(2 * (x * z + w * y)),
                        (float)(2 * (x * y + w * z)), (float)(1 - 2 * (x * x + z * z)), (float)(2 * (y * z - w * x)),
                        (float)(2 * (x * z - w * y)), (float)(2 * (y * z + w * x)), (float)(1 - 2 * (x * x + y * y))};
    if (n > 0) {
        k_sim3<<<grid_for(n), 256, 0, s>>>(n, in, out, sc, R[0], R[1], R[2], R[3], R[4], R[5], R[6], R[7], R[8], t[0],
                                           t[1], t[2], (float)w, (float)x, (float)y, (float)z, (float)log((double)sc));
        count_launches(1);
    }
    return check_launch();
}

}  // namespace gs
