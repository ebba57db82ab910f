// gs_kernels.cuh -- kernel argument blocks and host launchers of libgs.
#pragma once

#include "gs_internal.cuh"

namespace gs {

// ---------------- projection ----------------
struct ProjArgs {
    const ViewEntry *views;
    const gs_camera *cams;
    const float *means, *log_scales, *quats, *opacities, *colors;
    float4 *proj;               // [P,3] float4
    uint32_t *touched;          // [P]
    int W, H;
    float itw, ith, Tx, Ty;     // 1 / tile size (exact: tile sizes are powers of two), tiles per row / column
    float near_plane, dil, sigmas, alpha_min;
    uint32_t *tile_cnt;         // [G] key count per global tile (tile-bucket binning), else null
    int Txi, Ty_i;
    long long P;                // (view, Gaussian) pairs: the length of touched and slot
    DevStatus *st;              // errors; slot_ctr hands out the slots, num_visible their count
    uint32_t *slot;             // [P] slot of each visible pair in proj (kNoSlot when culled)
    long long vcap;             // slots in proj
    uint16_t *slane;            // [vcap] the chunk position of each slot's pair, | kSlotHole when the
                                //   decision chain culled it
    uint4 *blk;                 // [chunks] first slot and candidate count of each projection block
    long long chunks;           // projection blocks over all views (the length of blk)
};

struct ProjBwdArgs {
    const ViewEntry *views;
    const gs_camera *cams;
    const float *means, *log_scales, *quats;
    const uint16_t *slane;          // [vcap] chunk position of each slot's pair (| kSlotHole: a hole)
    const uint4 *blk;               // [chunks] first slot and candidate count of each projection block
    const float4 *g2d;              // [vcap,3] float4
    float *g_means, *g_ls, *g_quats, *g_op, *g_col;
    float *pose_part;               // [chunks, 8]
    int W, H;
    float dil;
    long long P, N, chunks;         // lengths of touched / slot, of the gradient arrays, of pose_part
    DevStatus *st;                  // bounds-checked build: where a violated index is recorded
    const uint32_t *slot;           // [P] slot of each visible pair in g2d
    long long vcap;                 // slots in g2d
};

void launch_project(const Layout &L, const ProjArgs &a, cudaStream_t s);
void launch_project_bwd(const Layout &L, const ProjBwdArgs &a, cudaStream_t s);
void launch_pose_reduce(const Layout &L, const ViewEntry *views, const float *part, float *out, DevStatus *st,
                        cudaStream_t s);

// ---------------- binning ----------------
struct BinArgs {
    const ViewEntry *views;
    uint32_t *touched;                 // in: counts; out: inclusive prefix sums
    unsigned long long *scan_state;
    const float4 *proj;
    float4 *g2d;
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t *hist;                    // [kMaxPasses][256]
    uint32_t *sort_state;              // [passes][sort_parts][256]
    uint32_t *ranges;                  // [G,2]
    float4 *srec;                      // [cap,3] records in list order
    DevStatus *st;
    int V, Tx, Ty, passes;
    float itw, ith;                    // 1 / tile size (exact: tile sizes are powers of two)
    long long P, cap, sort_parts, max_chunks, G;
    int fault_scan_part;               // -1 normally; >= 0: that scan partition never publishes
    void *clear_begin;                 // scan_state, hist, sort_state and ranges: one span cleared before
    size_t clear_bytes;                //   the onesweep binning
    unsigned long long spin_limit;
    int sort_mode;                     // GS_SORT_TILE_BUCKET or GS_SORT_ONESWEEP
    uint32_t *tile_cnt;                // [G + 1] per-tile key counts -> slice starts (bucket mode)
    uint32_t *tile_list;               // [G] tiles whose slices are sorted by k_tile_sort_long
    const uint32_t *slot;              // [P] slot of each visible pair in proj and g2d
    long long vcap;                    // slots in proj and g2d
    unsigned long long *tword;         // [G] start/end combining words of the ranges kernel
    uint32_t *clist;                   // [kClaimClasses, G] out: the items of each claim class
};

// onesweep: scan with key emission and digit histograms -> onesweep passes -> ranges; tile bucket: scan of the
// tile counts -> emission into tile slices -> per-tile sort.  Either way the sorted keys end in
// keys[passes % 2], the values in vals[passes % 2], the records in list order in srec
int run_bin_sort(const BinArgs &a, cudaStream_t s);
// scan alone (used by the bounded-wait test entry point)
int run_scan_only(const BinArgs &a, cudaStream_t s);

// ---------------- rendering ----------------
struct FwdArgs {
    const float4 *srec;                // [K,3] records in list order (r1.w = the pair's slot, as bits)
    const uint32_t *ranges;
    const uint32_t *clist;             // [kClaimClasses, G] items of each claim class (counts in st)
    float *rgb, *depth, *alpha, *finalT;
    int32_t *last;
    DevStatus *st;
    int W, H, Tx, Ty;
    long long G, P, cap;               // global tiles, pairs, key capacity (the length of srec)
    float amax, amin, tmin, bg0, bg1, bg2;
    // optional L1 epilogue (Eq. 4's photometric and depth terms): null rgb_t = none
    const float *rgb_t, *depth_t;
    float sc_rgb, sc_d;                // w / element count of each term
    float *d_rgb, *d_depth;
    double *loss;
};

struct BwdArgs {
    const float4 *srec;
    const uint32_t *ranges;
    const uint32_t *clist;             // [kClaimClasses, G] items of each claim class (counts in st)
    const float *finalT;
    const int32_t *last;
    const float *d_rgb, *d_depth, *d_alpha;
    float *g2d;                        // [P,12]
    DevStatus *st;
    int W, H, Tx, Ty;
    long long G, P, cap;               // global tiles, slots of g2d, key capacity (the length of srec)
    float amax, amin, bg0, bg1, bg2;
};

int launch_render_fwd(int tw, int th, int nb, const FwdArgs &a, cudaStream_t s);
int launch_render_bwd(int tw, int th, int nb, const BwdArgs &a, cudaStream_t s);

// ---------------- losses / optimiser ----------------
int launch_loss_l1(int V, int W, int H, const float *rgb, const float *rgb_t, const float *depth,
                   const float *depth_t, float w_rgb, float w_depth, float *d_rgb, float *d_depth, double *loss,
                   cudaStream_t s);
size_t ssim_scratch_bytes(int V, int W, int H);
int launch_loss_l1_ssim(int V, int W, int H, const float *rgb, const float *rgb_t, float w_l1, float w_ssim,
                        float *d_rgb, double *loss, void *scratch, cudaStream_t s);
int launch_loss_l1_ssim_noalloc(int V, int W, int H, const float *rgb, const float *rgb_t, float w_l1,
                                float w_ssim, float *d_rgb, double *loss, cudaStream_t s);
size_t refine_scratch_bytes(int V, int W, int H);
int launch_loss_refine(int V, int W, int H, const float *rgb, const float *rgb_t, const float *depth,
                       const float *depth_t, const float *expo, float w_l1, float w_ssim, float w_depth, float *d_rgb,
                       float *d_depth, float *d_expo, double *loss, void *scratch, cudaStream_t s);
size_t prune_scratch_bytes(long long n);
int launch_prune(long long n, const gs_gaussians &in, float thr, const gs_gaussian_arrays &out, long long *kept,
                 void *scratch, cudaStream_t s);
int launch_view_adam(int V, const gs_view_adam_state &st, const float *pose_grad, const float *expo_grad, float lr_pose,
                     float lr_expo, cudaStream_t s);
int launch_voxset_clear(void *mem, long long capacity, cudaStream_t s);
int launch_voxset_add_boxes(void *mem, long long capacity, long long n, const float *means, const float *log_scales,
                            float k, float v, cudaStream_t s);
int launch_voxset_add_rays(void *mem, long long capacity, int V, int W, int H, const gs_camera *cams,
                           const float *depth, int stride, float v, cudaStream_t s);
int launch_voxset_keep(long long n, const float *means, void *occ, long long occ_cap, void *fre, long long free_cap,
                       float v, uint8_t *keep, cudaStream_t s);
int launch_sim3(long long n, const gs_gaussians &in, const float q[4], const float t[3], float sc,
                const gs_gaussian_arrays &out, cudaStream_t s);
int launch_grads_zero(long long n, const gs_grads &g, cudaStream_t s);
int launch_adam(long long n, const gs_adam_state &st, const gs_grads &g, const float lr[5], int zero_grads,
                cudaStream_t s, float iso_weight = 0.f, double *iso_loss = nullptr);

// normal term of the mapping loss, Eq. 4 (gs_normal.cu)
struct NormalArgs {
    const float *depth;                // [V,H,W]
    const float *prior;                // [V,3,H,W] unit normals, camera frame
    const gs_camera *cams;             // [V] (intrinsics read)
    float *d_depth;                    // [V,H,W], +=
    double *loss;                      // +=
    int V, W, H;
    float scale;                       // weight / (V H W)
};
int launch_loss_normal(const NormalArgs &a, cudaStream_t s);

// Eq. 12 photometric residual blocks (gs_photometric.cu)
constexpr int kPhoMaxBlocksPerEdge = 1024;
struct PhoArgs {
    const gs_pho_edge *edges;
    int num_images, num_corr, width, height, stride;
    const float *images, *depths;
    const gs_camera *cams;
    const gs_sim3 *corrs;
    float huber_delta, near_plane;
    double *partials;                  // [edges, blocks per edge, 40]
    double *cost, *H, *g;
    int64_t *count;
};
size_t pho_scratch_bytes(int num_edges);
int launch_pho(const PhoArgs &a, int num_edges, cudaStream_t s);

}  // namespace gs
