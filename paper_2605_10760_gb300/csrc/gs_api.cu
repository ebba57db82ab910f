// gs_api.cu -- the C ABI of libgs: argument validation, workspace layout, stage launches.
#include <algorithm>

#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cstring>
#include <vector>

#include "gs_kernels.cuh"

namespace gs {

// One NVTX range per library call (visible under a profiler; a no-op without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define GS_RANGE(name) NvtxRange gs_nvtx_range_(name)


static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int tile_ok(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 32 && th == 16);
}

int compute_layout(const gs_problem *pb, Layout *L) {
    if (!pb || !L) return GS_ERR_INVALID_ARG;
    const gs_params &p = pb->params;
    if (pb->num_views < 1 || pb->num_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    if (pb->width < 1 || pb->height < 1 || pb->width > 16384 || pb->height > 16384) return GS_ERR_INVALID_ARG;
    if (!tile_ok(p.tile_w, p.tile_h)) return GS_ERR_INVALID_ARG;
    if (!pb->view_gauss_begin || !pb->view_gauss_count || pb->num_gaussians < 0) return GS_ERR_INVALID_ARG;
    if (pb->key_capacity < 1 || pb->key_capacity >= (1LL << 30)) return GS_ERR_INVALID_ARG;
    if (!(p.alpha_max > 0.f && p.alpha_max < 1.f) || !(p.t_min > 0.f && p.t_min < 1.f) || !(p.alpha_min >= 0.f) ||
        !(p.dilation >= 0.f) || !(p.radius_sigmas > 0.f) || !(p.near_plane > 0.f))
        return GS_ERR_INVALID_ARG;
    if (p.sort_mode != GS_SORT_TILE_BUCKET && p.sort_mode != GS_SORT_ONESWEEP) return GS_ERR_INVALID_ARG;
    const int pix = p.tile_w * p.tile_h;
    const int nb = p.batch_records == 0 ? std::min(256, pix) : p.batch_records;
    if ((nb != 64 && nb != 128 && nb != 256) || nb > pix) return GS_ERR_INVALID_ARG;
    std::memset(L, 0, sizeof(*L));
    L->sort_mode = p.sort_mode;
    L->nb = nb;
    L->V = pb->num_views;
    L->W = pb->width;
    L->H = pb->height;
    L->tw = p.tile_w;
    L->th = p.tile_h;
    L->Tx = (L->W + L->tw - 1) / L->tw;
    L->Ty = (L->H + L->th - 1) / L->th;
    L->G = (long long)L->V * L->Tx * L->Ty;
    L->N = pb->num_gaussians;
    L->cap = pb->key_capacity;
    long long P = 0, maxc = 0;
    for (int v = 0; v < L->V; ++v) {
        const long long b = pb->view_gauss_begin[v], c = pb->view_gauss_count[v];
        if (b < 0 || c < 0 || b + c > L->N) return GS_ERR_INVALID_ARG;
        P += c;
        maxc = std::max(maxc, c);
    }
    if (P >= 0xffffffffLL) return GS_ERR_INVALID_ARG;   // pair indices are 32-bit
    L->P = P;
    if (pb->visible_capacity < 0) return GS_ERR_INVALID_ARG;
    L->vcap = pb->visible_capacity > 0 ? (long long)pb->visible_capacity : std::max<long long>(1, P);
    L->max_count = maxc;
    L->max_chunks = std::max<long long>(1, (maxc + kChunk - 1) / kChunk);
    int gbits = 0;
    while ((1LL << gbits) < L->G) ++gbits;
    L->passes = (32 + gbits + 7) / 8;
    if (L->passes > kMaxPasses) return GS_ERR_INVALID_ARG;
    // the scan runs over the P touched-tile counts (onesweep) or the G tile key counts (bucket)
    L->scan_parts = std::max<long long>(1, (std::max(P, L->G) + kScanTile - 1) / kScanTile);
    const long long sort_tile = (long long)kSortThreads * kSortIPT;
    L->sort_parts = std::max<long long>(1, (L->cap + sort_tile - 1) / sort_tile);
    long long chunks_total = 0;
    for (int v = 0; v < L->V; ++v) chunks_total += (pb->view_gauss_count[v] + kChunk - 1) / kChunk;
    L->chunks_total = chunks_total;
    size_t o = 0;
    int ng = 0;   // a guard block of kGuardBytes follows each buffer that kernels index with data
    auto guard = [&]() {
        if (ng < kNumGuards) L->o_guard[ng] = o;
        ++ng;
        o += kGuardBytes;
    };
    L->o_status = o; o = align256(o + sizeof(DevStatus));
    L->o_views = o; o = align256(o + sizeof(ViewEntry) * L->V);
    L->o_proj = o; o = align256(o + sizeof(float) * 12 * (size_t)L->vcap);
    guard();
    L->o_touched = o; o = align256(o + sizeof(uint32_t) * (size_t)std::max<long long>(P, 1) + 64);
    guard();
    for (int k = 0; k < 2; ++k) { L->o_keys[k] = o; o = align256(o + sizeof(uint64_t) * (size_t)L->cap); guard(); }
    for (int k = 0; k < 2; ++k) { L->o_vals[k] = o; o = align256(o + sizeof(uint32_t) * (size_t)L->cap); guard(); }
    // scan_state .. ranges are adjacent: the onesweep binning clears them with one memset
    L->o_scan_state = o; o = align256(o + sizeof(unsigned long long) * L->scan_parts);
    L->o_hist = o; o = align256(o + sizeof(uint32_t) * kMaxPasses * 256);
    L->o_sort_state = o; o = align256(o + sizeof(uint32_t) * 256 * (size_t)L->sort_parts * L->passes);
    L->o_ranges = o; o = align256(o + sizeof(uint32_t) * 2 * (size_t)L->G);
    L->o_tword = o; o = align256(o + sizeof(unsigned long long) * (size_t)L->G);
    guard();
    L->o_tcnt = o; o = align256(o + sizeof(uint32_t) * ((size_t)L->G + 1) + 64);
    L->o_tlist = o; o = align256(o + sizeof(uint32_t) * (size_t)L->G);
    guard();
    L->o_srec = o; o = align256(o + sizeof(float) * 12 * (size_t)L->cap);
    guard();
    L->o_g2d = o; o = align256(o + sizeof(float) * 12 * (size_t)L->vcap);
    guard();
    L->o_pose_part = o; o = align256(o + sizeof(float) * 8 * (size_t)std::max<long long>(chunks_total, 1));
    guard();
    L->o_slot = o; o = align256(o + sizeof(uint32_t) * (size_t)std::max<long long>(P, 1));
    guard();
    L->o_clist = o; o = align256(o + sizeof(uint32_t) * kClaimClasses * (size_t)std::max<long long>(L->G, 1));
    guard();
    L->o_slane = o; o = align256(o + sizeof(uint16_t) * (size_t)L->vcap);
    guard();
    L->o_blk = o; o = align256(o + sizeof(uint4) * (size_t)std::max<long long>(chunks_total, 1));
    guard();
    if (ng != kNumGuards) return GS_ERR_INVALID_ARG;   // the layout and kNumGuards disagree: a build error
    L->total = o;
    return GS_OK;
}

static int ws_ok(const void *ws) { return ws && ((uintptr_t)ws & 255) == 0; }

}  // namespace gs

using namespace gs;

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char *gs_error_string(int code) {
    switch (code) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "key capacity exceeded";
    case GS_ERR_TIMEOUT: return "bounded device wait timed out";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_DEVICE_FAULT: return "device consistency check failed";
    case GS_ERR_TOO_LARGE: return "input larger than the static scratch area holds";
    default: return "unknown error";
    }
}

int gs_version(int *major, int *minor, int *arch) {
    if (major) *major = 1;
    if (minor) *minor = 0;
#ifdef GS_ARCH
    if (arch) *arch = GS_ARCH;
#else
    if (arch) *arch = 0;
#endif
    return GS_OK;
}

void gs_default_params(gs_params *out) {
    if (!out) return;
    out->tile_w = 16;
    out->tile_h = 16;
    out->near_plane = 0.2f;
    out->dilation = 0.3f;
    out->radius_sigmas = 3.0f;
    out->alpha_max = 0.99f;
    out->alpha_min = 1.0f / 255.0f;
    out->t_min = 1e-4f;
    out->bg[0] = out->bg[1] = out->bg[2] = 0.0f;
    out->sort_mode = GS_SORT_ONESWEEP;
    out->batch_records = 0;
}

int gs_workspace_size(const gs_problem *pb, size_t *bytes) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!bytes) return GS_ERR_INVALID_ARG;
    *bytes = L.total;
    return GS_OK;
}

__global__ void k_write_views(ViewEntry *dst, int first, int n, ViewEntry e0, ViewEntry e1, ViewEntry e2,
                              ViewEntry e3, ViewEntry e4, ViewEntry e5, ViewEntry e6, ViewEntry e7) {
    const ViewEntry es[8] = {e0, e1, e2, e3, e4, e5, e6, e7};
    if ((int)threadIdx.x < n) dst[first + threadIdx.x] = es[threadIdx.x];
}

int gs_workspace_init(const gs_problem *pb, void *ws, void *stream) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<ViewEntry> ve(L.V);
    long long pair = 0, chunk = 0;
    for (int v = 0; v < L.V; ++v) {
        ve[v].gauss_begin = pb->view_gauss_begin[v];
        ve[v].count = pb->view_gauss_count[v];
        ve[v].pair_off = pair;
        ve[v].chunk_off = chunk;
        pair += ve[v].count;
        chunk += (ve[v].count + kChunk - 1) / kChunk;
    }
    if (cudaMemsetAsync(ws_ptr<void>(ws, L.o_status), 0, sizeof(DevStatus), s) != cudaSuccess) return GS_ERR_CUDA;
    for (int k = 0; k < kNumGuards; ++k)
        if (cudaMemsetAsync(ws_ptr<void>(ws, L.o_guard[k]), kGuardByte, kGuardBytes, s) != cudaSuccess) return GS_ERR_CUDA;
    ViewEntry *dst = ws_ptr<ViewEntry>(ws, L.o_views);
    for (int v0 = 0; v0 < L.V; v0 += 8) {
        ViewEntry e[8];
        std::memset(e, 0, sizeof(e));
        const int n = std::min(8, L.V - v0);
        for (int k = 0; k < n; ++k) e[k] = ve[v0 + k];
        k_write_views<<<1, 8, 0, s>>>(dst, v0, n, e[0], e[1], e[2], e[3], e[4], e[5], e[6], e[7]);
        count_launches(1);
    }
    return check_launch();
}

int gs_workspace_view(const gs_problem *pb, void *ws, gs_ws_view *out) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !out) return GS_ERR_INVALID_ARG;
    out->proj = ws_ptr<float>(ws, L.o_proj);
    out->tiles_touched = ws_ptr<uint32_t>(ws, L.o_touched);
    out->sorted_keys = ws_ptr<uint64_t>(ws, L.o_keys[L.passes & 1]);
    out->sorted_vals = ws_ptr<uint32_t>(ws, L.o_vals[L.passes & 1]);
    out->tile_ranges = ws_ptr<uint32_t>(ws, L.o_ranges);
    out->grad2d = ws_ptr<float>(ws, L.o_g2d);
    out->num_keys = reinterpret_cast<uint32_t *>(&ws_ptr<DevStatus>(ws, L.o_status)->num_keys);
    out->num_pairs = L.P;
    out->num_tiles = L.G;
    out->sort_passes = L.passes;
    out->reserved = 0;
    out->pair_slot = ws_ptr<uint32_t>(ws, L.o_slot);
    out->visible_capacity = L.vcap;
    out->claim_count = ws_ptr<DevStatus>(ws, L.o_status)->claim_cnt;
    out->claim_list = ws_ptr<uint32_t>(ws, L.o_clist);
    return GS_OK;
}

int gs_check_status(const gs_problem *pb, void *ws, void *stream, int64_t *required_keys) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus h;
    DevStatus *d = ws_ptr<DevStatus>(ws, L.o_status);
    if (cudaMemcpyAsync(&h, d, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    if (required_keys) *required_keys = (int64_t)h.required_keys;
    if (h.code != 0) {
        int32_t zero[2] = {0, 0};
        if (cudaMemcpyAsync(d, zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return h.code;
}

}  // extern "C"

namespace gs {

struct GuardPtrs {
    const uint32_t *p[kNumGuards];
};

// one CTA: thread t compares word t of every guard block with the fill pattern
__global__ void k_check_guards(GuardPtrs g, int32_t *bad) {
    const uint32_t want = 0x01010101u * (uint32_t)kGuardByte;
    for (int k = 0; k < kNumGuards; ++k)
        for (int t = threadIdx.x; t < (int)(kGuardBytes / 4); t += blockDim.x)
            if (g.p[k][t] != want) atomicMin(bad, k);
}

int run_check_guards(const unsigned char *const *guards, DevStatus *st, int32_t *first_bad, cudaStream_t s) {
    GuardPtrs g;
    for (int k = 0; k < kNumGuards; ++k) g.p[k] = reinterpret_cast<const uint32_t *>(guards[k]);
    const int32_t none = kNumGuards;
    if (cudaMemcpyAsync(&st->guard_bad, &none, sizeof(none), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GS_ERR_CUDA;
    k_check_guards<<<1, 64, 0, s>>>(g, &st->guard_bad);
    count_launches(1);
    int32_t h = none;
    if (cudaMemcpyAsync(&h, &st->guard_bad, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    *first_bad = h < kNumGuards ? h : -1;
    return GS_OK;
}

}  // namespace gs

extern "C" {

int gs_check_guards(const gs_problem *pb, void *ws, void *stream, int32_t *first_bad) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char *g[kNumGuards];
    for (int k = 0; k < kNumGuards; ++k) g[k] = ws_ptr<const unsigned char>(ws, L.o_guard[k]);
    int32_t bad = -1;
    rc = run_check_guards(g, ws_ptr<DevStatus>(ws, L.o_status), &bad, s);
    if (first_bad) *first_bad = bad;
    if (rc) return rc;
    return bad >= 0 ? GS_ERR_DEVICE_FAULT : GS_OK;
}

int32_t gs_checked_build(void) { return GS_CHECKED ? 1 : 0; }

int gs_read_stats(const gs_problem *pb, void *ws, void *stream, gs_stats *out) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !out) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus h;
    if (cudaMemcpyAsync(&h, ws_ptr<DevStatus>(ws, L.o_status), sizeof(DevStatus), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    out->num_keys = (int64_t)h.num_keys;
    out->fwd_pairs = (int64_t)h.fwd_pairs;
    out->bwd_pairs = (int64_t)h.bwd_pairs;
    out->num_visible = (int64_t)h.num_visible;
    return GS_OK;
}

int gs_project(const gs_problem *pb, const gs_gaussians *g, void *ws, void *stream) {
    GS_RANGE("gs_project");
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !g || !pb->cameras) return GS_ERR_INVALID_ARG;
    if (L.N > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacities || !g->colors)) return GS_ERR_INVALID_ARG;
    if (((uintptr_t)g->quats & 15) != 0) return GS_ERR_INVALID_ARG;
    if (L.sort_mode == GS_SORT_TILE_BUCKET &&
        cudaMemsetAsync(ws_ptr<uint32_t>(ws, L.o_tcnt), 0, sizeof(uint32_t) * ((size_t)L.G + 1),
                        (cudaStream_t)stream) != cudaSuccess)
        return GS_ERR_CUDA;
    DevStatus *st = ws_ptr<DevStatus>(ws, L.o_status);
    if (L.P == 0)   // no projection launch: no slots taken
        return cudaMemsetAsync(&st->num_visible, 0, sizeof(st->num_visible), (cudaStream_t)stream) == cudaSuccess
                   ? GS_OK : GS_ERR_CUDA;
    ProjArgs a;
    a.views = ws_ptr<ViewEntry>(ws, L.o_views);
    a.cams = pb->cameras;
    a.means = g->means; a.log_scales = g->log_scales; a.quats = g->quats;
    a.opacities = g->opacities; a.colors = g->colors;
    a.proj = ws_ptr<float4>(ws, L.o_proj);
    a.touched = ws_ptr<uint32_t>(ws, L.o_touched);
    a.W = L.W; a.H = L.H;
    a.itw = 1.0f / (float)L.tw; a.ith = 1.0f / (float)L.th; a.Tx = (float)L.Tx; a.Ty = (float)L.Ty;
    a.near_plane = pb->params.near_plane; a.dil = pb->params.dilation; a.sigmas = pb->params.radius_sigmas;
    a.alpha_min = pb->params.alpha_min;
    a.tile_cnt = L.sort_mode == GS_SORT_TILE_BUCKET ? ws_ptr<uint32_t>(ws, L.o_tcnt) : nullptr;
    a.P = L.P;
    a.st = st;
    a.slot = ws_ptr<uint32_t>(ws, L.o_slot);
    a.vcap = L.vcap;
    a.slane = ws_ptr<uint16_t>(ws, L.o_slane);
    a.blk = ws_ptr<uint4>(ws, L.o_blk);
    a.chunks = L.chunks_total;
    a.Txi = L.Tx;
    a.Ty_i = L.Ty;
    launch_project(L, a, (cudaStream_t)stream);
    return check_launch();
}

static BinArgs make_bin_args(const Layout &L, void *ws) {
    BinArgs a;
    std::memset(&a, 0, sizeof(a));
    a.views = ws_ptr<ViewEntry>(ws, L.o_views);
    a.touched = ws_ptr<uint32_t>(ws, L.o_touched);
    a.scan_state = ws_ptr<unsigned long long>(ws, L.o_scan_state);
    a.proj = ws_ptr<float4>(ws, L.o_proj);
    a.g2d = ws_ptr<float4>(ws, L.o_g2d);
    for (int k = 0; k < 2; ++k) {
        a.keys[k] = ws_ptr<uint64_t>(ws, L.o_keys[k]);
        a.vals[k] = ws_ptr<uint32_t>(ws, L.o_vals[k]);
    }
    a.hist = ws_ptr<uint32_t>(ws, L.o_hist);
    a.sort_state = ws_ptr<uint32_t>(ws, L.o_sort_state);
    a.ranges = ws_ptr<uint32_t>(ws, L.o_ranges);
    a.srec = ws_ptr<float4>(ws, L.o_srec);
    a.st = ws_ptr<DevStatus>(ws, L.o_status);
    a.V = L.V; a.Tx = L.Tx; a.Ty = L.Ty; a.passes = L.passes;
    a.itw = 1.0f / (float)L.tw; a.ith = 1.0f / (float)L.th;
    a.P = L.P; a.cap = L.cap; a.sort_parts = L.sort_parts; a.max_chunks = L.max_chunks; a.G = L.G;
    a.slot = ws_ptr<const uint32_t>(ws, L.o_slot);
    a.vcap = L.vcap;
    a.fault_scan_part = -1;
    a.spin_limit = kSpinLimit;
    a.sort_mode = L.sort_mode;
    a.tile_cnt = ws_ptr<uint32_t>(ws, L.o_tcnt);
    a.tile_list = ws_ptr<uint32_t>(ws, L.o_tlist);
    a.tword = ws_ptr<unsigned long long>(ws, L.o_tword);
    a.clist = ws_ptr<uint32_t>(ws, L.o_clist);
    a.clear_begin = ws_ptr<unsigned char>(ws, L.o_scan_state);
    a.clear_bytes = L.o_tword + sizeof(unsigned long long) * (size_t)L.G - L.o_scan_state;
    return a;
}

int gs_bin_sort(const gs_problem *pb, void *ws, void *stream) {
    GS_RANGE("gs_bin_sort");
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws)) return GS_ERR_INVALID_ARG;
    BinArgs a = make_bin_args(L, ws);
    return run_bin_sort(a, (cudaStream_t)stream);
}

static int render_fwd_impl(const gs_problem *pb, void *ws, const gs_image *out, const gs_l1_target *l1,
                           void *stream) {
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !out || !out->final_T || !out->last_idx) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FwdArgs a;
    a.srec = ws_ptr<const float4>(ws, L.o_srec);
    a.ranges = ws_ptr<const uint32_t>(ws, L.o_ranges);
    a.clist = ws_ptr<const uint32_t>(ws, L.o_clist);
    a.rgb = out->rgb; a.depth = out->depth; a.alpha = out->alpha; a.finalT = out->final_T; a.last = out->last_idx;
    a.st = ws_ptr<DevStatus>(ws, L.o_status);
    a.W = L.W; a.H = L.H; a.Tx = L.Tx; a.Ty = L.Ty; a.G = L.G; a.P = std::max<long long>(L.P, 1);
    a.cap = L.cap;
    const gs_params &p = pb->params;
    a.amax = p.alpha_max; a.amin = p.alpha_min; a.tmin = p.t_min;
    a.bg0 = p.bg[0]; a.bg1 = p.bg[1]; a.bg2 = p.bg[2];
    a.rgb_t = nullptr; a.depth_t = nullptr; a.d_rgb = nullptr; a.d_depth = nullptr; a.loss = nullptr;
    a.sc_rgb = a.sc_d = 0.f;
    if (l1) {
        const double HWn = (double)L.W * L.H;
        a.rgb_t = l1->rgb_t;
        a.d_rgb = l1->d_rgb;
        a.loss = l1->loss;
        a.sc_rgb = (float)((double)l1->w_rgb / (3.0 * L.V * HWn));
        if (l1->w_depth != 0.f) {
            a.depth_t = l1->depth_t;
            a.d_depth = l1->d_depth;
            a.sc_d = (float)((double)l1->w_depth / ((double)L.V * HWn));
        }
    }
    return launch_render_fwd(L.tw, L.th, L.nb, a, s);
}

int gs_render_fwd(const gs_problem *pb, void *ws, const gs_image *out, void *stream) {
    GS_RANGE("gs_render_fwd");
    return render_fwd_impl(pb, ws, out, nullptr, stream);
}

int gs_render_fwd_l1(const gs_problem *pb, void *ws, const gs_image *out, const gs_l1_target *l1, void *stream) {
    GS_RANGE("gs_render_fwd_l1");
    if (!l1 || !l1->rgb_t || !l1->d_rgb || !l1->loss) return GS_ERR_INVALID_ARG;
    if (l1->w_depth != 0.f && (!l1->depth_t || !l1->d_depth)) return GS_ERR_INVALID_ARG;
    return render_fwd_impl(pb, ws, out, l1, stream);
}

int gs_render_bwd_composite(const gs_problem *pb, void *ws, const gs_image *fwd, const gs_image_grad *dimg,
                            void *stream) {
    GS_RANGE("gs_render_bwd_composite");
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !fwd || !fwd->final_T || !fwd->last_idx || !dimg) return GS_ERR_INVALID_ARG;
    BwdArgs a;
    a.srec = ws_ptr<const float4>(ws, L.o_srec);
    a.ranges = ws_ptr<const uint32_t>(ws, L.o_ranges);
    a.clist = ws_ptr<const uint32_t>(ws, L.o_clist);
    a.finalT = fwd->final_T; a.last = fwd->last_idx;
    a.d_rgb = dimg->d_rgb; a.d_depth = dimg->d_depth; a.d_alpha = dimg->d_alpha;
    a.g2d = ws_ptr<float>(ws, L.o_g2d);
    a.st = ws_ptr<DevStatus>(ws, L.o_status);
    a.W = L.W; a.H = L.H; a.Tx = L.Tx; a.Ty = L.Ty; a.G = L.G; a.P = L.vcap;   // g2d slots
    a.cap = L.cap;
    const gs_params &p = pb->params;
    a.amax = p.alpha_max; a.amin = p.alpha_min;
    a.bg0 = p.bg[0]; a.bg1 = p.bg[1]; a.bg2 = p.bg[2];
    return launch_render_bwd(L.tw, L.th, L.nb, a, (cudaStream_t)stream);
}

int gs_project_bwd(const gs_problem *pb, const gs_gaussians *g, void *ws, const gs_grads *grads, void *stream) {
    GS_RANGE("gs_project_bwd");
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !g || !grads || !pb->cameras) return GS_ERR_INVALID_ARG;
    if (L.N > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacities || !grads->colors))
        return GS_ERR_INVALID_ARG;
    if (L.P == 0) return GS_OK;
    ProjBwdArgs b;
    b.views = ws_ptr<ViewEntry>(ws, L.o_views);
    b.cams = pb->cameras;
    b.means = g->means; b.log_scales = g->log_scales; b.quats = g->quats;
    b.slane = ws_ptr<const uint16_t>(ws, L.o_slane);
    b.blk = ws_ptr<const uint4>(ws, L.o_blk);
    b.g2d = ws_ptr<const float4>(ws, L.o_g2d);
    b.g_means = grads->means; b.g_ls = grads->log_scales; b.g_quats = grads->quats;
    b.g_op = grads->opacities; b.g_col = grads->colors;
    b.pose_part = ws_ptr<float>(ws, L.o_pose_part);
    b.W = L.W; b.H = L.H;
    b.dil = pb->params.dilation;
    b.P = L.P;
    b.N = L.N;
    b.slot = ws_ptr<const uint32_t>(ws, L.o_slot);
    b.vcap = L.vcap;
    b.chunks = L.chunks_total;
    b.st = ws_ptr<DevStatus>(ws, L.o_status);
    launch_project_bwd(L, b, (cudaStream_t)stream);
    return check_launch();
}

int gs_render_bwd(const gs_problem *pb, const gs_gaussians *g, void *ws, const gs_image *fwd,
                  const gs_image_grad *dimg, const gs_grads *grads, void *stream) {
    GS_RANGE("gs_render_bwd");
    if (!g || !grads || !pb || !pb->cameras) return GS_ERR_INVALID_ARG;
    const int rc = gs_render_bwd_composite(pb, ws, fwd, dimg, stream);
    if (rc) return rc;
    return gs_project_bwd(pb, g, ws, grads, stream);
}

int gs_pose_grad(const gs_problem *pb, void *ws, float *pose_grad, void *stream) {
    GS_RANGE("gs_pose_grad");
    Layout L;
    int rc = compute_layout(pb, &L);
    if (rc) return rc;
    if (!ws_ok(ws) || !pose_grad) return GS_ERR_INVALID_ARG;
    launch_pose_reduce(L, ws_ptr<ViewEntry>(ws, L.o_views), ws_ptr<float>(ws, L.o_pose_part), pose_grad,
                       ws_ptr<DevStatus>(ws, L.o_status),
                       (cudaStream_t)stream);
    return check_launch();
}

int gs_loss_l1(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
               const float *depth, const float *depth_t, float w_rgb, float w_depth, float *d_rgb, float *d_depth,
               double *loss, void *stream) {
    GS_RANGE("gs_loss_l1");
    if (views < 1 || views > 65535 || width < 1 || height < 1 || !rgb || !rgb_t || !d_rgb || !loss)
        return GS_ERR_INVALID_ARG;
    if (w_depth != 0.f && (!depth || !depth_t || !d_depth)) return GS_ERR_INVALID_ARG;
    return launch_loss_l1(views, width, height, rgb, rgb_t, depth, depth_t, w_rgb, w_depth, d_rgb, d_depth, loss,
                          (cudaStream_t)stream);
}

int gs_loss_normal(int32_t views, int32_t width, int32_t height, const float *depth, const float *prior,
                   const gs_camera *cams, float weight, float *d_depth, double *loss, void *stream) {
    GS_RANGE("gs_loss_normal");
    if (views < 1 || views > GS_MAX_VIEWS || width < 1 || height < 1 || width > 16384 || height > 16384 || !depth ||
        !prior || !cams || !d_depth || !loss || !(weight == weight))
        return GS_ERR_INVALID_ARG;
    NormalArgs a;
    a.depth = depth;
    a.prior = prior;
    a.cams = cams;
    a.d_depth = d_depth;
    a.loss = loss;
    a.V = views;
    a.W = width;
    a.H = height;
    a.scale = (float)((double)weight / ((double)views * width * height));
    return launch_loss_normal(a, (cudaStream_t)stream);
}

size_t gs_ssim_scratch_size(int32_t views, int32_t width, int32_t height) {
    if (views < 1 || width < 1 || height < 1) return 0;
    return ssim_scratch_bytes(views, width, height);
}

int gs_loss_l1_ssim(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t, float w_l1,
                    float w_ssim, float *d_rgb, double *loss, void *scratch, void *stream) {
    GS_RANGE("gs_loss_l1_ssim");
    if (views < 1 || width < 1 || height < 1 || !rgb || !rgb_t || !d_rgb || !loss || !ws_ok(scratch))
        return GS_ERR_INVALID_ARG;
    return launch_loss_l1_ssim(views, width, height, rgb, rgb_t, w_l1, w_ssim, d_rgb, loss, scratch,
                               (cudaStream_t)stream);
}

int gs_loss_l1_ssim_noalloc(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
                            float w_l1, float w_ssim, float *d_rgb, double *loss, void *stream) {
    GS_RANGE("gs_loss_l1_ssim_noalloc");
    if (views < 1 || width < 1 || height < 1 || !rgb || !rgb_t || !d_rgb || !loss) return GS_ERR_INVALID_ARG;
    if ((long long)width * height > GS_SSIM_NOALLOC_MAX_PLANE) return GS_ERR_TOO_LARGE;
    return launch_loss_l1_ssim_noalloc(views, width, height, rgb, rgb_t, w_l1, w_ssim, d_rgb, loss,
                                       (cudaStream_t)stream);
}

size_t gs_refine_scratch_size(int32_t views, int32_t width, int32_t height) {
    if (views < 1 || width < 1 || height < 1) return 0;
    return refine_scratch_bytes(views, width, height);
}

int gs_loss_refine(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
                   const float *depth, const float *depth_t, const float *expo, float w_l1, float w_ssim,
                   float w_depth, float *d_rgb, float *d_depth, float *d_expo, double *loss, void *scratch,
                   void *stream) {
    GS_RANGE("gs_loss_refine");
    if (views < 1 || views > GS_MAX_VIEWS || width < 1 || height < 1 || !rgb || !rgb_t || !expo || !d_rgb ||
        !loss || !ws_ok(scratch))
        return GS_ERR_INVALID_ARG;
    if (w_depth != 0.f && (!depth || !depth_t || !d_depth)) return GS_ERR_INVALID_ARG;
    return launch_loss_refine(views, width, height, rgb, rgb_t, depth, depth_t, expo, w_l1, w_ssim, w_depth, d_rgb,
                              d_depth, d_expo, loss, scratch, (cudaStream_t)stream);
}

size_t gs_prune_scratch_size(int64_t n) { return n < 1 ? 0 : prune_scratch_bytes(n); }

int gs_prune(int64_t n, const gs_gaussians *in, float threshold, const gs_gaussian_arrays *out, int64_t *kept,
             void *scratch, void *stream) {
    GS_RANGE("gs_prune");
    if (n < 1 || n >= (1LL << 30) || !in || !out || !kept || !ws_ok(scratch)) return GS_ERR_INVALID_ARG;
    if (!in->means || !in->log_scales || !in->quats || !in->opacities || !in->colors || !out->means ||
        !out->log_scales || !out->quats || !out->opacities || !out->colors)
        return GS_ERR_INVALID_ARG;
    return launch_prune(n, *in, threshold, *out, reinterpret_cast<long long *>(kept), scratch, (cudaStream_t)stream);
}

int gs_view_adam_step(int32_t views, const gs_view_adam_state *st, const float *pose_grad, const float *expo_grad,
                      float lr_pose, float lr_expo, void *stream) {
    GS_RANGE("gs_view_adam_step");
    if (views < 1 || views > GS_MAX_VIEWS || !st || !st->cameras || !st->expo || !st->m || !st->v || !st->step ||
        !pose_grad || !expo_grad)
        return GS_ERR_INVALID_ARG;
    return launch_view_adam(views, *st, pose_grad, expo_grad, lr_pose, lr_expo, (cudaStream_t)stream);
}

static bool pow2(long long c) { return c >= 2 && (c & (c - 1)) == 0; }

int gs_sim3_apply(int64_t n, const gs_gaussians *in, const gs_sim3 *C, const gs_gaussian_arrays *out, void *stream) {
    GS_RANGE("gs_sim3_apply");
    if (n < 0 || !in || !C || !out || !(C->s > 0.f)) return GS_ERR_INVALID_ARG;
    const float nq = C->q[0] * C->q[0] + C->q[1] * C->q[1] + C->q[2] * C->q[2] + C->q[3] * C->q[3];
    if (!(nq > 0.f)) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!in->means || !in->log_scales || !in->quats || !in->opacities || !in->colors || !out->means ||
                  !out->log_scales || !out->quats || !out->opacities || !out->colors))
        return GS_ERR_INVALID_ARG;
    return launch_sim3(n, *in, C->q, C->t, C->s, *out, (cudaStream_t)stream);
}

size_t gs_voxset_bytes(int64_t capacity) { return pow2(capacity) ? 256 + 8 * (size_t)capacity : 0; }

int gs_voxset_clear(void *set, int64_t capacity, void *stream) {
    if (!ws_ok(set) || !pow2(capacity)) return GS_ERR_INVALID_ARG;
    return launch_voxset_clear(set, capacity, (cudaStream_t)stream);
}

__global__ void k_voxset_count(const unsigned long long *keys, long long capacity, unsigned long long *out) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < capacity; i += (long long)gridDim.x * blockDim.x)
        c += keys[i] != ~0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int gs_voxset_status(void *set, void *stream, int64_t *count, int64_t capacity) {
    if (!ws_ok(set)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t code = 0;
    if (count) {
        if (!pow2(capacity)) return GS_ERR_INVALID_ARG;
        // counter in the status block's spare bytes (offset 8)
        unsigned long long *c = reinterpret_cast<unsigned long long *>(static_cast<char *>(set) + 8);
        if (cudaMemsetAsync(c, 0, 8, s) != cudaSuccess) return GS_ERR_CUDA;
        k_voxset_count<<<std::max(1, std::min((int)((capacity + 255) / 256), device_sm_count() * 8)), 256, 0, s>>>(
            reinterpret_cast<const unsigned long long *>(static_cast<char *>(set) + 256), capacity, c);
        count_launches(1);
        unsigned long long h = 0;
        if (cudaMemcpyAsync(&h, c, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
        *count = (int64_t)h;
    }
    if (cudaMemcpyAsync(&code, set, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    return code;
}

int gs_voxset_add_boxes(void *set, int64_t capacity, int64_t n, const float *means, const float *log_scales, float k,
                        float voxel, void *stream) {
    GS_RANGE("gs_voxset_add_boxes");
    if (!ws_ok(set) || !pow2(capacity) || n < 0 || (n > 0 && (!means || !log_scales)) || !(voxel > 0.f) || !(k >= 0.f))
        return GS_ERR_INVALID_ARG;
    return launch_voxset_add_boxes(set, capacity, n, means, log_scales, k, voxel, (cudaStream_t)stream);
}

int gs_voxset_add_rays(void *set, int64_t capacity, int32_t views, int32_t width, int32_t height,
                       const gs_camera *cams, const float *depth, int32_t stride, float voxel, void *stream) {
    GS_RANGE("gs_voxset_add_rays");
    if (!ws_ok(set) || !pow2(capacity) || views < 1 || width < 1 || height < 1 || !cams || !depth || stride < 1 ||
        !(voxel > 0.f))
        return GS_ERR_INVALID_ARG;
    return launch_voxset_add_rays(set, capacity, views, width, height, cams, depth, stride, voxel, (cudaStream_t)stream);
}

int gs_voxset_keep(int64_t n, const float *means, void *occ, int64_t occ_capacity, void *free_set,
                   int64_t free_capacity, float voxel, uint8_t *keep, void *stream) {
    GS_RANGE("gs_voxset_keep");
    if (n < 0 || (n > 0 && (!means || !keep)) || !ws_ok(occ) || !pow2(occ_capacity) || !(voxel > 0.f))
        return GS_ERR_INVALID_ARG;
    if (free_set && (!ws_ok(free_set) || !pow2(free_capacity))) return GS_ERR_INVALID_ARG;
    return launch_voxset_keep(n, means, occ, occ_capacity, free_set, free_capacity, voxel, keep, (cudaStream_t)stream);
}

gs_pho_params gs_default_pho_params(void) {
    gs_pho_params p;
    p.stride = 1;
    p.huber_delta = 9.0f / 255.0f;
    p.near_plane = 0.2f;
    p.reserved = 0;
    return p;
}

size_t gs_pho_scratch_size(int32_t num_edges) { return num_edges > 0 ? pho_scratch_bytes(num_edges) : 0; }

int gs_pho_residual(int32_t num_edges, const gs_pho_edge *edges, int32_t num_images, int32_t width, int32_t height,
                    const float *images, const float *depths, const gs_camera *cameras, int32_t num_corr,
                    const gs_sim3 *corrections, const gs_pho_params *params, double *cost, int64_t *count,
                    double *H, double *g, void *scratch, size_t scratch_bytes, void *stream) {
    GS_RANGE("gs_pho_residual");
    if (num_edges < 0 || num_edges > 65535 || !params) return GS_ERR_INVALID_ARG;
    if (num_edges == 0) return GS_OK;
    if (!edges || !images || !depths || !cameras || !corrections || !cost || !count || !H || !g || !scratch)
        return GS_ERR_INVALID_ARG;
    if (num_images < 1 || num_corr < 1 || width < 2 || height < 2 || params->stride < 1) return GS_ERR_INVALID_ARG;
    if (scratch_bytes < pho_scratch_bytes(num_edges)) return GS_ERR_INVALID_ARG;
    PhoArgs a;
    a.edges = edges;
    a.num_images = num_images;
    a.num_corr = num_corr;
    a.width = width;
    a.height = height;
    a.stride = params->stride;
    a.images = images;
    a.depths = depths;
    a.cams = cameras;
    a.corrs = corrections;
    a.huber_delta = params->huber_delta;
    a.near_plane = params->near_plane;
    a.partials = static_cast<double *>(scratch);
    a.cost = cost;
    a.H = H;
    a.g = g;
    a.count = count;
    const int rc = launch_pho(a, num_edges, (cudaStream_t)stream);
    count_launches(2);
    return rc != GS_OK ? rc : check_launch();
}

int gs_adam_step(int64_t n, const gs_adam_state *st, const gs_grads *grads, const float lr[5], int32_t zero_grads,
                 void *stream) {
    GS_RANGE("gs_adam_step");
    if (n < 0 || !st || !grads || !lr || !st->step || !st->m || !st->v) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!st->means || !st->log_scales || !st->quats || !st->opacity_logits || !st->opacities ||
                  !st->colors || !grads->means || !grads->log_scales || !grads->quats || !grads->opacities ||
                  !grads->colors))
        return GS_ERR_INVALID_ARG;
    return launch_adam(n, *st, *grads, lr, zero_grads, (cudaStream_t)stream);
}

int gs_adam_step_reg(int64_t n, const gs_adam_state *st, const gs_grads *grads, const float lr[5], float iso_weight,
                     int32_t zero_grads, double *iso_loss, void *stream) {
    GS_RANGE("gs_adam_step_reg");
    if (n < 0 || !st || !grads || !lr || !st->step || !st->m || !st->v) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!st->means || !st->log_scales || !st->quats || !st->opacity_logits || !st->opacities ||
                  !st->colors || !grads->means || !grads->log_scales || !grads->quats || !grads->opacities ||
                  !grads->colors))
        return GS_ERR_INVALID_ARG;
    return launch_adam(n, *st, *grads, lr, zero_grads, (cudaStream_t)stream, iso_weight, iso_loss);
}

__global__ void k_debug_expf(const float *x, float *ys, float *yc, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = x[i];
        if (ys) ys[i] = spec_expf(v);
        if (yc) yc[i] = expf(v);
    }
}

int gs_grads_zero(int64_t n, const gs_grads *g, void *stream) {
    GS_RANGE("gs_grads_zero");
    if (n < 0 || !g) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!g->means || !g->log_scales || !g->quats || !g->opacities || !g->colors) return GS_ERR_INVALID_ARG;
    return launch_grads_zero(n, *g, (cudaStream_t)stream);
}

int64_t gs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int gs_debug_expf(const float *x, float *y_spec, float *y_cuda, int64_t n, void *stream) {
    if (!x || n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    k_debug_expf<<<grid, 256, 0, (cudaStream_t)stream>>>(x, y_spec, y_cuda, n);
    count_launches(1);
    return check_launch();
}

__global__ void k_fill_ones(uint32_t *p, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 1u;
}

size_t gs_debug_scan_scratch_size(int64_t n) {
    if (n < 1) return 0;
    const long long parts = (n + kScanTile - 1) / kScanTile;
    return align256(sizeof(DevStatus)) + align256(sizeof(uint32_t) * (size_t)n) +
           align256(sizeof(unsigned long long) * (size_t)parts);
}

int gs_debug_scan_timeout(void *scratch, int64_t n, int32_t silent_partition, void *stream, int64_t *total) {
    if (!ws_ok(scratch) || n < 1 || n > (1LL << 28)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BinArgs a;
    std::memset(&a, 0, sizeof(a));
    a.st = ws_ptr<DevStatus>(scratch, 0);
    a.touched = ws_ptr<uint32_t>(scratch, align256(sizeof(DevStatus)));
    a.scan_state = ws_ptr<unsigned long long>(scratch, align256(sizeof(DevStatus)) + align256(sizeof(uint32_t) * (size_t)n));
    a.P = n;
    a.cap = (1LL << 30) - 1;
    a.fault_scan_part = silent_partition;
    a.spin_limit = 1ull << 14;
    if (cudaMemsetAsync(a.st, 0, sizeof(DevStatus), s) != cudaSuccess) return GS_ERR_CUDA;
    k_fill_ones<<<64, 256, 0, s>>>(a.touched, n);
    count_launches(1);
    int rc = run_scan_only(a, s);
    if (rc) return rc;
    DevStatus h;
    if (cudaMemcpyAsync(&h, a.st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    if (total) *total = (int64_t)h.num_keys;
    return h.code;
}

}  // extern "C"
