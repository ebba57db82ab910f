"""GPU parity of libgs against the CPU oracle, through the C ABI (via the ctypes binding).

Bars: tile lists, keys and order bit-exact; projection decision quantities (mean2D, conic, depth,
radius, touched-tile count) and last_idx bit-exact; rgb / depth / alpha / final_T within 2e-4 max
abs; every gradient tensor within 1e-3 relative L2.
"""
import numpy as np
import pytest

from helpers import TOL_GRAD, TOL_IMAGE, gpu_problem, oracle_params_from, rel_l2, upstream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def run_gpu(R, wl, views=None, params=None, key_capacity=None, grads=True, seed=7, alpha_w=0.0):
    pb, g = gpu_problem(wl, views, params, key_capacity)
    pb.project(g)
    ws = pb.workspace()
    touched = ws["tiles_touched"].clone().cpu().numpy().view(np.uint32)
    proj = ws["proj"].clone().cpu().numpy()
    pb.bin_sort()
    rc, req = pb.check_status()
    out = dict(pb=pb, g=g, touched=touched, proj=proj, rc=rc, req=req)
    if rc != 0:
        return out
    ws = pb.workspace()
    K = int(ws["num_keys"][0].item()) & 0xffffffff
    out["K"] = K
    out["keys"] = ws["sorted_keys"][:K].cpu().numpy().view(np.uint64)
    out["vals"] = ws["sorted_vals"][:K].cpu().numpy().view(np.uint32)
    out["ranges"] = ws["tile_ranges"].cpu().numpy().view(np.uint32)
    out["claim"] = (ws["claim_count"].cpu().numpy().view(np.uint32), ws["claim_list"].cpu().numpy().view(np.uint32))
    img = pb.render_fwd()
    out["img"] = {k: v.cpu().numpy() for k, v in img.items()}
    if grads:
        V = pb.V
        d_rgb, d_depth, d_alpha = upstream(wl, V, seed, alpha_w=alpha_w)
        dev = lambda a: torch.from_numpy(a).cuda()
        gr = pb.render_bwd(g, img, dev(d_rgb), dev(d_depth), dev(d_alpha))
        pose = pb.pose_grad()
        out["g2d"] = pb.workspace()["grad2d"].cpu().numpy()
        out["grads"] = {k: getattr(gr, k).cpu().numpy() for k in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")}
        out["pose"] = pose.cpu().numpy()
        out["up"] = (d_rgb, d_depth, d_alpha)
    torch.cuda.synchronize()
    rc2, _ = pb.check_status()
    out["rc_end"] = rc2
    out["stats"] = pb.stats()
    assert pb.check_guards() == (0, -1), "a workspace guard block was overwritten"
    return out


def run_oracle(wl, views=None, params=None, up=None):
    orc = Oracle.from_workload(wl, oracle_params_from(params), views=views)
    res = dict(orc=orc, proj=orc.projection(), bins=orc.bins(), fwd=orc.forward())
    if up is not None:
        res["bwd"] = orc.backward(*[u.astype(np.float64) for u in up])
    return res


def claim_class(n):
    """Claim class of a list of n entries: 31 - (2 floor(log2 n) + the bit below the leading one),
    so class 0 holds the longest lists; lengths 0 and 1 are class 31, lengths from 2^16 on class 0."""
    n = np.maximum(np.asarray(n, np.int64), 1)
    e = np.floor(np.log2(n)).astype(np.int64)
    half = np.where(e >= 1, (n >> np.maximum(e - 1, 0)) & 1, 0)
    return np.where(e > 15, 0, 31 - (2 * e + half))


def check_claim_classes(count, lists, ranges):
    """The compositing kernels claim the (view, tile) items class by class, longest lists first: every
    item is listed exactly once, under the class of its list length (scheduling only: the images and
    gradients do not depend on it; the order inside a class is arbitrary)."""
    G = ranges.shape[0]
    assert count.shape == (32,) and lists.shape == (32, G)
    assert int(count.astype(np.int64).sum()) == G
    items = [lists[k, :count[k]].astype(np.int64) for k in range(32)]
    np.testing.assert_array_equal(np.sort(np.concatenate(items)), np.arange(G))
    cls = claim_class(np.diff(ranges.astype(np.int64), axis=1)[:, 0])
    for k in range(32):
        assert (cls[items[k]] == k).all(), k


def compare_all(gpu, orc, check_grads=True):
    op = orc["proj"]
    np.testing.assert_array_equal(gpu["touched"], op["touched"])
    vis = op["touched"] > 0
    gp = gpu["proj"]
    np.testing.assert_array_equal(gp[vis, 0:2].view(np.uint32), op["mean2d"][vis].view(np.uint32))
    np.testing.assert_array_equal(gp[vis, 2:5].view(np.uint32), op["conic"][vis].view(np.uint32))
    np.testing.assert_array_equal(gp[vis, 6].view(np.uint32), op["depth"][vis].view(np.uint32))
    np.testing.assert_array_equal(gp[vis, 7], op["radius"][vis])
    ob = orc["bins"]
    assert gpu["K"] == len(ob["keys"])
    np.testing.assert_array_equal(gpu["keys"], ob["keys"])
    np.testing.assert_array_equal(gpu["vals"], ob["vals"])
    np.testing.assert_array_equal(gpu["ranges"].reshape(-1, 2), ob["ranges"])
    check_claim_classes(*gpu["claim"], ob["ranges"])
    of, gi = orc["fwd"], gpu["img"]
    np.testing.assert_array_equal(gi["last_idx"], of["last"])
    for k, ko in (("rgb", "rgb"), ("depth", "depth"), ("alpha", "alpha"), ("final_T", "final_T")):
        err = np.abs(gi[k].astype(np.float64) - of[ko]).max()
        assert err <= TOL_IMAGE, (k, err)
    assert gpu["stats"]["fwd_pairs"] == of["pairs"]
    if not check_grads:
        return
    bw = orc["bwd"]
    g2d = gpu["g2d"]
    for name, sl in (("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                     ("depth", slice(6, 7)), ("color", slice(7, 10))):
        e = rel_l2(g2d[vis, sl], bw["g2d"][vis, sl])
        assert e <= TOL_GRAD, (name, e)
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        e = rel_l2(gpu["grads"][k], bw[k])
        assert e <= TOL_GRAD, (k, e)
    for v in range(gpu["pose"].shape[0]):
        e = rel_l2(gpu["pose"][v], bw["pose"][v])
        assert e <= TOL_GRAD, ("pose", v, e, gpu["pose"][v], bw["pose"][v])


def test_library_variant_is_the_requested_one(R):
    """GS_LIBGS_VARIANT=checked loads the bounds-checked build (tests/test_gpu_checked_build.py runs
    this module that way), anything else the release build."""
    import os
    want = 1 if os.environ.get("GS_LIBGS_VARIANT", "") == "checked" else 0
    assert R.L.load().gs_checked_build() == want


def test_debug_expf_bitwise_vs_oracle_and_cuda(R):
    from oracle.oracle import expf as oexpf
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-86.9, 87.9, 200_001), rng.uniform(-8, 1, 200_000),
                        [-87.0, -100.0, 88.5, 0.0, -0.0]]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    ys, yc = torch.empty_like(xd), torch.empty_like(xd)
    import ctypes as C
    rc = R.L.load().gs_debug_expf(C.c_void_p(xd.data_ptr()), C.c_void_p(ys.data_ptr()), C.c_void_p(yc.data_ptr()),
                                  x.size, R._stream())
    assert rc == 0
    ys, yc = ys.cpu().numpy(), yc.cpu().numpy()
    np.testing.assert_array_equal(ys.view(np.uint32), oexpf(x).view(np.uint32))
    fin = np.isfinite(yc) & (x > -87) & (x <= 88)
    ulp = np.spacing(np.abs(yc[fin])).astype(np.float64)
    assert (np.abs(ys[fin].astype(np.float64) - yc[fin]) / ulp).max() <= 3.0


SORT_MODES = [1, 0]   # GS_SORT_ONESWEEP, GS_SORT_TILE_BUCKET: both must give the oracle's lists


@pytest.mark.parametrize("mode", SORT_MODES)
@pytest.mark.parametrize("wname,scale", [("cloud10k", 1.0), ("room500k", 0.1)])
def test_parity_single_view(R, wname, scale, mode):
    wl = S.workload(wname, scale=scale)
    p = R.default_params(sort_mode=mode)
    gpu = run_gpu(R, wl, params=p)
    assert gpu["rc"] == 0 and gpu["rc_end"] == 0
    orc = run_oracle(wl, params=p, up=gpu["up"])
    compare_all(gpu, orc)


@pytest.mark.parametrize("mode", SORT_MODES)
def test_parity_tiles_longer_than_one_shared_memory_sort(R, mode):
    """20k small Gaussians in front of a 48x40 image: the central tiles hold about 10k entries
    each, so the tile-bucket sort goes through its sorted-runs-and-merge path."""
    sc = S.random_cloud(20_000, seed=21)
    sc.means[:, 0] *= 0.05
    sc.means[:, 1] *= 0.05
    wl = S.Workload("pile", sc, np.array([0, sc.n], np.int64), [S.identity_camera(48, 40, 60, 60, 24, 20)],
                    np.zeros(1, np.int32), 48, 40)
    p = R.default_params(sort_mode=mode)
    gpu = run_gpu(R, wl, params=p)
    assert gpu["rc"] == 0 and gpu["rc_end"] == 0
    orc = run_oracle(wl, params=p, up=gpu["up"])
    lens = np.diff(orc["bins"]["ranges"], axis=1)
    assert lens.max() > 4 * 4096
    compare_all(gpu, orc)


@pytest.mark.parametrize("mode", SORT_MODES)
def test_parity_room500k_full_size(R, mode):
    """The benchmark workload (500k-Gaussian room, one 1200x680 view) with about the benchmark's key
    capacity (270k keys), compared in full, in both binning modes."""
    wl = S.workload("room500k")
    gpu = run_gpu(R, wl, params=R.default_params(sort_mode=mode), key_capacity=400_000)
    assert gpu["rc"] == 0 and gpu["rc_end"] == 0
    orc = run_oracle(wl, up=gpu["up"])
    compare_all(gpu, orc)


@pytest.mark.parametrize("mode", SORT_MODES)
def test_parity_batched_agents(R, mode):
    """8 uneven submaps x 4 views in one problem (the batched launch), Gaussian counts scaled to
    5% so the oracle stays fast, full 1200x680 views."""
    wl = S.workload("agents8x4", scale=0.05)
    p = R.default_params(sort_mode=mode)
    gpu = run_gpu(R, wl, params=p, alpha_w=0.2)
    assert gpu["rc"] == 0 and gpu["rc_end"] == 0
    orc = run_oracle(wl, params=p, up=gpu["up"])
    compare_all(gpu, orc)


def test_batched_equals_per_view(R):
    """Rendering the 32 views in one batched problem gives the same decisions and images as
    rendering them one call at a time."""
    wl = S.workload("agents8x4", scale=0.03)
    full = run_gpu(R, wl, grads=False)
    for v in (0, 5, 13, 31):
        one = run_gpu(R, wl, views=[v], grads=False)
        np.testing.assert_array_equal(one["img"]["last_idx"][0], full["img"]["last_idx"][v])
        for k in ("rgb", "depth", "alpha", "final_T"):
            np.testing.assert_array_equal(one["img"][k][0], full["img"][k][v])


@pytest.mark.parametrize("mode", SORT_MODES)
@pytest.mark.parametrize("tw,th,nb", [(16, 8, 0), (32, 16, 0), (16, 16, 64), (16, 8, 64), (32, 16, 128)])
def test_parity_other_tiles(R, tw, th, nb, mode):
    """Other tile shapes and staged batch sizes (batch 0 = one record per pixel, at most 256)."""
    wl = S.workload("cloud10k", scale=0.5)
    p = R.default_params(tile_w=tw, tile_h=th, sort_mode=mode, batch_records=nb)
    gpu = run_gpu(R, wl, params=p)
    orc = run_oracle(wl, params=p, up=gpu["up"])
    compare_all(gpu, orc)


def test_parity_background_and_alpha_gradient(R):
    wl = S.workload("cloud10k", scale=0.3)
    p = R.default_params(bg=(0.2, 0.5, 0.8))
    gpu = run_gpu(R, wl, params=p, alpha_w=1.0)
    orc = run_oracle(wl, params=p, up=gpu["up"])
    compare_all(gpu, orc)


@pytest.mark.parametrize("mode", SORT_MODES)
def test_capacity_overflow_reports_required_keys(R, mode):
    wl = S.workload("cloud10k", scale=0.2)
    p = R.default_params(sort_mode=mode)
    gpu = run_gpu(R, wl, params=p, key_capacity=1000, grads=False)
    orc = Oracle.from_workload(wl)
    assert gpu["rc"] == R.L.GS_ERR_CAPACITY
    assert gpu["req"] == orc.K
    # a capacity that fits clears the status and gives the exact result
    ok = run_gpu(R, wl, params=p, key_capacity=orc.K, grads=False)
    assert ok["rc"] == 0 and ok["K"] == orc.K


@pytest.mark.parametrize("mode", SORT_MODES)
def test_visible_capacity_overflow_reports_and_recovers(R, mode):
    """A slot capacity below the number of visible pairs records GS_ERR_CAPACITY and reports the
    slots needed (the visible pairs and the pre-test's candidates that the decision chain culled);
    forward_checked then grows it, every visible pair holds a slot and the result is the oracle's."""
    wl = S.workload("cloud10k", scale=0.3)
    p = R.default_params(sort_mode=mode)
    pb, g = gpu_problem(wl, params=p)
    pb.set_capacity(pb.cap, visible=100)
    pb.project(g)
    pb.bin_sort()
    rc, _ = pb.check_status()
    nv = pb.stats()["num_visible"]
    orc = run_oracle(wl, params=p)
    vis_oracle = int((orc["proj"]["touched"] > 0).sum())
    assert rc == R.L.GS_ERR_CAPACITY and nv >= vis_oracle > 100
    img = pb.forward_checked(g)
    assert pb.vcap >= nv
    slots = pb.workspace()["pair_slot"].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(slots != 0xFFFFFFFF, orc["proj"]["touched"] > 0)
    np.testing.assert_array_equal(img["last_idx"].cpu().numpy(), orc["fwd"]["last"])
    assert np.abs(img["rgb"].cpu().numpy() - orc["fwd"]["rgb"]).max() <= TOL_IMAGE


def test_bounded_wait_times_out_and_recovers(R):
    import ctypes as C
    L = R.L.load()
    n = 3 * 4096 + 17
    scratch = torch.zeros(int(L.gs_debug_scan_scratch_size(n)), dtype=torch.uint8, device="cuda")
    tot = C.c_int64()
    rc = L.gs_debug_scan_timeout(C.c_void_p(scratch.data_ptr()), n, 0, R._stream(), C.byref(tot))
    assert rc == R.L.GS_ERR_TIMEOUT
    rc = L.gs_debug_scan_timeout(C.c_void_p(scratch.data_ptr()), n, -1, R._stream(), C.byref(tot))
    assert rc == 0 and tot.value == n
    # the context is still usable
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0


@pytest.mark.parametrize("mode", SORT_MODES)
def test_edge_cases_empty_and_culled(R, mode):
    # every Gaussian behind the camera: no keys, empty image, zero gradients
    p = R.default_params(sort_mode=mode)
    sc = S.random_cloud(64, seed=3)
    sc.means[:, 2] = -sc.means[:, 2]
    wl = S.Workload("behind", sc, np.array([0, sc.n], np.int64), [S.identity_camera(40, 30, 30, 30)],
                    np.zeros(1, np.int32), 40, 30)
    gpu = run_gpu(R, wl, params=p)
    assert gpu["rc"] == 0 and gpu["K"] == 0
    assert np.all(gpu["img"]["final_T"] == 1.0) and np.all(gpu["img"]["last_idx"] == 0)
    assert np.all(gpu["grads"]["means"] == 0) and np.all(gpu["pose"] == 0)
    # ragged image (not a multiple of the tile), one pixel wide
    sc2 = S.random_cloud(300, seed=4)
    for (W, H) in ((1, 1), (17, 33), (250, 7)):
        wl2 = S.Workload("ragged", sc2, np.array([0, sc2.n], np.int64),
                         [S.identity_camera(W, H, 40, 40, W / 2, H / 2)], np.zeros(1, np.int32), W, H)
        gpu2 = run_gpu(R, wl2, params=p)
        orc2 = run_oracle(wl2, params=p, up=gpu2["up"])
        compare_all(gpu2, orc2)


def test_autograd_function_matches_direct_calls(R):
    wl = S.workload("cloud10k", scale=0.3)
    pb, g = gpu_problem(wl)
    leaves = [getattr(g, k).clone().requires_grad_(True) for k in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")]
    pose = torch.zeros(1, 6, device="cuda", requires_grad=True)
    rgb, depth, alpha = R.rasterize(*leaves, problem=pb, pose_delta=pose)
    d_rgb, d_depth, d_alpha = upstream(wl, 1, 3, alpha_w=0.5)
    dev = lambda a: torch.from_numpy(a).cuda()
    loss = (rgb * dev(d_rgb)).sum() + (depth * dev(d_depth)).sum() + (alpha * dev(d_alpha)).sum()
    loss.backward()
    orc = run_oracle(wl, up=(d_rgb, d_depth, d_alpha))
    np.testing.assert_allclose(rgb.detach().cpu().numpy(), orc["fwd"]["rgb"], atol=TOL_IMAGE)
    for leaf, k in zip(leaves, ("means", "log_scales", "quats", "opacities", "colors")):
        assert rel_l2(leaf.grad.cpu().numpy(), orc["bwd"][k]) <= TOL_GRAD, k
    assert rel_l2(pose.grad.cpu().numpy(), orc["bwd"]["pose"]) <= TOL_GRAD


def test_repeated_launches_need_no_clearing(R):
    """The compositing launches return their work counters to zero themselves (no clearing between
    calls): forwards repeated on one binning give the same images and last indices every time and
    add the same pair count to the statistic (which counts the launches since the binning); a
    second backward walks the same pairs and adds the same 2-D gradients again (they accumulate
    until the next binning zeroes them)."""
    wl = S.workload("cloud10k", scale=0.3)
    pb, g = gpu_problem(wl)
    pb.project(g)
    pb.bin_sort()
    imgs, fwd_pairs = [], []
    for _ in range(3):
        img = pb.render_fwd()
        torch.cuda.synchronize()
        imgs.append({k: v.cpu().numpy().copy() for k, v in img.items()})
        fwd_pairs.append(pb.stats()["fwd_pairs"])
    for i in (1, 2):
        for k in imgs[0]:
            np.testing.assert_array_equal(imgs[i][k], imgs[0][k])
    assert fwd_pairs[0] > 0 and fwd_pairs[1] == 2 * fwd_pairs[0] and fwd_pairs[2] == 3 * fwd_pairs[0]
    d_rgb, d_depth, d_alpha = upstream(wl, pb.V, 7)
    dev = lambda a: torch.from_numpy(a).cuda()
    g2d, bwd_pairs = [], []
    for _ in range(2):
        pb.render_bwd(g, img, dev(d_rgb), dev(d_depth), dev(d_alpha))
        torch.cuda.synchronize()
        g2d.append(pb.workspace()["grad2d"].cpu().numpy())
        bwd_pairs.append(pb.stats()["bwd_pairs"])
    assert bwd_pairs[0] > 0 and bwd_pairs[1] == 2 * bwd_pairs[0]
    np.testing.assert_allclose(g2d[1], 2.0 * g2d[0], rtol=1e-5, atol=1e-9)
    rc, _ = pb.check_status()
    assert rc == 0


def test_views_without_gaussians(R):
    """A problem with no (view, Gaussian) pair at all: no projection or scan launch, an empty
    binning, the background everywhere, zero pose gradient, and the same again on a second call."""
    sc = S.random_cloud(0, seed=5)
    wl = S.Workload("empty", sc, np.array([0, 0], np.int64), [S.identity_camera(40, 30, 30, 30)],
                    np.zeros(1, np.int32), 40, 30)
    for _ in range(2):
        gpu = run_gpu(R, wl, params=R.default_params(bg=(0.25, 0.5, 0.75)))
        assert gpu["rc"] == 0 and gpu["rc_end"] == 0 and gpu["K"] == 0
        assert gpu["stats"]["num_visible"] == 0 and gpu["stats"]["fwd_pairs"] == 0
        assert np.all(gpu["img"]["final_T"] == 1.0) and np.all(gpu["img"]["last_idx"] == 0)
        np.testing.assert_array_equal(gpu["img"]["rgb"][0, 2], np.full((30, 40), 0.75, np.float32))
        assert np.all(gpu["pose"] == 0)
