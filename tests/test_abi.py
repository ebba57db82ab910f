"""CPU-side checks of the C ABI: the library loads, exports every function include/gs.h declares,
and validates arguments on the host (no GPU call is made by any of these)."""
import ctypes as C

import numpy as np
import pytest

from paper_2605_10760_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = L.header_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_version_reports_sm103a(lib):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    assert lib.gs_version(C.byref(a), C.byref(b), C.byref(c)) == 0
    assert c.value == 1030


def _problem(V=1, W=1200, H=680, N=500_000, cap=1 << 21, **par):
    p = L.gs_params()
    lib = L.load()
    lib.gs_default_params(C.byref(p))
    for k, v in par.items():
        setattr(p, k, v)
    vb = np.zeros(V, np.int64)
    vc = np.full(V, N, np.int64)
    pb = L.gs_problem()
    pb.num_views, pb.width, pb.height, pb.num_gaussians = V, W, H, N
    pb.view_gauss_begin = vb.ctypes.data_as(C.POINTER(C.c_int64))
    pb.view_gauss_count = vc.ctypes.data_as(C.POINTER(C.c_int64))
    pb.key_capacity = cap
    pb.params = p
    pb._keep = (vb, vc)
    return pb


def test_default_params(lib):
    p = L.gs_params()
    lib.gs_default_params(C.byref(p))
    assert (p.tile_w, p.tile_h) == (16, 16)
    assert p.alpha_max == np.float32(0.99) and p.alpha_min == np.float32(1) / np.float32(255)
    assert p.t_min == np.float32(1e-4) and p.dilation == np.float32(0.3)
    assert p.sort_mode == L.GS_SORT_ONESWEEP and p.batch_records == 0


def test_workspace_size_and_validation(lib):
    n = C.c_size_t()
    pb = _problem()
    assert lib.gs_workspace_size(C.byref(pb), C.byref(n)) == 0
    # proj + grad2d (48 B each per visible-pair slot: all 500k pairs by default), keys + values
    # (2 x 12 B per key) and the records in list order (48 B per key) dominate
    assert 500_000 * 96 + (1 << 21) * 72 < n.value < 500_000 * 140 + (1 << 21) * 90
    n_full = C.c_size_t(n.value)
    bad = [_problem(V=0), _problem(W=0), _problem(cap=0), _problem(cap=1 << 30), _problem(tile_w=8),
           _problem(alpha_max=1.5), _problem(t_min=0.0), _problem(near_plane=0.0), _problem(sort_mode=2),
           _problem(batch_records=100), _problem(batch_records=256, tile_h=8)]
    neg = _problem()
    neg.visible_capacity = -1
    bad.append(neg)
    for b in bad:
        assert lib.gs_workspace_size(C.byref(b), C.byref(n)) == L.GS_ERR_INVALID_ARG
    # a slot capacity below the pair count shrinks the records, the 2-D gradients and the slot
    # lanes (48 + 48 + 2 B per slot; each region is rounded up to 256 B)
    small = _problem()
    small.visible_capacity = 100_000
    m = C.c_size_t()
    assert lib.gs_workspace_size(C.byref(small), C.byref(m)) == 0
    assert 0 <= n_full.value - m.value - 400_000 * 98 < 3 * 256
    pb = _problem(V=2)
    vc = np.array([10, 20], np.int64)
    vb = np.array([0, 500_000 - 5], np.int64)       # second view overruns the arrays
    pb.view_gauss_begin = vb.ctypes.data_as(C.POINTER(C.c_int64))
    pb.view_gauss_count = vc.ctypes.data_as(C.POINTER(C.c_int64))
    assert lib.gs_workspace_size(C.byref(pb), C.byref(n)) == L.GS_ERR_INVALID_ARG


def test_sort_pass_count_follows_tile_bits(lib):
    for V, passes in ((1, 6), (64, 7)):
        pb = _problem(V=V, N=1000)
        v = L.gs_ws_view()
        # a fake 256-aligned non-null address: gs_workspace_view only does pointer arithmetic
        assert lib.gs_workspace_view(C.byref(pb), C.c_void_p(1 << 20), C.byref(v)) == 0
        assert v.sort_passes == passes and v.num_tiles == V * 75 * 43


def test_calls_reject_bad_arguments_without_launching(lib):
    pb = _problem()
    assert lib.gs_project(C.byref(pb), None, C.c_void_p(1 << 20), None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_bin_sort(C.byref(pb), C.c_void_p(3), None) == L.GS_ERR_INVALID_ARG   # misaligned
    assert lib.gs_render_fwd(C.byref(pb), C.c_void_p(1 << 20), None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_pose_grad(C.byref(pb), C.c_void_p(1 << 20), None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_loss_l1(0, 10, 10, None, None, None, None, 1.0, 0.0, None, None, None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_adam_step(-1, None, None, None, 0, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_debug_scan_timeout(None, 10, 0, None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_error_string(L.GS_ERR_CAPACITY) == b"key capacity exceeded"


def test_follow_up_calls_reject_bad_arguments_without_launching(lib):
    p = lib.gs_default_pho_params()
    assert p.stride == 1 and p.near_plane == np.float32(0.2) and p.huber_delta == np.float32(9.0 / 255.0)
    one = C.c_void_p(1 << 20)
    args = [one, 1, 16, 16, one, one, one, 1, one, C.byref(p), one, one, one, one, one, 1 << 30, None]
    assert lib.gs_pho_residual(0, *args) == L.GS_OK                    # no edges: nothing to do
    assert lib.gs_pho_residual(-1, *args) == L.GS_ERR_INVALID_ARG
    assert lib.gs_pho_residual(70000, *args) == L.GS_ERR_INVALID_ARG
    bad = list(args)
    bad[0] = None                                                      # edges
    assert lib.gs_pho_residual(1, *bad) == L.GS_ERR_INVALID_ARG
    bad = list(args)
    bad[15] = lib.gs_pho_scratch_size(4) - 1                           # scratch too small
    assert lib.gs_pho_residual(4, *bad) == L.GS_ERR_INVALID_ARG
    p.stride = 0
    assert lib.gs_pho_residual(1, *args) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxset_bytes(100) == 0 and lib.gs_voxset_bytes(128) == 256 + 8 * 128   # power of two
    assert lib.gs_voxset_clear(one, 100, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxset_add_boxes(one, 128, 1, None, None, 3.0, 0.05, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxset_keep(1, one, one, 128, None, 0, 0.0, one, None) == L.GS_ERR_INVALID_ARG   # voxel 0


def test_normal_loss_rejects_bad_arguments_without_launching(lib):
    one = C.c_void_p(1 << 20)
    args = [one, one, one, C.c_float(0.01), one, one, None]   # depth, prior, cams, weight, d_depth, loss, stream
    assert lib.gs_loss_normal(0, 16, 8, *args) == L.GS_ERR_INVALID_ARG            # no views
    assert lib.gs_loss_normal(1, 0, 8, *args) == L.GS_ERR_INVALID_ARG             # empty image
    for k in (0, 1, 2, 4, 5):                                                      # a missing pointer
        bad = list(args)
        bad[k] = None
        assert lib.gs_loss_normal(1, 16, 8, *bad) == L.GS_ERR_INVALID_ARG
    bad = list(args)
    bad[3] = C.c_float(float("nan"))                                               # weight
    assert lib.gs_loss_normal(1, 16, 8, *bad) == L.GS_ERR_INVALID_ARG


def test_both_library_builds_export_the_abi_and_name_their_variant():
    """libgs.so (release) and libgs_checked.so (bounds-checked) export the same calls; each says
    which build it is."""
    import os
    from paper_2605_10760_gb300 import build as B
    B.build()
    names = L.header_symbols()
    for fname, want in (("libgs.so", 0), ("libgs_checked.so", 1)):
        lib = C.CDLL(os.path.join(B.OUT, fname))
        for n in names:
            assert hasattr(lib, n), (fname, n)
        lib.gs_checked_build.restype = C.c_int32
        assert lib.gs_checked_build() == want
