"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* the FP32 exponential: against FP64 exp (ulp bound) and bit for bit against an independent
  restatement of its definition (numpy float32 arithmetic + the C library's fmaf);
* closed forms: an isotropic Gaussian at the principal point (alpha profile, colour, depth,
  transmittance, opacity gradient); an opaque, capped front pair that terminates the pixel;
* a textbook special case: with no dilation the alpha field of one axis-aligned Gaussian is o times
  2 pi sigma_x sigma_y times the bivariate normal density (scipy.stats);
* invariants: alpha-weights plus final transmittance sum to one, bounded colour;
* brute force: per-pixel compositing over all Gaussians (no binning) on tiny inputs, and the tile
  lists checked against a direct sort;
* central finite differences of the FP64 value chain for every gradient (means, log-scales,
  quaternions, opacities, colours, SE(3) pose), decisions held fixed.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from oracle.oracle import Oracle, Params, expf, exp_se3_left

_libm = ctypes.CDLL(ctypes.util.find_library("m"))
_libm.fmaf.restype = ctypes.c_float
_libm.fmaf.argtypes = [ctypes.c_float] * 3
_libm.rintf.restype = ctypes.c_float
_libm.rintf.argtypes = [ctypes.c_float]
F = np.float32


def fmaf(a, b, c):
    return F(_libm.fmaf(float(a), float(b), float(c)))


def py_expf(x):
    """Independent restatement of the decision-chain exponential (Cody-Waite + degree-7 Taylor)."""
    x = F(x)
    if not (x > F(-87.0)):
        return F(0.0)
    if x > F(88.0):
        return F(np.inf)
    ln2 = 0.6931471805599453
    hi = F(round(ln2 * 65536.0) / 65536.0)
    lo = F(ln2 - float(hi))
    kf = F(_libm.rintf(float(x * F(1.4426950408889634))))
    r = fmaf(-kf, hi, x)
    r = fmaf(-kf, lo, r)
    p = F(1.0) / F(5040.0)
    for c in (F(1.0) / F(720.0), F(1.0) / F(120.0), F(1.0) / F(24.0), F(1.0) / F(6.0), F(0.5), F(1.0), F(1.0)):
        p = fmaf(p, r, c)
    scale = np.array([(int(kf) + 127) << 23], dtype=np.uint32).view(np.float32)[0]
    return F(p * scale)


# ------------------------------------------------------------------------------------------
# exp
# ------------------------------------------------------------------------------------------

def test_expf_ulp_bound_vs_fp64():
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-86.9, 87.9, 400_001), rng.uniform(-10, 2, 200_000),
                        np.linspace(-6.0, 0.0, 100_001)]).astype(np.float32)
    y = expf(x).astype(np.float64)
    e = np.exp(x.astype(np.float64))
    ulp = np.spacing(e.astype(np.float32)).astype(np.float64)
    err = np.abs(y - e) / ulp
    assert err.max() <= 2.0, err.max()


def test_expf_bitwise_matches_independent_restatement():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-87, 88, 3000), rng.uniform(-6, 0, 3000), [-87.0, -86.99, 0.0, -0.0, 88.0,
                        88.5, -100.0, 1e-30]]).astype(np.float32)
    got = expf(x)
    ref = np.array([py_expf(v) for v in x], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------

def cam_row(R=np.eye(3), t=(0, 0, 0), fx=100.0, fy=100.0, cx=32.0, cy=32.0):
    return np.concatenate([np.asarray(R, float).reshape(9), np.asarray(t, float), [fx, fy, cx, cy]])


def single_view(means, ls, q, o, c, cam, W, H, params=None, **kw):
    n = len(means)
    return Oracle(np.asarray(means), np.asarray(ls), np.asarray(q), np.asarray(o), np.asarray(c),
                  cam[None], [0], [n], W, H, params, **kw)


# ------------------------------------------------------------------------------------------
# closed forms
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("o_val,s_val", [(0.7, 0.02), (1.0, 0.1)])
def test_isotropic_gaussian_at_principal_point(o_val, s_val):
    W = H = 64
    f, z = 100.0, 2.0
    col = np.array([[0.2, 0.5, 0.9]]).astype(np.float32).astype(np.float64)
    o_val = float(np.float32(o_val))
    orc = single_view([[0, 0, z]], [[np.log(s_val)] * 3], [[1, 0, 0, 0]], [o_val], col, cam_row(fx=f, fy=f),
                      W, H)
    out = orc.forward()
    s = np.exp(float(np.float32(np.log(s_val))))       # the FP64 chain widens the FP32 log-scale
    sig2 = (f * s / z) ** 2 + float(np.float32(0.3))
    xs = np.arange(W) + 0.5 - 32.0
    r2 = xs[None, :] ** 2 + xs[:, None] ** 2
    a_cf = o_val * np.exp(-r2 / (2 * sig2))
    capped = a_cf > 0.99
    a_cf = np.where(capped, float(np.float32(0.99)), a_cf)
    radius = np.ceil(3 * np.sqrt(sig2))
    tiles_lo = np.floor((32 - radius) / 16) * 16
    tiles_hi = (np.floor((32 + radius) / 16) + 1) * 16
    inrect = ((np.arange(W) >= tiles_lo) & (np.arange(W) < tiles_hi))
    inrect = inrect[None, :] & inrect[:, None]
    amin = 1.0 / 255.0
    on = (a_cf >= amin * (1 + 1e-5)) & inrect
    off = (a_cf < amin * (1 - 1e-5)) | ~inrect
    assert on.sum() > 10 and (on | off).sum() >= W * H - 8
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][0, ch][on], col[0, ch] * a_cf[on], rtol=1e-9, atol=1e-12)
        assert np.all(out["rgb"][0, ch][off] == 0)
    np.testing.assert_allclose(out["depth"][0][on], z * a_cf[on], rtol=1e-9)
    np.testing.assert_allclose(out["final_T"][0][on], 1 - a_cf[on], rtol=1e-9)
    assert np.all(out["last"][0][on] == 1) and np.all(out["last"][0][off] == 0)
    # dL/do for L = sum of red channel: sum over blended, uncapped pixels of c_r exp(-sigma)
    g = np.zeros((1, 3, H, W))
    g[0, 0] = 1.0
    bw = orc.backward(g)
    expect = col[0, 0] * (np.exp(-r2 / (2 * sig2)) * (on & ~capped)).sum()
    np.testing.assert_allclose(bw["opacities"][0], expect, rtol=1e-9)
    if o_val == 1.0:
        assert capped.sum() == 4
        np.testing.assert_array_equal(out["rgb"][0, 0][capped], col[0, 0] * float(np.float32(0.99)))


def test_occlusion_capped_pair_terminates():
    """Two coincident opaque copies in front: the first is capped at 0.99, the second drives the
    transmittance to (1-0.99f)^2 = 9.999981e-05 < 1e-4 in FP32, so the pixel stops without blending
    it and nothing behind contributes."""
    W = H = 32
    means = [[0, 0, 1.0], [0, 0, 1.0], [0, 0, 3.0]]
    ls = [[np.log(0.2)] * 3] * 3
    q = [[1, 0, 0, 0]] * 3
    o = [1.0, 1.0, 1.0]
    col = [[0.9, 0.1, 0.1], [0.9, 0.1, 0.1], [0.0, 1.0, 0.0]]
    orc = single_view(means, ls, q, o, col, cam_row(fx=50, fy=50, cx=16, cy=16), W, H)
    out = orc.forward()
    a = float(np.float32(0.99))
    assert np.float32(np.float32(1) - np.float32(0.99)) ** 2 < np.float32(1e-4)
    cen = (slice(15, 17), slice(15, 17))
    np.testing.assert_array_equal(out["rgb"][0, 0][cen], float(np.float32(0.9)) * a)
    np.testing.assert_array_equal(out["rgb"][0, 1][cen], float(np.float32(0.1)) * a)
    np.testing.assert_array_equal(out["final_T"][0][cen], 1.0 - a)
    assert np.all(out["last"][0][cen] == 1)


def test_textbook_bivariate_normal_without_dilation():
    from scipy.stats import multivariate_normal
    W, H, f, z = 48, 40, 80.0, 2.5
    sx, sy = 0.05, 0.11
    p = Params(dilation=0.0)
    orc = single_view([[0, 0, z]], [[np.log(sx), np.log(sy), np.log(0.01)]], [[1, 0, 0, 0]], [0.8],
                      [[1, 1, 1]], cam_row(fx=f, fy=f, cx=24, cy=20), W, H, params=p)
    out = orc.forward()
    sxp = f * np.exp(float(np.float32(np.log(sx)))) / z
    syp = f * np.exp(float(np.float32(np.log(sy)))) / z
    X, Y = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    pdf = multivariate_normal(mean=[24, 20], cov=np.diag([sxp ** 2, syp ** 2])).pdf(np.stack([X, Y], -1))
    a = float(np.float32(0.8)) * 2 * np.pi * sxp * syp * pdf
    on = out["last"][0] > 0
    assert on.sum() > 50
    np.testing.assert_allclose(out["alpha"][0][on], a[on], rtol=1e-9)


# ------------------------------------------------------------------------------------------
# invariants
# ------------------------------------------------------------------------------------------

def test_invariants_partition_of_unity_and_bounds():
    from paper_2605_10760_gb300 import scenes as S
    wl = S.workload("cloud10k", scale=0.3)
    ones = np.ones_like(wl.scene.colors, dtype=np.float64)
    orc = Oracle.from_workload(wl, values={"colors": ones})
    out = orc.forward()
    np.testing.assert_allclose(out["rgb"][0, 0] + out["final_T"][0], 1.0, atol=1e-12)
    assert np.all(out["alpha"] >= 0) and np.all(out["alpha"] <= 1)
    orc2 = Oracle.from_workload(wl)
    o2 = orc2.forward()
    assert np.all(o2["rgb"] <= wl.scene.colors.max() + 1e-12)
    assert np.all(o2["final_T"] >= 1e-4 * 0.99)   # never blended past the stop threshold
    np.testing.assert_allclose(o2["alpha"], out["alpha"], rtol=0, atol=0)


# ------------------------------------------------------------------------------------------
# brute force
# ------------------------------------------------------------------------------------------

def _tiny_problem(seed, n=14, V=2, W=32, H=32):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), rng.uniform(1.5, 3.0, n)], 1)
    means[3] = means[2]                                # identical depth bits: tie broken by index
    ls = rng.normal(-2.3, 0.4, (n, 3))
    q = rng.normal(0, 1, (n, 4))
    o = 1 / (1 + np.exp(-rng.normal(1.0, 1.5, n)))
    c = rng.uniform(0, 1, (n, 3))
    cams = []
    for v in range(V):
        ang = 0.15 * v
        R = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
        cams.append(cam_row(R=R, t=(0.05 * v, -0.03 * v, 0.1 * v), fx=30, fy=32, cx=W / 2, cy=H / 2))
    return means, ls, q, o, c, np.stack(cams), W, H


def test_brute_force_compositing_and_binning():
    means, ls, q, o, c, cams, W, H = _tiny_problem(3)
    n, V = len(means), len(cams)
    orc = Oracle(means, ls, q, o, c, cams, [0] * V, [n] * V, W, H)
    P = orc.params
    pr, bins, out = orc.projection(), orc.bins(), orc.forward()
    zbits = pr["depth"].view(np.uint32)
    Tx, Ty = orc.Tx, orc.Ty
    assert orc.K == int(pr["touched"].sum())
    for v in range(V):
        for ty in range(Ty):
            for tx in range(Tx):
                g = (v * Ty + ty) * Tx + tx
                cand = [v * n + i for i in range(n) if pr["touched"][v * n + i] > 0
                        and pr["rect"][v * n + i, 0] <= tx < pr["rect"][v * n + i, 1]
                        and pr["rect"][v * n + i, 2] <= ty < pr["rect"][v * n + i, 3]]
                cand.sort(key=lambda f: (int(zbits[f]), f))
                s, e = bins["ranges"][g]
                assert list(bins["vals"][s:e]) == cand
                for y in range(ty * 16, min(H, ty * 16 + 16)):
                    for x in range(tx * 16, min(W, tx * 16 + 16)):
                        px, py = F(x) + F(0.5), F(y) + F(0.5)
                        T32, T, C, D, last = F(1), 1.0, np.zeros(3), 0.0, 0
                        for pos, f in enumerate(cand):
                            i = f - v * n
                            dx, dy = px - pr["mean2d"][f, 0], py - pr["mean2d"][f, 1]
                            A, B, Cc = pr["conic"][f]
                            qq = fmaf(A * dx, dx, (Cc * dy) * dy)
                            sg = fmaf(B * dx, dy, F(0.5) * qq)
                            if sg < 0:
                                continue
                            araw = F(o.astype(np.float32)[i]) * py_expf(-sg)
                            cap = araw > F(P.alpha_max)
                            a32 = F(P.alpha_max) if cap else araw
                            if a32 < F(P.alpha_min):
                                continue
                            Tn = T32 * (F(1) - a32)
                            if Tn < F(P.t_min):
                                break
                            ddx = (x + 0.5) - pr["mean2d_d"][f, 0]
                            ddy = (y + 0.5) - pr["mean2d_d"][f, 1]
                            Ad, Bd, Cd = pr["conic_d"][f]
                            sgd = 0.5 * (Ad * ddx * ddx + Cd * ddy * ddy) + Bd * ddx * ddy
                            ad = float(F(P.alpha_max)) if cap else float(F(o[i])) * np.exp(-sgd)
                            C += c.astype(np.float32)[i].astype(np.float64) * ad * T
                            D += pr["depth_d"][f] * ad * T
                            T *= 1 - ad
                            T32 = Tn
                            last = pos + 1
                        np.testing.assert_allclose(out["rgb"][v, :, y, x], C, rtol=1e-13, atol=1e-15)
                        np.testing.assert_allclose(out["depth"][v, y, x], D, rtol=1e-13, atol=1e-15)
                        np.testing.assert_allclose(out["final_T"][v, y, x], T, rtol=1e-13)
                        assert out["last"][v, y, x] == last


# ------------------------------------------------------------------------------------------
# finite differences
# ------------------------------------------------------------------------------------------

def _loss(orc, w):
    out = orc.forward()
    return (w[0] * out["rgb"]).sum() + (w[1] * out["depth"]).sum() + (w[2] * out["alpha"]).sum()


@pytest.mark.parametrize("seed", [5, 6])
def test_finite_differences_all_gradients(seed):
    means, ls, q, o, c, cams, W, H = _tiny_problem(seed, n=10, V=2, W=40, H=36)
    n, V = len(means), len(cams)
    params = Params(bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(seed + 100)
    w = (rng.normal(0, 1, (V, 3, H, W)), rng.normal(0, 0.3, (V, H, W)), rng.normal(0, 1, (V, H, W)))
    base = dict(means=means.astype(np.float32).astype(float), log_scales=ls.astype(np.float32).astype(float),
                quats=q.astype(np.float32).astype(float), opacities=o.astype(np.float32).astype(float),
                colors=c.astype(np.float32).astype(float), cams=cams.astype(np.float32).astype(float))

    def make(vals):
        return Oracle(means, ls, q, o, c, cams, [0] * V, [n] * V, W, H, params, values=vals)

    orc = make(base)
    g = orc.backward(*w)
    checked = 0
    for key in ("means", "log_scales", "quats", "opacities", "colors"):
        arr = base[key]
        an = g[key].reshape(arr.shape)
        scale = np.abs(an).max() + 1e-30
        for idx in np.ndindex(arr.shape):
            h = 1e-6 * max(1.0, abs(arr[idx]))
            vp, vm = dict(base), dict(base)
            vp[key] = arr.copy(); vp[key][idx] += h
            vm[key] = arr.copy(); vm[key][idx] -= h
            fd = (_loss(make(vp), w) - _loss(make(vm), w)) / (2 * h)
            assert abs(fd - an[idx]) <= 1e-5 * abs(an[idx]) + 1e-6 * scale, (key, idx, fd, an[idx])
            checked += 1
    for v in range(V):
        scale = np.abs(g["pose"]).max()
        for k in range(6):
            h = 1e-6
            xi = np.zeros(6); xi[k] = h
            cp, cm = base["cams"].copy(), base["cams"].copy()
            cp[v] = exp_se3_left(base["cams"][v], xi)
            cm[v] = exp_se3_left(base["cams"][v], -xi)
            fd = (_loss(make({**base, "cams": cp}), w) - _loss(make({**base, "cams": cm}), w)) / (2 * h)
            assert abs(fd - g["pose"][v, k]) <= 1e-5 * abs(g["pose"][v, k]) + 1e-6 * scale, (v, k, fd, g["pose"][v, k])
            checked += 1
    assert checked == n * 14 + 6 * V
    assert np.abs(g["pose"]).max() > 0 and np.abs(g["quats"]).max() > 0


def test_shared_accumulator_mode_gives_same_gradients(monkeypatch):
    """The backward's shared atomic accumulator (used for large problems) only reorders FP64 sums."""
    means, ls, q, o, c, cams, W, H = _tiny_problem(8, n=12, V=2, W=40, H=36)
    n, V = len(means), len(cams)
    rng = np.random.default_rng(9)
    w = (rng.normal(0, 1, (V, 3, H, W)), rng.normal(0, 0.3, (V, H, W)), rng.normal(0, 1, (V, H, W)))
    a = Oracle(means, ls, q, o, c, cams, [0] * V, [n] * V, W, H).backward(*w)
    monkeypatch.setenv("GS_ORACLE_SHARED_ACC", "1")
    b = Oracle(means, ls, q, o, c, cams, [0] * V, [n] * V, W, H).backward(*w)
    for k in ("g2d", "means", "log_scales", "quats", "opacities", "colors", "pose"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-15)


def test_exp_se3_left_matches_matrix_exponential():
    """The SE(3) left update T <- Exp(xi) T equals scipy's matrix exponential of the twist."""
    from scipy.linalg import expm
    rng = np.random.default_rng(11)
    for _ in range(5):
        Rm = exp_se3_left(np.concatenate([np.eye(3).ravel(), [0, 0, 0], [1, 1, 1, 1]]),
                          np.concatenate([[0, 0, 0], rng.normal(0, 1, 3)]))[:9].reshape(3, 3)
        cam = np.concatenate([Rm.ravel(), rng.normal(0, 1, 3), [500, 500, 320, 240]])
        xi = rng.normal(0, 0.7, 6)
        rho, phi = xi[:3], xi[3:]
        Xi = np.zeros((4, 4))
        Xi[:3, :3] = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
        Xi[:3, 3] = rho
        T = np.eye(4)
        T[:3, :3] = cam[:9].reshape(3, 3)
        T[:3, 3] = cam[9:12]
        Tn = expm(Xi) @ T
        out = exp_se3_left(cam, xi)
        np.testing.assert_allclose(out[:9].reshape(3, 3), Tn[:3, :3], atol=1e-12)
        np.testing.assert_allclose(out[9:12], Tn[:3, 3], atol=1e-12)
        np.testing.assert_array_equal(out[12:], cam[12:])


# ------------------------------------------------------------------------------------------
# rotation conventions: the Gaussian's quaternion and the camera's world-to-camera rotation
# ------------------------------------------------------------------------------------------

def _quat_wxyz_to_scipy(q):
    from scipy.spatial.transform import Rotation
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])          # scipy stores (x, y, z, w)


@pytest.mark.parametrize("qcase", ["optical_axis_+35deg", "optical_axis_-50deg", "general"])
def test_textbook_rotated_gaussian_without_dilation(qcase):
    """Eq. 19's covariance form Sigma = R(q) S^2 R(q)^T for a rotated, anisotropic Gaussian.

    A Gaussian on the optical axis of an identity camera projects with J = (f/z) [I | 0], so with
    no dilation its alpha field is o * 2 pi |Sigma_2|^1/2 * N(x; c, Sigma_2) with Sigma_2 the upper
    2x2 block of (f/z)^2 R S^2 R^T.  R comes from scipy's quaternion map (Hamilton convention, the
    active rotation), not from the oracle.  The rotations about the optical axis put the long
    axis at +35 and -50 degrees from the image x axis towards +y, so the sign of the off-diagonal
    term (and of the conic's B) is fixed by the test; the general case also mixes in the z scale.
    """
    from scipy.stats import multivariate_normal
    W, H, f, z, cx, cy = 64, 56, 120.0, 2.5, 32.0, 28.0
    s_log = np.log([0.09, 0.025, 0.05])
    if qcase == "general":
        q = np.array([0.8, 0.3, -0.4, 0.5])
    else:
        th = np.deg2rad(35.0 if qcase.endswith("+35deg") else -50.0)
        q = np.array([np.cos(th / 2), 0.0, 0.0, np.sin(th / 2)])
    q32 = q.astype(np.float32)
    o = 0.8
    orc = single_view([[0, 0, z]], [s_log], [q32], [o], [[1, 1, 1]], cam_row(fx=f, fy=f, cx=cx, cy=cy), W, H,
                      params=Params(dilation=0.0))
    out = orc.forward()
    Rm = _quat_wxyz_to_scipy(q32.astype(np.float64)).as_matrix()
    s = np.exp(s_log.astype(np.float32).astype(np.float64))
    Sigma = Rm @ np.diag(s ** 2) @ Rm.T
    Sigma2 = (f / z) ** 2 * Sigma[:2, :2]
    corr = Sigma2[0, 1] / np.sqrt(Sigma2[0, 0] * Sigma2[1, 1])
    if qcase.endswith("+35deg"):
        assert corr > 0.3            # long axis towards +x +y: positive correlation
    elif qcase.endswith("-50deg"):
        assert corr < -0.3
    X, Y = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    pdf = multivariate_normal(mean=[cx, cy], cov=Sigma2).pdf(np.stack([X, Y], -1))
    a = float(np.float32(o)) * 2 * np.pi * np.sqrt(np.linalg.det(Sigma2)) * pdf
    on = out["last"][0] > 0
    assert on.sum() > 100
    np.testing.assert_allclose(out["alpha"][0][on], a[on], rtol=1e-9)
    # blended exactly where the textbook alpha reaches 1/255, within the 3-sigma bounding square
    r = 3.0 * np.sqrt(np.linalg.eigvalsh(Sigma2).max())
    inside = (np.abs(X - cx) <= r) & (np.abs(Y - cy) <= r)
    amin = 1.0 / 255.0
    assert np.all(on[inside & (a > amin * (1 + 1e-6))])
    assert not np.any(on & (a < amin * (1 - 1e-6)))
    conic = orc.projection()["conic_d"][0]
    np.testing.assert_allclose(conic, [np.linalg.inv(Sigma2)[0, 0], np.linalg.inv(Sigma2)[0, 1],
                                       np.linalg.inv(Sigma2)[1, 1]], rtol=1e-10)


def _scene_in_camera(rng, n, W, H, f):
    """n Gaussians whose camera-frame positions fall inside a W x H pinhole view at depths 1.5..3."""
    z = rng.uniform(1.5, 3.0, n)
    x = rng.uniform(-0.4, 0.4, n) * W / f * z
    y = rng.uniform(-0.4, 0.4, n) * H / f * z
    pc = np.stack([x, y, z], 1)
    ls = rng.normal(-2.6, 0.35, (n, 3)).astype(np.float32).astype(np.float64)
    q = rng.normal(0, 1, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = (1 / (1 + np.exp(-rng.normal(0.5, 1.0, n)))).astype(np.float32).astype(np.float64)
    c = rng.uniform(0, 1, (n, 3)).astype(np.float32).astype(np.float64)
    return pc, ls, q, o, c


def _orc_f32_f64(means, ls, q, o, c, cam, W, H):
    """Oracle whose FP32 inputs are the roundings of the given FP64 values and whose FP64 value
    chain runs on the FP64 values themselves (an exactly orthonormal R in particular)."""
    vals = dict(means=means, log_scales=ls, quats=q, opacities=o, colors=c, cams=cam[None])
    return Oracle(means, ls, q, o, c, cam[None], [0], [len(means)], W, H, values=vals)


def test_camera_rotation_equals_rotating_the_scene():
    """World-to-camera poses (Sec. III-B) and Eq. 19's rotation composition q' = q_R (x) q.

    Rendering Gaussians (mu, q) from a camera (R, t) must equal rendering (R mu + t, q_R (x) q) from
    the identity camera with the same intrinsics: same keys, same last index everywhere, images
    within 1e-12; the opacity, colour and log-scale gradients agree and the mean gradient maps by
    R^T.  q_R (x) q is scipy's rotation composition, independent of the oracle's quaternion map."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(21)
    W, H, f = 64, 48, 60.0
    n = 18
    pc, ls, q, o, c = _scene_in_camera(rng, n, W, H, f)
    Rot = Rotation.from_rotvec([0.45, -0.7, 0.3])
    R = Rot.as_matrix()
    t = np.array([0.3, -0.2, 0.5])
    mu_w = (R.T @ (pc - t).T).T                    # world points that the camera sees at pc
    mu_w = mu_w.astype(np.float32).astype(np.float64)
    q_w = (Rot.inv() * _quat_wxyz_to_scipy_batch(q)).as_quat()[:, [3, 0, 1, 2]]
    cam_rot = cam_row(R=R, t=t, fx=f, fy=f, cx=W / 2, cy=H / 2)
    a = _orc_f32_f64(mu_w, ls, q_w, o, c, cam_rot, W, H)
    # the same Gaussians expressed in the camera frame, seen by the identity camera
    mu_c = (R @ mu_w.T).T + t
    q_c = (Rot * _quat_wxyz_to_scipy_batch(q_w)).as_quat()[:, [3, 0, 1, 2]]
    b = _orc_f32_f64(mu_c, ls, q_c, o, c, cam_row(fx=f, fy=f, cx=W / 2, cy=H / 2), W, H)
    oa, ob = a.forward(), b.forward()
    assert a.K == b.K and a.K > 20
    np.testing.assert_array_equal(oa["last"], ob["last"])
    assert (oa["last"] > 0).sum() > 0.3 * W * H
    for k in ("rgb", "depth", "alpha", "final_T"):
        np.testing.assert_allclose(oa[k], ob[k], rtol=0, atol=1e-12, err_msg=k)
    g = (rng.normal(0, 1, (1, 3, H, W)), rng.normal(0, 0.3, (1, H, W)), rng.normal(0, 1, (1, H, W)))
    ga, gb = a.backward(*g), b.backward(*g)
    for k in ("opacities", "colors", "log_scales"):
        np.testing.assert_allclose(ga[k], gb[k], rtol=1e-9, atol=1e-12 * np.abs(gb[k]).max(), err_msg=k)
    np.testing.assert_allclose(ga["means"], gb["means"] @ R, rtol=1e-9, atol=1e-12 * np.abs(gb["means"]).max())


def _quat_wxyz_to_scipy_batch(q):
    from scipy.spatial.transform import Rotation
    q = np.asarray(q, np.float64)
    return Rotation.from_quat(q[:, [1, 2, 3, 0]])


def test_camera_roll_by_90_degrees_rotates_the_image():
    """A camera rolled by +90 degrees about its optical axis (R' = Rz R, t' = Rz t, Rz taking x to y)
    sees camera coordinates (x', y') = (-y, x); for a square image with the principal point at its
    centre, pixel (row i, column j) of the rolled view shows pixel (row W-1-j, column i) of the
    original.  RGB, depth, alpha and final transmittance must match within 1e-12 (last indices are
    not compared: they are positions in the per-tile lists)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(33)
    W = H = 64
    f = 55.0
    n = 20
    pc, ls, q, o, c = _scene_in_camera(rng, n, W, H, f)
    Rot = Rotation.from_rotvec([-0.2, 0.5, 0.35])
    R = Rot.as_matrix()
    t = np.array([-0.1, 0.25, 0.4])
    mu_w = (R.T @ (pc - t).T).T.astype(np.float32).astype(np.float64)
    q_w = (Rot.inv() * _quat_wxyz_to_scipy_batch(q)).as_quat()[:, [3, 0, 1, 2]]
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    base = _orc_f32_f64(mu_w, ls, q_w, o, c, cam_row(R=R, t=t, fx=f, fy=f, cx=W / 2, cy=H / 2), W, H)
    roll = _orc_f32_f64(mu_w, ls, q_w, o, c, cam_row(R=Rz @ R, t=Rz @ t, fx=f, fy=f, cx=W / 2, cy=H / 2), W, H)
    ob, orl = base.forward(), roll.forward()
    assert (ob["last"] > 0).sum() > 0.3 * W * H
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for k in ("depth", "alpha", "final_T"):
        np.testing.assert_allclose(orl[k][0], ob[k][0][W - 1 - jj, ii], rtol=0, atol=1e-12, err_msg=k)
    for ch in range(3):
        np.testing.assert_allclose(orl["rgb"][0, ch], ob["rgb"][0, ch][W - 1 - jj, ii], rtol=0, atol=1e-12)
    # the image really changed: a roll is not a symmetry of this scene
    assert np.abs(orl["rgb"][0] - ob["rgb"][0]).max() > 0.05
