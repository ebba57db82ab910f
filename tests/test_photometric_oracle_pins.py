"""Pins of the Eq. 12 photometric-residual oracle: a closed form on linear images, finite differences
of the residuals w.r.t. both Sim(3) twists, gauge invariance, a Gauss-Newton step, empty sets."""
import numpy as np
from scipy.linalg import expm

from oracle import photometric as PH


def _cam(W, H, f, R=np.eye(3), t=np.zeros(3)):
    return np.concatenate([np.asarray(R).ravel(), t, [f, f, W / 2, H / 2]]).astype(np.float32)


def _quat_of(R):
    """(w, x, y, z) of a rotation matrix (trace form; the test rotations are far from pi)."""
    w = np.sqrt(max(1e-12, 1 + np.trace(R))) / 2
    return np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])


def _retract(sim, xi):
    """Exp(xi) o C for a first-order-exact retraction: x -> e^sig R_phi (s R x + t) + rho."""
    q, t, s = sim
    Rp = expm(PH.skew(xi[3:6]))
    R = Rp @ PH.quat_matrix(q)
    es = np.exp(xi[6])
    return (_quat_of(R), es * Rp @ np.asarray(t, np.float64) + xi[0:3], es * s)


def _ramp(W, H, a, b, k):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return np.stack([a[c] * x + b[c] * y + k[c] for c in range(3)]).astype(np.float32)


IDENT = (np.array([1.0, 0, 0, 0]), np.zeros(3), 1.0)


def test_closed_form_translation_on_linear_images():
    """Identity cameras, fronto-parallel depth d, C_src a pure x-translation delta: every in-frame
    pixel moves by f delta / d, the residual is -a_c f delta / d, dr/drho_x = -a_c f / d,
    dr/dsigma = 0 (scaling about the camera centre keeps the projection), and U_e is the set of
    columns x with x + f delta / d in [0, W - 1) and rows y < H - 1."""
    W, H, f, d, delta = 40, 30, 50.0, 2.0, 0.125
    a, b, k = [2 ** -7, -2 ** -8, 2 ** -9], [2 ** -9, 2 ** -7, -2 ** -8], [0.25, 0.5, 0.75]   # exact in FP32
    img = _ramp(W, H, a, b, k)
    dep = np.full((H, W), d, np.float32)
    cam = _cam(W, H, f)
    sim_s = (np.array([1.0, 0, 0, 0]), np.array([delta, 0, 0]), 1.0)
    out = PH.edge_terms(img, dep, img, cam, cam, sim_s, IDENT, weight=1.0, per_pixel=True, delta=1.0)
    shift = f * delta / d                                   # 3.125 px
    ncols = sum(1 for x in range(W) if 0 <= x + shift < W - 1)
    assert out["n"] == ncols * (H - 1)
    r = out["r"]
    np.testing.assert_allclose(r, np.tile(-np.array(a) * shift, (out["n"], 1)), atol=1e-9)
    J = out["J"]
    np.testing.assert_allclose(J[:, :, 0], np.tile(-np.array(a) * f / d, (out["n"], 1)), atol=1e-9)
    np.testing.assert_allclose(J[:, :, 1], np.tile(-np.array(b) * f / d, (out["n"], 1)), atol=1e-9)
    np.testing.assert_allclose(J[:, :, 6], 0, atol=1e-9)
    assert abs(out["cost"] - float(np.sum((np.array(a) * shift) ** 2))) <= 1e-12


def _scene(seed, W=48, H=36):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W] / 9.0
    img_s = np.stack([0.5 + 0.3 * np.sin(x * (1 + c) + 0.7 * y + c) * np.cos(0.5 * y - c) for c in range(3)])
    img_t = np.stack([0.5 + 0.3 * np.sin(x * (1 + c) + 0.7 * y + c + 0.05) * np.cos(0.5 * y - c) for c in range(3)])
    dep = (2.0 + 0.3 * np.sin(x) * np.cos(y) + rng.uniform(0, 0.01, (H, W))).astype(np.float32)
    th = rng.normal(0, 0.03, 3)
    cam_s = _cam(W, H, 40.0, expm(PH.skew(th)), rng.normal(0, 0.05, 3))
    cam_t = _cam(W, H, 40.0, expm(PH.skew(-th)), rng.normal(0, 0.05, 3))
    sim_s = (rng.normal(0, 1, 4) * [1, 0.02, 0.02, 0.02] + [3, 0, 0, 0], rng.normal(0, 0.03, 3), 1.05)
    sim_t = (rng.normal(0, 1, 4) * [1, 0.02, 0.02, 0.02] + [3, 0, 0, 0], rng.normal(0, 0.03, 3), 0.97)
    sim_s = (np.asarray(sim_s[0], np.float32), np.asarray(sim_s[1], np.float32), np.float32(sim_s[2]))
    sim_t = (np.asarray(sim_t[0], np.float32), np.asarray(sim_t[1], np.float32), np.float32(sim_t[2]))
    return img_s.astype(np.float32), dep, img_t.astype(np.float32), cam_s, cam_t, sim_s, sim_t


def test_jacobian_matches_finite_differences_of_both_twists():
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(1)
    H_, W_ = dep.shape
    dec = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep)
    out = PH.edge_terms(img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t, decisions=dec, per_pixel=True)
    assert out["n"] > 800
    J = out["J"]
    # central differences of the FP64 residuals (decisions held fixed) under FP64-retracted
    # corrections; _r64 equals the oracle's residuals at the expansion point (test below)
    eps = 1e-6
    args = (img_s, dep, img_t, cam_s, cam_t)
    for side in range(2):
        for i in range(7):
            xi = np.zeros(7)
            xi[i] = eps
            sp, sm = (_retract(sim_s, xi), _retract(sim_s, -xi)) if side == 0 else (sim_s, sim_s)
            tp, tm = (sim_t, sim_t) if side == 0 else (_retract(sim_t, xi), _retract(sim_t, -xi))
            fd = (_r64(args, sp, tp, dec) - _r64(args, sm, tm, dec)) / (2 * eps)
            col = J[:, :, 7 * side + i]
            err = np.linalg.norm(fd - col) / max(1e-12, np.linalg.norm(col))
            assert err < 1e-5, (side, i, err)


def _r64(args, sim_s, sim_t, dec):
    """Residuals with the corrections taken in FP64 as given (no FP32 rounding of q, t, s)."""
    img_s, dep, img_t, cam_s, cam_t = args
    valid, x0, y0, _, _, xs, ys = dec
    xs, ys, x0, y0 = xs[valid], ys[valid], x0[valid], y0[valid]
    cs, ct = cam_s.astype(np.float64), cam_t.astype(np.float64)
    d = dep[ys, xs].astype(np.float64)
    pc = np.stack([(xs + 0.5 - cs[14]) / cs[12] * d, (ys + 0.5 - cs[15]) / cs[13] * d, d], 1) - cs[9:12]
    p = pc @ cs[:9].reshape(3, 3)
    As, bs = float(sim_s[2]) * PH.quat_matrix(sim_s[0]), np.asarray(sim_s[1], np.float64)
    At, bt = float(sim_t[2]) * PH.quat_matrix(sim_t[0]), np.asarray(sim_t[1], np.float64)
    q = np.linalg.solve(At, (p @ As.T + bs - bt).T).T
    c = q @ ct[:9].reshape(3, 3).T + ct[9:12]
    sx = ct[12] * c[:, 0] / c[:, 2] + ct[14] - 0.5
    sy = ct[13] * c[:, 1] / c[:, 2] + ct[15] - 0.5
    ax, ay = (sx - x0)[:, None], (sy - y0)[:, None]
    It = img_t.astype(np.float64)
    top = It[:, y0, x0].T * (1 - ax) + It[:, y0, x0 + 1].T * ax
    bot = It[:, y0 + 1, x0].T * (1 - ax) + It[:, y0 + 1, x0 + 1].T * ax
    return img_s.astype(np.float64)[:, ys, xs].T - (top * (1 - ay) + bot * ay)


def test_r64_restatement_agrees_with_oracle_residuals():
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(2)
    H_, W_ = dep.shape
    dec = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep)
    r = PH.edge_terms(img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t, decisions=dec, per_pixel=True)["r"]
    np.testing.assert_allclose(_r64((img_s, dep, img_t, cam_s, cam_t), sim_s, sim_t, dec), r, atol=1e-12)


def test_normal_equations_and_cost_gradient():
    """H = (w/n) sum omega J^T J is symmetric PSD with the [[S, -S], [-S, S]] block form, and 2 g is
    the gradient of the robust cost (central differences through the retraction)."""
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(3)
    H_, W_ = dep.shape
    dec = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep)
    out = PH.edge_terms(img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t, weight=2.5, decisions=dec)
    Hm, g = out["H"], out["g"]
    np.testing.assert_allclose(Hm, Hm.T, atol=1e-14)
    assert np.linalg.eigvalsh(Hm).min() > -1e-10
    np.testing.assert_allclose(Hm[:7, 7:], -Hm[:7, :7], atol=1e-14)
    args = (img_s, dep, img_t, cam_s, cam_t)

    def cost(ss, tt):
        r = _r64(args, ss, tt, dec)
        return 2.5 / out["n"] * PH.huber(r, PH.HUBER_DELTA)[0].sum()
    assert abs(cost(sim_s, sim_t) - out["cost"]) <= 1e-9 * out["cost"]
    eps = 1e-6
    fd = np.zeros(14)
    for i in range(7):
        xi = np.zeros(7)
        xi[i] = eps
        fd[i] = (cost(_retract(sim_s, xi), sim_t) - cost(_retract(sim_s, -xi), sim_t)) / (2 * eps)
        fd[7 + i] = (cost(sim_s, _retract(sim_t, xi)) - cost(sim_s, _retract(sim_t, -xi))) / (2 * eps)
    np.testing.assert_allclose(fd, 2 * g, rtol=1e-5, atol=1e-9)


def test_gauge_invariance_and_gauss_newton_step():
    """A common left Sim(3) on both corrections leaves every residual unchanged; one GN step on the
    source twist reduces the cost of a misaligned linear-image pair to (near) zero."""
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(4)
    H_, W_ = dep.shape
    dec = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep)
    args = (img_s, dep, img_t, cam_s, cam_t)
    G = np.array([0.01, -0.02, 0.03, 0.1, -0.05, 0.2, 0.3])
    np.testing.assert_allclose(_r64(args, _retract(sim_s, G), _retract(sim_t, G), dec), _r64(args, sim_s, sim_t, dec),
                               atol=1e-11)
    # GN on a linear image with a small misalignment (Huber threshold above every residual)
    W, Hh, f = 40, 30, 50.0
    img = _ramp(W, Hh, [0.010, -0.004, 0.002], [0.003, 0.006, -0.005], [0.2, 0.5, 0.7])
    dep2 = np.full((Hh, W), 2.0, np.float32)
    cam = _cam(W, Hh, f)
    s0 = (np.array([1.0, 0, 0, 0]), np.array([0.02, -0.01, 0.0]), 1.0)
    o0 = PH.edge_terms(img, dep2, img, cam, cam, s0, IDENT, delta=1.0)
    Hs, gs = o0["H"][:7, :7], o0["g"][:7]
    step = -np.linalg.lstsq(Hs, gs, rcond=None)[0]
    s1 = _retract(s0, step)
    o1 = PH.edge_terms(img, dep2, img, cam, cam, s1, IDENT, delta=1.0)
    assert o0["cost"] > 1e-6 and o1["cost"] < 1e-4 * o0["cost"]


def test_empty_and_invalid_depth():
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(5)
    zero = np.zeros_like(dep)
    out = PH.edge_terms(img_s, zero, img_t, cam_s, cam_t, sim_s, sim_t)
    assert out["n"] == 0 and out["cost"] == 0.0 and not out["H"].any() and not out["g"].any()
    bad = dep.copy()
    bad[:, ::2] = np.inf
    bad[::3, :] = np.nan
    H_, W_ = dep.shape
    v1 = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep)[0].reshape(H_, W_)
    v2 = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, bad)[0].reshape(H_, W_)
    assert not v2[:, ::2].any() and not v2[::3, :].any()
    keep = np.ones_like(v1)
    keep[:, ::2] = False
    keep[::3, :] = False
    np.testing.assert_array_equal(v2, v1 & keep)


def test_decision_chain_is_fp32_and_brute_force_membership():
    """Per-pixel scalar restatement of the FP32 chain (np.float32 scalars, same operation order)
    gives the same membership and cells; the FP32 projection agrees with FP64 to float precision."""
    img_s, dep, img_t, cam_s, cam_t, sim_s, sim_t = _scene(6, W=17, H=13)
    H_, W_ = dep.shape
    valid, x0, y0, sx, sy, xs, ys = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W_, H_, dep, stride=2)
    F = np.float32
    Q1, Q2 = PH.quat_matrix_f32(sim_s[0]), PH.quat_matrix_f32(sim_t[0])
    for k in range(len(xs)):
        x, y = xs[k], ys[k]
        d = F(dep[y, x])
        xn = F(F(F(F(x) + F(0.5)) - cam_s[14]) * F(F(1) / cam_s[12]))
        yn = F(F(F(F(y) + F(0.5)) - cam_s[15]) * F(F(1) / cam_s[13]))
        pc = [F(F(xn * d) - cam_s[9]), F(F(yn * d) - cam_s[10]), F(d - cam_s[11])]
        Rs = cam_s[:9].reshape(3, 3)
        p = [F(F(F(Rs[0, i] * pc[0]) + F(Rs[1, i] * pc[1])) + F(Rs[2, i] * pc[2])) for i in range(3)]
        rp = [F(F(F(Q1[i, 0] * p[0]) + F(Q1[i, 1] * p[1])) + F(Q1[i, 2] * p[2])) for i in range(3)]
        w = [F(F(sim_s[2] * rp[i]) + sim_s[1][i]) for i in range(3)]
        dw = [F(w[i] - sim_t[1][i]) for i in range(3)]
        rq = [F(F(F(Q2[0, i] * dw[0]) + F(Q2[1, i] * dw[1])) + F(Q2[2, i] * dw[2])) for i in range(3)]
        q = [F(rq[i] * F(F(1) / sim_t[2])) for i in range(3)]
        Ra = cam_t[:9].reshape(3, 3)
        c = [F(F(F(F(Ra[i, 0] * q[0]) + F(Ra[i, 1] * q[1])) + F(Ra[i, 2] * q[2])) + cam_t[9 + i]) for i in range(3)]
        iz = F(F(1) / c[2])
        px = F(F(cam_t[12] * F(c[0] * iz)) + cam_t[14])
        py = F(F(cam_t[13] * F(c[1] * iz)) + cam_t[15])
        assert px - F(0.5) == sx[k] and py - F(0.5) == sy[k]
        ok = d > 0 and np.isfinite(d) and c[2] > F(0.2) and 0 <= F(px - F(0.5)) < W_ - 1 and 0 <= F(py - F(0.5)) < H_ - 1
        assert bool(ok) == bool(valid[k])
        if ok:
            assert x0[k] == int(np.floor(F(px - F(0.5)))) and y0[k] == int(np.floor(F(py - F(0.5))))


def test_projection_of_a_known_plane_by_ray_intersection():
    """Independent geometry: the source depth map of the world plane z = 3 is built by intersecting
    each pixel ray (camera centre -R^T t, direction R^T K^-1 [u + 0.5, 1]) with the plane; the oracle's
    projected coordinate must equal the target camera's projection of C_tgt^-1 C_src X."""
    W, H, f = 32, 24, 30.0
    rng = np.random.default_rng(7)
    Rs, Ra = expm(PH.skew(rng.normal(0, 0.1, 3))), expm(PH.skew(rng.normal(0, 0.1, 3)))
    ts, ta = rng.normal(0, 0.1, 3), rng.normal(0, 0.1, 3)
    cam_s, cam_t = _cam(W, H, f, Rs, ts), _cam(W, H, f, Ra, ta)
    Rs, ts = cam_s[:9].reshape(3, 3).astype(np.float64), cam_s[9:12].astype(np.float64)
    Ra, ta = cam_t[:9].reshape(3, 3).astype(np.float64), cam_t[9:12].astype(np.float64)
    ctr = -Rs.T @ ts
    dep = np.zeros((H, W), np.float32)
    X = np.zeros((H, W, 3))
    for y in range(H):
        for x in range(W):
            ray = Rs.T @ np.array([(x + 0.5 - W / 2) / f, (y + 0.5 - H / 2) / f, 1.0])
            lam = (3.0 - ctr[2]) / ray[2]
            X[y, x] = ctr + lam * ray
            dep[y, x] = (Rs @ X[y, x] + ts)[2]
    sim_s = (np.array([0.999, 0.02, -0.01, 0.03], np.float32), np.array([0.05, -0.02, 0.01], np.float32),
             np.float32(1.02))
    sim_t = (np.array([0.998, -0.01, 0.03, 0.01], np.float32), np.array([-0.03, 0.01, 0.02], np.float32),
             np.float32(0.99))
    valid, _, _, sx, sy, xs, ys = PH.decision_chain(cam_s, cam_t, sim_s, sim_t, W, H, dep)
    As, bs = float(sim_s[2]) * PH.quat_matrix(sim_s[0]), sim_s[1].astype(np.float64)
    At, bt = float(sim_t[2]) * PH.quat_matrix(sim_t[0]), sim_t[1].astype(np.float64)
    assert valid.sum() > 0.5 * W * H
    for k in np.flatnonzero(valid):
        q = np.linalg.solve(At, As @ X[ys[k], xs[k]] + bs - bt)
        c = Ra @ q + ta
        assert abs(f * c[0] / c[2] + W / 2 - 0.5 - sx[k]) < 2e-4
        assert abs(f * c[1] / c[2] + H / 2 - 0.5 - sy[k]) < 2e-4
