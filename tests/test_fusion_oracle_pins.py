"""Pins of the fusion oracle (Eqs. 19-22) against closed forms and brute force."""
import numpy as np

from oracle import fusion as FU


def _cov(q, ls):
    R = FU.quat_to_matrix(q)
    S2 = np.exp(2 * np.asarray(ls))
    return R @ np.diag(S2) @ R.T


def test_sim3_covariance_closed_form_and_composition():
    rng = np.random.default_rng(0)
    n = 20
    mu, ls, q = rng.normal(0, 1, (n, 3)), rng.normal(-3, 0.4, (n, 3)), rng.normal(0, 1, (n, 4))
    s, qr, t = 1.7, rng.normal(0, 1, 4), rng.normal(0, 1, 3)
    mu2, ls2, q2 = FU.sim3_apply(mu, ls, q, s, qr, t)
    R = FU.quat_to_matrix(qr)
    np.testing.assert_allclose(mu2, s * mu @ R.T + t, atol=1e-12)
    for i in range(n):
        np.testing.assert_allclose(_cov(q2[i], ls2[i]), s * s * R @ _cov(q[i], ls[i]) @ R.T, atol=1e-12)
    # composition: C2 o C1 equals the composed similarity
    s2, qr2, t2 = 0.6, rng.normal(0, 1, 4), rng.normal(0, 1, 3)
    a = FU.sim3_apply(*FU.sim3_apply(mu, ls, q, s, qr, t), s2, qr2, t2)
    R2 = FU.quat_to_matrix(qr2)
    qc = FU.quat_mul(qr2 / np.linalg.norm(qr2), (qr / np.linalg.norm(qr))[None])[0]
    b = FU.sim3_apply(mu, ls, q, s * s2, qc, s2 * R2 @ t + t2)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=1e-11)


def test_occupied_box_of_one_gaussian():
    v, k = 0.05, 3.0
    mu = np.array([[0.512, -0.33, 1.2]], np.float32)
    ls = np.log(np.array([[0.02, 0.011, 0.004]], np.float32))
    occ = FU.occupied_set(mu, ls, k, v)
    s = np.exp(ls.astype(np.float64))
    lo = np.floor((mu - k * s) / v).astype(int)[0]
    hi = np.floor((mu + k * s) / v).astype(int)[0]
    assert len(occ) == np.prod(hi - lo + 1)
    assert int(FU.pack(*np.floor(mu[0] / np.float32(v)).astype(int))) in occ


def _dense_voxels(c, r, v, n=20000, guard=1e-4):
    """Voxels of dense FP64 samples of [c, r), skipping samples within `guard` of a voxel face."""
    c, r = np.asarray(c, np.float64), np.asarray(r, np.float64)
    ts = np.linspace(0.0, 1.0, n, endpoint=False)
    p = c[None] + ts[:, None] * (r - c)[None]
    q = p / v
    near = np.abs(q - np.round(q)).min(1) < guard
    return {tuple(x) for x in np.floor(q[~near]).astype(int).tolist()}


def test_dda_matches_dense_sampling_and_is_connected():
    rng = np.random.default_rng(1)
    v = 0.05
    for _ in range(40):
        c = rng.uniform(-1, 1, 3).astype(np.float32)
        r = (c + rng.normal(0, 0.6, 3)).astype(np.float32)
        vox = FU.dda_voxels(c, r, v)
        assert len(set(vox)) == len(vox)
        for a, b in zip(vox[:-1], vox[1:]):
            assert sum(abs(x - y) for x, y in zip(a, b)) == 1        # face-connected steps
        assert vox[0] == tuple(np.floor(c.astype(np.float64) / v).astype(int))
        dense = _dense_voxels(c, r, v)
        assert dense <= set(vox)
        # nothing beyond the endpoint's voxel
        end = tuple(np.floor(r.astype(np.float64) / v).astype(int))
        assert vox[-1] == end or abs((r.astype(np.float64) / v) - np.round(r / v)).min() < 1e-4


def test_backprojection_inverts_projection():
    from paper_2605_10760_gb300 import scenes as S
    cam = S.look_at([1.0, 2.0, 1.5], [4.0, 0.5, 1.0], 64, 48, 40.0, 40.0, 32.0, 24.0).as_row()
    R, t = cam[:9].reshape(3, 3).astype(np.float64), cam[9:12].astype(np.float64)
    for (x, y, d) in ((3, 5, 2.0), (60, 40, 3.3), (31, 23, 0.7)):
        p = FU.backproject(cam, x, y, d).astype(np.float64)
        pc = R @ p + t
        assert abs(pc[2] - d) < 1e-5
        assert abs(40.0 * pc[0] / pc[2] + 32.0 - (x + 0.5)) < 1e-3
        assert abs(40.0 * pc[1] / pc[2] + 24.0 - (y + 0.5)) < 1e-3
    c = FU.camera_center(cam).astype(np.float64)
    np.testing.assert_allclose(R @ c + t, 0.0, atol=1e-5)


def test_dedup_rules():
    v = 0.05
    tgt = np.array([[0.0, 0.0, 2.0]], np.float32)
    occ = FU.occupied_set(tgt, np.log(np.full((1, 3), 0.01, np.float32)), 3.0, v)
    from paper_2605_10760_gb300 import scenes as S
    cam = S.identity_camera(8, 8, 4.0, 4.0, 4.0, 4.0).as_row()
    depth = np.zeros((1, 8, 8), np.float32)
    depth[0, 4, 4] = 3.0                                  # one ray from the origin to (0.375, 0.375, 3)
    free = FU.free_set([cam], depth, v)
    borrowed = np.array([[0.001, 0.002, 2.001],           # inside the target's occupied box: dropped
                         [0.1880, 0.1880, 1.504],          # on the carved ray (x = y = z / 8): dropped
                         [1.0, 1.0, 1.0]], np.float32)    # unobserved: kept
    keep = FU.dedup_keep(borrowed, occ, free, v)
    assert keep.tolist() == [False, False, True]
