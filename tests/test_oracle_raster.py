"""Pins of the FP64 splatting oracle: scipy, closed forms, brute force, invariants, FD."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import synth
from oracle import raster as orc


def _real_sh_scipy(l, m, theta, phi):
    """Real SH from scipy's complex ones (Condon-Shortley phase removed)."""
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    y = sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2) * (-1) ** m * (y.real if m > 0 else y.imag)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ours = orc.sh_basis(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            ref = np.array([_real_sh_scipy(l, m, t, p) for t, p in zip(theta, phi)])
            np.testing.assert_allclose(ours[:, k], ref, rtol=0, atol=1e-13)


def test_quaternion_rotation_matches_scipy():
    q = np.random.default_rng(4).normal(size=(50, 4)) * 3.0
    ours = orc.quat_to_rot(q)
    ref = Rotation.from_quat(q, scalar_first=True).as_matrix()
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-14)


def _pinhole(mu, cam):
    vm = cam["viewmat"].astype(np.float64)
    t = vm[:, :3] @ mu + vm[:, 3]
    return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])


def test_projection_against_numerical_jacobian():
    g = synth.gaussians(30, 0, seed=9)
    cam = synth.camera_ring(3, resolutions=[(300, 200)] * 8)
    proj = orc.project(g, cam)
    rot = Rotation.from_quat(g["quats"].astype(np.float64), scalar_first=True).as_matrix()
    for i in range(30):
        if proj[i, orc.P_VALID] == 0:
            continue
        mu = g["means"][i].astype(np.float64)
        np.testing.assert_allclose(proj[i, [orc.P_MX, orc.P_MY]], _pinhole(mu, cam), rtol=1e-13)
        h = 1e-6
        jac = np.stack([(_pinhole(mu + h * e, cam) - _pinhole(mu - h * e, cam)) / (2 * h)
                        for e in np.eye(3)], axis=1)
        s = np.exp(g["log_scales"][i].astype(np.float64))
        sig = rot[i] @ np.diag(s * s) @ rot[i].T
        cov = jac @ sig @ jac.T + 0.3 * np.eye(2)
        ours = np.array([[proj[i, orc.P_COV_A], proj[i, orc.P_COV_B]],
                         [proj[i, orc.P_COV_B], proj[i, orc.P_COV_C]]])
        np.testing.assert_allclose(ours, cov, rtol=1e-6)
        con = np.array([[proj[i, orc.P_CON_A], proj[i, orc.P_CON_B]],
                        [proj[i, orc.P_CON_B], proj[i, orc.P_CON_C]]])
        np.testing.assert_allclose(con @ ours, np.eye(2), atol=1e-12)


def _single(scale, opacity_logit, dc, z=0.0, w=48, h=40):
    g = {"means": np.array([[0.0, 0.0, z]], np.float32),
         "log_scales": np.full((1, 3), math.log(scale), np.float32),
         "quats": np.array([[0.3, -0.5, 0.2, 0.7]], np.float32),
         "opacity_logits": np.array([opacity_logit], np.float32),
         "sh": np.array([[[dc, dc, dc]]], np.float32), "sh_degree": 0}
    return g, synth.camera_front(w, h)


def test_single_isotropic_gaussian_closed_form():
    g, cam = _single(0.05, 1.5, 0.8)
    out = orc.render(g, cam)
    f = float(cam["fx"])
    s = float(np.exp(np.float64(g["log_scales"][0, 0])))
    var = (f * s / 4.0) ** 2 + 0.3
    o = 1 / (1 + math.exp(-float(g["opacity_logits"][0])))
    col = max(0.0, float(g["sh"][0, 0, 0]) * 0.28209479177387814 + 0.5)
    ys, xs = np.mgrid[0:cam["height"], 0:cam["width"]]
    d2 = (xs + 0.5 - float(cam["cx"])) ** 2 + (ys + 0.5 - float(cam["cy"])) ** 2
    a = np.minimum(0.99, o * np.exp(-0.5 * d2 / var))
    a = np.where(a >= 1 / 255, a, 0.0)
    np.testing.assert_allclose(out["rgb"][..., 0], col * a, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["T"], 1 - a, rtol=0, atol=1e-14)
    assert (out["ncontrib"] == (a > 0)).all()


def test_zero_opacity_gives_background():
    g = synth.gaussians(200, 3, seed=5)
    g["opacity_logits"][:] = -40.0
    out = orc.render(g, synth.camera_front(64, 48), edge=np.ones((48, 64)))
    assert np.all(out["rgb"] == 0.0) and np.all(out["T"] == 1.0)
    assert np.all(out["ncontrib"] == 0) and np.all(out["score"] == 0.0)


def test_two_gaussians_hand_computed_transmittance():
    g = {"means": np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.5]], np.float32),
         "log_scales": np.full((2, 3), math.log(0.2), np.float32),
         "quats": np.array([[1.0, 0, 0, 0]] * 2, np.float32),
         "opacity_logits": np.array([0.0, 1.0], np.float32),
         "sh": np.array([[[1.0, 0.0, 0.5]], [[-1.0, 1.0, 0.25]]], np.float32), "sh_degree": 0}
    cam = synth.camera_front(32, 32)
    out = orc.render(g, cam)
    f = float(cam["fx"])
    c0 = 0.28209479177387814
    p = (16, 16)  # centre pixel: offset 0.5 from the image centre in x and y
    s = math.exp(float(g["log_scales"][0, 0]))  # the stored FP32 log-scale
    res = []
    for i, z in ((0, 4.0), (1, 4.5)):
        var = (f * s / z) ** 2 + 0.3
        o = 1 / (1 + math.exp(-float(g["opacity_logits"][i])))
        res.append(min(0.99, o * math.exp(-0.5 * 0.5 / var)))
    a1, a2 = res
    cols = [np.maximum(g["sh"][i, 0].astype(np.float64) * c0 + 0.5, 0) for i in range(2)]
    want = cols[0] * a1 + cols[1] * a2 * (1 - a1)
    np.testing.assert_allclose(out["rgb"][p], want, rtol=1e-13)
    assert abs(out["T"][p] - (1 - a1) * (1 - a2)) < 1e-15
    assert out["last_id"][p] == 1 and out["ncontrib"][p] == 2
    # equal depth key: the lower index composites first
    g["means"][1, 2] = 0.0
    out2 = orc.render(g, cam)
    var = (f * s / 4.0) ** 2 + 0.3
    b = [min(0.99, (1 / (1 + math.exp(-float(g["opacity_logits"][i])))) * math.exp(-0.25 / var))
         for i in range(2)]
    want2 = cols[0] * b[0] + cols[1] * b[1] * (1 - b[0])
    np.testing.assert_allclose(out2["rgb"][p], want2, rtol=1e-13)


def test_stop_before_transmittance_drops_below_threshold():
    n = 6
    logit = math.log(0.95 / 0.05)
    g = {"means": np.array([[0.0, 0.0, 0.1 * i] for i in range(n)], np.float32),
         "log_scales": np.full((n, 3), math.log(2.0), np.float32),
         "quats": np.array([[1.0, 0, 0, 0]] * n, np.float32),
         "opacity_logits": np.full(n, logit, np.float32),
         "sh": np.zeros((n, 1, 3), np.float32), "sh_degree": 0}
    cam = synth.camera_front(16, 16)
    out = orc.render(g, cam)
    # alpha ~ 0.95 at the centre pixel: T ~ 0.05, 2.6e-3, 1.4e-4, then ~7e-6 < 1e-4 stops
    f, s = float(cam["fx"]), math.exp(float(g["log_scales"][0, 0]))
    o = 1 / (1 + math.exp(-float(g["opacity_logits"][0])))
    z = [4.0 + float(np.float32(0.1 * i)) for i in range(n)]
    a = [o * math.exp(-0.25 / ((f * s / zk) ** 2 + 0.3)) for zk in z]
    t3 = (1 - a[0]) * (1 - a[1]) * (1 - a[2])
    assert out["ncontrib"][8, 8] == 3
    assert abs(out["T"][8, 8] - t3) < 1e-15 and t3 >= 1e-4 and t3 * (1 - a[3]) < 1e-4


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_equals_tiled(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 64))
    g = synth.gaussians(n, [0, 3][seed % 2], seed=100 + seed)
    g["log_scales"] += np.float32(rng.uniform(0.0, 1.5))
    w, h = int(rng.integers(16, 49)), int(rng.integers(16, 49))
    cam = synth.camera_look_at(rng.uniform(-1, 1, 3) + np.array([0, 0, -4.0]), w, h)
    e = rng.uniform(0, 3, (h, w))
    a = orc.render(g, cam, edge=e)
    b = orc.render(g, cam, edge=e, brute=True)
    for key in ("rgb", "T", "score"):
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-13)
    assert (a["ncontrib"] == b["ncontrib"]).all() and (a["last_id"] == b["last_id"]).all()


def test_score_invariant_with_unit_edge_map():
    g = synth.gaussians(2000, 0, seed=1)
    cam = synth.camera_front(128, 128)
    out = orc.render(g, cam, edge=np.ones((128, 128)))
    np.testing.assert_allclose(out["score"].sum(), (1.0 - out["T"]).sum(), rtol=1e-12)
    assert np.all(out["score"] >= 0)


def _fd_scene():
    rng = np.random.default_rng(5)
    g = synth.gaussians(40, 3, seed=3)
    g["log_scales"] = (g["log_scales"] + 1.2).astype(np.float32)
    g["quats"] = (g["quats"] * rng.uniform(0.5, 2.0, (40, 1))).astype(np.float32)
    return g, synth.camera_look_at((0.5, -0.3, -4.0), 48, 40), synth.image(40, 48, 2000)


def test_adjoint_matches_central_differences():
    g, cam, tgt = _fd_scene()
    out = orc.render(g, cam)
    _, dldc = orc.l1_loss(out["rgb"], tgt)
    gr = orc.render_bwd(g, cam, dldc)
    groups = {"means": 3, "log_scales": 3, "quats": 4, "opacity_logits": 1, "sh": 48}
    items = [(i, name, c) for i in range(40) for name, k in groups.items() for c in range(k)]
    fd1, fd2 = orc.fd_grad(g, cam, tgt, items)
    an = np.array([gr[n][i].ravel()[c] if gr[n].ndim > 1 else gr[n][i] for (i, n, c) in items])
    kink = np.abs(fd1 - fd2) > 0.1 * np.maximum(np.abs(fd1), 1e-12)
    assert kink.sum() < 0.02 * len(items)
    for name in groups:
        sel = np.array([it[1] == name for it in items])
        rms = np.sqrt(np.mean(an[sel] ** 2))
        assert rms > 0
        err = np.abs(an - fd1) / np.maximum(np.abs(fd1), 1e-3 * rms)
        assert err[sel & ~kink].max() < 1e-4, name


def test_masked_loss_differences_match_masked_adjoint():
    """fd_grad with a loss mask differentiates the L1 loss summed over the mask
    only: it must equal the adjoint of dL/dC zeroed outside the mask, and a
    full mask must give exactly the unmasked differences."""
    g, cam, tgt = _fd_scene()
    out = orc.render(g, cam)
    _, dldc = orc.l1_loss(out["rgb"], tgt)
    mask = np.zeros((40, 48), bool)
    mask[9:27, 13:37] = True
    gr = orc.render_bwd(g, cam, dldc * mask[:, :, None])
    items = [(i, name, c) for i in range(0, 40, 3) for name, c in
             (("means", 0), ("means", 2), ("log_scales", 1), ("quats", 0), ("opacity_logits", 0), ("sh", 0),
              ("sh", 47))]
    fd1, fd2 = orc.fd_grad(g, cam, tgt, items, loss_mask=mask)
    an = np.array([gr[n][i].ravel()[c] if gr[n].ndim > 1 else gr[n][i] for (i, n, c) in items])
    kink = np.abs(fd1 - fd2) > 0.1 * np.maximum(np.abs(fd1), 1e-12)
    assert kink.sum() <= 2
    rms = np.sqrt(np.mean(an ** 2))
    assert rms > 0 and np.count_nonzero(an) > len(items) // 2
    err = np.abs(an - fd1) / np.maximum(np.abs(fd1), 1e-3 * rms)
    assert err[~kink].max() < 1e-4
    full = orc.fd_grad(g, cam, tgt, items[:6], loss_mask=np.ones((40, 48), bool))
    plain = orc.fd_grad(g, cam, tgt, items[:6])
    np.testing.assert_array_equal(full[0], plain[0])


def test_l1_loss_sign_of_zero_is_zero():
    rgb = np.array([[[0.0, 1.0, 128 / 255.0]]])
    tgt = np.array([[[0, 0, 128]]], dtype=np.uint8)
    loss, d = orc.l1_loss(rgb, tgt)
    assert abs(loss - 1.0 / 3.0) < 1e-15
    np.testing.assert_array_equal(d, [[[0.0, 1.0 / 3.0, 0.0]]])


def _stack_scene(n=6):
    logit = math.log(0.95 / 0.05)
    return {"means": np.array([[0.0, 0.0, 0.1 * i] for i in range(n)], np.float32),
            "log_scales": np.full((n, 3), math.log(2.0), np.float32),
            "quats": np.array([[1.0, 0, 0, 0]] * n, np.float32),
            "opacity_logits": np.full(n, logit, np.float32),
            "sh": np.zeros((n, 1, 3), np.float32), "sh_degree": 0}


def test_gate_affected_marks_contributors_stop_candidate_and_next():
    # three composited, the fourth stops compositing, the fifth is the next
    # candidate past the stop, the sixth is never reached
    g, cam = _stack_scene(), synth.camera_front(16, 16)
    proj = orc.project(g, cam)
    mask = np.zeros((16, 16), bool)
    mask[8, 8] = True
    assert orc.render(g, cam)["ncontrib"][8, 8] == 3
    np.testing.assert_array_equal(orc.gate_affected(proj, mask, 0.0), [1, 1, 1, 1, 1, 0])
    assert not orc.gate_affected(proj, np.zeros((16, 16), bool), 0.0).any()


def test_gate_affected_with_wide_window_marks_every_tile_candidate():
    g = synth.gaussians(300, 0, seed=9)
    g["opacity_logits"][:] = -3.0  # faint: compositing never stops at the pixel
    cam = synth.camera_front(64, 48)
    proj = orc.project(g, cam)
    mask = np.zeros((48, 64), bool)
    mask[20, 37] = True  # tile (2, 1)
    assert orc.render(g, cam)["T"][20, 37] > 1e-2
    ok = (proj[:, orc.P_VALID] > 0) & (proj[:, orc.P_RADIUS] >= 0)
    member = ok & (proj[:, orc.P_TX0] <= 2) & (proj[:, orc.P_TX1] >= 2) & (proj[:, orc.P_TY0] <= 1) & \
        (proj[:, orc.P_TY1] >= 1)
    assert member.sum() > 10
    np.testing.assert_array_equal(orc.gate_affected(proj, mask, 2.0), member)  # relative gaps are <= 1


def test_order_is_depth_key_then_index():
    g = synth.gaussians(500, 0, seed=4)
    g["means"][::7, 2] = g["means"][0, 2]  # equal depth keys, broken by index
    cam = synth.camera_front(64, 64)
    proj = orc.project(g, cam)
    valid = np.nonzero(proj[:, orc.P_VALID] > 0)[0]
    keys = proj[valid, orc.P_ZKEY].astype(np.float32)
    expect = valid[np.lexsort((valid, keys))]
    np.testing.assert_array_equal(orc.order(proj), expect)
    a = orc.render(g, cam, proj=proj)
    b = orc.render(g, cam, proj=proj, order=expect)
    for key in ("rgb", "T", "ncontrib", "last_id"):
        np.testing.assert_array_equal(a[key], b[key])


def test_reorder_equals_sorting_with_the_new_key():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 20, 200).astype(np.float32)
    base = np.lexsort((np.arange(200), keys))
    for i in rng.choice(200, 20, replace=False):
        k2 = keys.copy()
        k2[i] = np.float32(rng.integers(0, 20))
        expect = np.lexsort((np.arange(200), k2))
        np.testing.assert_array_equal(orc._reorder(base, k2, int(i), float(k2[i]), True), expect)
        np.testing.assert_array_equal(orc._reorder(base, k2, int(i), 0.0, False), expect[expect != i])


def test_region_adjoint_equals_masked_upstream_gradient():
    g, cam, _ = _fd_scene()
    rng = np.random.default_rng(2)
    d = rng.normal(size=(40, 48, 3))
    box = (11, 7, 30, 25)
    m = np.zeros_like(d)
    m[box[1]:box[3], box[0]:box[2]] = d[box[1]:box[3], box[0]:box[2]]
    a = orc.render_bwd(g, cam, d, region=box)
    b = orc.render_bwd(g, cam, m)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-300)


def test_screen_space_mean_gradient_matches_differences_of_the_projected_mean():
    """g2d columns 0, 1 (dL/d mean2D, the input of the positional statistic of
    the gradient-threshold masking) against central differences that move the
    projected mean in the record itself, for a fixed linear upstream gradient."""
    g, cam, _ = _fd_scene()
    proj = orc.project(g, cam)
    rng = np.random.default_rng(21)
    dldc = rng.normal(size=(40, 48, 3))
    gr = orc.render_bwd(g, cam, dldc, proj=proj)

    def loss(p):
        return float(np.sum(orc.render(g, cam, proj=p)["rgb"] * dldc))

    checked = 0
    for i in range(40):
        if proj[i, orc.P_VALID] == 0:
            continue
        for col, c in ((orc.P_MX, 0), (orc.P_MY, 1)):
            fd = []
            for h in (1e-4, 5e-5):
                pp, pm = proj.copy(), proj.copy()
                pp[i, col] += h
                pm[i, col] -= h
                fd.append((loss(pp) - loss(pm)) / (2 * h))
            if abs(fd[0] - fd[1]) > 0.1 * max(abs(fd[0]), 1e-9):
                continue  # a gate moved inside the step
            an = gr["g2d"][i, c]
            assert abs(an - fd[0]) <= 1e-5 * max(abs(fd[0]), 1e-3), (i, c, an, fd[0])
            checked += 1
    assert checked > 40


# ---- magnitude adjoint (the condition of each gradient entry, used to bound
# what FP32 rounding can do to sums whose terms cancel)

def _mag_scene():
    g, cam, _ = _fd_scene()
    h, w = int(cam["height"]), int(cam["width"])
    dl = np.random.default_rng(21).normal(size=(h, w, 3)) / (h * w)
    return g, cam, dl


def test_magnitude_adjoint_bounds_the_adjoint_and_is_homogeneous():
    g, cam, dl = _mag_scene()
    gr = orc.render_bwd(g, cam, dl)
    gm = orc.render_bwd(g, cam, dl, magnitude=True)
    gm3 = orc.render_bwd(g, cam, -3.0 * dl, magnitude=True)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert np.all(gm[k] >= 0)
        assert np.all(gm[k] >= np.abs(gr[k]) * (1 - 1e-12))  # |sum| <= sum of |terms|
        np.testing.assert_allclose(gm3[k], 3.0 * gm[k], rtol=1e-12, atol=0)
    # the upstream gradient cancels across pixels: some entries are far below their magnitude
    assert (gm["opacity_logits"] > 10 * np.abs(gr["opacity_logits"])).any()


def test_magnitude_adjoint_of_sh_is_the_adjoint_of_the_absolute_upstream_gradient():
    """dL/dsh[k, ch] = Y_k(dir) sum_p alpha T g_ch(p): one product per pixel, so
    its magnitude is |Y_k| sum_p alpha T |g_ch(p)|, the plain adjoint of |g|
    up to the sign of Y_k (for the colour channels that are not clamped)."""
    g, cam, dl = _mag_scene()
    gm = orc.render_bwd(g, cam, dl, magnitude=True)
    ga = orc.render_bwd(g, cam, np.abs(dl))
    proj = orc.project(g, cam)
    for ch in range(3):
        live = (proj[:, orc.P_VALID] > 0) & (proj[:, orc.P_RAW_R + ch] >= 0)
        np.testing.assert_allclose(gm["sh"][live, :, ch], np.abs(ga["sh"][live, :, ch]), rtol=1e-12, atol=0)


def test_magnitude_adjoint_equals_the_adjoint_when_no_term_changes_sign():
    """With one Gaussian and a single pixel of positive upstream gradient, the
    colour and opacity entries are single products of positive factors."""
    g, cam = _single(0.08, 0.3, 0.4)
    h, w = int(cam["height"]), int(cam["width"])
    dl = np.zeros((h, w, 3))
    dl[h // 2, w // 2] = (1.0, 0.5, 0.25)
    gr = orc.render_bwd(g, cam, dl)
    gm = orc.render_bwd(g, cam, dl, magnitude=True)
    np.testing.assert_allclose(gm["sh"][0, 0], np.abs(gr["sh"][0, 0]), rtol=1e-14)
    np.testing.assert_allclose(gm["opacity_logits"], np.abs(gr["opacity_logits"]), rtol=1e-14)
