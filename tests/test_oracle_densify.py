"""Pins of the top-k / Long-Axis-Split oracle (Sec. 2.2, Alg. 1-2)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import densify as od

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "las_worked_example.json")


def _one(g, i):
    return {k: (v[i:i + 1] if isinstance(v, np.ndarray) else v) for k, v in g.items()}


def test_worked_example_with_paper_constants():
    ex = json.load(open(GOLDEN))
    p = ex["params"]
    # the paper's constants, Sec. 2.2 after Alg. 1
    assert p == {"k_off": 0.5, "long_factor": 0.5, "other_factor": 0.85, "beta": 0.6}
    assert od.PAPER_PRESET == p
    gs = ex["gaussians"]
    g = {"means": np.array([x["mean"] for x in gs]),
         "log_scales": np.log(np.array([x["scale"] for x in gs])),
         "quats": np.array([x["quat_wxyz"] for x in gs]),
         "opacity_logits": np.array([math.log(x["opacity"] / (1 - x["opacity"])) for x in gs]),
         "sh": np.zeros((len(gs), 1, 3)), "sh_degree": 0}
    out = od.las_split(g, np.ones(len(gs), bool), **p)
    n = len(gs)
    for i, x in enumerate(gs):
        assert int(np.argmax(g["log_scales"][i])) == x["expected_long_axis"]
        for slot, key in ((i, "expected_child0_mean"), (n + i, "expected_child1_mean")):
            np.testing.assert_allclose(out["means"][slot], x[key], rtol=0, atol=1e-15)
            np.testing.assert_allclose(np.exp(out["log_scales"][slot]), x["expected_scale"], rtol=1e-14)
            np.testing.assert_allclose(1 / (1 + np.exp(-out["opacity_logits"][slot])),
                                       x["expected_opacity"], rtol=1e-14)
            np.testing.assert_array_equal(out["quats"][slot], g["quats"][i])


@pytest.mark.parametrize("preset", ["paper", "config"])
def test_children_symmetric_and_offset_along_long_axis(preset):
    p = od.PAPER_PRESET if preset == "paper" else od.CONFIG_PRESET
    g = synth.gaussians(300, 3, seed=11)
    g["quats"] = g["quats"] * np.random.default_rng(1).uniform(0.5, 2.0, (300, 1)).astype(np.float32)
    mask = np.zeros(300, bool)
    mask[::3] = True
    out = od.las_split(g, mask, **p)
    sel = np.nonzero(mask)[0]
    n = 300
    rot = Rotation.from_quat(g["quats"].astype(np.float64), scalar_first=True).as_matrix()
    for rank, i in enumerate(sel):
        c0, c1 = out["means"][i], out["means"][n + rank]
        mu = g["means"][i].astype(np.float64)
        np.testing.assert_allclose(0.5 * (c0 + c1), mu, atol=1e-15)
        s = g["log_scales"][i].astype(np.float64)
        l = int(np.argmax(s))
        d = 0.5 * (c0 - c1)
        assert abs(np.linalg.norm(d) - p["k_off"] * math.exp(s[l])) < 1e-14
        # Alg. 2's column read equals R (off e_l) with R from scipy
        e = np.zeros(3)
        e[l] = p["k_off"] * math.exp(s[l])
        np.testing.assert_allclose(d, rot[i] @ e, atol=1e-14)
        ds = out["log_scales"][i] - s
        for a in range(3):
            want = math.log(p["long_factor"] if a == l else p["other_factor"])
            assert abs(ds[a] - want) < 1e-14
        sig_new = 1 / (1 + math.exp(-out["opacity_logits"][i]))
        sig_old = 1 / (1 + math.exp(-float(g["opacity_logits"][i])))
        assert abs(sig_new - p["beta"] * sig_old) < 1e-14
        np.testing.assert_array_equal(out["sh"][n + rank], g["sh"][i])
        np.testing.assert_array_equal(out["quats"][n + rank], g["quats"][i])
    untouched = ~mask
    np.testing.assert_array_equal(out["means"][:n][untouched], g["means"][untouched])
    np.testing.assert_array_equal(out["log_scales"][:n][untouched], g["log_scales"][untouched])


def test_config_preset_changes_only_the_long_axis():
    g = synth.gaussians(50, 0, seed=2)
    out = od.las_split(g, np.ones(50, bool), **od.CONFIG_PRESET)
    for i in range(50):
        s = g["log_scales"][i].astype(np.float64)
        l = int(np.argmax(s))
        changed = np.nonzero(out["log_scales"][i] != s)[0]
        assert list(changed) == [l]


def test_long_axis_ties_go_to_lowest_index():
    g = {"means": np.zeros((1, 3)), "log_scales": np.array([[-2.0, -1.0, -1.0]]),
         "quats": np.array([[1.0, 0, 0, 0]]), "opacity_logits": np.zeros(1),
         "sh": np.zeros((1, 1, 3)), "sh_degree": 0}
    out = od.las_split(g, np.ones(1, bool), **od.CONFIG_PRESET)
    np.testing.assert_allclose(out["means"][0], [0, math.exp(-1.0), 0], atol=1e-15)


def test_topk_ties_lowest_index_and_brute_force():
    s = np.array([0.5, 0.9, 0.5, 0.1, 0.9, 0.5, 0.7], dtype=np.float32)
    m = od.topk_mask(s, 4)
    # 0.9 (1, 4), 0.7 (6), then the lowest-index 0.5 (0)
    assert list(np.nonzero(m)[0]) == [0, 1, 4, 6]
    rng = np.random.default_rng(0)
    for trial in range(20):
        n = int(rng.integers(1, 200))
        s = rng.integers(0, 10, n).astype(np.float32)
        k = int(rng.integers(0, n + 1))
        ref = sorted(range(n), key=lambda i: (-float(s[i]), i))[:k]
        assert set(np.nonzero(od.topk_mask(s, k))[0]) == set(ref)
        assert od.topk_mask(s, k).sum() == k


def test_positional_statistic_worked_example():
    # view 1: (3, 4) -> 5, (0, 0) -> not counted; view 2: (0, -2) -> 2, (1e-30, 0) counted
    v1 = np.array([[3.0, 4.0, 9.0], [0.0, 0.0, 7.0]])
    v2 = np.array([[0.0, -2.0, 0.0], [1e-30, 0.0, 0.0]])
    s, c = od.pos_grad_stats([v1, v2])
    np.testing.assert_allclose(s, [7.0, 1e-30], rtol=0, atol=0)
    assert list(c) == [2, 1]
    s2, c2 = od.pos_grad_stats([v1], s, c)  # accumulates
    np.testing.assert_allclose(s2, [12.0, 1e-30])
    assert list(c2) == [3, 1]


def test_gated_topk_invariants_and_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = int(rng.integers(1, 300))
        s = rng.integers(0, 12, n).astype(np.float32)
        cnt = rng.integers(0, 4, n)
        sums = rng.uniform(0, 1, n) * cnt
        k = int(rng.integers(0, n + 1))
        # tau = 0 with every count > 0: plain top-k; tau = inf: nothing
        full = np.maximum(cnt, 1)
        assert np.array_equal(od.gated_topk_mask(s, k, sums, full, 0.0), od.topk_mask(s, k))
        assert not od.gated_topk_mask(s, k, sums, cnt, np.inf).any()
        tau = float(rng.uniform(0, 0.6))
        m = od.gated_topk_mask(s, k, sums, cnt, tau)
        # brute force over the candidates, in plain Python floats rounded to FP32
        cand = [i for i in range(n) if cnt[i] > 0 and
                float(np.float32(np.float32(sums[i]) / np.float32(cnt[i]))) >= float(np.float32(tau))]
        ref = sorted(cand, key=lambda i: (-float(s[i]), i))[:k]
        assert set(np.nonzero(m)[0]) == set(ref)
        assert m.sum() == min(k, len(cand))
    # a Gaussian never seen (count 0) is never a candidate, even at tau = 0
    assert not od.gated_topk_mask(np.ones(3, np.float32), 3, np.zeros(3), np.zeros(3, int), 0.0).any()


def test_sampling_first_draw_follows_the_scores():
    """Exponential clocks: the first Gaussian to ring is i with probability
    s_i / sum(s) (the minimum of independent Exp(s_i) clocks); 40,000 draws
    against the exact probabilities (chi-square, 5 degrees of freedom)."""
    s = np.array([0.5, 1.0, 2.0, 0.25, 4.0, 0.25], dtype=np.float32)
    p = s / s.sum()
    rng = np.random.default_rng(8)
    draws = 40000
    hits = np.zeros(6)
    for _ in range(draws // 2000):
        e = rng.exponential(size=(2000, 6)).astype(np.float32)
        for row in e:
            hits[np.nonzero(od.sample_mask(s, row, 1))[0][0]] += 1
    chi2 = np.sum((hits - draws * p) ** 2 / (draws * p))
    assert chi2 < 20.5  # 99.9 % quantile of chi-square with 5 dof


def test_sampling_limits_and_equal_scores():
    rng = np.random.default_rng(9)
    e = rng.exponential(size=500).astype(np.float32)
    s = rng.uniform(0, 2, 500).astype(np.float32)
    s[::7] = 0.0
    s[::11] = -1.0
    m = od.sample_mask(s, e, 10 ** 6)  # k beyond the positive scores: all of them
    assert np.array_equal(m, s > 0)
    assert not od.sample_mask(s, e, 0).any()
    # equal scores: uniform sampling, the k smallest variates
    eq = np.full(500, 3.0, np.float32)
    m = od.sample_mask(eq, e, 37)
    assert set(np.nonzero(m)[0]) == set(np.argsort(e, kind="stable")[:37])
    # the first draw of a sample of k is also a sample of 1; larger k nests
    for k in (1, 5, 50):
        assert np.all(od.sample_mask(s, e, k) <= od.sample_mask(s, e, k + 20))


def test_learning_rate_schedule_worked_values():
    from oracle import optim as oo
    l0, l1 = oo.PAPER_SCHEDULE["log_scales"]
    assert oo.lr_at(l0, l1, 30000, 0) == 0.020
    assert abs(oo.lr_at(l0, l1, 30000, 30000) - 0.002) < 1e-18
    assert abs(oo.lr_at(l0, l1, 30000, 10 ** 6) - 0.002) < 1e-18  # held after the horizon
    # half way: geometric mean of the ends (0.020 x 0.1^0.5)
    assert abs(oo.lr_at(l0, l1, 30000, 15000) - math.sqrt(0.020 * 0.002)) < 1e-15
    # constant ratio between consecutive steps: (final / init)^(1 / steps)
    r = [oo.lr_at(1.28e-4, 1.28e-5, 100, t + 1) / oo.lr_at(1.28e-4, 1.28e-5, 100, t) for t in range(100)]
    np.testing.assert_allclose(r, 0.1 ** 0.01, rtol=1e-12)
    assert oo.lr_at(0.5, 0.5, 10, 7) == 0.5
