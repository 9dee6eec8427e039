"""Pins for the oracle's binary64 gradient: the exact derivative of the frozen-decision forward
(contributor lists, alpha/colour/FOV clamp states of a reference render held fixed) must match
central finite differences of that forward in binary64 for every parameter group -- means,
log-scales, quaternions, opacity logits and SH coefficients.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth


@pytest.fixture(scope="module")
def setup(oracle_lib):
    scene, cam = synth.grad_subset(P=80, size=32)
    fz = oracle.Frozen(scene, cam, oracle.opts(bg=(0.2, 0.1, 0.4)))
    rng = np.random.default_rng(0)
    w = rng.normal(0, 1, (3, cam.height, cam.width))
    an = fz.backward(fz.p0, w)
    return scene, cam, fz, w, an


def loss(fz, p, w):
    rgb, _ = fz.forward(p)
    return float((rgb * w).sum())


@pytest.mark.parametrize("group,count", [("means", 30), ("scales", 30), ("quats", 30), ("opacity", 20), ("sh", 40)])
def test_gradient_matches_central_differences(setup, group, count):
    scene, cam, fz, w, an = setup
    rng = np.random.default_rng(hash(group) & 0xffff)
    used = np.unique(fz.gid[: fz.n_contrib])
    assert used.size > 20
    g = an[group]
    h = 1e-6
    checked = 0
    for _ in range(count):
        gi = int(rng.choice(used))
        idx = (gi,) + tuple(int(rng.integers(0, n)) for n in g.shape[1:])
        p_plus, p_minus = fz.p0.copy(), fz.p0.copy()
        getattr(p_plus, group)[idx] += h
        getattr(p_minus, group)[idx] -= h
        fd = (loss(fz, p_plus, w) - loss(fz, p_minus, w)) / (2 * h)
        assert abs(fd - g[idx]) <= 2e-6 + 1e-5 * abs(g[idx]), (group, idx, fd, g[idx])
        checked += 1
    assert checked == count
    assert np.abs(g).max() > 0


def test_gradient_is_zero_for_unused_gaussians(setup):
    scene, cam, fz, w, an = setup
    used = np.zeros(scene.P, bool)
    used[fz.gid[: fz.n_contrib]] = True
    for k in ("means", "scales", "quats", "opacity", "sh"):
        assert np.all(an[k][~used] == 0)


def test_frozen_forward_equals_the_render(setup):
    """At the reference parameters the frozen-decision forward is the binary64 render itself
    (the contributor lists and clamp states it holds fixed are the render's own)."""
    scene, cam, fz, w, an = setup
    rgb, T = fz.forward(fz.p0)
    assert np.abs(rgb - fz.ref.rgb).max() <= 1e-12
    assert np.abs(T - fz.ref.T).max() <= 1e-12
    assert fz.ref.rgb.max() > 0.05            # the view is not empty


def test_frozen_forward_equals_render_with_background_and_raw_inputs(oracle_lib):
    scene, cam = synth.grad_subset(P=120, size=40, seed=5)
    o = oracle.opts(bg=(0.3, 0.05, 0.6))
    fz = oracle.Frozen(scene, cam, o)
    rgb, T = fz.forward(fz.p0)
    ref = oracle.Frame(scene, cam, o, mode=64)
    assert np.abs(rgb - ref.rgb).max() <= 1e-12 and np.abs(T - ref.T).max() <= 1e-12
