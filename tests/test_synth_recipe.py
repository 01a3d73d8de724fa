"""The seeded input recipe (paper_2510_15602_gb300/synth.py), on the CPU: the same
seed gives the same image and another index another image; every workload has the
stated shapes, dtypes and window radii; the unplanted field has zero mean and unit
variance per channel (to sampling error) and the stated spatial correlation of a
Gaussian blur of width sigma; anomaly masks are non-empty and mark where the
features changed; class mixing matrices have the stated covariance spectrum."""
import numpy as np
import pytest

from paper_2510_15602_gb300 import synth


def test_seeded_and_reproducible():
    a = synth.make_image("plain_128_c64", 0)
    b = synth.make_image("plain_128_c64", 0)
    c = synth.make_image("plain_128_c64", 1)
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.mask, b.mask)
    assert a.seed == 1000 * 1 + 0 and c.seed == 1001
    assert not np.array_equal(a.X, c.X)


@pytest.mark.parametrize("name", ["plain_128_c64", "batch16_256_c256", "uneven64_c512", "serve_c256"])
def test_workload_shapes(name):
    wl = synth.WORKLOADS[name]
    img = synth.make_image(name, 3, C=16)  # a narrow copy of the recipe keeps this quick
    C, H, W = img.X.shape
    assert img.X.dtype == np.float32 and img.mask.dtype == np.uint8
    assert C == 16 and H == W and H in wl.sizes and img.mask.shape == (H, W)
    assert img.r in wl.radii
    assert wl.n_anom[0] <= len(img.kinds) <= wl.n_anom[1] and set(img.kinds) <= set(wl.kinds)


def test_field_is_unit_variance_and_blurred():
    rng = np.random.default_rng(7)
    sigma = 3.0
    X = synth.gaussian_field(rng, 64, 96, 96, sigma).astype(np.float64)
    assert abs(X.mean()) < 0.05
    assert abs(X.var() - 1.0) < 0.08
    # lag-1 correlation of a field blurred with a Gaussian of std sigma: exp(-1 / (4 sigma^2))
    rho = np.mean(X[:, :, 1:] * X[:, :, :-1]) / np.mean(X * X)
    assert abs(rho - np.exp(-1.0 / (4 * sigma ** 2))) < 0.02


@pytest.mark.parametrize("kind", ["square", "scratch", "blob", "rotcov"])
def test_anomaly_marks_where_features_change(kind):
    rng = np.random.default_rng(11)
    X = synth.gaussian_field(rng, 24, 64, 64, 2.0)
    X0 = X.copy()
    mask = np.zeros((64, 64), np.uint8)
    synth._PLANTERS[kind](rng, X, mask)
    changed = np.any(X != X0, axis=0)
    assert mask.any()
    assert not changed[mask == 0].any()   # nothing outside the mask moved
    assert changed[mask == 1].mean() > 0.9


def test_class_mixing_spectrum():
    C = 32
    M = synth.class_mixing(2, C).astype(np.float64)
    lam = np.sort(np.linalg.eigvalsh(M @ M.T))[::-1]
    want = 0.9 ** np.arange(C)
    want = want / want.mean()
    np.testing.assert_allclose(lam, want, rtol=1e-5)


def test_random_orthogonal_is_orthogonal():
    Q = synth.random_orthogonal(np.random.default_rng(3), 40)
    np.testing.assert_allclose(Q.T @ Q, np.eye(40), atol=1e-12)


@pytest.mark.parametrize("name,index", [("batch16_256_c256", 0), ("batch16_256_c256", 5), ("uneven64_c512", 7),
                                        ("plain_128_c64", 0)])
def test_kind_masks_replay_make_image(name, index):
    img = synth.make_image(name, index, C=24)
    km = synth.kind_masks(name, index, C=24)
    assert set(km) == set(img.kinds)
    union = np.zeros_like(img.mask)
    for m in km.values():
        assert m.dtype == np.uint8 and m.shape == img.mask.shape and m.any()
        union |= m
    np.testing.assert_array_equal(union, img.mask)
