"""Pins of the 1D mixture-fitting oracle (oracle/mixture1d.py): the signals' and models' closed
forms (App. A), the gradient by central differences, the first Adam step in closed form, and the
study's finding that a GEF mixture fits the square better than a Gaussian mixture with as many
components (Sec. 3.2, Fig. 1 b-c and the loss-stability figure)."""
import math

import numpy as np
import pytest

from oracle import mixture1d as om
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")


def test_signals_closed_forms():
    w = 1.0
    x = np.array([-0.75, -0.5, -0.25, 0.0, 0.25, 0.4999, 0.5, 0.8])
    inside = np.abs(x) < 0.5
    np.testing.assert_array_equal(om.signal("square", x, w), inside.astype(float))
    np.testing.assert_allclose(om.signal("triangle", x, w), np.where(inside, 0.5 - np.abs(x), 0), atol=1e-15)
    np.testing.assert_allclose(om.signal("parabolic", x, w), np.where(inside, 0.25 - x * x, 0), atol=1e-15)
    hs = om.signal("half_sinusoid", x, w)
    assert hs[3] == pytest.approx(1.0) and hs[2] == pytest.approx(math.sqrt(0.5)) and hs[0] == 0 and hs[-1] == 0
    np.testing.assert_allclose(om.signal("exponential", x, w), np.where(inside, np.exp(-np.abs(x)), 0), rtol=1e-15)
    g = om.signal("gaussian", np.array([0.0, 1.0, 2.0]), w)   # not truncated
    np.testing.assert_allclose(g, [1.0, math.exp(-0.5), math.exp(-2.0)], rtol=1e-15)
    # a wider support: the triangle's peak is width / 2 and the parabola's (width / 2)^2
    assert om.signal("triangle", np.array([0.0]), 3.0)[0] == 1.5 and om.signal("parabolic", np.array([0.0]), 3.0)[0] == 2.25


def test_models_closed_forms():
    x = np.linspace(-1, 1, 41)
    p = np.array([[0.7, -0.4], [0.1, -0.3], [0.2, 0.35]])
    eps = om.MIX_EPS
    gauss = om.model_eval("gaussian", p, x).numpy()
    ref = sum(p[0, i] * np.exp(-(x - p[1, i]) ** 2 / (2 * p[2, i] ** 2 + eps)) for i in range(2))
    np.testing.assert_allclose(om.model_eval("gaussian", p, x, positive=False).numpy(), ref, rtol=1e-14)
    assert np.all(gauss >= 0)                                    # |omega| keeps the weights positive
    # the GEF with beta = 2 is the Gaussian mixture (App. A, after Eq. genmixture)
    p4 = np.vstack([p, [2.0, 2.0]])
    np.testing.assert_allclose(om.model_eval("gef", p4, x).numpy(), gauss, rtol=1e-14)
    # a DoG with variance ratio 1 vanishes; a LoG is w at its mean and 0 at |x - mu| = gamma
    assert np.abs(om.model_eval("dog", p, x, nu=1.0).numpy()).max() == 0.0
    one = np.array([[0.6], [0.2], [0.3]])
    v = om.model_eval("log", one, np.array([0.2, 0.5, -0.1])).numpy()
    np.testing.assert_allclose(v, [0.6, 0.0, 0.0], atol=1e-15)
    # the GEF with beta = 1 is Laplace-shaped: w exp(-|d| / (2 s^2 + eps))
    p1 = np.array([[0.5], [0.0], [0.4], [1.0]])
    np.testing.assert_allclose(om.model_eval("gef", p1, x).numpy(), 0.5 * np.exp(-np.abs(x) / (0.32 + eps)), rtol=1e-14)


@pytest.mark.parametrize("model", om.MODELS)
@pytest.mark.parametrize("positive", [True, False])
def test_gradient_by_central_differences(model, positive):
    x = np.linspace(-1, 1, 301)
    y = om.signal("square", x)
    p0 = scenes.mixture_init(model, 4, 1, seed=3)[0]
    if not positive:
        p0[0] -= 0.5
    _, hist, g = om.fit(model, p0, x, y, 0, positive)
    def mse(p):
        return float(((om.model_eval(model, p, x, positive) - torch.tensor(y)) ** 2).mean())
    assert hist[0] == pytest.approx(mse(p0), rel=1e-14)
    h = 1e-6
    fd = np.zeros_like(p0)
    for idx in np.ndindex(*p0.shape):
        a, b = p0.copy(), p0.copy()
        a[idx] += h
        b[idx] -= h
        fd[idx] = (mse(a) - mse(b)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_first_adam_step_and_history():
    x = np.linspace(-1, 1, 200)
    y = om.signal("triangle", x)
    p0 = scenes.mixture_init("gef", 3, 1, seed=5)[0]
    _, _, g0 = om.fit("gef", p0, x, y, 0)
    p1, hist, _ = om.fit("gef", p0, x, y, 1, lr=0.01)
    assert np.all(np.abs((p1 - p0) + 0.01 * np.sign(g0)) <= 0.01 * (1e-8 / np.abs(g0) + 1e-12))
    p5, hist5, _ = om.fit("gef", p0, x, y, 5)
    assert hist5.shape == (6,) and hist5[0] == pytest.approx(hist[0], rel=1e-15)
    final = float(((om.model_eval("gef", p5, x) - torch.tensor(y)) ** 2).mean())
    assert hist5[-1] == pytest.approx(final, rel=1e-14)


def test_gef_fits_the_square_better_than_gaussians():
    """Sec. 3.2: a GEF mixture approximates the band-unlimited square with lower loss than a
    Gaussian mixture of as many components (here N = 2, 6 seeds, 600 epochs; mean final MSE)."""
    x = np.linspace(-1, 1, 1000)
    y = om.signal("square", x)
    res = {}
    for model in ("gaussian", "gef"):
        p0 = scenes.mixture_init(model, 2, 6, seed=11)
        res[model] = np.mean([om.fit(model, p0[r], x, y, 600)[1][-1] for r in range(6)])
    assert res["gef"] < 0.75 * res["gaussian"], res
