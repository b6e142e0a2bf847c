"""The preprocess backward (K8) is a deterministic function of each primitive's 2D gradients.

The 2D gradients that the backward composite leaves per primitive are sums of atomics, so their
last bits follow the order of the atomics; K8 then maps each primitive's row on its own.  So two
backward passes over the same frame must give bitwise equal scene gradients for every primitive
whose 2D gradients came out bitwise equal, and exact zeros for every culled primitive.  The cases
have ragged primitive counts (partial warps and CTAs) and culled primitives interleaved with
visible ones, at every SH degree.
"""
import numpy as np
import pytest

from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges, render
    return ges, render


@pytest.mark.parametrize("deg,n", [(3, 5003), (3, 31), (3, 64), (2, 777), (1, 1001), (0, 999)])
def test_preprocess_bwd_is_deterministic(lib, deg, n):
    ges, render = lib
    W, H = 160, 120
    sc = scenes.cube_scene(n, seed=70 + deg, sh_degree=deg, beta_range=(0.5, 8.0), beta_log=True)
    # close to the cube: primitives behind the camera and outside the view are culled
    cam = scenes.look_at((0.5, -0.4, -1.3), (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), W, H, 70.0)
    t = render.scene_tensors(sc, "cuda")
    fr = render.Frame(sc.n, W, H)
    img, T, nc = fr.forward(t, sc.sh_degree, cam)
    rng = np.random.default_rng(80 + deg)
    dL = torch.as_tensor(rng.standard_normal((3, H, W)).astype(np.float32), device="cuda")
    runs = []
    for _ in range(2):
        g = [x.clone() for x in fr.render_bwd(T, nc, dL)]
        torch.cuda.synchronize()
        runs.append((g, fr.inspect()))
    (g1, i1), (g2, i2) = runs
    culled = i1["depth_key"] == 0xFFFFFFFF
    assert culled.any() and (~culled).any()
    same = np.all(i1["grad2d"].view(np.uint32) == i2["grad2d"].view(np.uint32), axis=1) & ~culled
    # which primitives' atomics happen to sum in the same order differs from run to run: ask for a
    # few of them in the small cases, more in the large ones
    assert same.sum() >= (3 if n < 100 else 8), same.sum()
    for a, b in zip(g1, g2):
        a = a.cpu().numpy().reshape(n, -1).view(np.uint32)
        b = b.cpu().numpy().reshape(n, -1).view(np.uint32)
        assert np.array_equal(a[same], b[same])
        assert not a[culled].any() and not b[culled].any()
    st, _ = ges.ges_frame_status(fr.handle)
    assert st == ges.GES_OK
    fr.close()
