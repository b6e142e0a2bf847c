"""The GPU's tile lists and depth keys against FP64 geometry, independently of the key path.

The bit-exact key tests compare the kernels with the oracle's FP32 key module, which follows the
same specified operation order (FP32, no contraction).  These tests take the GPU's per-tile
lists (``ges_frame_keys``) and depth keys (``ges_frame_inspect``) and check them against the
extent ellipse and the camera depth computed in FP64 from the oracle's projection and the view
matrix, with none of the key path's arithmetic:

* every tile that the ellipse {q <= q*} meets (q* where kappa G = alpha_min, Sec. 3.1 Eq. ges with
  the compositing skip rule) is listed for its primitive: no pixel with alpha >= alpha_min is left
  out of a list;
* every listed tile meets the ellipse widened by the stated margins (q* (1 + 1e-3)^2, 1e-2 px);
* every depth key is the FP64 depth up to the FP32 rounding bound, and each tile's list is in
  FP64 depth order up to those bounds, equal keys by ascending primitive index.
"""
import numpy as np
import pytest

import oracle
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges
    return ges


def _small_cases():
    return {
        "ragged_lowbeta": (scenes.cube_scene(300, seed=11, beta_range=(0.3, 16.0), beta_log=True,
                                             scale_range=(0.02, 0.2)), scenes.tiny_camera(45, 37), None),
        "sh3_offaxis": (scenes.cube_scene(500, seed=12, sh_degree=3, beta_range=(0.5, 8.0), beta_log=True),
                        scenes.look_at((1.5, -1.0, -3.5), (0.0, 0.2, 0.0), (0.0, -1.0, 0.0), 100, 70, 65.0,
                                       bg=(0.2, 0.3, 0.1)), None),
        "exact_phi": (scenes.cube_scene(400, seed=14, beta_range=(0.8, 12.0), beta_log=True,
                                        scale_range=(0.01, 0.06)), scenes.tiny_camera(70, 50), dict(phi_mode=1)),
        "paper_form": (*scenes.tiny_workload(), dict(mode=1)),
        "dense_batches": (scenes.cube_scene(5000, seed=13, scale_range=(0.01, 0.06)), scenes.tiny_camera(160, 120),
                          None),
    }


CASES = _small_cases()


@pytest.mark.parametrize("case", list(CASES))
def test_gpu_tile_lists_follow_the_fp64_extent(lib, case):
    from gpu_helpers import gpu_run
    from helpers import check_depth_keys_fp64, check_tile_lists_fp64
    sc, cam, p = CASES[case]
    got = gpu_run(sc, cam, p)
    n, fails = check_tile_lists_fp64(sc, cam, p, got["keys"], got["vals"], oracle)
    assert n > 1000 and not fails, fails
    fails = check_depth_keys_fp64(sc, cam, got["inspect"]["depth_key"], oracle, got["keys"], got["vals"])
    assert not fails, fails


def test_gpu_tile_lists_follow_the_fp64_extent_full_size(lib):
    """A sample of 20,000 primitives of the scene-scale view (1.5M primitives, 1245x825): each
    one's complete set of listed tiles against its FP64 ellipse; every depth key and the order of
    every tile's list against the FP64 depths."""
    from gpu_helpers import gpu_run
    from helpers import check_depth_keys_fp64, check_tile_lists_fp64
    sc, cams = scenes.scene_scale_workload()
    cam = cams[0]
    got = gpu_run(sc, cam)
    prims = np.random.default_rng(31).choice(sc.n, 20_000, replace=False)
    n, fails = check_tile_lists_fp64(sc, cam, None, got["keys"], got["vals"], oracle, prims=prims)
    assert n > 100_000 and not fails, fails
    fails = check_depth_keys_fp64(sc, cam, got["inspect"]["depth_key"], oracle, got["keys"], got["vals"])
    assert not fails, fails
