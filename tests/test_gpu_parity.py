"""CUDA path (through the C-ABI) against the FP64 oracle, element by element.

Bars: integer work (visibility, depth keys, tile rectangles, sorted key/value lists, tile
ranges) bit-exact; images within 1e-4 max abs per channel on pixels the oracle does not flag
as sitting on a threshold (alpha within 1e-4 relative of 1/255 or 0.99, or T within 1e-4
relative of the stop value); gradients, per parameter tensor, within 1e-3 relative L2 error and
element by element within 1e-3 (|g_ref| + 1e-3 max|g_ref|) + 1e-5 c, c the oracle's sum of the
element's absolute per-pixel contributions (the rounding scale of a sum whose terms cancel), with
the upstream gradient zeroed on flagged pixels."""
import numpy as np
import pytest

import oracle
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
T_TOL = 1e-5


def _needles_and_discs(n=300, seed=17):
    """Elongated splats (one axis 40-60x the others) and discs (two exactly equal axes, the third
    thin), at random rotations: where the backward's covariance chain is ill-conditioned."""
    sc = scenes.cube_scene(n, seed=seed, beta_range=(0.7, 4.0))
    rng = np.random.default_rng(seed + 1)
    base = np.exp(rng.uniform(np.log(0.004), np.log(0.01), n)).astype(np.float32)
    long = base * rng.uniform(40.0, 60.0, n).astype(np.float32)
    needle = rng.random(n) < 0.5
    sc.scales[:] = np.where(needle[:, None], np.stack([long, base, base * 0.8], 1),
                            np.stack([long * 0.3, long * 0.3, base], 1))
    return sc


def _beta2_mixed(n=400, seed=18):
    """Half the primitives at beta = 2 exactly (the GEF kernels' exponent-free branch: p = q), the
    other half spread over [0.5, 8], mixed in depth so that both branches alternate in a tile; SH
    degree 1 (the other degrees have cases of their own)."""
    sc = scenes.cube_scene(n, seed=seed, sh_degree=1, beta_range=(0.5, 8.0), beta_log=True,
                           scale_range=(0.01, 0.07))
    rng = np.random.default_rng(seed + 1)
    sc.betas[rng.random(n) < 0.5] = np.float32(2.0)
    return sc


def _cases():
    return {
        "tiny": (*scenes.tiny_workload(), None),
        "ragged_lowbeta": (scenes.cube_scene(300, seed=11, beta_range=(0.3, 16.0), beta_log=True,
                                             scale_range=(0.02, 0.2)), scenes.tiny_camera(45, 37), None),
        "sh3_offaxis": (scenes.cube_scene(500, seed=12, sh_degree=3, beta_range=(0.5, 8.0), beta_log=True),
                        scenes.look_at((1.5, -1.0, -3.5), (0.0, 0.2, 0.0), (0.0, -1.0, 0.0), 100, 70, 65.0,
                                       bg=(0.2, 0.3, 0.1)), None),
        "paper_form": (*scenes.tiny_workload(), dict(mode=1)),
        "dense_batches": (scenes.cube_scene(5000, seed=13, scale_range=(0.01, 0.06)), scenes.tiny_camera(160, 120),
                          None),
        # the exact Gamma-ratio modification (Eq. probablity, normalised) on the scale vector and, with
        # the Gaussian-form rasterizer, on the variance; beta from 0.8 (phi_n = 11) to 12
        "exact_phi": (scenes.cube_scene(400, seed=14, beta_range=(0.8, 12.0), beta_log=True,
                                        scale_range=(0.01, 0.06)), scenes.tiny_camera(70, 50), dict(phi_mode=1)),
        "exact_phi_variance_paper_form": (scenes.cube_scene(400, seed=15, sh_degree=2, beta_range=(0.5, 12.0),
                                                            beta_log=True, scale_range=(0.01, 0.08)),
                                          scenes.tiny_camera(70, 50), dict(phi_mode=2, mode=1)),
        # the ablation's shape strengths: rho = 10 (phi_bar close to a step at beta = 2) and rho = 0
        "rho10": (scenes.cube_scene(400, seed=16, beta_range=(0.5, 8.0), beta_log=True), scenes.tiny_camera(70, 50),
                  dict(rho=10.0)),
        "rho0": (scenes.cube_scene(400, seed=16, beta_range=(0.5, 8.0), beta_log=True), scenes.tiny_camera(70, 50),
                 dict(rho=0.0)),
        "needles_and_discs": (_needles_and_discs(), scenes.tiny_camera(96, 80), None),
        "beta2_mixed": (_beta2_mixed(), scenes.tiny_camera(72, 56), None),
    }


CASES = _cases()


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges
    return ges


def _params_for(p):
    return p


@pytest.mark.parametrize("case", list(CASES))
def test_preprocess_integer_outputs_bitexact(lib, case):
    from gpu_helpers import gpu_run
    sc, cam, p = CASES[case]
    got = gpu_run(sc, cam, p)
    ref = oracle.keys(sc, cam, p)
    ins = got["inspect"]
    assert np.array_equal(ins["depth_key"], ref["depth_key"])
    assert np.array_equal(ins["rect"], ref["rect"])
    vis = ref["touched"] > 0
    # the 2D mean comes from the same FP32 key path
    assert np.array_equal(ins["record"][vis, 0:2], ref["mean2d"][vis])
    proj = oracle.project(sc, cam, p)
    # conic (FP32 from the key path vs FP64): error relative to the conic's scale, since the
    # off-diagonal term can be a small difference of large products; an inverse's relative
    # error grows with its condition number kappa, so the bound adds 16 FP32 ulps times kappa
    a, b, c = proj[vis, 2], proj[vis, 3], proj[vis, 4]
    disc = np.sqrt((a - c) ** 2 / 4 + b * b)
    kappa = (0.5 * (a + c) + disc) / (0.5 * (a + c) - disc)
    scale = np.maximum(np.abs(a), np.abs(c))
    bound = (1e-5 + 16 * np.finfo(np.float32).eps * kappa) * scale
    err = np.abs(ins["record"][vis, 4:7] - proj[vis, 2:5]).max(1)
    assert np.all(err <= bound), float((err / bound).max())
    np.testing.assert_allclose(ins["record"][vis, 8:11], proj[vis, 8:11], rtol=1e-5, atol=2e-6)
    np.testing.assert_allclose(ins["record"][vis, 7], sc.opacities[vis], rtol=0, atol=0)


@pytest.mark.parametrize("case", list(CASES))
def test_sorted_keys_and_ranges_bitexact(lib, case):
    from gpu_helpers import gpu_run
    sc, cam, p = CASES[case]
    got = gpu_run(sc, cam, p)
    kk, vv = oracle.sorted_keys(sc, cam, p)
    assert got["K_tiles"] == kk.size
    assert np.array_equal(got["keys"], kk)
    assert np.array_equal(got["vals"], vv)
    n_tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    ref_ranges = oracle.tile_ranges(kk, n_tiles)
    empty = ref_ranges[:, 0] == ref_ranges[:, 1]
    gr = got["inspect"]["ranges"]
    assert np.array_equal(gr[~empty], ref_ranges[~empty])
    assert np.all(gr[empty, 0] == gr[empty, 1])


@pytest.mark.parametrize("segment_tiles", [1, 2, 16, 1024])
@pytest.mark.parametrize("case", ["tiny", "ragged_lowbeta", "dense_batches"])
def test_segment_width_changes_neither_lists_nor_images(lib, case, segment_tiles):
    """The per-tile lists (expanded from the segment lists) are bit-exact against the oracle for
    every segment width, and the images are identical to those of the default width."""
    from gpu_helpers import gpu_run
    sc, cam, p = CASES[case]
    q = dict(p or {}, segment_tiles=segment_tiles)
    got = gpu_run(sc, cam, q)
    base = gpu_run(sc, cam, p, keys=False)
    kk, vv = oracle.sorted_keys(sc, cam, p)
    assert np.array_equal(got["keys"], kk) and np.array_equal(got["vals"], vv)
    assert np.array_equal(got["img"], base["img"]) and np.array_equal(got["T"], base["T"])
    if segment_tiles == 1:
        assert got["K"] == kk.size  # one entry per (tile, primitive)
    else:
        assert got["K"] <= kk.size


@pytest.mark.parametrize("case", list(CASES))
def test_image_matches_oracle(lib, case):
    from gpu_helpers import gpu_run
    sc, cam, p = CASES[case]
    got = gpu_run(sc, cam, p, keys=False)
    ref = oracle.render(sc, cam, p)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    err = np.abs(got["img"] - ref["img"])[:, ok]
    assert err.max() <= IMG_TOL, err.max()
    assert np.abs(got["T"] - ref["T"])[ok].max() <= T_TOL
    assert got["img"].min() >= 0.0


@pytest.mark.parametrize("case", list(CASES))
def test_gradients_match_oracle(lib, case):
    from gpu_helpers import grad_failures, gpu_run
    sc, cam, p = CASES[case]
    ref = oracle.render(sc, cam, p)
    rng = np.random.default_rng(5)
    g = rng.standard_normal((3, cam.height, cam.width)) * (ref["flags"] == 0)[None]
    got = gpu_run(sc, cam, p, backward_grad=g, keys=False)
    gref = oracle.backward(sc, cam, g, p, cond=True)
    # the compositing stage's per-primitive 2D gradients first (localises a failure)
    inter = got["inspect"]["grad2d"][:, :10].astype(np.float64)
    names2d = ["mx", "my", "ca", "cb", "cc", "kappa", "hb", "r", "g", "b"]
    if p and p.get("mode") == 1:
        names2d.remove("hb")
    cols = {n: inter[:, j] for j, n in enumerate(["mx", "my", "ca", "cb", "cc", "kappa", "hb", "r", "g", "b"])}
    refs = {n: gref["inter"][:, j] for j, n in enumerate(["mx", "my", "ca", "cb", "cc", "kappa", "hb", "r", "g", "b"])}
    conds = {n: gref["cond"]["inter"][:, j] for j, n in enumerate(["mx", "my", "ca", "cb", "cc", "kappa", "hb", "r",
                                                                    "g", "b"])}
    bad = grad_failures(cols, refs, names2d, cond=conds)
    assert not bad, "2D gradients: " + "; ".join(bad)
    bad = grad_failures(got["grads"], gref, cond=gref["cond"])
    assert not bad, "; ".join(bad)


def test_beta2_gef_equals_paper_form_bitwise(lib):
    from gpu_helpers import gpu_run
    sc, cam = scenes.tiny_workload()
    sc.betas[:] = 2.0
    a = gpu_run(sc, cam, None, keys=False)
    b = gpu_run(sc, cam, dict(mode=1), keys=False)
    assert np.array_equal(a["img"], b["img"]) and np.array_equal(a["T"], b["T"])


def test_empty_scene_renders_background(lib):
    from gpu_helpers import gpu_run
    sc = scenes.cube_scene(0, seed=0)
    cam = scenes.tiny_camera(33, 17, bg=(0.25, 0.5, 0.75))
    got = gpu_run(sc, cam)
    assert got["K"] == 0
    assert np.allclose(got["img"], np.array([0.25, 0.5, 0.75], np.float32)[:, None, None])
    assert np.all(got["T"] == 1.0) and np.all(got["nc"] == 0)


def test_all_culled_behind_camera(lib):
    from gpu_helpers import gpu_run
    sc, cam = scenes.tiny_workload()
    sc.means[:, 2] = -10.0  # behind the camera at z = -4
    got = gpu_run(sc, cam)
    assert got["K"] == 0 and np.all(got["inspect"]["depth_key"] == 0xFFFFFFFF)
    assert np.all(got["img"] == 0.0)


def test_single_primitive_one_pixel_image(lib):
    from gpu_helpers import gpu_run
    sc = scenes.cube_scene(1, seed=3)
    sc.means[0] = [0.0, 0.0, 0.0]
    sc.scales[0] = [0.3, 0.3, 0.3]
    cam = scenes.tiny_camera(1, 1)
    got = gpu_run(sc, cam)
    ref = oracle.render(sc, cam)
    assert got["K"] == 1
    assert np.abs(got["img"] - ref["img"]).max() <= IMG_TOL


def test_capacity_overflow_is_reported_then_retry_succeeds(lib):
    from gpu_helpers import gpu_run
    sc, cam = scenes.tiny_workload()
    small = gpu_run(sc, cam, key_capacity=100)
    assert small["status"] == lib.GES_ERR_CAPACITY and small["K"] > 100
    ok = gpu_run(sc, cam, key_capacity=small["K"])
    assert ok["status"] == lib.GES_OK
    kk, vv = oracle.sorted_keys(sc, cam)
    assert np.array_equal(ok["keys"], kk) and np.array_equal(ok["vals"], vv)


def test_invalid_arguments_rejected(lib):
    from paper_2402_10128_gb300 import render
    sc, cam = scenes.tiny_workload()
    t = render.scene_tensors(sc, "cuda")
    fr = render.Frame(sc.n, cam.width, cam.height)
    with pytest.raises(lib.GesError) as e:
        fr.preprocess(t, sc.sh_degree, scenes.tiny_camera(64, 64))
    assert e.value.status == lib.GES_ERR_INVALID_ARG
    with pytest.raises(lib.GesError):
        fr.preprocess(t, 4, cam)
    with pytest.raises(lib.GesError):
        fr.preprocess(t, sc.sh_degree, cam, dict(alpha_min=0.995))
    with pytest.raises(lib.GesError):
        fr.preprocess(t, sc.sh_degree, cam, dict(phi_mode=3))
    with pytest.raises(lib.GesError):
        fr.bin_sort()  # nothing preprocessed yet


def test_autograd_function_matches_oracle(lib):
    from paper_2402_10128_gb300 import render
    sc, cam, _ = CASES["sh3_offaxis"]
    t = [a.requires_grad_(True) for a in render.scene_tensors(sc, "cuda")]
    img, T, nc = render.rasterize(*t, sc.sh_degree, cam)
    ref = oracle.render(sc, cam)
    w = np.random.default_rng(9).standard_normal(img.shape) * (ref["flags"] == 0)[None]
    loss = (img * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    gref = oracle.backward(sc, cam, w, cond=True)
    from gpu_helpers import NAMES, grad_failures
    got = {n: a.grad.detach().cpu().double().numpy().reshape(gref[n].shape) for n, a in zip(NAMES, t)}
    bad = grad_failures(got, gref, cond=gref["cond"])
    assert not bad, "; ".join(bad)
