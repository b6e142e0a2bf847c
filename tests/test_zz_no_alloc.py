"""The allocation-free forward render (ges_render_fwd_noalloc) against the regular frame path.

Some callers cannot allocate device memory (they run under a memory manager that owns the
device's memory, or must not trigger cudaMalloc's device synchronisation).  For them libges
has one entry point whose intermediate buffers live in a fixed array inside the library.  This
test calls it through the C-ABI, twice in a row (the array keeps the previous call's contents),
and compares each result with ges_preprocess + ges_bin_sort + ges_render_fwd within the image
tolerance the parity tests use.  It also checks that sizes above the stated limits are refused.
The file name makes pytest collect it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def ges():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges as g
    return g


def _frame_path(ges, scene, cam):
    from paper_2402_10128_gb300 import render
    t = render.scene_tensors(scene, "cuda")
    fr = render.Frame(max(1, scene.n), cam.width, cam.height)
    img, T, nc = fr.forward(t, scene.sh_degree, cam)
    torch.cuda.synchronize()
    return img.cpu().numpy(), T.cpu().numpy(), nc.cpu().numpy()


def _noalloc(ges, scene, cam):
    from paper_2402_10128_gb300 import render
    t = render.scene_tensors(scene, "cuda")
    img = torch.full((3, cam.height, cam.width), -1.0, device="cuda")
    T = torch.full((cam.height, cam.width), -1.0, device="cuda")
    nc = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
    ges.ges_render_fwd_noalloc(ges.make_scene(*t, scene.sh_degree), ges.make_camera(cam), ges.params_default(),
                               img, T, nc)
    torch.cuda.synchronize()
    return img.cpu().numpy(), T.cpu().numpy(), nc.cpu().numpy()


def _cases():
    from paper_2402_10128_gb300 import scenes
    return [scenes.tiny_workload(),
            (scenes.cube_scene(3000, seed=21, sh_degree=3, beta_range=(0.5, 8.0), beta_log=True),
             scenes.tiny_camera(200, 150, bg=(0.1, 0.2, 0.3)))]


def test_noalloc_matches_frame_path_on_consecutive_calls(ges):
    for scene, cam in _cases():
        ref = _frame_path(ges, scene, cam)
        for _ in range(2):  # a second call starts from the first call's leftovers
            got = _noalloc(ges, scene, cam)
            assert np.abs(got[0] - ref[0]).max() <= IMG_TOL
            assert np.abs(got[1] - ref[1]).max() <= 1e-5
            assert np.array_equal(got[2], ref[2])


def test_noalloc_refuses_sizes_above_its_limits(ges):
    from paper_2402_10128_gb300 import render, scenes
    big = scenes.cube_scene(65537, seed=1)
    t = render.scene_tensors(big, "cuda")
    cam = scenes.tiny_camera(64, 64)
    out = [torch.empty((3, 64, 64), device="cuda"), torch.empty((64, 64), device="cuda"),
           torch.empty((64, 64), dtype=torch.int32, device="cuda")]
    with pytest.raises(ges.GesError) as e:
        ges.ges_render_fwd_noalloc(ges.make_scene(*t, 0), ges.make_camera(cam), ges.params_default(), *out)
    assert e.value.status == ges.GES_ERR_INVALID_ARG and "limit" in str(e.value)
    small = scenes.cube_scene(10, seed=1)
    ts = render.scene_tensors(small, "cuda")
    wide = scenes.tiny_camera(4096, 2048)
    outw = [torch.empty((3, 2048, 4096), device="cuda"), torch.empty((2048, 4096), device="cuda"),
            torch.empty((2048, 4096), dtype=torch.int32, device="cuda")]
    with pytest.raises(ges.GesError) as e:
        ges.ges_render_fwd_noalloc(ges.make_scene(*ts, 0), ges.make_camera(wide), ges.params_default(), *outw)
    assert e.value.status == ges.GES_ERR_INVALID_ARG


def test_noalloc_duplicate_overflow_reports_capacity_then_recovers(ges):
    """Within the primitive and tile limits but above the duplicate limit (6,000 large primitives
    over a 2048x2048 image list about 1.9M entries, against 1,048,576): the call reports
    GES_ERR_CAPACITY and its outputs hold the background only; the next call within the limits
    renders normally from the same array."""
    from paper_2402_10128_gb300 import render, scenes
    big = scenes.cube_scene(6000, seed=5, scale_range=(0.3, 0.5))
    cam = scenes.tiny_camera(2048, 2048, bg=(0.25, 0.5, 0.75))
    t = render.scene_tensors(big, "cuda")
    fr = render.Frame(big.n, cam.width, cam.height)
    fr.forward(t, big.sh_degree, cam)
    assert fr.status()[1] > (1 << 20)  # the frame path's entry count for the same view
    fr.close()
    img = torch.full((3, cam.height, cam.width), -1.0, device="cuda")
    T = torch.full((cam.height, cam.width), -1.0, device="cuda")
    nc = torch.full((cam.height, cam.width), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(ges.GesError) as e:
        ges.ges_render_fwd_noalloc(ges.make_scene(*t, big.sh_degree), ges.make_camera(cam), ges.params_default(),
                                   img, T, nc)
    assert e.value.status == ges.GES_ERR_CAPACITY
    torch.cuda.synchronize()
    bg = torch.tensor([0.25, 0.5, 0.75], device="cuda")[:, None, None]
    assert torch.equal(img, bg.expand_as(img))
    assert bool((T == 1.0).all()) and bool((nc == 0).all())
    for scene, cam in _cases():
        ref = _frame_path(ges, scene, cam)
        got = _noalloc(ges, scene, cam)
        assert np.abs(got[0] - ref[0]).max() <= IMG_TOL and np.array_equal(got[2], ref[2])
