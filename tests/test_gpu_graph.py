"""A frame's four calls (preprocess, bin_sort, render_fwd, render_bwd) captured into a CUDA graph
and replayed: the image and final transmittance equal the direct calls' bit for bit, and the
gradients agree with them as closely as two direct runs agree with each other (the order of the
atomics); the replay also matches the FP64 oracle like the direct path does."""
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
    from paper_2402_10128_gb300 import ges, render
    return ges, render


def test_captured_frame_replays_the_direct_calls(lib):
    ges, render = lib
    sc = scenes.cube_scene(3000, seed=61, sh_degree=1, beta_range=(0.5, 6.0), beta_log=True)
    cams = [scenes.tiny_camera(150, 110), scenes.look_at((1.5, -0.5, -3.5), (0, 0, 0), (0, -1, 0), 150, 110, 55.0)]
    t = render.scene_tensors(sc, "cuda")
    fr = render.Frame(sc.n, 150, 110, key_capacity=2_000_000)
    scene_c = ges.make_scene(*t, sc.sh_degree)
    params = ges.params_default()
    img = torch.empty((3, 110, 150), device="cuda")
    T = torch.empty((110, 150), device="cuda")
    nc = torch.empty((110, 150), dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(62)
    dL = torch.as_tensor(rng.standard_normal((3, 110, 150)).astype(np.float32) * 1e-3, device="cuda")
    grads = tuple(torch.empty_like(a) for a in t)
    grads_c = ges.make_grads(*grads)
    sp0 = torch.cuda.current_stream().cuda_stream

    def calls(cam, sp):
        ges.ges_preprocess(fr.handle, scene_c, cam, params, sp)
        ges.ges_bin_sort(fr.handle, sp)
        ges.ges_render_fwd(fr.handle, img, T, nc, sp)
        ges.ges_render_bwd(fr.handle, scene_c, T, nc, dL, grads_c, sp)

    def direct(cam):
        calls(cam, sp0)
        torch.cuda.synchronize()
        return [img.clone(), T.clone()] + [g.clone() for g in grads]

    gcams = [ges.make_camera(c) for c in cams]
    for cam in gcams:     # warm up (allocations, attributes) before capturing
        direct(cam)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graphs = []
    for cam in gcams:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            calls(cam, s.cuda_stream)
        graphs.append(g)

    def rel(a, b):
        return float((a - b).norm()) / max(float(a.norm()), 1e-30)

    for k, (cam, ocam) in enumerate(zip(gcams, cams)):
        ref, ref2 = direct(cam), direct(cam)
        img.zero_()
        graphs[k].replay()
        torch.cuda.synchronize()
        got = [img, T] + list(grads)
        assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
        for a, a2, b in zip(ref[2:], ref2[2:], got[2:]):
            assert rel(a, b) <= max(10 * rel(a, a2), 1e-5)
        out = oracle.render(sc, ocam)
        ok = out["flags"] == 0
        assert np.abs(got[0].cpu().numpy() - out["img"])[:, ok].max() <= 1e-4
    st, K = ges.ges_frame_status(fr.handle)
    assert st == ges.GES_OK and K > 0
    fr.close()
