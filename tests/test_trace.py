"""Kernel tracing (ges_trace_enable / ges_trace_read): names, launch counts and positive device
times for one forward + backward pass, and an empty record after a read."""
import numpy as np
import pytest

from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_trace_records_each_stage_once_per_pass():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_10128_gb300 import ges, render
    sc, cam = scenes.tiny_workload()
    ctx = render.Context(0)
    try:
        t = render.scene_tensors(sc, "cuda")
        fr = render.Frame(sc.n, cam.width, cam.height, ctx=ctx)
        ges.ges_trace_enable(ctx.handle, True)
        for _ in range(2):
            img, T, nc = fr.forward(t, sc.sh_degree, cam)
            fr.render_bwd(T, nc, torch.ones_like(img))
        got = ges.ges_trace_read(ctx.handle)
        ges.ges_trace_enable(ctx.handle, False)
        names = list(got)
        # the single-pass list sort of this view's segment ids also writes the segment ranges
        assert names == ["k_preprocess", "depth_sort", "scan_touched", "k_keygen", "list_sort",
                         "k_render_fwd", "tile_order", "k_render_bwd", "k_preprocess_bwd"]
        assert all(n == 2 for n, _ in got.values())
        assert all(ms > 0.0 for _, ms in got.values())
        assert ges.ges_trace_read(ctx.handle) == {}
        fr.close()
    finally:
        ctx.close()
