"""The training-side updates on the GPU (ges_adam_step, ges_activate, ges_densify_stats,
ges_density_control, resets) against the FP64 oracle (oracle/train.py), on the same seeded inputs.

Bars (FP32 against FP64 on FP32 inputs):
* Adam (both sides step from the same seeded state, each on its own trajectory): per step,
  moments within 1e-6 of (|old moment| + |term added|), variables within 2e-7 |p| +
  1e-5 lr (1 + |update / lr| + the update's sensitivity to the first moment's rounding), these
  bars times the number of steps taken; physical values within 1e-6 relative plus the variable's
  error carried through the activation;
* densification statistics: counts exact, sums within 1e-3 relative (they are gradient norms);
* density control: the row decisions and counts exact (both sides decide in FP32 against the same
  FP32 thresholds); copied rows and moments bit-exact; the children's means within 1e-6 of their
  magnitude, their log-scales within 2 ulp;
* resets exact up to the threshold's rounding.
Row counts are ragged (not multiples of 4) so the kernels' 4-element tails run.
"""
import numpy as np
import pytest

import oracle
from oracle import train as ot
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = ot.GROUPS


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges, render
    return ges, render.default_context(0)


def _dev(d):
    return {k: torch.as_tensor(np.ascontiguousarray(d[k])).cuda() for k in G}


def _host(d):
    return {k: d[k].cpu().numpy() for k in G}


def _set(ges, n, sh, p, m, v):
    return ges.make_train_set(n, sh, [p[k] for k in G], [m[k] for k in G], [v[k] for k in G])


def _f64(d):
    return {k: np.asarray(a, np.float64) for k, a in d.items()}


@pytest.mark.parametrize("n,sh", [(1037, 3), (333, 0), (50, 2)])
def test_adam_steps_match_the_oracle(lib, n, sh):
    """Four steps from the same seeded state on both sides (the oracle follows its own trajectory);
    the per-step bars grow linearly with the step count, as FP32 rounding adds up step by step."""
    ges, ctx = lib
    w = scenes.optimizer_workload(n, sh, seed=n)
    p, m, v = _dev(w["raw"]), _dev(w["m"]), _dev(w["v"])
    phys = {k: torch.empty_like(p[k]) for k in G}
    ts = _set(ges, n, sh, p, m, v)
    hp = ges.adam_params_default()
    hpd = dict(lr_means=float(hp.lr[0]), lr_scales=float(hp.lr[1]), lr_quats=float(hp.lr[2]),
               lr_betas=float(hp.lr[3]), lr_opacities=float(hp.lr[4]), lr_sh_dc=float(hp.lr[5]),
               lr_sh_rest=float(hp.lr_sh_rest), beta1=float(hp.beta1), beta2=float(hp.beta2), eps=float(hp.eps))
    b1, b2 = float(hp.beta1), float(hp.beta2)
    r0, m0, v0 = _f64(w["raw"]), _f64(w["m"]), _f64(w["v"])
    rng = np.random.default_rng(n + 1)
    for k_step, step in enumerate((1, 2, 3, 10), start=1):
        gr = {k: (w["grads"][k] * rng.uniform(0.5, 1.5, w["grads"][k].shape)).astype(np.float32) for k in G}
        gd = _dev(gr)
        ges.ges_adam_step(ctx.handle, ts, ges.make_grads(*[gd[k] for k in G]),
                          ges.make_scene_out(*[phys[k] for k in G]), hp, step)
        torch.cuda.synchronize()
        r1, m1, v1, ph1 = ot.adam_step(r0, m0, v0, _f64(gr), step, hpd)
        graw = ot.raw_gradient(r0, _f64(gr))
        hp_lr = {"means": hp.lr[0], "scales": hp.lr[1], "quats": hp.lr[2], "betas": hp.lr[3], "opacities": hp.lr[4]}
        c1, c2 = 1.0 - b1 ** step, 1.0 - b2 ** step
        for k in G:
            gp, gm, gv, gph = (a[k].cpu().double().numpy() for a in (p, m, v, phys))
            assert np.all(np.abs(gm - m1[k]) <= k_step * 1e-6 * (np.abs(b1 * m0[k]) + np.abs((1 - b1) * graw[k]))
                          + 1e-30), k
            assert np.all(np.abs(gv - v1[k]) <= k_step * 1e-6 * (np.abs(b2 * v0[k]) + np.abs((1 - b2) * graw[k] ** 2))
                          + 1e-30), k
            if k == "shs":
                lr = np.full(r0[k].reshape(n, -1).shape, float(hp.lr_sh_rest))
                lr[:, :3] = float(hp.lr[5])
                lr = lr.reshape(r0[k].shape)
            else:
                lr = float(hp_lr[k])
            upd = np.abs(r0[k] - r1[k]) / lr
            # how far the update moves when the new first moment does by its rounding (cancellation)
            sens = (np.abs(b1 * m0[k]) + np.abs((1 - b1) * graw[k])) / c1 / (np.sqrt(v1[k] / c2) + float(hp.eps))
            dp = np.abs(gp - r1[k])
            assert np.all(dp <= k_step * (2e-7 * np.abs(r1[k]) + 1e-5 * lr * (1 + upd + sens))), k
            slope = {"scales": np.abs(ph1[k]), "opacities": 0.25}.get(k, 1.0)
            assert np.all(np.abs(gph - ph1[k]) <= 1e-6 * np.abs(ph1[k]) + slope * dp + 1e-30), k
        r0, m0, v0 = r1, m1, v1


def test_activate_matches_the_oracle(lib):
    ges, ctx = lib
    w = scenes.optimizer_workload(777, 3, seed=3)
    p, m, v = _dev(w["raw"]), _dev(w["m"]), _dev(w["v"])
    phys = {k: torch.empty_like(p[k]) for k in G}
    ges.ges_activate(ctx.handle, _set(ges, 777, 3, p, m, v), ges.make_scene_out(*[phys[k] for k in G]))
    torch.cuda.synchronize()
    ref = ot.activate(_f64(w["raw"]))
    for k in G:
        np.testing.assert_allclose(phys[k].cpu().double().numpy(), ref[k], rtol=1e-6, atol=0)
    for k in G:   # the variables and moments are untouched
        assert np.array_equal(p[k].cpu().numpy(), w["raw"][k]) and np.array_equal(m[k].cpu().numpy(), w["m"][k])


def test_densify_stats_match_the_oracle(lib):
    """Two views of a small scene, each rendered, differentiated and added to the statistics."""
    ges, ctx = lib
    from paper_2402_10128_gb300 import render
    sc = scenes.cube_scene(601, seed=31, scale_range=(0.02, 0.1))
    # the second view sees about half of the primitives
    cams = [scenes.tiny_camera(90, 70), scenes.look_at((0.6, -0.3, -2.0), (0.9, 0, 0), (0, -1, 0), 90, 70, 50.0)]
    t = render.scene_tensors(sc, "cuda")
    acc = torch.zeros(sc.n, device="cuda")
    cnt = torch.zeros(sc.n, dtype=torch.int32, device="cuda")
    ref_acc, ref_cnt = None, None
    fr = render.Frame(sc.n, 90, 70)
    for i, cam in enumerate(cams):
        ref = oracle.render(sc, cam)
        g = np.random.default_rng(40 + i).standard_normal((3, cam.height, cam.width)) * (ref["flags"] == 0)[None]
        img, T, nc = fr.forward(t, sc.sh_degree, cam)
        fr.render_bwd(T, nc, torch.as_tensor(g, dtype=torch.float32, device="cuda"))
        ges.ges_densify_stats(fr.handle, acc, cnt)
        touched = oracle.keys(sc, cam)["touched"]
        inter = oracle.backward(sc, cam, g)["inter"]
        ref_acc, ref_cnt = ot.densify_stats(touched, inter, cam.width, cam.height, ref_acc, ref_cnt)
    torch.cuda.synchronize()
    fr.close()
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    a = acc.cpu().double().numpy()
    assert np.linalg.norm(a - ref_acc) <= 1e-3 * np.linalg.norm(ref_acc)
    assert np.all(np.abs(a - ref_acc) <= 1e-3 * np.abs(ref_acc) + 1e-3 * np.abs(ref_acc).max())
    assert (ref_cnt == 2).sum() > 100 and (ref_cnt < 2).sum() > 0


def _run_density(ges, ctx, w, n, sh, cap, **kw):
    p, m, v = _dev(w["raw"]), _dev(w["m"]), _dev(w["v"])
    ts = _set(ges, n, sh, p, m, v)
    op = {k: torch.full((cap,) + tuple(p[k].shape[1:]), np.nan, device="cuda") for k in G}
    om = {k: torch.full_like(op[k], np.nan) for k in G}
    ov = {k: torch.full_like(op[k], np.nan) for k in G}
    tout = _set(ges, cap, sh, op, om, ov)
    names = dict(grad_threshold="grad_threshold", percent_dense="percent_dense", extent="scene_extent",
                 min_opacity="min_opacity", min_beta="min_beta", max_world="max_world_size")
    dp = ges.density_params_default(**{names[k]: val for k, val in kw.items()})
    acc = torch.as_tensor(w["accum"]).cuda()
    cnt = torch.as_tensor(w["count"]).cuda()
    xi = torch.as_tensor(w["xi"]).cuda()
    k_out = ges.ges_density_control(ctx.handle, ts, acc, cnt, xi, dp, tout)
    torch.cuda.synchronize()
    return k_out, _host(op), _host(om), _host(ov)


@pytest.mark.parametrize("kw", [dict(), dict(min_beta=0.5, max_world=0.1, extent=1.0),
                                dict(extent=3.0, percent_dense=0.005), dict(grad_threshold=1e9, min_beta=0.5)])
def test_density_control_matches_the_oracle(lib, kw):
    ges, ctx = lib
    n, sh = 4099, 3
    w = scenes.optimizer_workload(n, sh, seed=17)
    k_out, op, om, ov = _run_density(ges, ctx, w, n, sh, 3 * n, **kw)
    ref, rm, rv, d = ot.density_control(_f64(w["raw"]), _f64(w["m"]), _f64(w["v"]), w["accum"], w["count"],
                                        w["xi"].astype(np.float64), **kw)
    assert k_out == ref["means"].shape[0]
    nk, nc, ns = int(d["keep"].sum()), int(d["clone"].sum()), int(d["child"].sum())
    assert nk + nc + 2 * ns == k_out
    if kw.get("grad_threshold", 0) < 1:
        assert nc > 0 and ns > 0
    copied = slice(0, nk + nc)
    for k in G:
        assert np.array_equal(op[k][copied], ref[k][copied].astype(np.float32)), k
        assert np.array_equal(om[k][:k_out], rm[k].astype(np.float32)), k
        assert np.array_equal(ov[k][:k_out], rv[k].astype(np.float32)), k
        if k not in ("means", "scales"):
            assert np.array_equal(op[k][nk + nc:k_out], ref[k][nk + nc:].astype(np.float32)), k
        assert np.all(np.isnan(op[k][k_out:])), k      # nothing written past the rows it reports
    kids = slice(nk + nc, k_out)
    mu = ref["means"][kids]
    assert np.all(np.abs(op["means"][kids] - mu) <= 1e-6 * (1.0 + np.abs(mu)))
    ls = ref["scales"][kids]
    assert np.all(np.abs(op["scales"][kids] - ls) <= 2 * np.spacing(np.abs(ls).astype(np.float32)))


def test_density_control_capacity_and_edge_cases(lib):
    ges, ctx = lib
    n, sh = 513, 1
    w = scenes.optimizer_workload(n, sh, seed=19)
    ref, _, _, _ = ot.density_control(_f64(w["raw"]), _f64(w["m"]), _f64(w["v"]), w["accum"], w["count"],
                                      w["xi"].astype(np.float64))
    need = ref["means"].shape[0]
    with pytest.raises(ges.GesError) as e:
        _run_density(ges, ctx, w, n, sh, need - 1)
    assert e.value.status == ges.GES_ERR_CAPACITY and e.value.n_out == need
    k_out, _, _, _ = _run_density(ges, ctx, w, n, sh, need)          # exactly enough
    assert k_out == need
    # everything transparent: nothing survives
    w0 = dict(w, raw=dict(w["raw"], opacities=np.full(n, -20.0, np.float32)))
    k_out, _, _, _ = _run_density(ges, ctx, w0, n, sh, 2 * n)
    assert k_out == 0


def test_resets_match_the_oracle(lib):
    ges, ctx = lib
    n = 1001
    w = scenes.optimizer_workload(n, 0, seed=23)
    p, m, v = _dev(w["raw"]), _dev(w["m"]), _dev(w["v"])
    ts = _set(ges, n, 0, p, m, v)
    ges.ges_reset_opacity(ctx.handle, ts, 0.01)
    ges.ges_reset_shape(ctx.handle, ts, 2.0)
    torch.cuda.synchronize()
    r, mm, vv = ot.reset_opacity(_f64(w["raw"]), _f64(w["m"]), _f64(w["v"]))
    r, mm, vv = ot.reset_shape(r, mm, vv)
    gp, gm, gv = _host(p), _host(m), _host(v)
    np.testing.assert_allclose(gp["opacities"], r["opacities"], rtol=1e-7)
    assert np.all(gp["betas"] == 0.0)
    for k in G:
        assert np.array_equal(gm[k], mm[k].astype(np.float32)) and np.array_equal(gv[k], vv[k].astype(np.float32)), k
        if k not in ("opacities", "betas"):
            assert np.array_equal(gp[k], w["raw"][k]), k


def test_training_loop_reduces_the_loss(lib):
    """Forty steps of render -> image loss -> backward -> statistics -> Adam through the C-ABI fit a
    perturbed scene toward a target image rendered from the original (the loss falls by half)."""
    ges, ctx = lib
    from paper_2402_10128_gb300 import render
    sc = scenes.cube_scene(800, seed=51, scale_range=(0.03, 0.1))
    cam = scenes.tiny_camera(96, 80)
    target, _, _ = render.Frame(sc.n, 96, 80).forward(render.scene_tensors(sc, "cuda"), sc.sh_degree, cam)
    target = target.clone()
    rng = np.random.default_rng(52)
    raw = dict(means=sc.means + rng.normal(0, 0.03, sc.means.shape), scales=np.log(sc.scales),
               quats=sc.quats, betas=sc.betas - 2.0, opacities=np.log(sc.opacities / (1 - sc.opacities)),
               shs=sc.shs + rng.normal(0, 0.3, sc.shs.shape))
    raw = {k: np.asarray(a, np.float32) for k, a in raw.items()}
    p = _dev(raw)
    m = {k: torch.zeros_like(p[k]) for k in G}
    v = {k: torch.zeros_like(p[k]) for k in G}
    phys = {k: torch.empty_like(p[k]) for k in G}
    ts = _set(ges, sc.n, sc.sh_degree, p, m, v)
    so = ges.make_scene_out(*[phys[k] for k in G])
    ges.ges_activate(ctx.handle, ts, so)
    hp = ges.adam_params_default()
    hp.lr[0] = 1e-3
    hp.lr[5] = 0.02
    fr = render.Frame(sc.n, 96, 80)
    mask = torch.ones((80, 96), dtype=torch.uint8, device="cuda")
    loss = torch.empty(4, device="cuda")
    dL = torch.empty((3, 80, 96), device="cuda")
    acc = torch.zeros(sc.n, device="cuda")
    cnt = torch.zeros(sc.n, dtype=torch.int32, device="cuda")
    grads = tuple(torch.empty_like(phys[k]) for k in G)
    losses = []
    steps = 40
    for step in range(1, steps + 1):
        img, T, nc = fr.forward(tuple(phys[k] for k in G), sc.sh_degree, cam)
        ges.ges_image_loss(ctx.handle, img, target, mask, 96, 80, loss, dL, lambda_ssim=0.2, lambda_omega=0.0)
        fr.render_bwd(T, nc, dL, grads)
        ges.ges_densify_stats(fr.handle, acc, cnt)
        ges.ges_adam_step(ctx.handle, ts, ges.make_grads(*grads), so, hp, step)
        losses.append(float(loss[0]))
    torch.cuda.synchronize()
    fr.close()
    assert losses[-1] < 0.5 * losses[0], losses
    assert int(cnt.max()) == steps
