"""The batched 1D mixture fits on the GPU (ges_signal1d, ges_fit1d) against the FP64 oracle
(oracle/mixture1d.py), each side computing its own samples and targets from the same definitions
and starting from the same seeded parameters.

Bars:
* signals: FP64 within 1e-14, FP32 within 1e-6, away from the support's edges;
* the loss and gradient at the initial parameters: FP64 within 1e-12 / 1e-10 relative, FP32 within
  1e-5 / 1e-4 relative (per run, L2 over the parameters);
* 20 Adam steps: FP64 parameters within 1e-9 relative and the loss history within 1e-10.  FP32:
  the history within 1e-4 relative for the first 5 steps and 1e-2 after (FP32 GEF fits drift
  fastest: up to 3e-3 measured), 95% of the parameters within 1e-4 (|p| + 20 lr) and all within
  Adam's reach (2 x 20 lr: where a gradient is near 0 its FP32 sign may differ);
* 1000 steps: runs can branch on rounding where their dynamics are not smooth (see the test), so
  FP64 is held to: the same runs unstable (NaN), every final loss below the initial one, and at
  least half of the runs equal to 1e-9; FP32 to the statistics: its final loss within a factor 2
  of the oracle's for at least 75% of the runs, and the same ranking of the GEF against the
  Gaussian mixture on the square.
"""
import numpy as np
import pytest

from oracle import mixture1d as om
from paper_2402_10128_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

S = 1000


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_2402_10128_gb300 import ges, render
    return ges, render.default_context(0)


def _gpu_signals(ges, ctx, kinds, n, dtype, width=1.0):
    x = torch.empty(n, dtype=dtype, device="cuda")
    ys = torch.empty((len(kinds), n), dtype=dtype, device="cuda")
    for i, k in enumerate(kinds):
        ges.ges_signal1d(ctx.handle, k, x, ys[i], width=width)
    return x, ys


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [1000, 777])
def test_signals_match_the_oracle(lib, dtype, n):
    ges, ctx = lib
    x, ys = _gpu_signals(ges, ctx, om.SIGNALS, n, dtype, width=1.0)
    torch.cuda.synchronize()
    xr = np.linspace(-1.0, 1.0, n)
    tol = 1e-14 if dtype == torch.float64 else 1e-6
    np.testing.assert_allclose(x.cpu().double().numpy(), xr, rtol=0, atol=tol)
    sure = np.abs(np.abs(xr) - 0.5) > 1e-6
    for i, k in enumerate(om.SIGNALS):
        np.testing.assert_allclose(ys[i].cpu().double().numpy()[sure], om.signal(k, xr)[sure], rtol=0, atol=tol)


def _fit_gpu(ges, ctx, model, n_comp, p0, kinds, epochs, dtype, positive=True, hist=True, grad=True):
    runs = p0.shape[0]
    x, ys = _gpu_signals(ges, ctx, om.SIGNALS, S, dtype)
    idx = torch.as_tensor([om.SIGNALS.index(k) for k in kinds], device="cuda")
    y = ys[idx].contiguous()
    params = torch.as_tensor(p0, dtype=dtype, device="cuda").contiguous()
    fl = torch.empty(runs, dtype=dtype, device="cuda")
    lh = torch.empty((runs, epochs + 1), dtype=dtype, device="cuda") if hist else None
    gr = torch.empty_like(params) if grad else None
    prec = 64 if dtype == torch.float64 else 32
    p = ges.fit1d_params_default(model=ges.MIX_MODELS[model], n_components=n_comp, positive_weights=int(positive),
                                 epochs=epochs, precision=prec)
    ges.ges_fit1d(ctx.handle, p, x, y, params, fl, lh, gr)
    torch.cuda.synchronize()
    out = dict(params=params.cpu().double().numpy(), final=fl.cpu().double().numpy())
    if hist:
        out["hist"] = lh.cpu().double().numpy()
    if grad:
        out["grad"] = gr.cpu().double().numpy()
    return out


def _fit_ref(model, p0, kinds, epochs, positive=True):
    x = np.linspace(-1.0, 1.0, S)
    res = [om.fit(model, p0[r], x, om.signal(k, x), epochs, positive) for r, k in enumerate(kinds)]
    return dict(params=np.stack([r[0] for r in res]), hist=np.stack([r[1] for r in res]),
                grad=np.stack([r[2] for r in res]))


def _kinds(runs):
    return [om.SIGNALS[r % len(om.SIGNALS)] for r in range(runs)]


@pytest.mark.parametrize("model", om.MODELS)
@pytest.mark.parametrize("n_comp", [1, 5, 20, 128])
@pytest.mark.parametrize("positive", [True, False])
def test_loss_and_gradient_at_the_start(lib, model, n_comp, positive):
    ges, ctx = lib
    runs = 6
    p0 = scenes.mixture_init(model, n_comp, runs, seed=n_comp)
    kinds = _kinds(runs)
    ref = _fit_ref(model, p0, kinds, 0, positive)
    for dtype, tl, tg in ((torch.float64, 1e-12, 1e-10), (torch.float32, 1e-5, 1e-4)):
        got = _fit_gpu(ges, ctx, model, n_comp, p0, kinds, 0, dtype, positive)
        np.testing.assert_allclose(got["final"], ref["hist"][:, 0], rtol=tl)
        for r in range(runs):
            err = np.linalg.norm(got["grad"][r] - ref["grad"][r]) / np.linalg.norm(ref["grad"][r])
            assert err <= tg, (dtype, r, err)


@pytest.mark.parametrize("model", om.MODELS)
def test_twenty_steps(lib, model):
    ges, ctx = lib
    runs, n_comp, E = 12, 8, 20
    p0 = scenes.mixture_init(model, n_comp, runs, seed=7)
    kinds = _kinds(runs)
    ref = _fit_ref(model, p0, kinds, E)
    got = _fit_gpu(ges, ctx, model, n_comp, p0, kinds, E, torch.float64)
    np.testing.assert_allclose(got["hist"], ref["hist"], rtol=1e-10)
    np.testing.assert_allclose(got["params"], ref["params"], rtol=1e-9, atol=1e-12)
    got = _fit_gpu(ges, ctx, model, n_comp, p0, kinds, E, torch.float32)
    rel = np.abs(got["hist"] - ref["hist"]) / np.abs(ref["hist"])
    assert rel[:, :5].max() <= 1e-4 and rel.max() <= 1e-2, rel.max(0)
    # Adam moves a parameter by about lr whatever its gradient's size, so where a gradient is near 0
    # its FP32 sign may differ: most parameters agree closely, none by more than Adam's reach
    dp = np.abs(got["params"] - ref["params"])
    assert np.mean(dp <= 1e-4 * (np.abs(ref["params"]) + E * 0.01)) >= 0.95
    assert dp.max() <= 2 * E * 0.01


@pytest.fixture(scope="module")
def long_runs(lib):
    """1000 steps, N = 5, every model on every signal (24 runs; the oracle takes about 15 s)."""
    ges, ctx = lib
    out = {}
    for model in om.MODELS:
        p0 = scenes.mixture_init(model, 5, 6, seed=21)
        kinds = list(om.SIGNALS)
        ref = _fit_ref(model, p0, kinds, 1000)
        g64 = _fit_gpu(ges, ctx, model, 5, p0, kinds, 1000, torch.float64, hist=False, grad=False)
        g32 = _fit_gpu(ges, ctx, model, 5, p0, kinds, 1000, torch.float32, hist=False, grad=False)
        out[model] = (ref, g64, g32)
    return out


def test_thousand_steps_fp64_match(long_runs):
    """Over 1000 steps a run can pass a point where its dynamics are not smooth (a weight through 0,
    where d|omega|/d omega jumps, or a gradient through 0 under Adam's normalisation); from there
    rounding decides the branch, in FP64 as well (measured: a 3e-11 difference at step 50 grew to
    0.1 by step 100).  So: every run stable or unstable on both sides alike, every final loss below
    the initial one on both sides, and most runs (at least half; 18 of 24 measured) equal to 1e-9."""
    same, total = 0, 0
    for model, (ref, g64, _) in long_runs.items():
        a, b = ref["hist"][:, -1], g64["final"]
        assert np.array_equal(np.isnan(a), np.isnan(b)), model
        ok = ~np.isnan(a)
        assert np.all(a[ok] < ref["hist"][ok, 0]) and np.all(b[ok] < ref["hist"][ok, 0]), model
        same += int((np.abs(b[ok] - a[ok]) <= 1e-9 * a[ok]).sum())
        total += int(ok.sum())
    assert same >= total / 2, (same, total)


def test_thousand_steps_fp32_statistics(long_runs):
    ratios = []
    for model, (ref, _, g32) in long_runs.items():
        a, b = ref["hist"][:, -1], g32["final"]
        ok = ~np.isnan(a) & ~np.isnan(b)
        ratios += list(np.maximum(a[ok], b[ok]) / np.maximum(np.minimum(a[ok], b[ok]), 1e-30))
    assert np.mean(np.array(ratios) <= 2.0) >= 0.75, ratios
    sq = om.SIGNALS.index("square")
    assert long_runs["gef"][2]["final"][sq] < long_runs["gaussian"][2]["final"][sq]
    assert long_runs["gef"][0]["hist"][sq, -1] < long_runs["gaussian"][0]["hist"][sq, -1]


def test_unstable_run_reports_nan(lib):
    """A LoG component of zero scale divides by zero: the oracle's loss is NaN from the start, and
    so is the GPU's, with NaN parameters; the other runs of the batch are unaffected."""
    ges, ctx = lib
    p0 = scenes.mixture_init("log", 3, 2, seed=1)
    p0[0, 2, 1] = 0.0
    ref = _fit_ref("log", p0, ["square", "square"], 10)
    got = _fit_gpu(ges, ctx, "log", 3, p0, ["square", "square"], 10, torch.float64)
    assert np.isnan(ref["hist"][0]).all() and np.isnan(got["hist"][0]).all() and np.isnan(got["params"][0]).all()
    np.testing.assert_allclose(got["hist"][1], ref["hist"][1], rtol=1e-10)
