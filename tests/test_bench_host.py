"""Host-side pieces of bench.py that need no GPU: the composites' FP32 operation counts behind the
roofline's FP32 floor, restated here from the equations they count."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_composite_fp32_counts():
    b = _bench()
    # falloff per in-extent pair: d (2), q = (a dx + 2b dy) dx + c dy^2 (5), beta/2 log2 q (1),
    # -log2(e)/2 p (1), kappa G (1); the Gaussian form has no q^(beta/2)
    assert (b.FP32_EVAL_GEF, b.FP32_EVAL_GAUSS) == (2 + 5 + 1 + 1 + 1, 2 + 5 + 1 + 1)
    # forward per composited pair: 1 - alpha, T (1 - alpha), alpha T, three colour FMAs
    assert b.FP32_FWD == 1 + 1 + 1 + 3
    # backward per composited pair: T recovery and alpha T (3), D (3), dL/dalpha (2), U (1),
    # kappa (1), p (2), q (3) and beta (1) for the GEF only, dq/dd (2), mean (4), conic (3),
    # colour (3), and the 10 adds summing the pair's 10 terms
    gef = 3 + 3 + 2 + 1 + 1 + 2 + 3 + 1 + 2 + 4 + 3 + 3 + 10
    assert (b.FP32_BWD_GEF, b.FP32_BWD_GAUSS) == (gef, gef - 4)
    fwd, bwd = b.composite_fp32_ops(True, 100, 80)
    assert (fwd, bwd) == (100 * b.FP32_EVAL_GEF + 80 * b.FP32_FWD, 100 * b.FP32_EVAL_GEF + 80 * b.FP32_BWD_GEF)
    fwd, bwd = b.composite_fp32_ops(False, 100, 80)
    assert (fwd, bwd) == (100 * b.FP32_EVAL_GAUSS + 80 * b.FP32_FWD, 100 * b.FP32_EVAL_GAUSS + 80 * b.FP32_BWD_GAUSS)
