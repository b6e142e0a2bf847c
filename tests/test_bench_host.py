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


def test_headline_line_is_short_and_complete():
    """The headline is the last line of the bench's output; a log tail of a few KB must hold it
    whole, with the keys the measurement is judged by."""
    import json
    b = _bench()
    roof = {"kernel": "k_render_bwd (backward composite)", "bound": "alu", "binding": "fp32",
            "achieved": 13.123456789, "peak": 37.81234567, "unit": "Tops/s (FP32 pipe)", "frac": 0.3712345678,
            "traffic": 44123456.0, "floors_ms": {"mufu": 0.371234567, "fp32": 0.591234567}}
    graph = {"ms_per_step": 2.9081234567, "fwd_mpix_s": 902.123456789, "fwd_ms_per_frame": 1.1381234567}
    e2e = {"value": 349.123456, "unit": "Mpix/s", "h2d_bytes_per_step": 12325500, "d2h_bytes_per_step": 372325500,
           "what": "scene resident (uploaded once, as weights); per step: dL/dI in; image and all gradients out",
           "ms_per_step": 2.95}
    cpu = {"value": 0.0086123456, "unit": "Mpix/s", "cores": 16, "kind": "oracle", "seconds": 11.5,
           "sample": "100000 uniformly random pixels of one 1245x825 view of the 1.5M-primitive scene, fwd+bwd "
                     "(FP64 brute force over all primitives); Mpix/s extrapolated from the sampled pixels"}
    rates = [{"rate_mult": m, "batched": {"p50_ms": 2.123456, "p99_ms": 10.123456, "req_s": 353.123456},
              "per_request": {"p50_ms": 6.123456, "p99_ms": 15.123456, "req_s": 350.123456}} for m in (0.5, 1.0, 2.0)]
    serving = {"requests": 2000, "rates": rates}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 120}
    head = b.headline(1, 20, 5, 353.123456789, graph, 7.0e6, roof, 340, clocks, e2e, cpu, serving)
    line = b.headline_line(head)
    assert len(line) <= 2000
    d = json.loads(line)
    for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "n_gpus", "higher_is_better", "dtype",
              "config", "roofline", "cpu_baseline", "e2e", "fwd_mpix_s", "clocks", "gpu_launches", "serving"):
        assert k in d, k
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["roofline"]["frac"] == 0.37123


def test_leg_lines_fit():
    b = _bench()
    big = {"a": list(range(3000)), "b": {"x": 1.23456789}, "c": "y" * 500}
    import json
    d = b._fit(dict({"leg": "x"}, **big))
    assert len(json.dumps(d)) <= 1900 and d["leg"] == "x" and d["omitted"] == ["a"] and d["b"]["x"] == 1.235
