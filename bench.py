"""Benchmark of the GEF rasterizer hot path on GB300.

A step is one full pass of the hot path over one view: preprocess (projection, SH colour,
extent), binning (depth sort, scan, keygen, tile sort, ranges), forward composite, backward
composite and preprocess backward -- with a fixed synthetic upstream gradient.  The default
workload is the scene-scale case: 1.5M clustered GEF primitives (SH degree 3, beta
log-uniform [0.5, 8]) rendered at 1245x825 from 20 orbit cameras, cycled step by step.

Printed (rank 0, one JSON line): Mpix/s of the fwd+bwd step (``value``), the forward-only
rate, per-stage times, the dominant kernel's roofline, the end-to-end rate through the C-ABI
with host buffers, the FP64 oracle timed on the host cores (``cpu_baseline``) and the SM clocks
seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: independent replicas (each rank renders its own views; no collective), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpix/s fwd & fwd+bwd at 1.5M GEF prims 1245×825; serving p50/p99 ms/frame"
N_PRIMS = 1_500_000
WIDTH, HEIGHT = 1245, 825


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running.  Entering waits
    (up to 5 s) for the first sample, so that sampling is live when the timed region starts."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.lines = []
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.monotonic()
            while not self.lines and time.monotonic() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()  # keep only samples taken after entry
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel's
    sources have changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha1()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return float(rec["dram_bytes_per_launch"]) if h.hexdigest() == rec["sources_sha1"] else None
    except (OSError, KeyError, ValueError):
        return None


def replica_cameras(cams, rank):
    """Replicas only: rank r renders the camera sequence rotated by r, so that ranks start on
    different views and together cover the orbit."""
    k = rank % len(cams)
    return cams[k:] + cams[:k]


def max_over_ranks(ms, dist, dev):
    """The slowest rank's time (every rank gets it); ms unchanged without a process group."""
    if dist is None:
        return ms
    import torch
    x = torch.tensor([float(ms)], device=dev)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def aggregate_mpix_s(ws, pixels_per_step, steps, ms):
    """Whole-job throughput: every rank renders `steps` views of `pixels_per_step` pixels."""
    return ws * pixels_per_step * steps / (ms / 1e3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, ws, rank):
    """The oracle (FP64 CPU brute force, as it stands) on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_2402_10128_gb300 import scenes
    sc, cams = scenes.scene_scale_workload(N_PRIMS)
    rng = np.random.default_rng(0)
    cores = os.cpu_count() or 1
    per_step = args.ref_pixels
    times = []
    for i in range(args.warmup + args.steps):
        cam = cams[i % len(cams)]
        pix = rng.choice(WIDTH * HEIGHT, per_step, replace=False)
        g = rng.standard_normal((3, per_step))
        t0 = time.perf_counter()
        oracle.backward(sc, cam, g, pixels=pix, nthreads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "scene-scale: 1.5M clustered GEF primitives, SH3, 1245x825, "
                                                       "20 orbit cameras; fwd+bwd", "sample_pixels_per_step": per_step},
           "cpu_baseline": {"kind": "oracle", "value": value, "unit": "Mpix/s", "cores": cores,
                            "sample": f"{per_step} uniformly random pixels per step of one 1245x825 view "
                                      f"(fwd+bwd, FP64 brute force over all 1.5M primitives)"},
           "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# FP32 arithmetic (adds, multiplies, FMAs; not compares or selects) that the composites' math needs,
# counted from the equations:
# * per in-extent (fragment, pixel) pair, the falloff: d = p - mean (2), q = (a dx + 2b dy) dx + c dy^2
#   (5), the exponent's scale beta/2 log2 q (1), G's scale -log2(e)/2 p (1), kappa G (1): 10; 9 in the
#   Gaussian form (no q^(beta/2));
# * forward, per composited pair: 1 - alpha, T (1 - alpha), alpha T and the three colour FMAs: 6;
# * backward, per composited pair: 1 - alpha, T_i = T_(i+1) / (1 - alpha), w = alpha T (3); D = sum_c
#   dL/dC_c c_c (3); dL/dalpha = D T - U / (1 - alpha) (2); U += D w (1); dL/dkappa (1); dL/dp (2); dL/dq
#   (3) and dL/dbeta (1), GEF only; dq/d(dx, dy) (2); the mean (4), conic (3) and colour (3) terms; and
#   the 10 adds that sum each pair's 10 terms into the fragment's totals: 38 (34 in the Gaussian form)
FP32_EVAL_GEF, FP32_EVAL_GAUSS, FP32_FWD, FP32_BWD_GEF, FP32_BWD_GAUSS = 10, 9, 6, 38, 34


def composite_fp32_ops(gef, in_extent, composited):
    """(forward, backward) FP32 op counts of one frame's composites from its pair counts."""
    ev = (FP32_EVAL_GEF if gef else FP32_EVAL_GAUSS) * in_extent
    return ev + FP32_FWD * composited, ev + (FP32_BWD_GEF if gef else FP32_BWD_GAUSS) * composited


def sfu_rates():
    """Measured MUFU rates (results per SM per clock) from the SFU microbenchmark."""
    from paper_2402_10128_gb300 import build
    exe = build.build_microbench()
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def cpu_baseline(sc, cams, pixels, cores):
    import oracle
    rng = np.random.default_rng(1)
    cam = cams[0]
    pix = rng.choice(cam.width * cam.height, pixels, replace=False)
    g = rng.standard_normal((3, pixels))
    t0 = time.perf_counter()
    oracle.backward(sc, cam, g, pixels=pix, nthreads=cores)
    dt = time.perf_counter() - t0
    # one thread on a smaller sample; the tiled FP64 renderer (the same algorithm as the GPU) on a
    # whole frame (fwd); the small 128x128 case end to end (fwd + bwd, brute force)
    from paper_2402_10128_gb300 import scenes
    n1 = max(1, pixels // 50)
    t0 = time.perf_counter()
    oracle.backward(sc, cam, g[:, :n1], pixels=pix[:n1], nthreads=1)
    dt1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.render(sc, cam, tiled=True, nthreads=cores)
    dtt = time.perf_counter() - t0
    tsc, tcam = scenes.tiny_workload()
    t0 = time.perf_counter()
    tref = oracle.render(tsc, tcam, nthreads=cores)
    oracle.backward(tsc, tcam, np.ones_like(tref["img"]), nthreads=cores)
    dts = time.perf_counter() - t0
    return {"value": pixels / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "seconds": dt,
            "sample": f"{pixels} uniformly random pixels of one 1245x825 view of the 1.5M-primitive scene, "
                      f"fwd+bwd (FP64 brute force over all primitives); Mpix/s extrapolated from the sampled pixels",
            "one_thread": {"value": n1 / dt1 / 1e6, "unit": "Mpix/s", "sample": f"{n1} of the same pixels, fwd+bwd"},
            "tiled_full_frame_fwd": {"value": cam.width * cam.height / dtt / 1e6, "unit": "Mpix/s", "seconds": dtt,
                                     "sample": "the whole view, the oracle's tiled FP64 renderer (tile lists from its "
                                               "key module), forward"},
            "small_case_fwd_bwd_s": {"value": dts, "unit": "s",
                                     "sample": "the 2,000-primitive 128x128 case end to end, brute force fwd + bwd"}}


def serving_bench(n_requests, rate_mults, slots, dev, seed=40, hbm_budget_gib=48):
    """Serving workload: 4 resident scenes (cube generator, SH3: 0.3M/0.8M/1.5M/3M primitives),
    requests at 800x800 / 1245x825 / 1920x1080 from random cameras, Poisson arrivals.  The same
    arrival trace is served (a) by the batched server (continuous batching, captured-graph
    batches) and (b) by plain per-request launches of the frame API in arrival order.  Latency is
    arrival to image-in-host-memory."""
    import torch
    from paper_2402_10128_gb300 import ges, render, scenes
    sizes = [300_000, 800_000, 1_500_000, 3_000_000]
    scs = [scenes.cube_scene(n, seed=seed + i, sh_degree=3) for i, n in enumerate(sizes)]
    cams = scenes.random_sphere_cameras(n_requests, seed + 10, radius=(3.0, 5.0),
                                        sizes=((800, 800), (1245, 825), (1920, 1080)))
    rng = np.random.default_rng(seed + 20)
    which = rng.integers(0, len(scs), n_requests)
    gcams = [ges.make_camera(c) for c in cams]
    ctx = render.default_context(dev.index or 0)
    # (b) per-request path: one frame per resolution (sized for the largest scene), images copied to host
    dev_scenes = [render.scene_tensors(sc, dev) for sc in scs]
    frames = {}
    n_max = max(sc.n for sc in scs)
    # host images: a free list per resolution; a buffer goes back once its request has been polled
    pool = {}
    pool_lock = threading.Lock()

    def take(c):
        with pool_lock:
            free = pool.setdefault((c.width, c.height), [])
            return free.pop() if free else np.empty((3, c.height, c.width), np.float32)

    def give(a):
        with pool_lock:
            pool[(a.shape[2], a.shape[1])].append(a)

    pr_out = {}

    def per_request(i):
        w = which[i]
        c = cams[i]
        key = (c.width, c.height)
        fr = frames.get(key)
        if fr is None:
            fr = frames[key] = render.Frame(n_max, c.width, c.height, key_capacity=0, ctx=ctx)
            pr_out[key] = np.empty((3, c.height, c.width), np.float32)
        img, _, _ = fr.forward(dev_scenes[w], 3, gcams[i])
        pr_out[key][...] = img.cpu().numpy()

    for i in range(min(12, n_requests)):  # warm-up: frames, capacities
        per_request(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_requests):
        per_request(i)
    service = (time.perf_counter() - t0) / n_requests
    capacity = 1.0 / service  # requests/s of back-to-back per-request launches

    # the server's own context: its HBM budget bounds the resident scenes and both workspaces
    budget = hbm_budget_gib << 30
    sctx = render.Context(dev.index or 0, hbm_budget_bytes=budget)
    srv = ges.ges_serve_create(sctx.handle, ges.params_default(), slots)
    keep = []
    for sc in scs:
        arrs = [np.ascontiguousarray(a, np.float32) for a in sc.arrays()]
        keep.append(arrs)
        ges.ges_serve_add_scene(srv, ges.make_scene(*arrs, sc.sh_degree))
    resident = sum(a.nbytes for arrs in keep for a in arrs)
    # warm-up of the server (workspaces, graphs)
    for i in range(min(16, n_requests)):
        o = take(cams[i])
        t = ges.ges_serve_submit(srv, int(which[i]), gcams[i], o)
        ges.ges_serve_poll(srv, t, 120_000_000)
        give(o)

    results = []
    for mult in rate_mults:
        rate = mult * capacity
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
        # (a) server
        tickets = [None] * n_requests
        bufs = [None] * n_requests
        t_start = time.perf_counter() + 0.01

        def submitter():
            for i in range(n_requests):
                dt = t_start + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                bufs[i] = take(cams[i])
                tickets[i] = ges.ges_serve_submit(srv, int(which[i]), gcams[i], bufs[i])

        th = threading.Thread(target=submitter)
        th.start()
        lat_srv = []
        for i in range(n_requests):
            while tickets[i] is None:
                time.sleep(0.0002)
            st, lat = ges.ges_serve_poll(srv, tickets[i], 120_000_000)
            assert st == ges.GES_OK
            lat_srv.append(lat)
            give(bufs[i])
            bufs[i] = None
        th.join()
        t_end_srv = time.perf_counter()
        span_srv = t_end_srv - t_start
        # (b) per-request launches, FIFO, same arrivals
        lat_pr = []
        t_start = time.perf_counter() + 0.01
        for i in range(n_requests):
            dt = t_start + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            per_request(i)
            lat_pr.append(1e3 * (time.perf_counter() - (t_start + arrivals[i])))
        span_pr = time.perf_counter() - t_start
        pix = sum(c.width * c.height for c in cams)
        results.append({
            "rate_mult": mult, "rate_req_s": rate,
            "batched": {"p50_ms": float(np.percentile(lat_srv, 50)), "p99_ms": float(np.percentile(lat_srv, 99)),
                        "req_s": n_requests / span_srv, "mpix_s": pix / span_srv / 1e6},
            "per_request": {"p50_ms": float(np.percentile(lat_pr, 50)), "p99_ms": float(np.percentile(lat_pr, 99)),
                            "req_s": n_requests / span_pr, "mpix_s": pix / span_pr / 1e6}})
    ges.ges_serve_destroy(srv)
    sctx.close()
    for fr in frames.values():
        fr.close()
    return {"workload": "4 resident cube scenes (0.3M/0.8M/1.5M/3M prims, SH3); 800x800/1245x825/1920x1080 "
                        "requests, random cameras at radius 3-5, Poisson arrivals",
            "requests": n_requests, "slots": slots, "hbm_budget_bytes": budget, "resident_scene_bytes": resident,
            "admission": "two workspaces share what the budget leaves after the resident scenes; each batch "
                         "takes queued requests in order while they fit a workspace's primitive, tile, pixel "
                         "and slot capacities",
            "per_request_service_ms": 1e3 * service,
            "per_request_capacity_req_s": capacity, "rates": results}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-pixels", type=int, default=4096)
    ap.add_argument("--cpu-pixels", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_PRIMS)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the differentiation and stress legs")
    ap.add_argument("--extra", default="image_loss,differentiation,scale_modification,training,mixture_study,stress,"
                                       "stress_beta2",
                    help="comma-separated extra legs to run (default: all)")
    ap.add_argument("--segment-tiles", type=int, default=16, help="binning granularity (ges_params.segment_tiles)")
    ap.add_argument("--full-json", default="", help="write every leg in full to this JSON file")
    ap.add_argument("--profile", action="store_true",
                    help="minimal run for ncu: no work counters, e2e or CPU baseline; warmup + steps fwd+bwd")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference" or os.environ.get("GES_BENCH_ALLOW_SHORT")
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2402_10128_gb300 import ges, render, scenes

    sc, cams = scenes.scene_scale_workload(args.n)
    # each rank renders its own views (replicas): rotate the camera sequence by rank
    cams = replica_cameras(cams, rank)
    dev = torch.device("cuda", local)
    t = render.scene_tensors(sc, dev)
    stream = torch.cuda.current_stream()
    ctx = render.default_context(local)

    # key capacity: the largest K over the camera set, plus headroom (no host sync per frame)
    probe = render.Frame(sc.n, WIDTH, HEIGHT, key_capacity=0, ctx=ctx)
    Ks, Fs = [], []
    for cam in (cams[:1] if args.profile else cams):
        probe.forward(t, sc.sh_degree, cam, {"segment_tiles": args.segment_tiles})
        if args.profile:
            Ks.append(int(ges.ges_frame_status(probe.handle)[1] * 1.3))
            Fs.append((0, 0, 0))
        else:
            ev, inr, comp, K = ges.ges_frame_count_work(probe.handle)
            Ks.append(K)
            Fs.append((ev, inr, comp))
    probe.close()
    del probe
    cap = int(max(Ks) * 1.05) + 4096
    frame = render.Frame(sc.n, WIDTH, HEIGHT, key_capacity=cap, ctx=ctx)
    gcam = [ges.make_camera(c) for c in cams]
    params = ges.params_default()
    params.segment_tiles = args.segment_tiles
    img = torch.empty((3, HEIGHT, WIDTH), device=dev)
    T = torch.empty((HEIGHT, WIDTH), device=dev)
    nc = torch.empty((HEIGHT, WIDTH), dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(7)
    dL = (torch.rand((3, HEIGHT, WIDTH), device=dev, generator=gen) - 0.5) * (2.0 / (WIDTH * HEIGHT))
    grads = tuple(torch.empty_like(a) for a in t)
    scene_c = ges.make_scene(*t, sc.sh_degree)
    grads_c = ges.make_grads(*grads)
    sp = stream.cuda_stream
    nst = 5
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(args.steps)]

    def step(i, events=None, bwd=True):
        cam = gcam[i % len(gcam)]
        if events:
            events[0].record(stream)
        ges.ges_preprocess(frame.handle, scene_c, cam, params, sp)
        if events:
            events[1].record(stream)
        ges.ges_bin_sort(frame.handle, sp)
        if events:
            events[2].record(stream)
        ges.ges_render_fwd(frame.handle, img, T, nc, sp)
        if events:
            events[3].record(stream)
        if bwd:
            ges.ges_render_bwd(frame.handle, scene_c, T, nc, dL, grads_c, sp)
        if events:
            events[4].record(stream)

    def timed(fn_steps, bwd, trace=False):
        for i in range(args.warmup):
            step(i, bwd=bwd)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if trace:
            ges.ges_trace_enable(ctx.handle, True)  # starts an empty record
        l0 = ges.ges_kernel_launches()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for i in range(args.steps):
            step(i, ev[i] if bwd else None, bwd=bwd)
        s1.record(stream)
        torch.cuda.synchronize()
        launches = ges.ges_kernel_launches() - l0
        ms = max_over_ranks(s0.elapsed_time(s1), dist, dev)
        return ms, launches

    if args.profile:
        timed(args.steps, bwd=True)
        print(json.dumps({"profile_run": True, "K": Ks[0]}))
        return
    with ClockSampler(local) as clk:
        # per-kernel device times of the timed fwd+bwd steps: library tracing (events on `stream`)
        ms_fb, launches = timed(args.steps, bwd=True, trace=True)
        trace = ges.ges_trace_read(ctx.handle)
        ges.ges_trace_enable(ctx.handle, False)
        stage = np.array([[ev[i][k].elapsed_time(ev[i][k + 1]) for k in range(nst - 1)] for i in range(args.steps)])
        ms_f, _ = timed(args.steps, bwd=False)
        err = ges.ges_frame_status(frame.handle)[0]
        assert err == ges.GES_OK, "key capacity overflowed during the timed region"
        # the headline: the same step replayed from one CUDA graph per camera
        graph = graph_replay_bench(frame, scene_c, gcam, params, img, T, nc, dL, grads, grads_c, args.steps,
                                   args.warmup, dev, ws, dist)
    clocks = clk.summary()

    pix = WIDTH * HEIGHT
    direct = aggregate_mpix_s(ws, pix, args.steps, ms_fb)
    value = graph["mpix_s"]
    fwd_direct = aggregate_mpix_s(ws, pix, args.steps, ms_f)
    fwd_rate = graph["fwd_mpix_s"]
    st_mean = stage.mean(0)

    # roofline of the dominant kernel: the composites' algorithmic work per (fragment, pixel) pair is
    # transcendental (MUFU) and FP32 arithmetic; both pipes' rates are measured live by the SFU
    # microbenchmark, and the binding one is reported
    peaks, src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    stage_names = ["preprocess", "bin_sort", "render_fwd", "render_bwd+preprocess_bwd"]
    dom = int(np.argmax(st_mean))
    mean_eval = float(np.mean([f[0] for f in Fs]))
    mean_inr = float(np.mean([f[1] for f in Fs]))
    mean_comp = float(np.mean([f[2] for f in Fs]))
    mean_K = float(np.mean(Ks))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sfu = sfu_rates()
    r_ex2, r_lg2, r_rcp = (sfu["per_sm_per_clk"][k] for k in ("ex2", "lg2", "rcp"))
    clk = nsm * sm_mhz * 1e6

    r_fma = float(sfu["per_sm_per_clk"].get("fma", 128.0))

    def composite_roofline(kernel, ms, n_lg2, n_ex2, n_rcp, n_fp32, work):
        """Two floors for a launch: its MUFU ops at the measured per-instruction rates, and its FP32
        ops (adds, multiplies, FMAs) at the measured FMA-pipe rate; the larger one binds."""
        mufu_ops = n_lg2 + n_ex2 + n_rcp
        t_mufu = (n_lg2 / r_lg2 + n_ex2 / r_ex2 + n_rcp / r_rcp) / clk  # seconds at the measured rates
        t_fp32 = n_fp32 / r_fma / clk
        sec = ms / 1e3
        res = {"mufu": {"ops": mufu_ops, "achieved": mufu_ops / sec / 1e12,
                        "peak": (mufu_ops / t_mufu / 1e12) if t_mufu > 0 else None, "unit": "Tops/s",
                        "frac": t_mufu / sec, "floor_ms": t_mufu * 1e3},
               "fp32": {"ops": n_fp32, "achieved": n_fp32 / sec / 1e12, "peak": r_fma * clk / 1e12, "unit": "Tops/s",
                        "frac": t_fp32 / sec, "floor_ms": t_fp32 * 1e3}}
        bind = "fp32" if t_fp32 >= t_mufu else "mufu"
        r = res[bind]
        return {"kernel": kernel, "bound": "alu", "binding": bind, "achieved": r["achieved"], "peak": r["peak"],
                "unit": "Tops/s (%s)" % ("FP32 pipe" if bind == "fp32" else "MUFU"), "frac": r["frac"],
                "traffic": _traffic(kernel.split()[0]), "work": work, "resources": res,
                "peak_source": (f"{nsm} SMs x {sm_mhz:.0f} MHz ({src} max clock) x rates per SM per clock measured "
                                f"by the sfu_rates microbenchmark: FP32 FMA {r_fma:.1f}; MUFU ex2 {r_ex2:.1f}, "
                                f"lg2 {r_lg2:.1f}, rcp {r_rcp:.1f}, weighted by the kernel's MUFU mix")}

    # average device time per launch of each traced kernel over the timed steps
    kernel_ms = {k: ms / n for k, (n, ms) in trace.items()}
    bwd_ms = kernel_ms["k_render_bwd"]
    fwd_ms = kernel_ms["k_render_fwd"]
    fp32_fwd, fp32_bwd = composite_fp32_ops(True, mean_inr, mean_comp)
    roofline = composite_roofline("k_render_bwd (backward composite)", bwd_ms,
                                  mean_inr, 2 * mean_inr, 2 * mean_comp, fp32_bwd,
                                  f"per frame: lg2 + 2 ex2 and {FP32_EVAL_GEF} FP32 ops per in-extent pair "
                                  f"({mean_inr:.3e}); 2 rcp and {FP32_BWD_GEF} FP32 ops per composited pair "
                                  f"({mean_comp:.3e})")
    roofline_fwd = composite_roofline("k_render_fwd (forward composite)", fwd_ms, mean_inr, 2 * mean_inr, 0, fp32_fwd,
                                      f"per frame: lg2 + 2 ex2 and {FP32_EVAL_GEF} FP32 ops per in-extent pair "
                                      f"({mean_inr:.3e}); {FP32_FWD} FP32 ops per composited pair ({mean_comp:.3e})")
    # preprocess: HBM bytes per primitive (read 240 B at SH3; write 88 B: depth key x2, sort value,
    # rect, 48-B record, extent shape, tile count)
    pre_bytes = sc.n * (240 + 88)
    pre_gbs = pre_bytes / (kernel_ms["k_preprocess"] / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    full = {}  # every leg in full; written to --full-json

    def leg(name, d, summary=None):
        """Record a leg and print its line (rank 0): the summary, or the leg itself cut to fit."""
        full[name] = d
        if rank == 0:
            print(json.dumps(_fit(dict({"leg": name}, **(summary if summary is not None else d)))), flush=True)

    roof = {k: roofline[k] for k in ("kernel", "bound", "binding", "achieved", "peak", "unit", "frac", "traffic")}
    roof["floors_ms"] = {k: v["floor_ms"] for k, v in roofline["resources"].items()}
    leg("composite_rooflines", {"k_render_bwd": roofline, "k_render_fwd": roofline_fwd, "sfu_rates": sfu,
                                "preprocess_hbm": {"kernel": "k_preprocess", "achieved_gbs": pre_gbs, "peak_gbs": hbm,
                                                   "frac": pre_gbs / hbm, "bytes_per_prim": 328}},
        summary={"k_render_bwd": roof,
                 "k_render_fwd": {k: roofline_fwd[k] for k in ("binding", "achieved", "peak", "unit", "frac")},
                 "k_render_fwd_floors_ms": {k: v["floor_ms"] for k, v in roofline_fwd["resources"].items()},
                 "work_per_frame": roofline["work"],
                 "rates_per_sm_per_clk": sfu.get("per_sm_per_clk"),
                 "k_preprocess": {"bound": "hbm", "achieved_gbs": pre_gbs, "peak_gbs": hbm, "frac": pre_gbs / hbm,
                                  "bytes_per_prim": 328}})
    leg("kernels", {"kernel_ms": kernel_ms, "stage_ms": dict(zip(stage_names, [float(x) for x in st_mean])),
                    "dominant_stage": stage_names[dom],
                    "frame_stats": {"K_mean": mean_K, "evaluated_pairs_mean": mean_eval,
                                    "in_extent_pairs_mean": mean_inr, "composited_pairs_mean": mean_comp},
                    "direct_calls": {"mpix_s": direct, "ms_per_step": ms_fb / args.steps, "fwd_mpix_s": fwd_direct,
                                     "fwd_ms_per_frame": ms_f / args.steps,
                                     "what": "the same steps as four C-ABI calls each, traced"},
                    "graph_replay": {k: graph[k] for k in ("mpix_s", "ms_per_step", "fwd_mpix_s", "fwd_ms_per_frame")},
                    "graph_check": graph["check"]["image"]})
    leg("graph_replay_check", graph["check"])

    e2e_res = None
    if not args.no_e2e:
        e2e_res = e2e(args, sc, gcam, frame, params, dev, stream, ws, dist)
        leg("e2e", e2e_res)
        leg("e2e_full_transfer", e2e(args, sc, gcam, frame, params, dev, stream, ws, dist, full_transfer=True))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, cams, args.cpu_pixels, os.cpu_count() or 1)
        leg("cpu_baseline", cpu)
    if not args.no_extra:
        legs = set(x for x in args.extra.split(",") if x)
        if "image_loss" in legs:
            leg("image_loss", loss_bench(50, 3, dev, img))
        if "differentiation" in legs:
            leg("differentiation", differentiation_bench(20, 3, dev))
        if "scale_modification" in legs:
            r = scale_modification_bench(10, 3, dev, sc, t, cams[0], args.segment_tiles, composite_roofline)
            leg("scale_modification", r, summary={
                "workload": r["workload"],
                "variants": {k: {"fwd_bwd_ms": v["fwd_bwd"]["ms_per_frame"], "fwd_ms": v["fwd"]["ms_per_frame"],
                                 "K": v["K_entries"], "composited": v["pairs"]["composited_pairs"],
                                 "bwd_ms": v["k_render_bwd_ms"],
                                 "bwd_frac": v.get("roofline_bwd", {}).get("frac"),
                                 "oracle_mpix_s": v["cpu_baseline"]["value"]}
                             for k, v in r["variants"].items()}})
        torch.cuda.empty_cache()
        if "mixture_study" in legs:
            leg("mixture_study", mixture_study_bench(dev))
        if "training" in legs:
            leg("training", training_bench(20, 3, dev, sc, cams, args.segment_tiles))
            torch.cuda.empty_cache()
        if "stress" in legs:
            leg("stress", stress_bench(5, 3, dev, beta2=False, segment_tiles=256))
            torch.cuda.empty_cache()
        if "stress_beta2" in legs:
            leg("stress_beta2", stress_bench(5, 3, dev, beta2=True, segment_tiles=args.segment_tiles))
            torch.cuda.empty_cache()
    serving = None
    if not args.no_serve:
        del t, grads
        frame.close()
        torch.cuda.empty_cache()
        serving = serving_bench(args.serve_requests, (0.5, 1.0, 2.0), args.serve_slots, dev)
        leg("serving", serving)

    head = headline(ws, args.steps, args.warmup, value, graph, mean_K, roof, launches, clocks, e2e_res, cpu,
                    serving)
    full["headline"] = head
    if rank == 0 and args.full_json:
        with open(args.full_json, "w") as f:
            json.dump(full, f, indent=1)
    if rank == 0:
        print(headline_line(head), flush=True)
    if dist:
        dist.destroy_process_group()


def headline(ws, steps, warmup, value, graph, mean_K, roof, launches, clocks, e2e_res, cpu, serving):
    """The headline record: the fwd+bwd rate of the scene-scale step with the forward rate, the
    dominant kernel's roofline, the end-to-end rate, the oracle's rate on the host, the serving
    latencies at each arrival rate and the clocks seen."""
    head = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": steps,
            "warmup": warmup, "ms_per_step": graph["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "scene-scale fwd+bwd: 1.5M clustered GEF primitives, SH3, beta log-U[0.5,8], "
                                   "1245x825, 20 orbit cameras; one view per step",
                       "l2": "inputs larger than L2 (scene 360 MB, lists ~%d MB)" % int(mean_K * 16 / 1e6),
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "fwd_mpix_s": graph["fwd_mpix_s"], "fwd_ms_per_frame": graph["fwd_ms_per_frame"],
            "roofline": roof,
            "gpu_launches": int(launches), "clocks": clocks}
    if e2e_res is not None:
        head["e2e"] = {k: e2e_res[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step",
                                                "what")}
    if cpu is not None:
        head["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if serving is not None:
        head["serving"] = {"requests_per_rate": serving["requests"],
                           **{f"x{r['rate_mult']:g}": {m: [r[m]["p50_ms"], r[m]["p99_ms"], r[m]["req_s"]]
                                                       for m in ("batched", "per_request")}
                              for r in serving["rates"]},
                           "fields": "p50 ms, p99 ms, req/s"}
    return head


def headline_line(head, limit=2000):
    """The headline as one JSON line of at most `limit` characters (floats to 5 significant
    digits; the serving summary, then the roofline's floors, give way if it is longer)."""
    head = dict(head)
    line = json.dumps(_round(head, 5))
    for drop in ("serving", "floors_ms"):
        if len(line) <= limit:
            break
        if drop == "floors_ms":
            head["roofline"] = {k: v for k, v in head["roofline"].items() if k != "floors_ms"}
        else:
            head.pop(drop, None)
        line = json.dumps(_round(head, 5))
    return line


def _round(o, sig=4):
    """Floats rounded to `sig` significant digits, recursively (for short printed lines)."""
    if isinstance(o, float):
        return float(f"{o:.{sig}g}") if np.isfinite(o) else None
    if isinstance(o, dict):
        return {k: _round(v, sig) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_round(v, sig) for v in o]
    return o


def _fit(d, limit=1900):
    """A leg's printed form: floats to 4 significant digits; while the line is longer than
    `limit` characters, the largest top-level entry is replaced by the note that it is only in
    the full record."""
    d = _round(d)
    cut = []
    while len(json.dumps(d)) > limit:
        big = max((k for k in d if k != "leg"), key=lambda k: len(json.dumps(d[k])))
        d.pop(big)
        cut.append(big)
        d["omitted"] = cut
    return d


def _ssim(x, y):
    """Mean SSIM of two [3,H,W] images: 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2."""
    import torch
    import torch.nn.functional as F
    g = torch.exp(-((torch.arange(11, device=x.device, dtype=torch.float32) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    w = (g[:, None] * g[None, :]).expand(3, 1, 11, 11).contiguous()

    def blur(a):
        return F.conv2d(a[None], w, padding=5, groups=3)[0]

    mx, my = blur(x), blur(y)
    sxx, syy, sxy = blur(x * x) - mx * mx, blur(y * y) - my * my, blur(x * y) - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return s.mean()


def differentiation_bench(steps, warmup, dev):
    """fwd+bwd through the torch.autograd.Function on the differentiation workload (cube
    distribution, 1.5M primitives, SH0, 1245x825).  The upstream gradient is that of
    0.8 L1 + 0.2 (1 - SSIM) against a seeded uniform target, computed once by torch outside the
    timed region; each timed step is rasterize() + torch.autograd.grad() (K1-K8)."""
    import torch
    from paper_2402_10128_gb300 import render, scenes
    sc, cam = scenes.differentiation_workload()
    params = [p.requires_grad_(True) for p in render.scene_tensors(sc, dev)]
    probe = render.Frame(sc.n, cam.width, cam.height, key_capacity=0)
    probe.forward(tuple(p.detach() for p in params), sc.sh_degree, cam)
    K = probe.status()[1]
    probe.close()
    frame = render.Frame(sc.n, cam.width, cam.height, key_capacity=int(K * 1.05) + 4096)
    gen = torch.Generator(device=dev).manual_seed(3)
    target = torch.rand((3, cam.height, cam.width), device=dev, generator=gen)
    img, _, _ = render.rasterize(*params, sc.sh_degree, cam, frame=frame)
    loss = 0.8 * (img - target).abs().mean() + 0.2 * (1.0 - _ssim(img, target))
    dL = torch.autograd.grad(loss, img)[0].detach().contiguous()
    for p in params:
        p.grad = None

    def step():
        im, _, _ = render.rasterize(*params, sc.sh_degree, cam, frame=frame)
        return torch.autograd.grad(im, params, grad_outputs=dL)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        grads = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st, _ = frame.status()
    assert st == 0 and all(torch.isfinite(g).all() for g in grads)
    frame.close()
    return {"workload": "differentiation: cube distribution, 1.5M primitives, SH0, 1245x825; upstream gradient of "
                        "0.8 L1 + 0.2 (1 - SSIM) vs a seeded uniform target; step = rasterize + autograd.grad",
            "fwd_bwd_mpix_s": cam.width * cam.height / (ms / 1e3) / 1e6, "ms_per_step": ms, "steps": steps,
            "K": int(K), "loss": float(loss.detach())}


def loss_bench(steps, warmup, dev, img):
    """The training image loss on the rendered 1245x825 view: ges_freq_mask (omega 0.7, scale 0.2)
    and ges_image_loss (lambda_ssim 0.2, lambda_omega 0.5) against a perturbed copy as the
    ground truth.  Roofline: HBM, on the algorithmic bytes (mask: read I_gt, write the mask; loss:
    read I, I_gt and the mask, write dL/dI)."""
    import torch
    from paper_2402_10128_gb300 import ges, render
    ctx = render.default_context(dev.index or 0)
    C, H, W = img.shape
    gen = torch.Generator(device=dev).manual_seed(9)
    gt = (img + 0.05 * torch.randn(img.shape, device=dev, generator=gen)).contiguous()
    mask = torch.empty((H, W), dtype=torch.uint8, device=dev)
    loss = torch.empty(4, device=dev)
    grad = torch.empty_like(img)

    def step():
        ges.ges_freq_mask(ctx.handle, gt, W, H, 0.7, mask)
        ges.ges_image_loss(ctx.handle, img, gt, mask, W, H, loss, grad)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(steps):
        ges.ges_freq_mask(ctx.handle, gt, W, H, 0.7, mask)
    e[1].record()
    for _ in range(steps):
        ges.ges_image_loss(ctx.handle, img, gt, mask, W, H, loss, grad)
    e[2].record()
    torch.cuda.synchronize()
    ms_mask, ms_loss = e[0].elapsed_time(e[1]) / steps, e[1].elapsed_time(e[2]) / steps
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    px = W * H
    b_mask, b_loss = px * (12 + 1), px * (12 + 12 + 1 + 12)
    # the oracle (FP64, numpy / torch on the host) on the same images, once each
    from oracle import loss as ol
    gt_h, img_h = gt.cpu().numpy().astype(np.float64), img.cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    m_ref, _ = ol.freq_mask(gt_h, 0.7, 0.2)
    t_mask = time.perf_counter() - t0
    t0 = time.perf_counter()
    ol.image_loss(img_h, gt_h, m_ref)
    t_loss = time.perf_counter() - t0
    return {"workload": "training image loss of the rendered 1245x825 view: frequency mask (omega 0.7, scale 0.2) "
                        "and L = 0.3 L1 + 0.2 (1 - SSIM) + 0.5 L_omega with dL/dI",
            "mask_ms": ms_mask, "loss_ms": ms_loss, "loss": [float(v) for v in loss.cpu()],
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                         "mask_achieved": b_mask / (ms_mask / 1e3) / 1e9, "mask_frac": b_mask / (ms_mask / 1e3) / 1e9 / hbm,
                         "loss_achieved": b_loss / (ms_loss / 1e3) / 1e9, "loss_frac": b_loss / (ms_loss / 1e3) / 1e9 / hbm,
                         "bytes_per_pixel": {"mask": 13, "loss": 37}},
            "cpu_baseline": {"kind": "oracle", "mask_ms": t_mask * 1e3, "loss_ms": t_loss * 1e3,
                             "cores": torch.get_num_threads(),
                             "sample": "the same 1245x825 images once: oracle.loss.freq_mask and image_loss (FP64)"}}


def graph_replay_bench(frame, scene_c, gcam, params, img, T, nc, dL, grads, grads_c, steps, warmup, dev, ws=1,
                       dist=None):
    """The same fwd+bwd step (ges_preprocess, ges_bin_sort, ges_render_fwd, ges_render_bwd on the
    same frame and tensors) captured once per camera as a CUDA graph and replayed: the same kernels
    with the launch gaps between them removed.  Before timing, one replay per camera is checked to
    give the direct calls' image bit for bit and their gradients up to the order of the atomics."""
    import torch
    from paper_2402_10128_gb300 import ges
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    sp0 = torch.cuda.current_stream().cuda_stream
    graphs, fwd_graphs = [], []
    for cam in gcam:
        for bwd in (True, False):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                sp = s.cuda_stream
                ges.ges_preprocess(frame.handle, scene_c, cam, params, sp)
                ges.ges_bin_sort(frame.handle, sp)
                ges.ges_render_fwd(frame.handle, img, T, nc, sp)
                if bwd:
                    ges.ges_render_bwd(frame.handle, scene_c, T, nc, dL, grads_c, sp)
            (graphs if bwd else fwd_graphs).append(g)
    # the replays do the direct calls' work: equal outputs, bit for bit, for every camera
    def direct(cam):
        ges.ges_preprocess(frame.handle, scene_c, cam, params, sp0)
        ges.ges_bin_sort(frame.handle, sp0)
        ges.ges_render_fwd(frame.handle, img, T, nc, sp0)
        ges.ges_render_bwd(frame.handle, scene_c, T, nc, dL, grads_c, sp0)
        torch.cuda.synchronize()
        return [img.clone()] + [g.clone() for g in grads]

    def rel(a, b):
        return float((a - b).norm()) / max(float(a.norm()), 1e-30)

    names = ("means", "scales", "quats", "betas", "opacities", "shs")
    worst = {n: [0.0, 0.0] for n in names}  # largest replay-vs-direct and direct-vs-direct differences
    for k, cam in enumerate(gcam):
        ref, ref2 = direct(cam), direct(cam)
        graphs[k].replay()
        torch.cuda.synchronize()
        got = [img] + list(grads)
        # the image is deterministic; the gradients are sums of atomics, equal up to their order: the
        # replay must differ from the direct calls no more than two direct runs do (x10), or than the
        # gradients' parity tolerance (1e-3 relative)
        assert torch.equal(ref[0], got[0]), f"graph replay image differs from the direct calls ({k})"
        for n, a, a2, b in zip(names, ref[1:], ref2[1:], got[1:]):
            d, noise = rel(a, b), rel(a, a2)
            worst[n] = [max(worst[n][0], d), max(worst[n][1], noise)]
            assert d <= max(10 * noise, 1e-3), f"graph replay gradients differ ({k}, {n}): {d} (direct runs: {noise})"
        img.zero_()
        fwd_graphs[k].replay()
        torch.cuda.synchronize()
        assert torch.equal(ref[0], img), f"forward graph replay image differs from the direct calls ({k})"
    def timed(gs):
        for i in range(warmup):
            gs[i % len(gs)].replay()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        e0.record(cur)
        for i in range(steps):
            gs[i % len(gs)].replay()
        e1.record(cur)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    ms = timed(graphs)
    ms_f = timed(fwd_graphs)
    assert ges.ges_frame_status(frame.handle)[0] == ges.GES_OK
    del graphs, fwd_graphs
    px = img.shape[1] * img.shape[2]
    return {"mpix_s": aggregate_mpix_s(ws, px, steps, ms), "ms_per_step": ms / steps,
            "fwd_mpix_s": aggregate_mpix_s(ws, px, steps, ms_f), "fwd_ms_per_frame": ms_f / steps,
            "what": "the fwd+bwd step (and the fwd alone) captured per camera as a CUDA graph and replayed "
                    "(checked against the direct calls)",
            "check": {"image": "bitwise equal to the direct calls, every camera",
                      "gradients_rel_l2_max": {n: {"replay_vs_direct": v[0], "direct_vs_direct": v[1]}
                                               for n, v in worst.items()}}}


def training_bench(steps, warmup, dev, sc, cams, segment_tiles):
    """One training iteration of the paper's loop per step on the scene-scale workload (1.5M
    primitives, SH3, 1245x825, cycling through the 20 views): ges_preprocess, ges_bin_sort,
    ges_render_fwd, ges_freq_mask of the view's target (omega 0.7), ges_image_loss (0.2 SSIM,
    0.5 L_omega), ges_render_bwd, ges_densify_stats and ges_adam_step over all 1.5M primitives.  The
    targets are the views rendered once from the scene; the optimizer starts from the scene's own
    parameters (log-scales, logits, beta - 2).  Then one ges_density_control over the statistics
    of the timed steps (App. B.2 thresholds, extent 1, split normals from a seeded generator).
    Roofline of k_adam: HBM, 32 B per element (read variable, moments, gradient; write variable,
    moments, physical value), 60 elements per primitive at SH3."""
    import torch
    from paper_2402_10128_gb300 import ges, render
    ctx = render.default_context(dev.index or 0)
    n, sh = sc.n, sc.sh_degree
    W, H = cams[0].width, cams[0].height
    t = render.scene_tensors(sc, dev)
    probe = render.Frame(n, W, H, key_capacity=0)
    targets, K = [], 0
    for cam in cams:
        img, _, _ = probe.forward(t, sh, cam, {"segment_tiles": segment_tiles})
        targets.append(img.clone())
        K = max(K, probe.status()[1])
    probe.close()
    raw = [t[0].clone(), torch.log(t[1]), t[2].clone(), t[3] - 2.0, torch.logit(t[4]), t[5].clone()]
    mom = [torch.zeros_like(a) for a in raw]
    vel = [torch.zeros_like(a) for a in raw]
    phys = [torch.empty_like(a) for a in raw]
    grads = tuple(torch.empty_like(a) for a in raw)
    del t
    tset = ges.make_train_set(n, sh, raw, mom, vel)
    so = ges.make_scene_out(*phys)
    ges.ges_activate(ctx.handle, tset, so)
    hp = ges.adam_params_default()
    frame = render.Frame(n, W, H, key_capacity=int(K * 1.05) + 4096)
    gcams = [ges.make_camera(c) for c in cams]
    params = ges.params_default()
    params.segment_tiles = segment_tiles
    scene_c, grads_c = ges.make_scene(*phys, sh), ges.make_grads(*grads)
    img = torch.empty((3, H, W), device=dev)
    T = torch.empty((H, W), device=dev)
    nc = torch.empty((H, W), dtype=torch.int32, device=dev)
    mask = torch.empty((H, W), dtype=torch.uint8, device=dev)
    loss = torch.empty(4, device=dev)
    dL = torch.empty((3, H, W), device=dev)
    acc = torch.zeros(n, device=dev)
    cnt = torch.zeros(n, dtype=torch.int32, device=dev)
    it = [0]

    def step():
        i = it[0]
        it[0] += 1
        k = i % len(cams)
        ges.ges_preprocess(frame.handle, scene_c, gcams[k], params)
        ges.ges_bin_sort(frame.handle)
        ges.ges_render_fwd(frame.handle, img, T, nc)
        ges.ges_freq_mask(ctx.handle, targets[k], W, H, 0.7, mask)
        ges.ges_image_loss(ctx.handle, img, targets[k], mask, W, H, loss, dL)
        ges.ges_render_bwd(frame.handle, scene_c, T, nc, dL, grads_c)
        ges.ges_densify_stats(frame.handle, acc, cnt)
        ges.ges_adam_step(ctx.handle, tset, grads_c, so, hp, i + 1)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ges.ges_trace_enable(ctx.handle, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    trace = ges.ges_trace_read(ctx.handle)
    ges.ges_trace_enable(ctx.handle, False)
    ms = e0.elapsed_time(e1) / steps
    assert frame.status()[0] == 0 and bool(torch.isfinite(loss).all())
    frame.close()
    kernel_ms = {k: v[1] / steps for k, v in trace.items()}
    adam_ms = trace["k_adam"][1] / trace["k_adam"][0]
    elems = n * (12 + 3 * (sh + 1) ** 2)
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    adam_gbs = elems * 32 / (adam_ms / 1e3) / 1e9

    # one density control over the statistics gathered above
    gen = torch.Generator(device=dev).manual_seed(11)
    xi = torch.randn((n, 2, 3), device=dev, generator=gen)
    dp = ges.density_params_default()
    cap = 3 * n
    out = [torch.empty((cap,) + tuple(a.shape[1:]), device=dev) for a in raw]
    om = [torch.empty_like(a) for a in out]
    ov = [torch.empty_like(a) for a in out]
    tout = ges.make_train_set(cap, sh, out, om, ov)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record()
    n_out = ges.ges_density_control(ctx.handle, tset, acc, cnt, xi, dp, tout)
    d1.record()
    torch.cuda.synchronize()
    # the oracle's Adam step and density control (numpy FP64 on the host) on the same state
    from oracle import train as ot
    names = ("means", "scales", "quats", "betas", "opacities", "shs")
    r_h = {k: a.cpu().double().numpy() for k, a in zip(names, raw)}
    m_h = {k: a.cpu().double().numpy() for k, a in zip(names, mom)}
    v_h = {k: a.cpu().double().numpy() for k, a in zip(names, vel)}
    g_h = {k: a.cpu().double().numpy() for k, a in zip(names, grads)}
    t0 = time.perf_counter()
    ot.adam_step(r_h, m_h, v_h, g_h, steps + warmup + 1)
    t_adam = time.perf_counter() - t0
    t0 = time.perf_counter()
    ot.density_control(r_h, m_h, v_h, acc.cpu().numpy(), cnt.cpu().numpy(), xi.cpu().double().numpy())
    t_dens = time.perf_counter() - t0
    return {"workload": "training iteration: scene-scale, 1.5M primitives, SH3, 1245x825, 20 views; fwd + frequency "
                        "mask + image loss + bwd + densification statistics + Adam over all primitives",
            "steps": steps, "ms_per_step": ms, "iterations_per_s": 1e3 / ms,
            "kernel_ms_per_step": kernel_ms, "loss_last": [float(v) for v in loss.cpu()],
            "adam": {"ms": adam_ms, "elements": elems,
                     "roofline": {"bound": "hbm", "achieved": adam_gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": adam_gbs / hbm, "bytes_per_element": 32}},
            "density_control": {"ms": d0.elapsed_time(d1), "rows_in": n, "rows_out": int(n_out),
                                "views_accumulated": steps + warmup},
            "cpu_baseline": {"kind": "oracle", "adam_ms": t_adam * 1e3, "density_control_ms": t_dens * 1e3,
                             "cores": torch.get_num_threads(),
                             "sample": "one Adam step and one density control over the same 1.5M primitives "
                                       "(oracle.train, numpy FP64)"}}


def mixture_study_bench(dev, epochs=1000, runs_per=20, n_points=1000, cpu_fits=2):
    """The 1D mixture study of App. A on the GPU: every model (Gaussian, DoG, LoG, GEF) x N in
    {2, 5, 8, 10, 15, 20} x positive or unrestricted weights x the six signals x 20 seeded runs
    (5,760 fits), 1000 full-batch Adam steps each on 1000 samples of [-1, 1], signal width 1.
    One ges_fit1d launch per (model, N, weight mode) with the 120 runs of the six signals, spread
    over 8 streams.  Reported: the study's wall time in FP32 and FP64, fits/s, component
    evaluations/s (forward and gradient passes), and the study's result per model and signal
    (mean final MSE over the stable runs, and the share of stable runs), as in its figures.
    cpu_baseline: the oracle (torch FP64 on the host) on `cpu_fits` fits of the same kind."""
    import time
    import torch
    from paper_2402_10128_gb300 import ges, render, scenes
    ctx = render.default_context(dev.index or 0)
    models, Ns, signals = ["gaussian", "dog", "log", "gef"], [2, 5, 8, 10, 15, 20], list(ges.SIGNAL_KINDS)
    out = {}
    for prec, dtype in ((32, torch.float32), (64, torch.float64)):
        x = torch.empty(n_points, dtype=dtype, device=dev)
        ys = torch.empty((len(signals), n_points), dtype=dtype, device=dev)
        for i, k in enumerate(signals):
            ges.ges_signal1d(ctx.handle, k, x, ys[i])
        y = ys.repeat_interleave(runs_per, dim=0).contiguous()          # run r fits signal r // runs_per
        jobs = []
        for model in models:
            for n in Ns:
                for pos in (1, 0):
                    p0 = scenes.mixture_init(model, n, len(signals) * runs_per, seed=1000 * n + pos)
                    prm = torch.as_tensor(p0, dtype=dtype, device=dev).contiguous()
                    fl = torch.empty(prm.shape[0], dtype=dtype, device=dev)
                    fp = ges.fit1d_params_default(model=ges.MIX_MODELS[model], n_components=n, positive_weights=pos,
                                                  epochs=epochs, precision=prec)
                    jobs.append((model, n, pos, p0, prm, fl, fp))
        streams = [torch.cuda.Stream(device=dev) for _ in range(8)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for j, (model, n, pos, p0, prm, fl, fp) in enumerate(jobs):
            st = streams[j % len(streams)]
            st.wait_event(e0)
            ges.ges_fit1d(ctx.handle, fp, x, y, prm, fl, stream=st.cuda_stream)
        for st in streams:
            torch.cuda.current_stream().wait_stream(st)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fits = sum(j[4].shape[0] for j in jobs)
        evals = sum(j[4].shape[0] * n_points * j[1] * 2 * (epochs + 1) for j in jobs)
        res = {}
        for model, n, pos, p0, prm, fl, fp in jobs:
            if not pos:
                continue
            f = fl.cpu().double().numpy().reshape(len(signals), runs_per)
            for i, k in enumerate(signals):
                ok = np.isfinite(f[i])
                r = res.setdefault(model, {}).setdefault(k, {"N": Ns, "mean_mse": [], "stable": []})
                r["mean_mse"].append(float(f[i][ok].mean()) if ok.any() else None)
                r["stable"].append(float(ok.mean()))
        entry = {"ms": ms, "fits": fits, "fits_per_s": fits / (ms / 1e3),
                 "component_evals_per_s": evals / (ms / 1e3), "positive_weights_result": res}
        if prec == 32:
            # MUFU work per (sample, component, epoch), forward + gradient pass, in SM clocks at the
            # measured per-SM rates: Gaussian and LoG 2 ex2, DoG 4 ex2, GEF 4 ex2 + 3 lg2 + 1 rcp
            sfu = sfu_rates()
            per = sfu.get("per_sm_per_clk", {})
            ex2, lg2, rcp = per.get("ex2", 31.4), per.get("lg2", 15.9), per.get("rcp", 15.9)
            clk = {"gaussian": 2 / ex2, "dog": 4 / ex2, "log": 2 / ex2, "gef": 4 / ex2 + 3 / lg2 + 1 / rcp}
            sm_clk = sum(j[4].shape[0] * n_points * j[1] * (epochs + 1) * clk[j[0]] for j in jobs)
            t_peak = sm_clk / (sfu.get("sms", 152) * sfu.get("max_clock_mhz", 2070) * 1e6)
            entry["roofline"] = {"kernel": "k_fit1d", "bound": "alu", "unit": "ms (MUFU-limited time)",
                                 "peak_time_ms": t_peak * 1e3, "achieved_ms": ms, "frac": t_peak * 1e3 / ms,
                                 "work": "ex2/lg2/rcp per (sample, component, epoch) by model at the measured MUFU "
                                         "rates; 152 SMs at the maximum clock"}
        out["fp%d" % prec] = entry
    # the oracle on a bounded sample of the same work
    from oracle import mixture1d as om
    xs = np.linspace(-1.0, 1.0, n_points)
    t0 = time.perf_counter()
    for r in range(cpu_fits):
        p0 = scenes.mixture_init("gef", 10, 1, seed=r)[0]
        om.fit("gef", p0, xs, om.signal("square", xs), epochs)
    cpu_s = time.perf_counter() - t0
    out["workload"] = ("1D mixture study: 4 models x N in {2,5,8,10,15,20} x 2 weight modes x 6 signals x 20 runs, "
                       "1000 Adam steps on 1000 samples")
    out["cpu_baseline"] = {"value": cpu_fits / cpu_s, "unit": "fits/s", "kind": "oracle",
                           "cores": torch.get_num_threads(),
                           "sample": f"{cpu_fits} GEF fits, N = 10, square, {epochs} steps (torch FP64 on the host)"}
    return out


def _time_c_abi_steps(sc, t, cam, params, steps, warmup, dev, detail=None):
    """fwd (K1-K4) and fwd+bwd (K1-K8) through the C-ABI on device-resident scene tensors `t`,
    timed with CUDA events; returns (K entries, {"fwd": ..., "fwd_bwd": ...}).  With a dict
    `detail`, also fills in the frame's (fragment, pixel) pair counts and the traced per-launch
    device time of every kernel of the fwd+bwd steps."""
    import torch
    from paper_2402_10128_gb300 import ges, render
    probe = render.Frame(sc.n, cam.width, cam.height, key_capacity=0)
    probe.forward(t, sc.sh_degree, cam, {"segment_tiles": params.segment_tiles, "mode": params.falloff,
                                         "rho": params.rho, "phi_mode": params.phi_mode})
    K = probe.status()[1]
    if detail is not None:
        ev, inr, comp, _ = ges.ges_frame_count_work(probe.handle)
        detail.update(evaluated_pairs=int(ev), in_extent_pairs=int(inr), composited_pairs=int(comp))
    probe.close()
    frame = render.Frame(sc.n, cam.width, cam.height, key_capacity=int(K * 1.02) + 4096)
    gcam = ges.make_camera(cam)
    H, W = cam.height, cam.width
    img = torch.empty((3, H, W), device=dev)
    T = torch.empty((H, W), device=dev)
    nc = torch.empty((H, W), dtype=torch.int32, device=dev)
    dL = torch.full((3, H, W), 1.0 / (W * H), device=dev)
    grads = tuple(torch.empty_like(a) for a in t)
    scene_c, grads_c = ges.make_scene(*t, sc.sh_degree), ges.make_grads(*grads)

    def step(bwd):
        ges.ges_preprocess(frame.handle, scene_c, gcam, params)
        ges.ges_bin_sort(frame.handle)
        ges.ges_render_fwd(frame.handle, img, T, nc)
        if bwd:
            ges.ges_render_bwd(frame.handle, scene_c, T, nc, dL, grads_c)

    out = {}
    ctx = render.default_context(dev.index or 0)
    for bwd in (False, True):
        for _ in range(warmup):
            step(bwd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step(bwd)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["fwd_bwd" if bwd else "fwd"] = {"mpix_s": W * H / (ms / 1e3) / 1e6, "ms_per_frame": ms}
    if detail is not None:  # per-kernel times from a separate traced run (tracing adds events per launch)
        ges.ges_trace_enable(ctx.handle, True)
        for _ in range(steps):
            step(True)
        torch.cuda.synchronize()
        tr = ges.ges_trace_read(ctx.handle)
        ges.ges_trace_enable(ctx.handle, False)
        detail["kernel_ms"] = {k: ms / n for k, (n, ms) in tr.items()}
    assert frame.status()[0] == 0
    assert all(torch.isfinite(g).all() for g in grads)
    frame.close()
    return int(K), out


def stress_bench(steps, warmup, dev, beta2, segment_tiles):
    """The stress configuration (6M cube primitives, SH3, 3840x2160): fwd and fwd+bwd, either with
    beta log-U[0.3,16] (very sharp and very wide kernels; listed per tile row, segment_tiles =
    256) or with beta = 2 everywhere (the Gaussian degenerate case)."""
    from paper_2402_10128_gb300 import ges, render, scenes
    sc, cam = scenes.stress_beta2_workload() if beta2 else scenes.stress_workload()
    t = render.scene_tensors(sc, dev)
    params = ges.params_default()
    params.segment_tiles = segment_tiles
    K, out = _time_c_abi_steps(sc, t, cam, params, steps, warmup, dev)
    form = "beta = 2" if beta2 else "beta log-U[0.3,16]"
    return {"workload": f"stress, {form}: 6M cube primitives, SH3, 3840x2160", "segment_tiles": segment_tiles,
            "K_entries": K, "steps": steps, **out}


def scale_modification_bench(steps, warmup, dev, sc, t, cam, segment_tiles, roofline_fn=None, cpu_pixels=1000):
    """The scale-modification variants (Sec. 4.2 and the ablation's shape strengths) on one view of
    the scene-scale workload: phi_bar_rho at rho = 0.1 (default), 0 and 10, the exact normalised
    Gamma ratio on the scale vector and on the variance, and the Gaussian-form rasterizer.  The
    exact ratio makes small-beta primitives far larger (240x at beta = 1/2), hence more list entries
    and more pairs to composite."""
    from paper_2402_10128_gb300 import ges
    variants = {"phi_bar_rho0.1": {}, "phi_bar_rho0": {"rho": 0.0}, "phi_bar_rho10": {"rho": 10.0},
                "phi_exact": {"phi_mode": ges.GES_PHI_EXACT},
                "phi_exact_variance": {"phi_mode": ges.GES_PHI_EXACT_VARIANCE},
                "gaussian_form_phi_bar": {"falloff": ges.GES_FALLOFF_PAPER_APPROX}}
    import oracle
    rng = np.random.default_rng(5)
    pix = rng.choice(cam.width * cam.height, cpu_pixels, replace=False)
    gpx = rng.standard_normal((3, cpu_pixels))
    res = {}
    for name, kw in variants.items():
        params = ges.params_default()
        params.segment_tiles = segment_tiles
        for k, v in kw.items():
            setattr(params, k, v)
        detail = {}
        K, out = _time_c_abi_steps(sc, t, cam, params, steps, warmup, dev, detail)
        entry = {"K_entries": K, **out, "pairs": {k: detail[k] for k in ("evaluated_pairs", "in_extent_pairs",
                                                                        "composited_pairs")},
                 "k_render_bwd_ms": detail["kernel_ms"].get("k_render_bwd"),
                 "k_render_fwd_ms": detail["kernel_ms"].get("k_render_fwd")}
        if roofline_fn is not None:
            inr, comp = detail["in_extent_pairs"], detail["composited_pairs"]
            gef = params.falloff == ges.GES_FALLOFF_GEF
            # per pair: GEF lg2 + 2 ex2 (fwd and bwd) and 2 rcp (bwd); Gaussian form 1 ex2 and 1 rcp (bwd)
            entry["roofline_bwd"] = roofline_fn("k_render_bwd", entry["k_render_bwd_ms"], inr if gef else 0,
                                                2 * inr if gef else inr, 2 * comp if gef else comp,
                                                composite_fp32_ops(gef, inr, comp)[1],
                                                "MUFU and FP32 work of this variant's pairs")
        # the oracle (FP64 brute force on the host) on a sample of pixels of the same view and variant
        op = {"rho": float(params.rho), "mode": int(params.falloff), "phi_mode": int(params.phi_mode)}
        t0 = time.perf_counter()
        oracle.backward(sc, cam, gpx, params=op, pixels=pix, nthreads=os.cpu_count() or 1)
        entry["cpu_baseline"] = {"kind": "oracle", "value": cpu_pixels / (time.perf_counter() - t0) / 1e6,
                                 "unit": "Mpix/s", "sample": f"{cpu_pixels} random pixels, fwd+bwd, FP64 brute force"}
        res[name] = entry
    return {"workload": "scene-scale view 0: 1.5M clustered primitives, SH3, beta log-U[0.5,8], 1245x825",
            "steps": steps, "segment_tiles": segment_tiles, "variants": res}


def e2e(args, sc, gcam, frame, params, dev, stream, ws, dist, full_transfer=False):
    """The fwd+bwd step through the C-ABI with host buffers.  Default: the scene is the model,
    uploaded once from pinned host memory before the timed region (as weights are); every step
    copies its input in (the upstream gradient dL/dI, 12 MB; the camera travels by value) and its
    results out: the rendered image (12 MB) and the gradients of every primitive parameter
    (360 MB at SH3), the step's product.  full_transfer: the scene is copied in every step as well
    (372 MB in, 372 MB out).  The copies are pipelined against the kernels: two slots of device
    buffers; step i's inputs travel on one copy stream while step i-1 computes, and its results
    travel back on another while step i+1 computes."""
    import torch
    from paper_2402_10128_gb300 import ges
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in sc.arrays()]
    gen = torch.Generator().manual_seed(3)
    dL_h = ((torch.rand((3, HEIGHT, WIDTH), generator=gen) - 0.5) * (2.0 / (WIDTH * HEIGHT))).pin_memory()
    resident = None if full_transfer else [h.to(dev, non_blocking=False) for h in host]
    slots = []
    for _ in range(2):
        dev_in = [torch.empty(h.shape, dtype=h.dtype, device=dev) for h in host] if full_transfer else resident
        grads = [torch.empty_like(a) for a in dev_in]
        slots.append(dict(dev_in=dev_in, dL=torch.empty_like(dL_h, device=dev), grads=grads,
                          img=torch.empty((3, HEIGHT, WIDTH), device=dev),
                          img_h=torch.empty((3, HEIGHT, WIDTH)).pin_memory(),
                          grads_h=[torch.empty(h.shape).pin_memory() for h in host],
                          scene=ges.make_scene(*dev_in, sc.sh_degree), grads_c=ges.make_grads(*grads),
                          in_ready=torch.cuda.Event(), computed=torch.cuda.Event(), out_done=torch.cuda.Event(),
                          used=False))
    T = torch.empty((HEIGHT, WIDTH), device=dev)
    nc = torch.empty((HEIGHT, WIDTH), dtype=torch.int32, device=dev)
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    h2d = dL_h.numel() * 4 + (sum(h.numel() * 4 for h in host) if full_transfer else 0)
    d2h = slots[0]["img_h"].numel() * 4 + sum(h.numel() * 4 for h in slots[0]["grads_h"])

    def step(i):
        sl = slots[i % 2]
        with torch.cuda.stream(s_in):
            if sl["used"]:
                s_in.wait_event(sl["computed"])  # the kernels of step i-2 are done with this slot's inputs
            if full_transfer:
                for d, h in zip(sl["dev_in"], host):
                    d.copy_(h, non_blocking=True)
            sl["dL"].copy_(dL_h, non_blocking=True)
            sl["in_ready"].record(s_in)
        stream.wait_event(sl["in_ready"])
        if sl["used"]:
            stream.wait_event(sl["out_done"])  # step i-2's results have left this slot's outputs
        cam = gcam[i % len(gcam)]
        ges.ges_preprocess(frame.handle, sl["scene"], cam, params, sp)
        ges.ges_bin_sort(frame.handle, sp)
        ges.ges_render_fwd(frame.handle, sl["img"], T, nc, sp)
        ges.ges_render_bwd(frame.handle, sl["scene"], T, nc, sl["dL"], sl["grads_c"], sp)
        sl["computed"].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(sl["computed"])
            sl["img_h"].copy_(sl["img"], non_blocking=True)
            for h, d in zip(sl["grads_h"], sl["grads"]):
                h.copy_(d, non_blocking=True)
            sl["out_done"].record(s_out)
        sl["used"] = True

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    s_in.wait_stream(stream)  # no copy of the timed steps starts before s0
    for i in range(args.steps):
        step(i)
    stream.wait_stream(s_in)
    stream.wait_stream(s_out)  # the last results are in host memory
    s1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(s0.elapsed_time(s1), dist, dev)
    what = ("per step: scene and dL/dI in; image and all gradients out" if full_transfer
            else "scene resident (uploaded once, as weights); per step: dL/dI in; image and all gradients out")
    return {"value": aggregate_mpix_s(ws, WIDTH * HEIGHT, args.steps, ms), "unit": "Mpix/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / args.steps,
            "what": what,
            "overlap": "copies pipelined against the kernels (two buffer slots, one copy stream per direction)"}


if __name__ == "__main__":
    main()
