"""Benchmark: 2-D DWT by non-separable lifting on one GB300 (and N replicas under torchrun).

Workload: one 8192 x 8192 seeded 1/f^2 field in [0, 255], 5 decomposition levels.  The headline
value is the forward CDF 9/7 (fp32) transform in Gpixel/s (level-0 pixels per second); the same
line carries the reversible integer CDF 5/3 forward, both inverses and the separable-lifting
comparators (one-pass Eq. 3 steps and the two-pass row/column transform), each with its HBM
GB/s against the measured copy roofline.

Timing: W untimed warm-up steps, then K timed steps; before every timed step L2 is flushed (a
2xL2 buffer written, a second one read); each step is timed with CUDA events on the stream the library
launches on.  Clocks and throttle reasons are sampled with nvidia-smi during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (fp64, all host cores) on the same workload and prints the
same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import subprocess
import tempfile
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

H = W = 8192
LEVELS = 5
METRIC = "Gpixel/s & HBM GB/s (% of peak), 2-D DWT non-separable vs separable, 1 GB300"
CONFIG = {"workload": "8192x8192 seeded 1/f^2 field in [0,255], 5-level 2-D DWT, forward CDF 9/7 "
                      "fp32 (headline) + reversible CDF 5/3 int32, non-separable vs separable",
          "image": [H, W], "levels": LEVELS,
          "l2": "flushed before every timed step: a 2xL2 buffer is written, then a second 2xL2 "
                "buffer is read, so the timed step starts with no data of its own and no dirty "
                "lines in L2"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alg_bytes(h: int, w: int, levels: int, esize: int = 4) -> int:
    """One read and one write of every level's input plane."""
    tot = 0
    for _ in range(levels):
        tot += 2 * h * w * esize
        h, w = (h + 1) // 2, (w + 1) // 2
    return tot


# Sources the level-1 forward kernel is compiled from: a recorded ncu capture counts only while
# their code is unchanged.
KERNEL_SOURCES = {"fwd_l1_cdf97_f32": ["dwt2_device.cuh", "dwt2_lifting.cuh", "dwt2_stream.cuh",
                                       "dwt2_fwd_f97.cu"]}


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed (string literals in these
    files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def src_hash(kernel_key: str) -> str:
    """Hash of the code (not the comments) of a kernel's sources."""
    d = os.path.join(ROOT, "paper_1708_07853_gb300", "csrc")
    m = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel_key]:
        m.update(_code_only(open(os.path.join(d, f)).read()).encode())
    return m.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel_key)
    if not e or e.get("src_hash") != src_hash(kernel_key):
        return None
    return e.get("dram_bytes_per_launch")


class L2Flush:
    """Evicts everything from L2 before a timed step: writes one buffer of twice the L2 size,
    then reads a second one (the read pass writes the first buffer's dirty lines back to HBM
    outside the timed region)."""

    def __init__(self, nbytes: int, dev):
        self.w = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(nbytes // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.fill_(1.0)
        self.r.sum()


class ClockSampler:
    """nvidia-smi samples (every 20 ms) kept with their wall time; summarised for a window."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.samples, self.proc, self.err = index, [], None, None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError as e:
            self.err = str(e)
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        """Samples inside [t0, t1].  A window too short for 3 samples is extended forward by up
        to 0.5 s, into the timed cases that follow it (the GPU stays busy), and the extension
        is reported."""
        margin = 0.0
        rows = [s for t, s in self.samples if t0 <= t <= t1]
        while len(rows) < 3 and margin < 0.5:
            margin += 0.05
            rows = [s for t, s in self.samples if t0 <= t <= t1 + margin]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0, "note": self.err or "no sample inside the timed window"}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, smax, reasons = [], [], set()
        for r in rows:
            p = [v.strip() for v in r.split(",")]
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, p[2:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "window_margin_s": round(margin, 2)}


# ------------------------------------------------------------------------------ reference arm
# ------------------------------------------------------------------------------ multi-rank runs
# With N ranks (one per GPU, under torchrun) every rank runs the whole workload on its own image:
# replicas, since one image is not split across GPUs.  The job's time is the slowest rank's,
# and its rate counts every rank's pixels.

def max_over_ranks(ms: float, world: int, device) -> float:
    """The largest of the ranks' times (a collective over the default process group)."""
    if world <= 1:
        return ms
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job rate in giga-units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def host_cpu():
    """(usable host cores, CPU model from lscpu)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - Linux has it
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model


def oracle_forward_seconds(O, img: np.ndarray, threads: int, reps: int):
    """Median wall time of `reps` oracle forwards (CDF 9/7 fp64, LEVELS levels) of img."""
    O.set_threads(threads)
    try:
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            O.forward(img, "cdf97", LEVELS)
            ts.append(time.perf_counter() - t)
    finally:
        O.set_threads(1)
    return float(np.median(ts))


# Longest the reference arm may take (warm-up + timed steps) before it times a crop instead.
REFERENCE_BUDGET_S = 180.0


def run_reference(args, rank: int, world: int):
    """The oracle over all host cores on the workload image, one full forward per step."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1708_07853_gb300 import inputs as I

    O.build()
    cores, model = host_cpu()
    img = I.field(H, W, I.seed_for(1)).astype(np.float64)
    est = oracle_forward_seconds(O, img, cores, 1)  # one probe run, untimed
    side = H
    if est * (args.steps + args.warmup) > REFERENCE_BUDGET_S:  # too many steps: a crop
        side = int(H * np.sqrt(REFERENCE_BUDGET_S / (est * (args.steps + args.warmup))))
        side = max(256, side // 256 * 256)
        img = np.ascontiguousarray(img[:side, :side])
    O.set_threads(cores)
    times = []
    try:
        for i in range(args.warmup + args.steps):
            t = time.perf_counter()
            O.forward(img, "cdf97", LEVELS)
            if i >= args.warmup:
                times.append(time.perf_counter() - t)
    finally:
        O.set_threads(1)
    ms = 1e3 * float(np.median(times))
    gpix = side * side / (ms * 1e-3) / 1e9
    sample = (f"{'the full' if side == H else f'a {side}x{side} top-left crop of the'} "
              f"{H}x{W} workload image per step, CDF 9/7 fp64, {LEVELS} levels, "
              f"{cores} host threads (median of {args.steps})")
    line = {"impl": "reference", "metric": METRIC, "value": round(gpix, 5), "unit": "Gpixel/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, parallelism="host cores"),
            "cpu_baseline": {"kind": "oracle", "value": round(gpix, 5), "unit": "Gpixel/s",
                             "cores": cores, "cpu_model": model, "sample": sample},
            "e2e": {"value": round(gpix, 5), "unit": "Gpixel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ our arm
def run_only(args, D, dev, x_f32, x_i32, flush, stream):
    """One case, W warm-up and K timed calls (the command the profiler captures)."""
    wv, x, lv, inv, scheme = {
        "fwd_l1_cdf97": ("cdf97", x_f32, 1, False, "nonsep"),
        "fwd_cdf97": ("cdf97", x_f32, LEVELS, False, "nonsep"),
        "inv_cdf97": ("cdf97", x_f32, LEVELS, True, "nonsep"),
        "fwd_cdf53_int": ("cdf53_int", x_i32, LEVELS, False, "nonsep"),
        "inv_cdf53_int": ("cdf53_int", x_i32, LEVELS, True, "nonsep"),
        "fwd_dd137": ("dd137", x_f32, LEVELS, False, "nonsep"),
        "inv_dd137": ("dd137", x_f32, LEVELS, True, "nonsep"),
        "twopass_cdf97": ("cdf97", x_f32, LEVELS, False, "sep_twopass"),
        "sepfused_cdf97": ("cdf97", x_f32, LEVELS, False, "sep_fused"),
        "adapted_cdf97": ("cdf97", x_f32, LEVELS, False, "adapted"),
        "conv_cdf97": ("cdf97", x_f32, LEVELS, False, "conv"),
        "plan_cdf97": ("cdf97", x_f32, LEVELS, False, "plan"),
        "plan_cdf53_int": ("cdf53_int", x_i32, LEVELS, False, "plan"),
        "batch_plan_cdf97": ("cdf97", x_f32, 4, False, "batch_plan"),
        "batch_plan_cdf53_int": ("cdf53_int", x_i32, 4, False, "batch_plan"),
    }[args.only]
    if args.levels:
        lv = args.levels
    bdt = D.TORCH_DT[x.dtype]
    out = torch.empty_like(x)
    ab = alg_bytes(H, W, lv)
    if scheme == "plan":
        # the same image through a one-image plan: all levels in one persistent launch
        plan, (c,) = D.plan_forward([x], wv, lv)
        ws = plan.workspace

        def step():
            plan.run()
    elif scheme == "batch_plan":
        # the default run's 512 uneven images (or the first --images of them) through one plan
        # (default tile rows, no autotuner launches before the timed ones)
        from paper_1708_07853_gb300 import inputs as I
        sizes = I.batch_sizes(512, I.seed_for(3))[:args.images]
        imgs = [I.field_device(h, w, I.seed_for(3, k), dev).to(x.dtype)
                for k, (h, w) in enumerate(sizes)]
        plan, _ = D.plan_forward(imgs, wv, lv)
        ws = plan.workspace
        ab = sum(alg_bytes(h, w, lv) for h, w in sizes)

        def step():
            plan.run()
    else:
        c = D.alloc_coeffs(H, W, lv, wv, bdt, dev)
        ws = D.new_workspace(D.workspace_bytes(H, W, lv, wv, bdt, scheme), dev)
        D.forward(x, wv, lv, scheme=scheme, out=c, workspace=ws)

        def step():
            if inv:
                D.inverse(c, out=out, workspace=ws)
            else:
                D.forward(x, wv, lv, scheme=scheme, out=c, workspace=ws)

    for _ in range(args.warmup):
        step()
    evs = []
    for _ in range(args.steps):
        flush()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        step()
        e.record(stream)
        evs.append((s, e))
    torch.cuda.synchronize()
    ms = float(np.mean([s.elapsed_time(e) for s, e in evs]))
    print(json.dumps({"only": args.only, "ms": ms, "levels": lv,
                      "gb_s": ab / (ms * 1e-3) / 1e9,
                      "plan": plan.info() if scheme in ("plan", "batch_plan") else None,
                      "status": D.check_status(ws)}), flush=True)


def run_levels_table(args, D, dev, x_f32, x_i32, flush, stream):
    """Per-level times of the 8192 x 8192 forward and inverse transforms: the median of K calls
    of the J-level transform for J = 1 .. LEVELS, L2 flushed before each call; level j's time is
    the J = j median minus the J = j - 1 one (PDL lets a level overlap the previous one's tail,
    so a level's share is what adding it costs the transform)."""
    def med(fn):
        for _ in range(args.warmup):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for s0, e0 in evs:
            flush()
            s0.record(stream)
            fn()
            e0.record(stream)
        torch.cuda.synchronize()
        return 1e3 * float(np.median([a.elapsed_time(b) for a, b in evs]))  # us

    report = {}
    for wv, x in (("cdf97", x_f32), ("cdf53_int", x_i32), ("cdf53", x_f32)):
        bdt = D.TORCH_DT[x.dtype]
        out = torch.empty_like(x)
        fwd, inv = [], []
        for lv in range(1, LEVELS + 1):
            c = D.alloc_coeffs(H, W, lv, wv, bdt, dev)
            ws = D.new_workspace(D.workspace_bytes(H, W, lv, wv, bdt), dev)
            fwd.append(med(lambda: D.forward(x, wv, lv, out=c, workspace=ws)))
            inv.append(med(lambda: D.inverse(c, out=out, workspace=ws)))
            del c, ws
        per = lambda t: [round(t[0], 1)] + [round(t[k] - t[k - 1], 1) for k in range(1, len(t))]
        report[wv] = {"forward_level_us": per(fwd), "forward_total_us": round(fwd[-1], 1),
                      "inverse_level_us": per(inv), "inverse_total_us": round(inv[-1], 1),
                      "level_bytes": [2 * x.element_size() * (H >> j) * (W >> j)
                                      for j in range(LEVELS)]}
    print(json.dumps({"levels_table": f"{H}x{W}, 1..{LEVELS} levels, median of {args.steps} "
                                      "calls per transform, L2 flushed before each",
                      "report": report}), flush=True)


def storage_bytes(h: int, w: int, levels: int, in_es: int, band_es: int, ll_es: int = 4) -> int:
    """Algorithmic bytes of a forward with band storage band_es: per level one read of the
    input plane and one write of the four bands (LL planes fp32)."""
    tot = 0
    for j in range(levels):
        ner, nec = (h + 1) // 2, (w + 1) // 2
        tot += h * w * (in_es if j == 0 else ll_es) + ner * nec * ll_es + (h * w - ner * nec) * band_es
        h, w = ner, nec
    return tot


def run_precision(args, D, I, dev, flush, stream):
    """Config 3: 16384 x 16384, field + uniform noise in [0, 255], CDF 9/7, 5 levels."""
    from oracle import oracle as O
    O.build()
    n, lv = 16384, LEVELS
    x = I.field_plus_noise(n, n, I.seed_for(2))
    want = O.forward(x.astype(np.float64), "cdf97", lv)
    shapes = O.band_shapes(n, n, lv)
    xg = torch.from_numpy(x).to(dev)
    report = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        c = D.forward(xg, "cdf97", lv, band_dtype=dt)
        bands = {}
        for (kind, j, h, w), v, wv in zip(shapes, c.band_views(), want):
            if wv.size == 0:
                continue
            d = v.float().cpu().numpy().astype(np.float64) - wv
            bands[f"{kind}{j}"] = {"max": float(np.abs(d).max()), "rms": float(np.sqrt((d * d).mean()))}
        r = D.inverse(c, img_dtype=torch.float32)
        rd = (r.double() - xg.double())
        ws = D.new_workspace(D.workspace_bytes(n, n, lv, "cdf97", D.TORCH_DT[dt]), dev)
        for _ in range(args.warmup):
            D.forward(xg, "cdf97", lv, band_dtype=dt, out=c, workspace=ws)
        evs = []
        for _ in range(args.steps):
            flush()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            D.forward(xg, "cdf97", lv, band_dtype=dt, out=c, workspace=ws)
            e0.record(stream)
            evs.append((s0, e0))
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        nbytes = storage_bytes(n, n, lv, 4, 2 if dt != torch.float32 else 4)
        report[name] = {"bands": bands, "roundtrip_max": float(rd.abs().max()),
                        "roundtrip_rms": float(rd.pow(2).mean().sqrt()), "ms": round(ms, 4),
                        "gpix_s": round(n * n / (ms * 1e-3) / 1e9, 2),
                        "algorithmic_bytes": nbytes, "gb_s": round(nbytes / (ms * 1e-3) / 1e9, 1)}
    print(json.dumps({"precision": "16384x16384 field+noise in [0,255], CDF 9/7, 5 levels, "
                                   "fp32 arithmetic; band storage fp32 / bf16 / fp16, LL fp32",
                      "report": report}), flush=True)



# ------------------------------------------------------------------------------------------------
# The other workloads of the scope table, timed in the default run beside the headline:
# a batch of 512 uneven images (one persistent launch from a CUDA graph vs one call per image),
# the autograd step on 64 x 3 x 1024^2, and 16384^2 band storage in fp32 / bf16 / fp16.

def run_batch_workload(D, I, dev, run_case, steps, warmup):
    """512 images, sides log-uniform on [63, 4096], 4 levels; int 5/3 and fp32 9/7."""
    sizes = I.batch_sizes(512, I.seed_for(3))
    lv = 4
    npix = sum(h * w for h, w in sizes)
    ab = sum(alg_bytes(h, w, lv) for h, w in sizes)
    res = {"images": len(sizes), "levels": lv, "pixels": npix,
           "algorithmic_bytes_per_step": ab,
           "sizes": "each side round(exp(U[ln 63, ln 4096])), independent, seeded"}
    for wv, dt in (("cdf53_int", torch.int32), ("cdf97", torch.float32)):
        imgs = [I.field_device(h, w, I.seed_for(3, k), dev).to(dt) for k, (h, w) in
                enumerate(sizes)]
        with tempfile.TemporaryDirectory() as td:
            plan, coeffs = D.plan_forward(imgs, wv, lv, tune_cache=os.path.join(td, "tune.txt"))
        ms_plan = run_case(plan.run, steps, warmup)
        status = D.check_status(plan.workspace)
        bdt = D.TORCH_DT[dt]
        ws = D.new_workspace(max(D.workspace_bytes(h, w, lv, wv, bdt) for h, w in sizes), dev)

        def loop():
            for x, c in zip(imgs, coeffs):
                D.forward(x, wv, lv, out=c, workspace=ws)

        ms_loop = run_case(loop, max(3, steps // 4), warmup)
        ms_graph = None
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                loop()
            ms_graph = run_case(g.replay, steps, warmup)
        except RuntimeError as e:  # report, do not hide, a capture failure
            ms_graph = f"capture failed: {str(e).splitlines()[0]}"
        # the plan's bits equal the per-image calls' bits
        plan.run()
        snap = [coeffs[k].buffer.clone() for k in (0, 255, 511)]
        loop()
        torch.cuda.synchronize()
        same = all(torch.equal(a, coeffs[k].buffer) for a, k in zip(snap, (0, 255, 511)))

        def rate(ms):
            if not isinstance(ms, float):
                return ms
            return {"ms": round(ms, 4), "gpix_s": round(npix / (ms * 1e-3) / 1e9, 2),
                    "gb_s": round(ab / (ms * 1e-3) / 1e9, 1)}

        res[wv] = {"plan_graph": rate(ms_plan), "per_image_calls": rate(ms_loop),
                   "per_image_calls_graph": rate(ms_graph), "plan": plan.info(),
                   "plan_equals_per_image_calls": same, "device_status": status}
        plan.close()
        del imgs, coeffs, ws, plan
        torch.cuda.empty_cache()
    return res


def run_autograd_workload(D, A, I, dev, run_case, steps, warmup):
    """64 x 3 x 1024^2 fp32 in [0, 1], 3-level 9/7: loss = L1 of every high-pass band plus the
    MSE of the reconstruction; one step = forward + backward through the autograd Functions."""
    B, C, H, W, lv = 64, 3, 1024, 1024, 3
    x = torch.empty((B, C, H, W), device=dev)
    flat = x.view(-1, H, W)
    for k in range(B * C):
        flat[k] = I.field_device(H, W, I.seed_for(4, k), dev) / 255.0
    x.requires_grad_(True)
    n = A.coeff_floats(H, W, lv)
    lay, _ = D.layout(H, W, lv, D.DT_F32)
    mask = torch.ones(n, device=dev)
    ll = lay[0]
    mask[ll.offset_bytes // 4: ll.offset_bytes // 4 + ll.h * ll.pitch_bytes // 4] = 0.0

    def step():
        c = A.dwt2(x, "cdf97", lv)
        y = A.idwt2(c, H, W, "cdf97", lv)
        loss = (c.abs() * mask).sum() + (y - x).pow(2).mean()
        loss.backward()
        x.grad = None

    ms_step = run_case(step, steps, warmup)
    # the four transforms of a step alone, through the batched entry points
    xs = x.detach().view(-1, H, W)
    N = xs.shape[0]
    cbuf = torch.zeros((N, n), device=dev)
    ybuf = torch.empty_like(xs)
    gc = torch.zeros_like(cbuf)
    gx = torch.empty_like(xs)
    ws = D.new_workspace(D.workspace_bytes_batch(N, H, W, lv, "cdf97", D.DT_F32), dev)

    def transforms():
        D.forward_batch(xs, "cdf97", lv, D.DT_F32, out=cbuf, workspace=ws)
        D.inverse_batch(cbuf, H, W, "cdf97", lv, D.DT_F32, out=ybuf, workspace=ws)
        D.inverse_adjoint_batch(ybuf, "cdf97", lv, out=gc, workspace=ws)
        D.forward_adjoint_batch(gc, H, W, "cdf97", lv, out=gx, workspace=ws)

    ms_tr = run_case(transforms, steps, warmup)
    ms_fwd = run_case(lambda: D.forward_batch(xs, "cdf97", lv, D.DT_F32, out=cbuf, workspace=ws),
                      steps, warmup)
    status = D.check_status(ws)
    npix = N * H * W
    ab = N * alg_bytes(H, W, lv)
    return {"batch": [B, C, H, W], "levels": lv, "pixels": npix,
            "fwd_bwd_step": {"ms": round(ms_step, 4),
                             "gpix_s": round(npix / (ms_step * 1e-3) / 1e9, 2)},
            "four_transforms": {"ms": round(ms_tr, 4),
                                "gb_s": round(4 * ab / (ms_tr * 1e-3) / 1e9, 1),
                                "share_of_step": round(ms_tr / ms_step, 3)},
            "forward_only_plain_f32": {"ms": round(ms_fwd, 4),
                                       "gpix_s": round(npix / (ms_fwd * 1e-3) / 1e9, 2),
                                       "gb_s": round(ab / (ms_fwd * 1e-3) / 1e9, 1)},
            "algorithmic_bytes_per_transform": ab, "device_status": status}


def run_storage_workload(D, I, dev, run_case, steps, warmup):
    """16384^2, 0.5 * field + 0.5 * U[0, 255), CDF 9/7, 5 levels: fp32 vs bf16 / fp16 band
    storage (fp32 arithmetic, fp32 LL), forward and inverse times.  The per-band errors against
    the fp64 oracle come from --precision."""
    n, lv = 16384, LEVELS
    g = torch.Generator(device=dev).manual_seed(I.seed_for(2) + 50)
    x = 0.5 * I.field_device(n, n, I.seed_for(2), dev, integer=False) + \
        0.5 * 255.0 * torch.rand((n, n), generator=g, device=dev)
    res = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        bdt = D.TORCH_DT[dt]
        c = D.alloc_coeffs(n, n, lv, "cdf97", bdt, dev)
        ws = D.new_workspace(D.workspace_bytes(n, n, lv, "cdf97", bdt), dev)
        y = torch.empty_like(x)
        ms_f = run_case(lambda: D.forward(x, "cdf97", lv, band_dtype=bdt, out=c, workspace=ws),
                        steps, warmup)
        ms_i = run_case(lambda: D.inverse(c, out=y, workspace=ws), steps, warmup)
        nb = storage_bytes(n, n, lv, 4, 4 if dt == torch.float32 else 2)
        res[name] = {"fwd_ms": round(ms_f, 4), "fwd_gpix_s": round(n * n / (ms_f * 1e-3) / 1e9, 2),
                     "inv_ms": round(ms_i, 4), "inv_gpix_s": round(n * n / (ms_i * 1e-3) / 1e9, 2),
                     "storage_bytes": nb, "fwd_gb_s": round(nb / (ms_f * 1e-3) / 1e9, 1),
                     "roundtrip_max_abs": float((y - x).abs().max()),
                     "device_status": D.check_status(ws)}
        del c, ws, y
    del x
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the batched, autograd and storage workloads")
    ap.add_argument("--precision", action="store_true",
                    help="16384x16384 CDF 9/7, 5 levels: per-band error of fp32 / bf16 / fp16 band "
                         "storage against the fp64 oracle, and the time of each")
    ap.add_argument("--only", default=None,
                    choices=["fwd_l1_cdf97", "fwd_cdf97", "inv_cdf97", "fwd_cdf53_int",
                             "inv_cdf53_int", "fwd_dd137", "inv_dd137", "twopass_cdf97", "sepfused_cdf97", "adapted_cdf97",
                             "conv_cdf97", "plan_cdf97", "plan_cdf53_int", "batch_plan_cdf97",
                             "batch_plan_cdf53_int"],
                    help="run one case only (for profiler captures); prints a short line")
    ap.add_argument("--levels-table", action="store_true",
                    help="8192x8192: per-level forward and inverse times of each wavelet")
    ap.add_argument("--images", type=int, default=512,
                    help="with --only batch_plan_*: the first N images of the 512-image batch")
    ap.add_argument("--levels", type=int, default=0,
                    help="with --only: decomposition levels instead of the case's own")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch.distributed as dist
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1708_07853_gb300 import build as B
    B.build()
    from paper_1708_07853_gb300 import dwt2 as D
    from paper_1708_07853_gb300 import inputs as I

    def barrier():
        if world > 1:
            dist.barrier()

    peak, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream()
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = L2Flush(2 * l2, dev)

    if args.precision:
        return run_precision(args, D, I, dev, flush, stream)

    field = I.field(H, W, I.seed_for(1))
    x_f32 = torch.from_numpy(field).to(dev)
    x_i32 = torch.from_numpy(field.astype(np.int32)).to(dev)
    npix = H * W

    if args.only:
        return run_only(args, D, dev, x_f32, x_i32, flush, stream)
    if args.levels_table:
        return run_levels_table(args, D, dev, x_f32, x_i32, flush, stream)

    def run_case(fn, steps, warmup):
        """Median CUDA-event time (ms) of `steps` calls, L2 flushed before each."""
        for _ in range(warmup):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for s, e in evs:
            flush()
            s.record(stream)
            fn()
            e.record(stream)
        torch.cuda.synchronize()
        return float(np.median([s.elapsed_time(e) for s, e in evs]))  # ms

    cases = {}

    def make(wv, x, scheme="nonsep", levels=LEVELS):
        bdt = D.TORCH_DT[x.dtype]
        c = D.alloc_coeffs(H, W, levels, wv, bdt, dev)
        ws = D.new_workspace(D.workspace_bytes(H, W, levels, wv, bdt, scheme), dev)
        return c, ws, bdt

    # ---- headline: forward CDF 9/7 fp32, non-separable, 5 levels (timed region) ----
    c97, ws97, _ = make("cdf97", x_f32)

    def fwd97():
        D.forward(x_f32, "cdf97", LEVELS, out=c97, workspace=ws97)

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    time.sleep(0.3)  # let the sampler start delivering
    # about a second of back-to-back transforms first, so that the timed steps do not start on
    # clocks still ramping up from idle
    t_warm = time.time()
    while time.time() - t_warm < 1.0:
        for _ in range(50):
            fwd97()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        fwd97()
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    ms_main = run_case(fwd97, args.steps, 0)
    torch.cuda.synchronize()
    barrier()
    t1 = time.time()
    ms_main = max_over_ranks(ms_main, world, dev)
    status = D.check_status(ws97)

    ab = alg_bytes(H, W, LEVELS)
    gpix_main = job_rate(npix, world, ms_main)

    def summarise(ms, nbytes=ab):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"ms": round(ms, 4), "gpix_s": round(npix / (ms * 1e-3) / 1e9, 2),
                "gb_s": round(gbs, 1), "frac_measured": round(gbs / peak, 3),
                "frac_nominal_8tbs": round(gbs / 8000.0, 3)}

    cases["fwd_cdf97_f32_nonsep"] = summarise(ms_main)

    # ---- the other cases (same harness, not the headline) ----
    ci, wsi, _ = make("cdf53_int", x_i32)
    cases["fwd_cdf53_int_nonsep"] = summarise(run_case(
        lambda: D.forward(x_i32, "cdf53_int", LEVELS, out=ci, workspace=wsi), args.steps,
        args.warmup))
    out_f = torch.empty_like(x_f32)
    out_i = torch.empty_like(x_i32)
    cases["inv_cdf97_f32_nonsep"] = summarise(run_case(
        lambda: D.inverse(c97, out=out_f, workspace=ws97), args.steps, args.warmup))
    cases["inv_cdf53_int_nonsep"] = summarise(run_case(
        lambda: D.inverse(ci, out=out_i, workspace=wsi), args.steps, args.warmup))
    # the Deslauriers-Dubuc wavelets (four-tap steps) through the same non-separable kernels
    for wv in ("dd97", "dd137"):
        cd, wsd, _ = make(wv, x_f32)
        cases[f"fwd_{wv}_f32_nonsep"] = summarise(run_case(
            lambda: D.forward(x_f32, wv, LEVELS, out=cd, workspace=wsd), args.steps,
            args.warmup))
        cases[f"inv_{wv}_f32_nonsep"] = summarise(run_case(
            lambda: D.inverse(cd, out=out_f, workspace=wsd), args.steps, args.warmup))
        del cd, wsd
    for scheme in ("sep_fused", "sep_twopass"):
        for wv, x in (("cdf97", x_f32), ("cdf53_int", x_i32)):
            c, ws, _ = make(wv, x, scheme)
            ms = run_case(lambda: D.forward(x, wv, LEVELS, scheme=scheme, out=c, workspace=ws),
                          args.steps, args.warmup)
            cases[f"fwd_{wv}_{scheme}"] = summarise(ms)
    # the two-pass comparator of the four-tap Deslauriers-Dubuc 13/7
    cd2, wsd2, _ = make("dd137", x_f32, "sep_twopass")
    cases["fwd_dd137_sep_twopass"] = summarise(run_case(
        lambda: D.forward(x_f32, "dd137", LEVELS, scheme="sep_twopass", out=cd2, workspace=wsd2),
        args.steps, args.warmup))
    del cd2, wsd2
    # the adapted non-separable scheme (Sec. 3; float wavelets): the ablation of its split
    c, ws, _ = make("cdf97", x_f32, "adapted")
    cases["fwd_cdf97_adapted"] = summarise(run_case(
        lambda: D.forward(x_f32, "cdf97", LEVELS, scheme="adapted", out=c, workspace=ws),
        args.steps, args.warmup))
    # the separable convolution (Eq. 4; float wavelets): the filter-bank comparator
    cc, wsc, _ = make("cdf97", x_f32, "conv")
    cases["fwd_cdf97_conv"] = summarise(run_case(
        lambda: D.forward(x_f32, "cdf97", LEVELS, scheme="conv", out=cc, workspace=wsc),
        args.steps, args.warmup))
    # the non-separable kernel against both separable comparators (time ratios, > 1: faster)
    comparison = {
        f"{wv}_nonsep_speedup_vs_{sc}": round(
            cases[f"fwd_{wv}_{sc}"]["ms"] / cases[f"fwd_{wv}_{ref}"]["ms"], 3)
        for wv, ref in (("cdf97", "f32_nonsep"), ("cdf53_int", "nonsep"))
        for sc in ("sep_fused", "sep_twopass")}
    comparison["dd137_nonsep_speedup_vs_sep_twopass"] = round(
        cases["fwd_dd137_sep_twopass"]["ms"] / cases["fwd_dd137_f32_nonsep"]["ms"], 3)
    correct_inv = bool(torch.equal(D.inverse(ci, out=out_i, workspace=wsi), x_i32))
    clocks = sampler.summary(t0, t1)  # the headline window (extended into these cases if short)
    sampler.stop()

    # ---- dominant kernel: the level-1 forward launch (one launch = one 1-level transform) ----
    c1, ws1, _ = make("cdf97", x_f32, levels=1)
    ms_l1 = run_case(lambda: D.forward(x_f32, "cdf97", 1, out=c1, workspace=ws1), args.steps,
                     args.warmup)
    l1_bytes = alg_bytes(H, W, 1)
    achieved = l1_bytes / (ms_l1 * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 3), "traffic": recorded_traffic("fwd_l1_cdf97_f32"),
                "kernel": "k_forward<CDF97, NONSEP, f32, TMA> (level 1, 8192x8192)",
                "algorithmic_bytes_per_launch": l1_bytes, "peak_kind": peak_kind}

    # ---- end to end through host buffers (pinned), copies inside the timed region ----
    # A caller streaming images through the public API: two buffer sets and three streams, so
    # the upload of step k + 1 overlaps the download of step k (separate copy engines).  Each
    # step's own host->device copy of its image, its transform and the device->host copy of its
    # coefficients all lie inside the timed region; the rate is steps x pixels over that time.
    host_in = [torch.from_numpy(field).pin_memory() for _ in range(2)]
    host_out = [torch.empty(c97.buffer.numel(), dtype=torch.uint8).pin_memory() for _ in range(2)]
    dev_in = [torch.empty_like(x_f32) for _ in range(2)]
    cbufs = [c97, make("cdf97", x_f32)[0]]
    wss = [ws97, D.new_workspace(D.workspace_bytes(H, W, LEVELS, "cdf97", D.DT_F32), dev)]
    s_up, s_tf, s_down = (torch.cuda.Stream(dev) for _ in range(3))
    ev_up, ev_tf, ev_down = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))

    def e2e_run(k):
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(s_up)
        for i in range(k):
            b = i % 2
            with torch.cuda.stream(s_up):
                if i >= 2:
                    s_up.wait_event(ev_tf[b])  # dev_in[b] is read by transform i - 2
                dev_in[b].copy_(host_in[b], non_blocking=True)
                ev_up[b].record(s_up)
            s_tf.wait_event(ev_up[b])
            if i >= 2:
                s_tf.wait_event(ev_down[b])  # cbufs[b] is read by download i - 2
            D.forward(dev_in[b], "cdf97", LEVELS, out=cbufs[b], workspace=wss[b], stream=s_tf)
            ev_tf[b].record(s_tf)
            with torch.cuda.stream(s_down):
                s_down.wait_event(ev_tf[b])
                host_out[b].copy_(cbufs[b].buffer, non_blocking=True)
                ev_down[b].record(s_down)
        end.record(s_down)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / k

    e2e_run(3)  # warm-up
    e2e_steps = max(4, min(args.steps, 50))
    barrier()
    ms_e2e = max_over_ranks(e2e_run(e2e_steps), world, dev)
    e2e_ok = bool(torch.equal(host_out[(e2e_steps - 1) % 2].to(dev), c97.buffer)) and \
        D.check_status(wss[1]) == 0
    e2e = {"value": round(job_rate(npix, world, ms_e2e), 3), "unit": "Gpixel/s",
           "h2d_bytes_per_step": host_in[0].numel() * host_in[0].element_size(),
           "d2h_bytes_per_step": host_out[0].numel(), "ms_per_step": round(ms_e2e, 4),
           "pipeline": "double-buffered: upload of step k+1 overlaps download of step k",
           "result_matches_device_run": e2e_ok}

    # ---- the other workloads (batched plan, autograd, reduced-precision storage) ----
    workloads = None
    if not args.headline_only:
        from paper_1708_07853_gb300 import autograd as A
        wsteps = max(3, min(args.steps, 20))
        workloads = {
            "batch_512_uneven_4lv": run_batch_workload(D, I, dev, run_case, wsteps, args.warmup),
            "autograd_64x3x1024sq_3lv": run_autograd_workload(D, A, I, dev, run_case, wsteps,
                                                                args.warmup),
            "storage_16384sq_cdf97_5lv": run_storage_workload(D, I, dev, run_case, wsteps,
                                                              args.warmup)}

    # ---- CPU baseline: the oracle on the host, bounded sample ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cores, model = host_cpu()
        img = field.astype(np.float64)
        t_all = oracle_forward_seconds(O, img, cores, 3)
        t_one = oracle_forward_seconds(O, img, 1, 3)
        cpu = {"value": round(npix / t_all / 1e9, 5), "unit": "Gpixel/s", "cores": cores,
               "cpu_model": model, "kind": "oracle",
               "sample": f"full 8192x8192 forward, CDF 9/7 fp64, 5 levels, {cores} host "
                         f"threads, median of 3", "seconds": round(t_all, 3),
               "single_thread": {"value": round(npix / t_one / 1e9, 5), "unit": "Gpixel/s",
                                 "seconds": round(t_one, 3), "sample": "the same, one thread, "
                                                                       "median of 3"}}

    line = {"metric": METRIC, "value": round(gpix_main, 2), "unit": "Gpixel/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_main, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(CONFIG, parallelism=f"replicas{world}" if world > 1 else "single",
                           algorithmic_bytes_per_step=ab),
            "hbm_gb_s": cases["fwd_cdf97_f32_nonsep"]["gb_s"],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * LEVELS, "clocks": clocks, "cases": cases,
            "comparison": comparison,
            "workloads": workloads,
            "device_status": status, "int53_roundtrip_exact": correct_inv}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
