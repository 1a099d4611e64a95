"""Benchmark of the co-sparse data term on GB300.

One step = the whole hot path on one synthetic image: patches, codes and
co-support bitmasks (cs_codes), exact scribble distances, sample tables, the
pixel x sample likelihood sum and the label normalisation (cs_likelihood).
Workload: 481x321 RGB, 5 labels x 2000 scribble samples, 7x7 patches,
Omega 98x49 (1.544e9 pixel x sample pairs per step).

Metric: pixel x sample likelihood pairs per second, whole job.
  value  device time of the K timed steps (CUDA events around each step on
         the launching stream; inputs resident in HBM; L2 flushed between
         steps by writing a 256 MB buffer outside the timed events)
  e2e    the same steps through the C ABI starting from pinned host buffers:
         host->device copy of the inputs, the step, device->host copy of the
         data term f_i (neglog), all inside the timed region
Secondary blocks of the same line (not the headline): "forms" (the BF16
tensor-core and the plain FP32 forms beside the FP8 one, each with its error
against the FP64 oracle at sampled pixels, computed outside the timed
region), "batch" (64 uneven images through cs_batch_*, graph-replayed and
autotuned), "large" (the 1024x1024 and 4096x4096 workloads, both forms,
with their errors) and "surrogate" (the learned surrogate on the 1024x1024
workload: fit and evaluation times, fallback shares and errors against the
exact sums, per fallback rule). The ALU roofline's denominators come from
cs_unit_rates, a microbenchmark of the pipes run at the start ("unit_rates").
Under torchrun (N > 1) every rank runs its own image (weak scaling, no
collective on the data path); rank 0 prints the max-over-ranks line.

--impl reference times the FP64 CPU oracle (the method's plain definition)
on the host cores, on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = 2
WORKLOAD_NAME = "481x321 RGB, 5 labels x 2000 samples, 7x7 patches, Omega 98x49"


def rank_seed(rank: int) -> int:
    """Weak scaling: every rank draws its own image of the bench workload."""
    return 1000 + WORKLOAD + 7919 * rank


def combine(dev_ms, e2e_ms, pairs_rank, steps, world, reduce_max):
    """Whole-job numbers from this rank's times: the max over ranks of the
    device and end-to-end times (reduce_max: list of floats -> list of the
    maxima over ranks), and the pairs of all ranks divided by them."""
    dev_ms, e2e_ms = reduce_max([dev_ms, e2e_ms])
    total = pairs_rank * world * steps
    return {"value": total / (dev_ms * 1e-3), "e2e_value": total / (e2e_ms * 1e-3),
            "ms_per_step": dev_ms / steps, "dev_ms": dev_ms, "e2e_ms": e2e_ms}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Nominal per-SM, per-clock rates of the pipes the pair loops use on GB300
# (152 SMs): 128 FP32 lanes, 64 INT32, 16 popc and 32 ex2 (special-function)
# results per clock. The roofline uses the rates cs_unit_rates measures on
# the device where it has them (FP32, popc, ex2) and these nominal figures
# for the rest (INT32), and reports both.
PIPE_LANES = {"fp32": 128, "int32": 64, "mufu": 32, "popc": 16}


def measured_lanes(rates):
    """Per-SM per-clock rates for the roofline: measured where probed."""
    lanes = dict(PIPE_LANES)
    if rates:
        lanes.update({"fp32": rates["ffma"], "popc": rates["popc"], "mufu": rates["ex2"]})
    return lanes


def pair_ops(form: str, Wk: int) -> dict:
    """Algorithmic operations per pixel x sample pair.

    fp32 (CUDA cores): location 2 sub + mul + fma, colour 3 sub + mul + 2 fma,
    combine 3, running max, exponent offset and sum (16 FP32); Wk xor and
    Wk - 1 adds (INT32); Wk popc; one ex2.
    tensor-core forms: the dot products run on the tensor cores; the CUDA
    cores do 2 FFMA (texture/colour scale, location scale) and one add per
    pair (3 FP32) and one ex2.
    """
    if form == "fp32":
        return {"fp32": 16, "int32": 2 * Wk - 1, "popc": Wk, "mufu": 1}
    return {"fp32": 3, "mufu": 1}


def alu_peak_pairs(form: str, Wk: int, sm_mhz: float, n_sm: int = 152,
                   lanes: dict | None = None) -> tuple[float, str]:
    lanes = lanes or PIPE_LANES
    ops = pair_ops(form, Wk)
    rates = {k: lanes[k] / v for k, v in ops.items()}
    pipe = min(rates, key=rates.get)
    return rates[pipe] * n_sm * sm_mhz * 1e6, pipe


def errors(L, post, ref):
    """A form's error against the oracle at the sampled pixels: max relative
    error on L (max |L - L_o| / max(|L_o|, 1)), max probability error and
    argmax agreement (oracle ties within 1e-12 count as agreement)."""
    L = np.asarray(L, np.float64)
    post = np.asarray(post, np.float64)
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(post - ref["post"])))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12 if srt.shape[0] > 1 else np.ones(srt.shape[1], bool)
    agree = float(np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie))
    return {"max_rel_err_L": rel, "max_prob_err": perr, "argmax_agreement": agree}


def sample_pixels(pr, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(rng.integers(0, pr.H * pr.W, n)).astype(np.int32)


def gather_px(torch, t, nl, pix):
    """(nl, len(pix)) host copy of the sampled pixels of a (nl, H, W) tensor."""
    idx = torch.from_numpy(pix.astype(np.int64)).to(t.device)
    return t.reshape(nl, -1).index_select(1, idx).cpu().numpy()


def run_reference(args):
    """Oracle timed on the host cores on a bounded pixel sample per step."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1312_4746_gb300 import synth

    oracle.build()
    pr = synth.make_workload(WORKLOAD)
    prm = pr.params
    rng = np.random.default_rng(0)
    P = pr.H * pr.W
    n_pix = args.ref_pixels
    cores = os.cpu_count()
    times = []
    for step in range(args.warmup + args.steps):
        pix = np.sort(rng.choice(P, n_pix, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.data_term(pr, pix=pix)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    pairs = n_pix * pr.n_samples
    value = pairs * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "pixel x sample likelihood pairs/s",
        "value": value, "unit": "pairs/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample_pixels_per_step": n_pix},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_pix} random pixels x all {pr.n_samples} samples per step "
                                   f"(codes of those pixels and of every sample included)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline(pr, budget_s=15.0):
    """The oracle as it stands on a bounded pixel sample (about budget_s)."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(1)
    P = pr.H * pr.W
    n_pix = 256
    pix = np.sort(rng.choice(P, n_pix, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.data_term(pr, pix=pix)
    dt = time.perf_counter() - t0
    # grow the sample to about budget_s of CPU work
    n2 = int(min(P, max(n_pix, n_pix * budget_s / max(dt, 1e-3) * 0.8)))
    pix = np.sort(rng.choice(P, n2, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.data_term(pr, pix=pix)
    dt = time.perf_counter() - t0
    return {"value": n2 * pr.n_samples / dt, "unit": "pairs/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{n2} random pixels x all {pr.n_samples} samples, {dt:.1f} s "
                      f"(FP64 C oracle, OpenMP over pixels)"}


# DRAM bytes per launch of the sum kernels on this workload
# (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the
# kernels as they are now)
TRAFFIC = {"sum_tc_kernel": 9.01e6, "sum_plain_kernel": 7.83e6}

FORMS = {"fp32": 0, "bf16": 1, "fp8": 2}
FORM_NAMES = {"fp32": "plain FP32 (CUDA cores, popc TSM)",
              "bf16": "tensor cores (tcgen05): BF16 exact texture dot, split-BF16 colour, location from exact offset pieces (one FP32 accumulator)",
              "fp8": "tensor cores (tcgen05): FP8 exact texture dot, split-BF16 colour, location from exact offset pieces (one FP32 accumulator)"}
# kernels one step launches (cs_data_term, per-sample form): offsets, seed,
# row scan, column envelope; row norms, operator split, tcgen05 codes, guard;
# gather; then either the plain sum, or Morton sort, tile build, the tcgen05
# sum and the FP64 recompute of rows below the FP32 floor
LAUNCHES = {"fp32": 10, "bf16": 13, "fp8": 13}


def measure(ctx, cs, torch, pr, form, steps, warmup, dev, stream, flush, clk=None, mode=None):
    """Device time (ms) of `steps` data-term steps with inputs resident, the
    per-stage times, and the end-to-end time from pinned host buffers."""
    P = pr.H * pr.W
    nl = pr.n_labels
    prm = cs.Params.from_synth(pr.params, precision=FORMS[form])
    if mode is not None:
        prm.mode = mode
    img = torch.from_numpy(pr.image).to(dev)
    om = torch.from_numpy(pr.omega).to(dev)
    mask = torch.from_numpy(pr.mask).to(dev)
    smp = torch.from_numpy(pr.sample_pix).to(dev)
    out = {"neglog": torch.empty((nl, pr.H, pr.W), dtype=torch.float32, device=dev),
           "post": torch.empty((nl, pr.H, pr.W), dtype=torch.float32, device=dev)}

    def step(img_d, om_d, mask_d, smp_d):
        ctx.data_term(img_d, om_d, mask_d, pr.label_off, smp_d, prm, out=out)

    for _ in range(warmup):
        flush.fill_(1.0)
        step(img, om, mask, smp)
    ctx.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        step(img, om, mask, smp)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    refined = ctx.refined_count()  # pixels of the last step recomputed in FP64
    # per-stage times from a second, profiled pass (stage events cost a few
    # microseconds and run the launches one by one instead of as the replayed
    # graph, so they stay out of the timed steps)
    ctx.profile(True)
    for i in range(steps):
        flush.fill_(float(i))
        step(img, om, mask, smp)
    torch.cuda.synchronize()
    ctx.profile(False)
    ctx.sync()
    stage = {}
    for name, st in (("codes", cs.STAGE_CODES), ("dist", cs.STAGE_DIST),
                     ("gather", cs.STAGE_GATHER), ("sum", cs.STAGE_SUM)):
        ms, n = ctx.profile_read(st)
        stage[name] = ms / max(n, 1)
    # end to end through the C ABI from pinned host buffers
    h_img = torch.from_numpy(pr.image).pin_memory()
    h_om = torch.from_numpy(pr.omega).pin_memory()
    h_mask = torch.from_numpy(pr.mask).pin_memory()
    h_smp = torch.from_numpy(pr.sample_pix).pin_memory()
    h_out = torch.empty((nl, pr.H, pr.W), dtype=torch.float32).pin_memory()
    d_img, d_om, d_mask, d_smp = (torch.empty_like(img), torch.empty_like(om),
                                  torch.empty_like(mask), torch.empty_like(smp))
    h2d = sum(t.numel() * t.element_size() for t in (h_img, h_om, h_mask, h_smp)) + 4 * (nl + 1)
    d2h = h_out.numel() * 4
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        e2e_ev[i][0].record(stream)
        d_img.copy_(h_img, non_blocking=True)
        d_om.copy_(h_om, non_blocking=True)
        d_mask.copy_(h_mask, non_blocking=True)
        d_smp.copy_(h_smp, non_blocking=True)
        step(d_img, d_om, d_mask, d_smp)
        h_out.copy_(out["neglog"], non_blocking=True)
        e2e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev)
    stage["refined_pixels"] = refined
    return dev_ms, e2e_ms, stage, h2d, d2h, out


def measure_segment(ctx, cs, torch, pr, dev, stream, iterations=300, runs=3):
    """Convex multilabel segmentation (cs_segment) of this workload's FP8 data
    term: device time of `iterations` primal-dual iterations plus argmax."""
    prm = cs.Params.from_synth(pr.params, precision=FORMS["fp8"])
    f = ctx.data_term(torch.from_numpy(pr.image).to(dev), torch.from_numpy(pr.omega).to(dev),
                      torch.from_numpy(pr.mask).to(dev), pr.label_off,
                      torch.from_numpy(pr.sample_pix).to(dev), prm)["neglog"]
    img = torch.from_numpy(pr.image).to(dev)
    sp = cs.SegParams.default(lam=4.0, iterations=iterations)
    out = ctx.segment(f, img, sp)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        ctx.segment(f, img, sp, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    return {"what": f"cs_segment on the FP8 data term: {iterations} primal-dual iterations "
                    f"(lambda {sp.lam}, nu {sp.nu}, gamma {sp.gamma}) and argmax",
            "ms": ms, "ms_per_iteration": ms / iterations}


def measure_unsup(ctx, cs, torch, pr, dev, stream, runs=3):
    """Unsupervised segmentation of this workload's image (Sec. 3.2 with the
    Berkeley settings: 16 initial segments = 4 colour x 4 texture classes,
    lambda 6, nu 1100): cs_unsup_data_term, then cs_segment; device time of
    each part, and how many labels the label cost leaves."""
    import numpy as np

    P = pr.H * pr.W
    prm = cs.Params.from_synth(pr.params)
    prm.sigma_c2 = 0.02
    up = cs.UnsupParams.default(beta=0.5)
    ci = np.random.default_rng(2).choice(P, up.n_colour, replace=False).astype(np.int32)
    ti = np.random.default_rng(3).choice(P, up.n_texture, replace=False).astype(np.int32)
    img = torch.from_numpy(pr.image).to(dev)
    om = torch.from_numpy(pr.omega).to(dev)
    mk = torch.from_numpy(pr.mask).to(dev)
    sp = cs.SegParams.default(lam=6.0, nu=1100.0, iterations=300)
    out = ctx.unsup_data_term(img, om, mk, prm, up, ci, ti)  # warm-up
    seg = ctx.segment(out["neglog"], img, sp)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_dt = t_seg = 0.0
    for _ in range(runs):
        ev[0].record(stream)
        ctx.unsup_data_term(img, om, mk, prm, up, ci, ti, out=out)
        ev[1].record(stream)
        ctx.segment(out["neglog"], img, sp, out=seg)
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_dt += ev[0].elapsed_time(ev[1]) / runs
        t_seg += ev[1].elapsed_time(ev[2]) / runs
    used = int(torch.unique(seg["labels"]).numel())
    return {"what": "unsupervised segmentation: iota of every pixel, k-means (4 colour classes, "
                    "10 rounds), k-medians (4 texture classes, 10 rounds), 16-segment data term "
                    "(sigma_c2 0.02, beta 0.5), then 300 solver iterations with lambda 6, nu 1100",
            "data_term_ms": t_dt, "segment_ms": t_seg, "total_ms": t_dt + t_seg,
            "labels_left": used}


def measure_batch(ctx, cs, torch, dev, n_images, reduce_max, world, runs=5):
    """The batch workload (uneven images, one persistent tensor-core sum over
    all of them) through cs_batch_*: autotuned, captured in a CUDA graph,
    timed with CUDA events over `runs` replays after the tuning run."""
    import dataclasses

    from paper_1312_4746_gb300 import synth

    probs = synth.make_batch(n_images)
    probs = [dataclasses.replace(q, omega=probs[0].omega, mask=probs[0].mask) for q in probs]
    pairs = float(sum(q.H * q.W * q.n_samples for q in probs))
    om = torch.from_numpy(probs[0].omega).to(dev)
    mask = torch.from_numpy(probs[0].mask).to(dev)
    inp = [{"img": torch.from_numpy(q.image).to(dev),
            "sample_pix": torch.from_numpy(q.sample_pix).to(dev), "label_off": q.label_off}
           for q in probs]
    prm = cs.Params.from_synth(probs[0].params, precision=FORMS["fp8"])
    b = ctx.batch(inp, om, mask, prm, flags=cs.BATCH_GRAPH | cs.BATCH_AUTOTUNE)
    b.run()  # tunes, then captures the graph
    b.run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    (ms,) = reduce_max([e0.elapsed_time(e1) / runs])
    cfg = b.config()
    b.close()
    return {"workload": f"{n_images} images 240-640 x 160-480, 2-10 labels x 500-5000 "
                        "samples, 7x7 patches, Omega 98x49 (seeds 100000+b)",
            "form": FORM_NAMES["fp8"], "pairs_per_run": pairs, "ms_per_run": ms,
            "pairs_per_s": pairs * world / (ms * 1e-3), "runs": runs,
            "graph": True, "autotuned": {"n_streams": cfg["n_streams"],
                                         "order": "by cost" if cfg["order"] == 0 else "given",
                                         "sum_kernel": (
                                             f"variant {cfg['sum_variant']}: "
                                             f"{cfg['sum_shape']['ctas_per_sm']} CTA(s) per SM, "
                                             f"{cfg['sum_shape']['epilogue_warps']} epilogue warps, "
                                             f"{cfg['sum_shape']['ring_stages']}-stage sample ring, "
                                             f"{cfg['sum_shape']['texture_buffers']} pixel-tile "
                                             "texture buffer(s)"),
                                         "tuning_ms": cfg["tuned_ms"]},
            "l2": "not flushed: each run reads and writes about 1 GB (images, bitmasks, distances, outputs), far above L2"}


def measure_large(ctx, cs, torch, dev, reduce_max, world, steps=3):
    """The 1024 x 1024 (10 labels x 20000 samples) and 4096 x 4096 (16 x 6250,
    9x9 patches, Omega 162x81) workloads through cs_data_term, both forms:
    CUDA events over `steps` steps after one warm-up step (inputs of several
    hundred MB to GB per step, above L2)."""
    from paper_1312_4746_gb300 import synth

    import oracle

    out = {}
    stream = torch.cuda.current_stream()
    for wl in (4, 5):
        pr = synth.make_workload(wl)
        pix = sample_pixels(pr, 256, 40 + wl)
        img = torch.from_numpy(pr.image).to(dev)
        om = torch.from_numpy(pr.omega).to(dev)
        mask = torch.from_numpy(pr.mask).to(dev)
        smp = torch.from_numpy(pr.sample_pix).to(dev)
        pairs = float(pr.H * pr.W * pr.n_samples)
        entry = {"workload": pr.name or f"{pr.W}x{pr.H}", "pairs_per_step": pairs}
        for form in ("fp8", "fp32"):
            prm = cs.Params.from_synth(pr.params, precision=FORMS[form])
            res = ctx.data_term(img, om, mask, pr.label_off, smp, prm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.data_term(img, om, mask, pr.label_off, smp, prm, out=res)
            e1.record(stream)
            torch.cuda.synchronize()
            (ms,) = reduce_max([e0.elapsed_time(e1) / steps])
            entry[form] = {"ms_per_step": ms, "pairs_per_s": pairs * world / (ms * 1e-3),
                           "fp64_recomputed_pixels": ctx.refined_count() if form != "fp32" else 0,
                           "_got": (-gather_px(torch, res["neglog"], pr.n_labels, pix),
                                    gather_px(torch, res["post"], pr.n_labels, pix))}
            del res
        ref = oracle.data_term(pr, pix=pix)
        for form in ("fp8", "fp32"):
            entry[form]["error_vs_oracle"] = errors(*entry[form].pop("_got"), ref)
        entry["error_sample"] = f"{len(pix)} random pixels x all samples (FP64 oracle)"
        out[f"{pr.W}x{pr.H}"] = entry
        del img, om, mask, smp
        torch.cuda.empty_cache()
    return out


def measure_surrogate(ctx, cs, torch, dev, reduce_max, world, steps=1000, runs=2):
    """The learned surrogate on the 1024 x 1024 workload (10 labels x 20000
    samples): fit on exact FP32 likelihoods at 5% of the pixels (tensor-core
    training, `steps` Adam steps), then evaluation under each fallback rule,
    against the exact sums of the same call (cs_likelihood, plain FP32 and
    FP8 tensor-core forms) as the reference: fallback share, max posterior
    error and argmax agreement over all pixels and over the pixels the
    network answers, and the time of fit + eval as pairs/s-equivalent.
    Per mode (per-sample and factorised texture) and feature set. CUDA
    events around each call, `runs` timed runs after one warm-up."""
    from paper_1312_4746_gb300 import synth

    pr = synth.make_workload(4)
    P, nl = pr.H * pr.W, pr.n_labels
    pairs = float(P * pr.n_samples)
    img = torch.from_numpy(pr.image).to(dev)
    om = torch.from_numpy(pr.omega).to(dev)
    mask = torch.from_numpy(pr.mask).to(dev)
    smp = torch.from_numpy(pr.sample_pix).to(dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(runs):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        (ms,) = reduce_max([e0.elapsed_time(e1) / runs])
        return ms, r

    def err(post, ex_post, sel=None):
        d = (post - ex_post).abs().amax(0)
        agree = post.argmax(0) == ex_post.argmax(0)
        if sel is not None:
            if not bool(sel.any()):
                return {"max_prob_err": None, "argmax_agreement": None}
            d, agree = d[sel], agree[sel]
        return {"max_prob_err": float(d.max()), "argmax_agreement": float(agree.float().mean())}

    out = {"workload": pr.name, "pairs_per_image": pairs, "training_fraction": 0.05,
           "steps": steps, "errors_against": "exact FP32 sums of the whole image (cs_likelihood)"}
    for mode in (0, 1):
        prm = cs.Params.from_synth(pr.params, mode=mode)
        c = ctx.codes(img, om, mask, prm, want_lead16=True)
        ms32, ex = timed(lambda: ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, smp, prm))
        prm8 = cs.Params.from_synth(pr.params, mode=mode, precision=FORMS["fp8"])
        ms8, _ = timed(lambda: ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, smp, prm8))
        ex_post = ex["post"].reshape(nl, P)
        entry = {"exact_fp32_ms": ms32, "exact_fp8_ms": ms8}
        for feat, fname in ((cs.SURR_BASIC, "basic"), (cs.SURR_EXTENDED, "extended")):
            def fit():
                ctx.surrogate_fit(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                                  frac=0.05, steps=steps, features=feat, seed=11)
            ctx.profile(True)
            fit_ms, _ = timed(fit)
            train_ms, _ = ctx.profile_read(cs.STAGE_TRAIN)
            for st in range(cs.STAGE_TRAIN):  # forget the other stages' records
                ctx.profile_read(st)
            ctx.profile(False)
            info = ctx.surrogate_info(nl)
            e = {"features": info["n_in"], "fit_ms": fit_ms, "train_ms": train_ms / (runs + 1),
                 "train_ms_per_step": train_ms / (runs + 1) / steps, "eta_nats": info["eta"],
                 "final_loss": info["loss"], "rules": {}}
            for rule, rname in ((cs.FALLBACK_NONE, "none"), (cs.FALLBACK_MARGIN, "margin 0.1"),
                                (cs.FALLBACK_GUARANTEED, "guaranteed")):
                def ev():
                    return ctx.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off,
                                              smp, prm, rule=rule, margin=0.1, count=False)
                ev_ms, (o, _) = timed(ev)
                post = o["post"].reshape(nl, P)
                # the pixels the network answered: not bit-identical to the exact sum
                answered = (o["neglog"].reshape(nl, P) != ex["neglog"].reshape(nl, P)).any(0)
                e["rules"][rname] = {
                    "eval_ms": ev_ms, "fallback_share": 1.0 - float(answered.float().mean()),
                    "all_pixels": err(post, ex_post), "answered_pixels": err(post, ex_post, answered),
                    "pairs_per_s_equiv_fit_plus_eval": pairs * world / ((fit_ms + ev_ms) * 1e-3),
                    "pairs_per_s_equiv_eval_only": pairs * world / (ev_ms * 1e-3)}
                del o, post
            entry[fname] = e
        out["per-sample" if mode == 0 else "factorised"] = entry
        del c, ex, ex_post
        torch.cuda.empty_cache()
    return out


def profile_kernels():
    """A small, fixed case for ncu captures of the hot kernels: after
    untimed warm-ups (the FP8 data term on the 481x321 workload three times,
    a 200-step surrogate fit on the 1024x1024 workload), one FP8 data term,
    one network gradient over 19456 rows and one surrogate evaluation of the
    1024x1024 image run inside the NVTX range "kernels". Prints nothing
    measured: the numbers come from the profiler."""
    import numpy as np
    import torch

    from paper_1312_4746_gb300 import build as csbuild

    csbuild.build()
    import paper_1312_4746_gb300 as cs
    from paper_1312_4746_gb300 import synth

    dev = torch.device("cuda:0")
    ctx = cs.Context(0)
    pr = synth.make_workload(WORKLOAD)
    img = torch.from_numpy(pr.image).to(dev)
    om = torch.from_numpy(pr.omega).to(dev)
    mask = torch.from_numpy(pr.mask).to(dev)
    smp = torch.from_numpy(pr.sample_pix).to(dev)
    prm = cs.Params.from_synth(pr.params, precision=FORMS["fp8"])
    out = None
    for _ in range(3):
        out = ctx.data_term(img, om, mask, pr.label_off, smp, prm, out=out)
    p4 = synth.make_workload(4)
    img4 = torch.from_numpy(p4.image).to(dev)
    smp4 = torch.from_numpy(p4.sample_pix).to(dev)
    prm4 = cs.Params.from_synth(p4.params, mode=1)
    c4 = ctx.codes(img4, torch.from_numpy(p4.omega).to(dev), torch.from_numpy(p4.mask).to(dev),
                   prm4, want_lead16=True)
    ctx.surrogate_fit(img4, c4["bitmask"], c4["lead16"], p4.k, p4.label_off, smp4, prm4,
                      frac=0.05, steps=200, features=cs.SURR_EXTENDED, seed=11)
    n_in = ctx.surrogate_info(p4.n_labels)["n_in"]
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.normal(0, 1, (19456, n_in)).astype(np.float32)).to(dev)
    T = torch.from_numpy(rng.normal(0, 1, (19456, p4.n_labels)).astype(np.float32)).to(dev)
    params = torch.from_numpy(ctx.surrogate_params()).to(dev)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernels")
    ctx.data_term(img, om, mask, pr.label_off, smp, prm, out=out)
    ctx.mlp_grad(params, p4.n_labels, X, T)
    ctx.surrogate_eval(img4, c4["bitmask"], c4["lead16"], p4.k, p4.label_off, smp4, prm4,
                       rule=cs.FALLBACK_NONE, count=False)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ctx.close()
    print("profile-kernels: done")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="fp8", choices=list(FORMS))
    ap.add_argument("--ref-pixels", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-images", type=int, default=64,
                    help="also time a batch of this many uneven images (0: skip)")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="run only the small fixed case for ncu captures (see profile_kernels)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 1024x1024 and 4096x4096 workloads and the surrogate")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_kernels:
        profile_kernels()
        return

    import torch

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    from paper_1312_4746_gb300 import build as csbuild

    csbuild.build()
    import paper_1312_4746_gb300 as cs
    from paper_1312_4746_gb300 import synth

    # weak scaling: every rank gets its own image of the same shape
    pr = synth.make_workload(WORKLOAD, seed=rank_seed(rank))
    P = pr.H * pr.W
    Wk = (pr.k + 31) // 32
    ctx = cs.Context(local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    pairs_rank = P * pr.n_samples

    forms = [args.form] + [f for f in ("bf16", "fp32") if f != args.form]
    res = {}
    rates = ctx.unit_rates() if rank == 0 else None  # pipe rates for the roofline
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        for form in forms:
            res[form] = measure(ctx, cs, torch, pr, form, args.steps, args.warmup, dev, stream,
                                flush)
        # the smooth co-sparse texture (mode 2): FP8 Parzen sum + smooth texture posterior
        res_smooth = measure(ctx, cs, torch, pr, "fp8", args.steps, args.warmup, dev, stream,
                             flush, mode=cs.MODE_SMOOTH)
        seg = measure_segment(ctx, cs, torch, pr, dev, stream)
        uns = measure_unsup(ctx, cs, torch, pr, dev, stream)
    if world > 1:
        torch.distributed.barrier()

    def reduce_max(vals):
        t = torch.tensor(vals, dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return [float(v) for v in t]

    head = args.form
    comb = combine(res[head][0], res[head][1], pairs_rank, args.steps, world, reduce_max)
    dev_ms, value, e2e_value = comb["dev_ms"], comb["value"], comb["e2e_value"]
    batch = None
    if args.batch_images > 0:
        batch = measure_batch(ctx, cs, torch, dev, args.batch_images, reduce_max, world)
    large = None if args.no_large else measure_large(ctx, cs, torch, dev, reduce_max, world)
    surr = None if args.no_large else measure_surrogate(ctx, cs, torch, dev, reduce_max, world)
    if rank == 0:
        peaks, src = _peaks()
        clocks = clk.summary()
        sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        import oracle

        lanes = measured_lanes(rates)
        # errors against the FP64 oracle at sampled pixels (outside the timed region)
        pix = sample_pixels(pr, 2000, 17)
        ref = oracle.data_term(pr, pix=pix)
        nl = pr.n_labels
        forms_out = {}
        refined = {f: res[f][2].pop("refined_pixels") for f in forms}
        for form in forms:
            d_ms, e_ms, stage, h2d, d2h, o = res[form]
            peak, pipe = alu_peak_pairs(form, Wk, sm_mhz, n_sm, lanes)
            achieved = pairs_rank / (stage["sum"] * 1e-3)
            forms_out[form] = {
                "form": FORM_NAMES[form], "pairs_per_s": pairs_rank * args.steps / (d_ms * 1e-3),
                "ms_per_step": d_ms / args.steps, "stage_ms": stage,
                "sum_kernel_pairs_per_s": achieved, "sum_kernel_peak": peak,
                "sum_kernel_frac": achieved / peak, "binding_pipe": pipe,
                "fp64_recomputed_pixels": refined[form],
                "error_vs_oracle": errors(-gather_px(torch, o["neglog"], nl, pix),
                                          gather_px(torch, o["post"], nl, pix), ref)}
        pr_s = synth.make_workload(WORKLOAD, seed=rank_seed(rank))
        pr_s.params.mode = 2
        ref_s = oracle.data_term(pr_s, pix=pix)
        o = res_smooth[5]
        smooth_err = errors(-gather_px(torch, o["neglog"], nl, pix),
                            gather_px(torch, o["post"], nl, pix), ref_s)
        d_ms, e_ms, stage, h2d, d2h, _ = res[head]
        peak, pipe = alu_peak_pairs(head, Wk, sm_mhz, n_sm, lanes)
        achieved = pairs_rank / (stage["sum"] * 1e-3)
        kernel = "sum_plain_kernel" if head == "fp32" else "sum_tc_kernel"
        line = {
            "metric": "pixel x sample likelihood pairs/s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if head == "fp32" else head + "+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "form": FORM_NAMES[head], "mode": "per-sample",
                       "pairs_per_step": pairs_rank,
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "stage_ms": stage},
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": LAUNCHES[head] * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "pairs/s",
                         "frac": achieved / peak, "traffic": TRAFFIC.get(kernel), "kernel": kernel,
                         "binding_pipe": pipe,
                         "peak_basis": f"{lanes[pipe]:.1f} {pipe} results/SM/clk "
                                       f"({'measured by cs_unit_rates' if rates and pipe != 'int32' else 'nominal'}; "
                                       f"nominal {PIPE_LANES[pipe]}) / "
                                       f"{pair_ops(head, Wk)[pipe]} per pair x {n_sm} SMs x "
                                       f"{sm_mhz:.0f} MHz (median SM clock sampled under load)",
                         "peak_nominal": alu_peak_pairs(head, Wk, sm_mhz, n_sm)[0]},
            "error_vs_oracle": forms_out[head]["error_vs_oracle"],
            "error_sample": f"{len(pix)} random pixels x all {pr.n_samples} samples (FP64 oracle, "
                            "outside the timed region)",
            "unit_rates": rates,
            "forms": forms_out,
            "smooth": {
                "form": "mode 2: FP8 tensor-core Parzen colour-location sum, then the smooth "
                        "co-sparse texture posterior (iota of FP32 codes, sigma "
                        f"{pr.params.iota_sigma}, median representatives, l1 softmax)",
                "ms_per_step": res_smooth[0] / args.steps,
                "pairs_per_s": pairs_rank * args.steps / (res_smooth[0] * 1e-3),
                "stage_ms": res_smooth[2], "error_vs_oracle": smooth_err},
            "segment": seg,
            "unsupervised": uns,
            "clocks": clocks,
        }
        if batch is not None:
            line["batch"] = batch
        if large is not None:
            line["large"] = large
        if surr is not None:
            line["surrogate"] = surr
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(pr)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
