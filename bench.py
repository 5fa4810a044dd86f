#!/usr/bin/env python
"""Throughput of the patch-hashing zoom on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference] [--no-cpu-baseline] [--no-extras]

Default workload: the 2x zoom of a 512 x 512 LR image with a 1,000,000-pair
dictionary (5x5 LR / 10x10 HR patches, L=16, k=16, K=8, 5 back-projection
steps).  One step = one zoom_upscale (features, hashing, bin lookup,
neighbour search, LLE, blend + overlap average, back-projection), inputs
resident in HBM; `value` is HR megapixels/s of the exact FP32 form.  The
same line reports the BF16 form (recall and PSNR against the exact form),
one step of the plain SIMT scan, per-kernel rooflines, the end-to-end rate
through the Python API with host buffers, and the FP64 oracle timed on a
bounded sample on the host cores.

--workload batch64_mixed: 64 LR images (96..768 x 128..1024, half 2x, half
3x) with one 1,000,000-pair dictionary per scale, zoomed by one
zoom_upscale_batch call (recorded CUDA graph) in the BF16 form; one step =
one batch; reports aggregate HR MP/s, per-image p50/p99 latency, and the
exact FP32 form batched and looped image by image for comparison.

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its
own copy of the workload on its own GPU (replicas, weak scaling); the
reported time is the max over ranks.
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

import synth_inputs as S  # noqa: E402

METRIC = "HR megapixels/s"
UNIT = "MP/s"
GRAD_W = 8.0   # bin width of the gradient-feature extra


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="zoom2x_512_dict1m")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--cpu-sample-queries", type=int, default=24)
    return ap.parse_args()


def profiled_traffic(kernel_src: str, summary: str):
    """DRAM bytes per launch from the committed ncu summary, or None once the
    kernel source differs from the one the counters were taken on."""
    import hashlib
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()[:16]
        fields = dict(ln.split(":", 1) for ln in open(os.path.join(ROOT, summary)) if ":" in ln)
        if fields.get("kernel_source_sha256_16", "").strip() != sha:
            return None
        return int(fields["traffic_bytes_per_launch"].strip())
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback (no measured peaks file)"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi takes a while to start: wait for its first sample, then
        # keep only the samples taken from here on (the timed region)
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload_inputs(wl: S.Workload):
    train = S.training_images(wl)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, wl.patch ** 2, wl.w)
    lr = S.test_image(wl)
    return train, pos, alpha, beta, lr


def cpu_oracle_setup(wl: S.Workload, train, pos, alpha, beta):
    """The oracle's dictionary and index of the workload (not timed as part
    of the metric; built once per run)."""
    from oracle import zoom_oracle as O
    t0 = time.perf_counter()
    od = O.build_dictionary(train, pos, wl.scale, wl.patch, wl.blur_sigma)
    oi = O.build_index(od, alpha, beta, wl.w, wl.L, wl.k)
    return od, oi, time.perf_counter() - t0


def cpu_oracle_sample(wl: S.Workload, train, pos, alpha, beta, lr, n_sample: int, built=None):
    """Times the oracle, as it stands, on a bounded sample of the workload and
    extrapolates to HR megapixels/s: n_sample evenly spaced queries through
    the per-patch steps (hash, candidates, top-K, LLE), the blend of those
    patches, and back-projection on a 64-row HR band.  `built`: the result of
    cpu_oracle_setup, else it is built here."""
    from oracle import zoom_oracle as O
    od, oi, setup_s = built if built is not None else cpu_oracle_setup(wl, train, pos, alpha, beta)
    P, s = wl.patch, wl.scale
    nq = (wl.lr_h - P + 1) * (wl.lr_w - P + 1)
    rows = np.linspace(0, nq - 1, n_sample).astype(np.int64)
    t0 = time.perf_counter()
    qr = O.query(lr, od, oi, wl.K, wl.reg_rel, rows=rows)
    t_query = (time.perf_counter() - t0) / n_sample
    t0 = time.perf_counter()
    O.blend_patches(qr.nbr, qr.wgt, qr.mu, od.hr_res)
    t_blend = (time.perf_counter() - t0) / n_sample
    band = min(64, s * wl.lr_h)
    lrb = lr[:band // s].astype(np.float64)
    xb = np.kron(lrb, np.ones((s, s)))
    t0 = time.perf_counter()
    O.back_project(xb, lrb, s, wl.blur_sigma, wl.bp_iters, wl.sigma_spatial, wl.sigma_range, wl.bp_radius)
    t_bp_px = (time.perf_counter() - t0) / xb.size
    hr_px = s * wl.lr_h * s * wl.lr_w
    total = nq * (t_query + t_blend) + hr_px * t_bp_px
    return {"value": hr_px / 1e6 / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{n_sample} of {nq} queries (hash, candidate union, FP64 top-{wl.K}, LLE, blend) "
                       f"+ back-projection of a {band}-row HR band, extrapolated per query and per HR pixel"),
            "seconds_per_query": t_query, "mean_candidates_per_query": float(qr.n_cand.mean()),
            "setup_s": setup_s}


def launches_per_step(wl: S.Workload, tc: bool) -> int:
    # features, hash, lookup; the exact tensor search: operand, single-term
    # filter, rerank, then the second stage (gather, split operand, split
    # filter, rerank), the SIMT re-run and the fallback-count update (9), or
    # the SIMT scan (1); LLE, the two overlap-average passes (blend, average),
    # 2 per back-projection step
    return 3 + (9 if tc else 1) + 3 + 2 * wl.bp_iters


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's time (replicas: the job ends when the last one does);
    `device` is the tensor device of the process group's backend."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Units all ranks processed per second (weak scaling: every replica does
    the same per-rank work in the step)."""
    return world * units_per_rank / (ms_per_step / 1e3)


def timed_steps(fn, steps, st, torch, world: int = 1):
    """Mean ms per step of `fn` with CUDA events on `st`; with several ranks
    the region is bracketed by barriers and the slowest rank's time is kept."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    return max_over_ranks(e0.elapsed_time(e1) / steps, world, "cuda")


def reference_arm(a, wl, config, hr_px, rank):
    if rank != 0:
        return
    train, pos, alpha, beta, lr = workload_inputs(wl)
    built = cpu_oracle_setup(wl, train, pos, alpha, beta)
    vals = []
    r = None
    for i in range(a.warmup + a.steps):
        r = cpu_oracle_sample(wl, train, pos, alpha, beta, lr, max(4, a.cpu_sample_queries // 4), built)
        if i >= a.warmup:
            vals.append(r["value"])
    v = statistics.median(vals)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                      "steps": a.steps, "warmup": a.warmup, "ms_per_step": hr_px / 1e6 / v * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": config,
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def run_single(a, wl, config, rank, world, local):
    import torch

    import paper_1004_3980_gb300 as Z
    hbm_peak, tc_peak, peak_src = peaks()
    hr_px = wl.scale * wl.lr_h * wl.scale * wl.lr_w
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    train, pos, alpha, beta, lr_np = workload_inputs(wl)
    ctx = Z.Context(local)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    imgs = [torch.from_numpy(x).cuda() for x in train]
    e0.record(st)
    d = Z.Dictionary(ctx, imgs, pos, wl.scale, wl.patch, wl.blur_sigma)
    e1.record(st)
    torch.cuda.synchronize()
    dict_ms = e0.elapsed_time(e1)
    e0.record(st)
    ix = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta)
    e1.record(st)
    torch.cuda.synchronize()
    index_ms = e0.elapsed_time(e1)
    del imgs

    def params(**kw):
        p = Z.UpscaleParams(K=wl.K, reg_rel=wl.reg_rel, bp_iters=wl.bp_iters, sigma_spatial=wl.sigma_spatial,
                            sigma_range=wl.sigma_range, bp_radius=wl.bp_radius)
        for k2, v in kw.items():
            setattr(p, k2, v)
        return p

    prm = params()
    lr = torch.from_numpy(lr_np).cuda()
    out = torch.empty((wl.scale * wl.lr_h, wl.scale * wl.lr_w), device="cuda")
    for _ in range(a.warmup):
        Z.upscale(ix, lr, prm, out=out)
    ctx.sync_status()
    stats0 = ctx.stats()

    # ---- timed region: K steps of the exact FP32 form, inputs resident ------
    ctx.set_stage_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stage_ms = {}
    e0.record(st)
    for _ in range(a.steps):
        torch.cuda.nvtx.range_push("zoom_step")
        Z.upscale(ix, lr, prm, out=out)
        torch.cuda.nvtx.range_pop()
        for k2, v in ctx.stats()["ms_stage"].items():   # this step's stage events
            stage_ms[k2] = stage_ms.get(k2, 0.0) + v
    e1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    ctx.set_stage_timing(False)
    ms_step = ms_total / a.steps
    value = whole_job_rate(hr_px / 1e6, world, ms_step)
    stage = {k2: v / a.steps for k2, v in stage_ms.items()}
    hr_exact = out.clone()

    # ---- end to end through the public API with host buffers ----------------
    lr_host = torch.from_numpy(lr_np).pin_memory()
    hr_host = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    lr_dev = torch.empty_like(lr)

    def e2e_step():
        lr_dev.copy_(lr_host, non_blocking=True)
        Z.upscale(ix, lr_dev, prm, out=out)
        hr_host.copy_(out, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        e2e_step()
        st.synchronize()
    e2e_s = (time.perf_counter() - t0) / a.steps
    e2e = {"value": world * hr_px / 1e6 / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": lr_host.numel() * 4, "d2h_bytes_per_step": hr_host.numel() * 4}

    # ---- rooflines ------------------------------------------------------------
    filt_ms = stage.get("knn_filter_kernel", 0.0)
    mma_flops = nq * wl.n_pairs * 2.0 * 32        # one FP16 term: K = 32 per (query, entry) pair
    achieved = mma_flops / (filt_ms / 1e3) / 1e12 if filt_ms > 0 else None
    traffic = profiled_traffic("paper_1004_3980_gb300/csrc/kernels_tc.cu",
                               "profiles/knn_tc_single_zoom2x_512_dict1m.md")
    roofline = {"kernel": "k_knn_tc<4,16,0> (tcgen05 single-term FP16 distance filter of the exact form)",
                "bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": achieved / tc_peak if achieved else None, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                  "(profiles/knn_tc_single_zoom2x_512_dict1m.md)",
                "peak_source": peak_src + ", bf16 dense (fp16 runs at the bf16 rate)",
                "work": "258,064 queries x 1,000,000 entries x 2 x 32 flops (K = 32 per pair)",
                "kernel_ms": filt_ms, "stage_share": filt_ms / ms_step if ms_step else None,
                "note": "at K = 32 a tile's MMAs take about as long as 40 % of its accumulator hand-off "
                        "(TMEM loads and chunk minima), which sets the pace; the split filter alone "
                        "(K = 80, key exact_split_filter) is tensor-bound"}
    PH2 = (wl.scale * wl.patch) ** 2
    oa_bytes = nq * wl.K * PH2 * 4 + hr_px * 4 + nq * (wl.K * 8 + 4)
    bp_bytes = wl.bp_iters * (hr_px * 4 * 3 + wl.lr_h * wl.lr_w * 4 * 3)
    kernels = {}
    for name, byts in (("overlap_add", oa_bytes), ("backproject", bp_bytes)):
        ms = stage.get(name, 0.0)
        if ms > 0:
            gbs = byts / (ms / 1e3) / 1e9
            kernels[name] = {"ms": ms, "algorithmic_bytes": byts, "GB/s": gbs, "frac_hbm": gbs / hbm_peak}
    if "overlap_add" in kernels:
        # blend pass + average pass; DRAM traffic from the committed ncu summary
        kernels["overlap_add"]["kernels"] = "k_blend_rows + k_overlap_average"
        kernels["overlap_add"]["traffic"] = profiled_traffic("paper_1004_3980_gb300/csrc/kernels_image.cu",
                                                             "profiles/overlap_average_zoom2x_512_dict1m.md")

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
           "lr_patch_queries_per_s": world * nq / (ms_step / 1e3),
           "roofline": roofline, "kernels_hbm": kernels, "e2e": e2e,
           "gpu_launches": launches_per_step(wl, True) * a.steps, "clocks": clk,
           "stage_ms_per_step": stage, "mean_bucket_sum_per_query": stats0["mean_bucket_sum"],
           "dictionary_build_ms": dict_ms, "index_build_ms": index_ms,
           "stats": {k2: v for k2, v in stats0.items() if k2 != "ms_stage"}}

    if not a.no_extras:
        # BF16 form: same inputs; recall of its neighbours and PSNR of its
        # output against the exact form
        p1 = params(precision=1, rerank_mult=2)
        for _ in range(2):
            Z.upscale(ix, lr, p1, out=out)
        ms1 = timed_steps(lambda: Z.upscale(ix, lr, p1, out=out), a.steps, st, torch, world)
        mse = float(((out - hr_exact) ** 2).mean())
        qe = Z.query(ix, lr, prm)["nbr"].cpu().numpy()
        qb = Z.query(ix, lr, p1)["nbr"].cpu().numpy()
        rec = float(np.mean([len(np.intersect1d(qe[i], qb[i])) for i in range(len(qe))]) / wl.K)
        res["bf16"] = {"value": world * hr_px / 1e6 / (ms1 / 1e3), "unit": UNIT, "ms_per_step": ms1,
                       "recall_vs_exact": rec, "psnr_vs_exact_db": 10 * np.log10(1.0 / max(mse, 1e-30))}
        # the FP16-split filter alone (K = 80; the exact form's second stage)
        p3 = params(search=3)
        for _ in range(2):
            Z.upscale(ix, lr, p3, out=out)
        ms6 = timed_steps(lambda: Z.upscale(ix, lr, p3, out=out), a.steps, st, torch, world)
        ctx.set_stage_timing(True)
        f3 = []
        for _ in range(3):
            Z.upscale(ix, lr, p3, out=out)
            f3.append(ctx.stats()["ms_stage"].get("knn_filter_kernel", 0.0))
        ctx.set_stage_timing(False)
        f3m = float(np.mean(f3))
        ach3 = nq * wl.n_pairs * 2.0 * 80 / (f3m / 1e3) / 1e12 if f3m > 0 else None
        res["exact_split_filter"] = {
            "value": world * hr_px / 1e6 / (ms6 / 1e3), "unit": UNIT, "ms_per_step": ms6,
            "identical_to_exact_form": bool(torch.equal(out, hr_exact)),
            "roofline": {"kernel": "k_knn_tc<10,16,0> (FP16 hi/lo split, K = 80)", "bound": "tensor",
                         "achieved": ach3, "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": ach3 / tc_peak if ach3 else None, "kernel_ms": f3m,
                         "traffic": profiled_traffic("paper_1004_3980_gb300/csrc/kernels_tc.cu",
                                                     "profiles/knn_tc_exact_zoom2x_512_dict1m.md")}}
        # one step of the plain SIMT scan (exact, no tensor cores)
        p2 = params(search=1)
        ms2 = timed_steps(lambda: Z.upscale(ix, lr, p2, out=out), 1, st, torch, world)
        res["fp32_simt_scan"] = {"value": world * hr_px / 1e6 / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2,
                                 "identical_to_exact_form": bool(torch.equal(out, hr_exact))}
        # the paper's early stop: candidate set capped at 3L IDs (tables in
        # order, IDs ascending within a bin), K nearest among them
        cap = 3 * wl.L
        ixc = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta, max_candidates=cap)
        for _ in range(2):
            Z.upscale(ixc, lr, prm, out=out)
        ms3 = timed_steps(lambda: Z.upscale(ixc, lr, prm, out=out), a.steps, st, torch, world)
        mse3 = float(((out - hr_exact) ** 2).mean())
        res["capped_3L"] = {"value": world * hr_px / 1e6 / (ms3 / 1e3), "unit": UNIT, "ms_per_step": ms3,
                            "max_candidates": cap, "distances_per_query": cap,
                            "psnr_vs_uncapped_db": 10 * np.log10(1.0 / max(mse3, 1e-30))}
        ixc.close()
        # gradient features (Sec. 4.1): the same workload with the 2 P^2 = 50
        # first-order gradients of each LR patch as its feature; w = 8 puts
        # about the pixel form's share of the dictionary in the candidate set.
        # Exact form: the single-term FP16 filter at K = 64, the split filter
        # (K = 160) as its second stage.
        d_g = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, wl.scale, wl.patch,
                           wl.blur_sigma, feature=1)
        D_g = 2 * wl.patch ** 2
        a_g, b_g = S.lsh_draws(wl.proj_seed, wl.L, wl.k, D_g, GRAD_W)
        ixg = Z.Index(d_g, wl.L, wl.k, GRAD_W, a_g, b_g)
        for _ in range(2):
            Z.upscale(ixg, lr, prm, out=out)
        ms4 = timed_steps(lambda: Z.upscale(ixg, lr, prm, out=out), a.steps, st, torch, world)
        ctx.set_stage_timing(True)
        filt_g = []
        for _ in range(3):
            Z.upscale(ixg, lr, prm, out=out)
            filt_g.append(ctx.stats()["ms_stage"].get("knn_filter_kernel", 0.0))
        ctx.set_stage_timing(False)
        st_g = ctx.stats()
        fg = float(np.mean(filt_g))
        ach_g = nq * wl.n_pairs * 2.0 * 64 / (fg / 1e3) / 1e12 if fg > 0 else None
        res["gradient_features"] = {
            "value": world * hr_px / 1e6 / (ms4 / 1e3), "unit": UNIT, "ms_per_step": ms4,
            "feature_dim": D_g, "w": GRAD_W, "mean_bucket_sum_per_query": st_g["mean_bucket_sum"],
            "filter_fallback_queries": st_g["n_filter_fallback"],
            "roofline": {"kernel": "k_knn_tc<8,16,0> (single-term FP16, K = 64)", "bound": "tensor",
                         "achieved": ach_g, "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": ach_g / tc_peak if ach_g else None, "kernel_ms": fg,
                         "work": f"{nq} queries x {wl.n_pairs} entries x 2 x 64 flops"}}
        ixg.close()
        d_g.close()
        # training-crop sampling (Sec. 5.1): 25 crops of 100 x 100 per training
        # image of the workload, drawn by gradient mass (the paper's recipe)
        imgs_t = [torch.from_numpy(x).cuda() for x in train]
        n_draw, side = 25, 100
        u_s = np.random.default_rng(17).random((len(train), n_draw))
        crops_out = torch.empty((len(train) * n_draw, side, side), device="cuda")
        for _ in range(2):
            Z.sample_crops(ctx, imgs_t, u_s, side, side)
        ms5 = timed_steps(lambda: Z.sample_crops(ctx, imgs_t, u_s, side, side), a.steps, st, torch, world)
        px = sum(x.size for x in train)
        byts = px * 4 + len(train) * n_draw * (1024 * 4 + 2 * side * side * 4)
        res["crop_sampling"] = {
            "value": world * len(train) * n_draw / (ms5 / 1e3), "unit": "crops/s", "ms_per_step": ms5,
            "images": len(train), "pixels": px, "crops_per_image": n_draw, "crop": [side, side],
            "algorithmic_bytes": byts, "GB/s": byts / (ms5 / 1e3) / 1e9,
            "frac_hbm": byts / (ms5 / 1e3) / 1e9 / hbm_peak,
            "note": "one call: draws copied in, tile masses, prefix, draws, crop gather, windows copied out"}
        del imgs_t, crops_out
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        res["cpu_baseline"] = cpu_oracle_sample(wl, train, pos, alpha, beta, lr_np, a.cpu_sample_queries)
    return res


def run_batch(a, config, rank, world, local):
    """64 mixed images through zoom_upscale_batch (BF16 form, recorded graph)."""
    import torch

    import paper_1004_3980_gb300 as Z
    shapes = S.batch_shapes(64)
    ctx = Z.Context(local)
    indexes = []
    for s, hrs, nimg in ((2, 512, 64), (3, 768, 128)):
        wl = S.Workload(f"dict{s}x", 0, 0, s, 5, nimg, hrs, 1_000_000, L=16, k=16, K=8, bp_iters=5,
                        train_seed0=1000 if s == 2 else 5000)
        train = S.training_images(wl)
        lrs = hrs // s
        pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, 5, wl.n_pairs)
        alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, 25, wl.w)
        imgs = [torch.from_numpy(x).cuda() for x in train]
        d = Z.Dictionary(ctx, imgs, pos, s, 5)
        indexes.append(Z.Index(d, wl.L, wl.k, wl.w, alpha, beta))
        del imgs, train
    lrs = [(s, torch.from_numpy(S.make_image(seed, h, w)).cuda()) for seed, h, w, s in shapes]
    hr_px = sum(s * s * x.shape[0] * x.shape[1] for s, x in lrs)
    nq = sum((x.shape[0] - 4) * (x.shape[1] - 4) for _, x in lrs)
    p1 = Z.UpscaleParams(K=8, bp_iters=5, precision=1, rerank_mult=2)
    st = torch.cuda.current_stream()
    outs, _ = Z.upscale_batch(indexes, lrs, p1)            # autotune + record
    for _ in range(max(0, a.warmup - 1)):
        Z.upscale_batch(indexes, lrs, p1, outs=outs)
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(lambda: Z.upscale_batch(indexes, lrs, p1, outs=outs), a.steps, st, torch, world)
    clk = clocks.stop()
    _, lat = Z.upscale_batch(indexes, lrs, p1, outs=outs, want_latency=True)
    value = whole_job_rate(hr_px / 1e6, world, ms)
    # the exact FP32 form looped image by image, for comparison
    p0 = Z.UpscaleParams(K=8, bp_iters=5)
    by = {ix.dictionary.scale: ix for ix in indexes}
    loop_outs = [torch.empty_like(o) for o in outs]

    def loop():
        for (s, x), o in zip(lrs, loop_outs):
            Z.upscale(by[s], x, p0, out=o)

    loop()
    ms_loop = timed_steps(loop, 1, st, torch, world)
    mse = float(sum(((o - lo) ** 2).sum() for o, lo in zip(outs, loop_outs)) / hr_px)
    # the exact FP32 form batched (three-stage tensor search, recorded graph)
    outs0, _ = Z.upscale_batch(indexes, lrs, p0)
    Z.upscale_batch(indexes, lrs, p0, outs=outs0)
    ms_exact = timed_steps(lambda: Z.upscale_batch(indexes, lrs, p0, outs=outs0), min(a.steps, 5), st, torch,
                           world)
    same = all(bool(torch.equal(o, lo)) for o, lo in zip(outs0, loop_outs))
    Z.batch_release(ctx)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": config,
            "lr_patch_queries_per_s": world * nq / (ms / 1e3), "hr_megapixels_per_batch": hr_px / 1e6,
            "per_image_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "fp32_exact_loop": {"value": world * hr_px / 1e6 / (ms_loop / 1e3), "ms_per_batch": ms_loop},
            "fp32_exact_batch": {"value": world * hr_px / 1e6 / (ms_exact / 1e3), "ms_per_batch": ms_exact,
                                 "identical_to_exact_loop": same},
            "psnr_bf16_batch_vs_fp32_exact_db": 10 * np.log10(1.0 / max(mse, 1e-30)),
            "clocks": clk, "gpu_launches": None,
            "e2e": None}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    batch = a.workload == "batch64_mixed"
    wl = None if batch else S.WORKLOADS[a.workload]
    if batch:
        config = {"workload": "batch64_mixed: 64 LR images 96..768 x 128..1024, half 2x / half 3x, "
                              "1M-pair dictionary per scale, K=8, 5 back-projection steps, BF16 form",
                  "parallelism": f"replicas{world}" if world > 1 else "single"}
    else:
        config = {"workload": wl.name, "lr": [wl.lr_h, wl.lr_w], "scale": wl.scale, "dict_pairs": wl.n_pairs,
                  "lr_patch": wl.patch, "L": wl.L, "k": wl.k, "K": wl.K, "bp_iters": wl.bp_iters,
                  "precision": "fp32-exact", "parallelism": f"replicas{world}" if world > 1 else "single",
                  "l2": "inputs larger than L2 (dictionary operands, features and HR patches: 0.9 GB)"}
    if a.impl == "reference":
        if batch:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-image "
                                  "workloads only"}), flush=True)
            return
        reference_arm(a, wl, config, wl.scale * wl.lr_h * wl.scale * wl.lr_w, rank)
        return

    import torch
    from paper_1004_3980_gb300 import build as B
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if rank == 0:
            B.build()
        dist.barrier()
    B.build()
    torch.cuda.set_device(local)
    res = run_batch(a, config, rank, world, local) if batch else run_single(a, wl, config, rank, world, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
