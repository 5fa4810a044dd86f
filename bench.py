#!/usr/bin/env python
"""Throughput of the patch-hashing zoom on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference] [--no-cpu-baseline] [--no-batch]
                    [--all-extras]

Default workload: the 3x zoom of a 1920 x 1080 LR image with a
4,000,000-pair dictionary (5x5 LR / 15x15 HR patches, L=16, k=18, K=8, 5
back-projection steps), the precision form against the plain one on the
same inputs.  One step = one zoom_upscale (features, hashing, bin lookup,
neighbour search, LLE, blend + overlap average, back-projection), inputs
resident in HBM.  `value` is HR megapixels/s of the precision form (BF16
tensor-core distance filter, FP32 exact rerank of the best 32 chunks);
`fp32_exact` is the plain form (exact FP32 neighbours) timed the same way.
The line also carries: the BF16 form's neighbour recall and PSNR against the
exact form over the whole image, and against the FP64 oracle on sampled
blocks of queries (neighbours, weights, and the reconstructed HR pixels that
only those queries cover); per-kernel rooflines; the end-to-end rate through
the Python API with host buffers; the paper's early stop (cap 3L); the
batched form (64 mixed images, key batch64_mixed); and the FP64 oracle timed
on the host cores on the sampled blocks.

--workload batch64_mixed: only the batched form (64 LR images 96..768 x
128..1024, half 2x, half 3x, one 1,000,000-pair dictionary per scale, one
zoom_upscale_batch call per step, recorded CUDA graph).

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
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth_inputs as S  # noqa: E402

METRIC = "HR megapixels/s"
UNIT = "MP/s"
DEFAULT_WORKLOAD = "zoom3x_1920x1080_dict4m"
GRAD_W = 8.0        # bin width of the gradient-feature extra
BLOCK = 16          # side of a sampled block of queries (oracle comparison)
TOP32_MULT = 4      # rerank_mult * K = 32: the precision form reranks the best 32 chunks


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--all-extras", action="store_true",
                    help="also the split filter alone, one step of the SIMT scan, gradient features, crop sampling")
    ap.add_argument("--cpu-blocks", type=int, default=0,
                    help="16x16 query blocks the oracle runs (0: by workload size)")
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads (0: all host cores)")
    return ap.parse_args()


def profiled_traffic(kernel_src: str, summary: str, key: str = "traffic_bytes_per_launch"):
    """DRAM bytes per launch from the committed ncu summary, or None once the
    kernel source differs from the one the counters were taken on."""
    import hashlib
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()[:16]
        fields = dict(ln.split(":", 1) for ln in open(os.path.join(ROOT, summary)) if ":" in ln)
        if fields.get("kernel_source_sha256_16", "").strip() != sha:
            return None
        return int(fields[key].strip())
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    """(HBM GB/s, bf16 TFLOP/s burst, bf16 TFLOP/s sustained, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return (float(p["hbm_gbs"]), float(p["bf16_tflops"]),
                float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "measured (MEASURED_PEAKS.json)")
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback (no measured peaks file)"


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


def n_queries(wl: S.Workload) -> int:
    return (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)


def default_blocks(wl: S.Workload) -> int:
    """Sampled 16x16 query blocks: about 1000 queries where the oracle takes
    ~0.2 s a query (1M entries), 256 at 4M entries (~4x that)."""
    return 4 if wl.n_pairs <= 1_000_000 else 1


def block_origins(wl: S.Workload, n_blocks: int, seed: int = 23):
    """Query-block origins (LR row, col), seeded, inside the query grid."""
    nh, nw = wl.lr_h - wl.patch + 1, wl.lr_w - wl.patch + 1
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, nh - BLOCK + 1)), int(rng.integers(0, nw - BLOCK + 1))) for _ in range(n_blocks)]


def block_rows(wl: S.Workload, i0: int, j0: int) -> np.ndarray:
    """Query numbers (row order) of the block at (i0, j0)."""
    nw = wl.lr_w - wl.patch + 1
    ii, jj = np.meshgrid(np.arange(i0, i0 + BLOCK), np.arange(j0, j0 + BLOCK), indexing="ij")
    return (ii * nw + jj).ravel()


def covered_window(wl: S.Workload, i0: int, j0: int):
    """HR pixels (slices of the full HR image) covered only by the patches of
    the block at (i0, j0): local rows/cols [s P - 1, s BLOCK) of the block's
    own HR frame (the first patch origin's HR position)."""
    s, PH = wl.scale, wl.scale * wl.patch
    lo, hi = PH - 1, s * BLOCK
    return (slice(s * i0 + lo, s * i0 + hi), slice(s * j0 + lo, s * j0 + hi)), (slice(lo, hi), slice(lo, hi))


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (CPU baseline and parity sample)
# ---------------------------------------------------------------------------
def oracle_setup(wl: S.Workload, train, pos, alpha, beta):
    """The oracle's dictionary (LR side) and index of the workload; built
    once per run, not part of the timed metric."""
    from oracle import zoom_oracle as O
    t0 = time.perf_counter()
    od = O.build_dictionary(train, pos, wl.scale, wl.patch, wl.blur_sigma, with_hr=False)
    oi = O.build_index(od, alpha, beta, wl.w, wl.L, wl.k)
    return od, oi, time.perf_counter() - t0


def oracle_block_queries(wl, lr, od, oi, origins, threads: int, side: int = BLOCK, cols: int | None = None):
    """The oracle's per-patch steps (Sec. 4.2: hash, candidate union, FP64
    K+1 nearest) on every query of the sampled blocks, one query row of a
    block per task, `threads` tasks at a time.  The weights are solved over
    the K nearest (Eq. 12-13).  Returns per block (nbr [Q][K+1], dist, wgt
    [Q][K], mu, margin, n_cand) and the wall seconds of the query steps."""
    from oracle import zoom_oracle as O
    P, K = wl.patch, wl.K

    cols = side if cols is None else cols   # a block of side rows x cols columns of queries

    def task(args):
        i0, j0, r = args
        sub = lr[i0 + r:i0 + r + P, j0:j0 + cols + P - 1]
        q = O.query(sub, od, oi, K + 1, wl.reg_rel)
        wgt = np.stack([O.lle_weights(q.feat[n], od.feat[q.nbr[n, :K]], wl.reg_rel, q.dist[n, 0])[0]
                        for n in range(len(q.nbr))])
        return q, wgt

    jobs = [(i0, j0, r) for i0, j0 in origins for r in range(side)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(task, jobs))
    wall = time.perf_counter() - t0
    out = []
    for b in range(len(origins)):
        part = res[b * side:(b + 1) * side]
        cat = lambda f: np.concatenate([getattr(q, f) for q, _ in part])
        out.append({"nbr": cat("nbr"), "dist": cat("dist"), "mu": cat("mu"), "margin": cat("margin"),
                    "n_cand": cat("n_cand"), "feat": cat("feat"), "wgt": np.concatenate([w for _, w in part])})
    return out, wall


def oracle_block_hr(wl, train, pos, blk, side: int = BLOCK, cols: int | None = None):
    """The oracle's HR estimate before back-projection (Eq. 14 + the overlap
    average) over a block's own HR frame, from its K nearest and weights;
    the HR residuals of the entries used come from the oracle's dictionary
    build on those entries' positions."""
    from oracle import zoom_oracle as O
    K = wl.K
    ids = np.unique(blk["nbr"][:, :K])
    dh = O.build_dictionary(train, pos[ids], wl.scale, wl.patch, wl.blur_sigma)
    local = np.searchsorted(ids, blk["nbr"][:, :K])
    cols = side if cols is None else cols
    return O.reconstruct(local, blk["wgt"], blk["mu"], dh, side + wl.patch - 1, cols + wl.patch - 1)


def block_exclusions(blocks, od, oi, threads):
    """Per block, the queries left out of the bit-exact neighbour comparison
    (the oracle's neighbour_exclusions: a bin boundary of the query or of an
    entry that could enter its K nearest, or an FP64 near-tie), one query row
    per task."""
    from oracle import zoom_oracle as O
    fn = (od.feat * od.feat).sum(axis=1)

    def task(args):
        b, r = args
        sl = slice(r * BLOCK, (r + 1) * BLOCK)
        blk = blocks[b]
        return O.neighbour_exclusions(blk["feat"][sl], blk["margin"][sl], blk["dist"][sl], od, oi, feat_norm2=fn)

    jobs = [(b, r) for b in range(len(blocks)) for r in range(BLOCK)]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(task, jobs))
    return [np.concatenate(res[b * BLOCK:(b + 1) * BLOCK]) for b in range(len(blocks))]


def oracle_bp_seconds_per_px(wl, lr):
    """Oracle back-projection (Sec. 4, Eq. 6-7, 15-17) of a 64-row HR band:
    seconds per HR pixel."""
    from oracle import zoom_oracle as O
    s = wl.scale
    band = min(64 - 64 % s, s * wl.lr_h)
    lrb = lr[:band // s].astype(np.float64)
    xb = np.kron(lrb, np.ones((s, s)))
    t0 = time.perf_counter()
    O.back_project(xb, lrb, s, wl.blur_sigma, wl.bp_iters, wl.sigma_spatial, wl.sigma_range, wl.bp_radius)
    return (time.perf_counter() - t0) / xb.size, band


def cpu_rate(wl, q_wall_per_query, blend_s_per_query, bp_s_per_px):
    """Extrapolated oracle HR MP/s: every query's per-patch steps and blend at
    the sampled rate, and the back-projection of every HR pixel."""
    hr_px = wl.scale * wl.lr_h * wl.scale * wl.lr_w
    total = n_queries(wl) * (q_wall_per_query + blend_s_per_query) + hr_px * bp_s_per_px
    return hr_px / 1e6 / total


def cpu_baseline_and_parity(wl, train, pos, alpha, beta, lr, n_blocks, threads):
    """The oracle, as it stands, on n_blocks sampled 16x16 query blocks with
    `threads` host threads: its timing (the CPU baseline) and its results
    (neighbours, weights, the HR pixels only the blocks cover) for the
    comparison with the GPU."""
    from oracle import zoom_oracle as O
    od, oi, setup_s = oracle_setup(wl, train, pos, alpha, beta)
    origins = block_origins(wl, n_blocks)
    blocks, wall = oracle_block_queries(wl, lr, od, oi, origins, threads)
    nq_s = n_blocks * BLOCK * BLOCK
    t0 = time.perf_counter()
    hrs = [oracle_block_hr(wl, train, pos, b) for b in blocks]
    blend_s = (time.perf_counter() - t0) / nq_s
    bp_px, band = oracle_bp_seconds_per_px(wl, lr)
    value = cpu_rate(wl, wall / nq_s, blend_s, bp_px)
    base = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{nq_s} of {n_queries(wl)} queries in {n_blocks} seeded {BLOCK}x{BLOCK} blocks "
                       f"(hash, candidate union, FP64 top-{wl.K + 1}, LLE; {threads} threads), their blend and "
                       f"overlap average (1 thread), back-projection of a {band}-row HR band (1 thread); "
                       f"extrapolated per query and per HR pixel"),
            "seconds_per_query_wall": wall / nq_s, "mean_candidates_per_query": float(
                np.mean([b["n_cand"].mean() for b in blocks])),
            "setup_s": setup_s, "host_cores": os.cpu_count(), "cpu_model": cpu_model()}
    return base, {"origins": origins, "blocks": blocks, "hr": hrs, "n": od.n,
                  "excluded": block_exclusions(blocks, od, oi, threads)}


def cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def compare_with_oracle(wl, par, nbr_gpu, wgt_gpu, x0_gpu):
    """GPU results (one form) against the oracle on the sampled blocks:
    neighbour agreement on the non-excluded queries, recall of the K nearest,
    weights where the neighbours agree, and PSNR / max-abs of the HR pixels
    only the blocks cover."""
    K = wl.K
    agree = excl = total = 0
    rec = []
    werr = 0.0
    se = 0.0
    npx = 0
    mx = 0.0
    for (i0, j0), blk, xo, ex in zip(par["origins"], par["blocks"], par["hr"], par["excluded"]):
        rows = block_rows(wl, i0, j0)
        g = nbr_gpu[rows]
        o = blk["nbr"][:, :K]
        same = (g == o).all(axis=1)
        agree += int((same & ~ex).sum())
        excl += int(ex.sum())
        total += len(rows)
        rec.extend(len(np.intersect1d(a, b)) / K for a, b in zip(g[~ex], o[~ex]))
        if same.any():
            werr = max(werr, float(np.abs(wgt_gpu[rows][same] - blk["wgt"][same]).max()))
        full, loc = covered_window(wl, i0, j0)
        d = x0_gpu[full].astype(np.float64) - xo[loc]
        se += float((d * d).sum())
        npx += d.size
        mx = max(mx, float(np.abs(d).max()))
    mse = se / max(npx, 1)
    return {"queries": total, "excluded_tie_or_boundary": excl, "identical_neighbours": agree,
            "recall": float(np.mean(rec)) if rec else None, "weights_max_abs": werr,
            "hr_pixels": npx, "psnr_db": 10 * np.log10(1.0 / max(mse, 1e-30)), "max_abs": mx}


# ---------------------------------------------------------------------------
# GPU timing helpers
# ---------------------------------------------------------------------------
def launches_per_step(wl: S.Workload, precision: int) -> int:
    """Kernels of one zoom_upscale: features, hash, lookup; the search --
    exact form: operand, single-term filter, rerank, then the second stage
    (gather, split operand, split filter, rerank), the SIMT re-run and the
    fallback-count update (9); BF16 form: operand, filter, rerank, SIMT
    re-run, fallback count (5) --; LLE, the two overlap-average passes, and
    two per back-projection step."""
    return 3 + (9 if precision == 0 else 5) + 3 + 2 * wl.bp_iters


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


def timed_steps(fn, steps, st, torch, world: int = 1, nvtx: str = "bench_extra"):
    """Mean ms per step of `fn` with CUDA events on `st`; with several ranks
    the region is bracketed by barriers and the slowest rank's time is kept.
    Every step is an NVTX range named `nvtx` (for profiler filters)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        torch.cuda.nvtx.range_push(nvtx)
        fn()
        torch.cuda.nvtx.range_pop()
    e1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    return max_over_ranks(e0.elapsed_time(e1) / steps, world, "cuda")


def stage_profile(ctx, fn, reps: int = 3) -> dict:
    """Mean per-stage device ms of `fn` over `reps` calls (CUDA events the
    library records between its stages, on the call's stream)."""
    ctx.set_stage_timing(True)
    acc = {}
    for _ in range(reps):
        fn()
        for k, v in ctx.stats()["ms_stage"].items():
            acc[k] = acc.get(k, 0.0) + v / reps
    ctx.set_stage_timing(False)
    return acc


def mean_candidate_fraction(ix, qkeys, torch, n_sample: int = 512, seed: int = 31) -> float:
    """Mean |C(q)| / N over n_sample seeded queries: an entry is a candidate
    when one of its L bucket keys equals the query's (a measurement of the
    method's work per query; torch on the device, outside the timed path)."""
    dk = torch.from_numpy(ix.export_keys()[0].view(np.int64)).cuda()        # [N][L]
    rows = np.random.default_rng(seed).choice(qkeys.shape[0], min(n_sample, qkeys.shape[0]), replace=False)
    qs = qkeys[torch.from_numpy(rows).cuda()]
    tot = 0
    for q in qs:
        tot += int((dk == q[None, :]).any(dim=1).sum())
    del dk
    return tot / len(rows) / ix.dictionary.n


# ---------------------------------------------------------------------------
# the single-image workloads
# ---------------------------------------------------------------------------
def run_single(a, wl, config, rank, world, local):
    import torch

    import paper_1004_3980_gb300 as Z
    hbm_peak, tc_peak, tc_sus, peak_src = peaks()
    hr_px = wl.scale * wl.lr_h * wl.scale * wl.lr_w
    nq = n_queries(wl)
    train, pos, alpha, beta, lr_np = workload_inputs(wl)
    # the oracle first (threads; before any GPU work), on the sampled blocks
    cpu, par = None, None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        threads = a.cpu_threads or os.cpu_count() or 1
        cpu, par = cpu_baseline_and_parity(wl, train, pos, alpha, beta, lr_np,
                                           a.cpu_blocks or default_blocks(wl), threads)
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

    p_bf = params(precision=1, rerank_mult=TOP32_MULT)
    p_ex = params()
    lr = torch.from_numpy(lr_np).cuda()
    shape = (wl.scale * wl.lr_h, wl.scale * wl.lr_w)
    out_bf = torch.empty(shape, device="cuda")
    out_ex = torch.empty(shape, device="cuda")
    # each form warms up right before its own timed region (the caching
    # allocator then holds that form's scratch blocks)
    for _ in range(a.warmup):
        Z.upscale(ix, lr, p_bf, out=out_bf)
    ctx.sync_status()

    # ---- timed region: K steps of the precision form, inputs resident -------
    clocks = ClockSampler(local)
    clocks.start()
    ms_bf = timed_steps(lambda: Z.upscale(ix, lr, p_bf, out=out_bf), a.steps, st, torch, world, "zoom_step")
    clk = clocks.stop()
    value = whole_job_rate(hr_px / 1e6, world, ms_bf)
    # ---- the plain form (exact FP32 neighbours), timed the same way ---------
    for _ in range(a.warmup):
        Z.upscale(ix, lr, p_ex, out=out_ex)
    ctx.sync_status()
    clocks_ex = ClockSampler(local)
    clocks_ex.start()
    ms_ex = timed_steps(lambda: Z.upscale(ix, lr, p_ex, out=out_ex), a.steps, st, torch, world, "zoom_step_fp32")
    clk_ex = clocks_ex.stop()
    ctx.sync_status()
    stage_bf = stage_profile(ctx, lambda: Z.upscale(ix, lr, p_bf, out=out_bf))
    stats_bf = ctx.stats()
    stage_ex = stage_profile(ctx, lambda: Z.upscale(ix, lr, p_ex, out=out_ex))
    stats_ex = ctx.stats()

    # ---- BF16 against the exact form over the whole image ----------------------
    q_ex = Z.query(ix, lr, p_ex)
    q_bf = Z.query(ix, lr, p_bf)
    nb_e, nb_b = q_ex["nbr"], q_bf["nbr"]
    hits = torch.zeros(nq, dtype=torch.int32, device="cuda")
    for m in range(wl.K):
        hits += (nb_b == nb_e[:, m:m + 1]).any(dim=1).int()
    recall_vs_exact = float(hits.double().mean()) / wl.K
    diff = (out_bf.double() - out_ex.double())
    mse = float((diff * diff).mean())
    bf_vs_ex = {"recall": recall_vs_exact, "psnr_db": 10 * np.log10(1.0 / max(mse, 1e-30)),
                "max_abs": float(diff.abs().max()), "queries": nq}
    frac_c = mean_candidate_fraction(ix, q_ex["keys"], torch)

    # ---- the oracle's sampled blocks against both forms ---------------------
    vs_oracle = None
    if par is not None:
        vs_oracle = {"sample": f"{len(par['origins'])} seeded {BLOCK}x{BLOCK} query blocks; HR pixels covered "
                               f"only by a block's patches, before back-projection",
                     "tolerances": "neighbours bit-exact outside FP64 ties (1e-6 rel) and queries whose own bins, "
                                   "or the membership of an entry within their (K+1)-th distance, a projection "
                                   "within 1e-5 w of a bin boundary makes uncertain"}
        for name, q, prm in (("fp32_exact", q_ex, p_ex), ("bf16", q_bf, p_bf)):
            x0 = Z.reconstruct(ix, q["nbr"], q["wgt"], q["mu"], wl.lr_h, wl.lr_w).cpu().numpy()
            vs_oracle[name] = compare_with_oracle(wl, par, q["nbr"].cpu().numpy(), q["wgt"].cpu().numpy(), x0)
    del q_ex, q_bf

    # ---- end to end through the public API with host buffers ----------------
    lr_host = torch.from_numpy(lr_np).pin_memory()
    hr_host = torch.empty(shape, dtype=torch.float32).pin_memory()
    lr_dev = torch.empty_like(lr)

    def e2e_step():
        lr_dev.copy_(lr_host, non_blocking=True)
        Z.upscale(ix, lr_dev, p_bf, out=out_bf)
        hr_host.copy_(out_bf, non_blocking=True)

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
    pairs = nq * frac_c * wl.n_pairs       # the method's work: sum over queries of |C(q)|
    dense = float(nq) * wl.n_pairs

    def filt_roofline(kernel, kms, kdepth, form):
        if kms <= 0:
            return None
        ach = pairs * 2.0 * kdepth / (kms / 1e3) / 1e12
        ach_dense = dense * 2.0 * kdepth / (kms / 1e3) / 1e12
        return {"kernel": kernel, "bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": ach / tc_peak, "kernel_ms": kms,
                "work": (f"sum_q |C(q)| = {nq} queries x {frac_c:.4f} x {wl.n_pairs} entries (mean candidate "
                         f"fraction of 512 sampled queries) x 2 x {kdepth} flops ({form})"),
                "dense_achieved": ach_dense, "dense_frac": ach_dense / tc_peak,
                "dense_note": f"the kernel computes all {nq} x {wl.n_pairs} pairs; dense_* counts them all",
                "peak_source": peak_src + ", bf16 dense burst (fp16 runs at the bf16 rate)",
                "sustained_peak": tc_sus}

    rf_bf = filt_roofline("k_knn_tw<4,32,1,packed> (tcgen05 M128 x N256 BF16 distance filter, "
                          "32-chunk packed lists)",
                          stage_bf.get("knn_filter_kernel", 0.0), 32, "one BF16 term, K = 32 per pair")
    rf_ex = filt_roofline("k_knn_tw<4,16,0> (tcgen05 M128 x N256 single-term FP16 filter of the exact form)",
                          stage_ex.get("knn_filter_kernel", 0.0), 32, "one FP16 term, K = 32 per pair")
    if rf_bf:
        rf_bf["traffic"] = profiled_traffic("paper_1004_3980_gb300/csrc/kernels_tc.cu",
                                            "profiles/knn_tw_bf16_zoom3x_1920x1080_dict4m.md")
        rf_bf["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                                   "(profiles/knn_tw_bf16_zoom3x_1920x1080_dict4m.md); null once the kernel "
                                   "source differs from the captured one")
    PH2 = (wl.scale * wl.patch) ** 2
    oa_bytes = nq * wl.K * PH2 * 4 + hr_px * 4 + nq * (wl.K * 8 + 4)
    bp_bytes = wl.bp_iters * (hr_px * 4 * 3 + wl.lr_h * wl.lr_w * 4 * 3)
    kernels = {}
    for name, byts in (("overlap_add", oa_bytes), ("backproject", bp_bytes)):
        ms = stage_bf.get(name, 0.0)
        if ms > 0:
            gbs = byts / (ms / 1e3) / 1e9
            kernels[name] = {"ms": ms, "algorithmic_bytes": byts, "GB/s": gbs, "frac_hbm": gbs / hbm_peak}
    # the precision form's rerank: the search stage after its filter kernel (the SIMT re-run there has no
    # queries).  Algorithmic bytes: the FP32 rows of the top 4K candidates gathered per query; the kernel
    # reads whole 32-row chunks instead (from L2 mostly), about 8 of them per query
    rr_ms = stage_bf.get("knn", 0.0) - stage_bf.get("knn_filter_kernel", 0.0)
    if rr_ms > 0:
        rr_bytes = nq * 4 * wl.K * wl.patch ** 2 * 4
        gbs = rr_bytes / (rr_ms / 1e3) / 1e9
        kernels["rerank"] = {"ms": rr_ms, "algorithmic_bytes": rr_bytes, "GB/s": gbs, "frac_hbm": gbs / hbm_peak,
                             "kernels": f"k_rerank<{wl.patch ** 2},32>",
                             "note": "algorithmic bytes: 4K rows of 4d bytes per query; the kernel stages "
                                     "whole 32-entry chunks of 112-byte rows, about 8 per query (about 9x "
                                     "those bytes), mostly from L2"}
    if "overlap_add" in kernels:
        kernels["overlap_add"]["kernels"] = "k_blend_rows + k_overlap_average"
        kernels["overlap_add"]["note"] = ("algorithmic bytes count every gathered HR residual value; repeated "
                                          "neighbours are served by L2, so this can exceed the DRAM peak")

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_bf, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": config,
           "lr_patch_queries_per_s": world * nq / (ms_bf / 1e3),
           "fp32_exact": {"value": whole_job_rate(hr_px / 1e6, world, ms_ex), "unit": UNIT, "ms_per_step": ms_ex,
                          "lr_patch_queries_per_s": world * nq / (ms_ex / 1e3), "dtype": "f32",
                          "roofline": rf_ex, "stage_ms_per_step": stage_ex, "clocks": clk_ex,
                          "filter_fallback_queries": stats_ex["n_filter_fallback"],
                          "gpu_launches_per_step": launches_per_step(wl, 0)},
           "bf16_speedup_over_fp32_exact": ms_ex / ms_bf,
           "bf16_vs_fp32_exact": bf_vs_ex, "vs_oracle": vs_oracle,
           "roofline": rf_bf, "kernels_hbm": kernels, "e2e": e2e,
           "gpu_launches": launches_per_step(wl, 1) * a.steps, "clocks": clk,
           "stage_ms_per_step": stage_bf, "mean_candidate_fraction": frac_c,
           "mean_bucket_sum_per_query": stats_bf["mean_bucket_sum"],
           "dictionary_build_ms": dict_ms, "index_build_ms": index_ms,
           "stats": {k2: v for k2, v in stats_bf.items() if k2 != "ms_stage"}}

    if not a.no_extras:
        # the paper's early stop: candidate set capped at 3L IDs (tables in
        # order, IDs ascending within a bin), K nearest among them in FP32
        cap = 3 * wl.L
        ixc = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta, max_candidates=cap)
        out = torch.empty(shape, device="cuda")
        for _ in range(2):
            Z.upscale(ixc, lr, p_ex, out=out)
        ms3 = timed_steps(lambda: Z.upscale(ixc, lr, p_ex, out=out), a.steps, st, torch, world)
        mse3 = float(((out.double() - out_ex.double()) ** 2).mean())
        res["capped_3L"] = {"value": world * hr_px / 1e6 / (ms3 / 1e3), "unit": UNIT, "ms_per_step": ms3,
                            "max_candidates": cap, "distances_per_query": cap,
                            "psnr_vs_uncapped_exact_db": 10 * np.log10(1.0 / max(mse3, 1e-30))}
        ixc.close()
        del out
    if a.all_extras:
        res.update(all_extras(a, wl, ctx, d, ix, lr, out_ex, params, train, pos, st, world, hr_px, nq,
                              tc_peak, hbm_peak))
    ix.close()
    d.close()
    if cpu is not None:
        res["cpu_baseline"] = cpu
    return res


def all_extras(a, wl, ctx, d, ix, lr, hr_exact, params, train, pos, st, world, hr_px, nq, tc_peak, hbm_peak):
    """The split filter alone, one step of the SIMT scan, gradient features
    and crop sampling (not in the default line: minutes at the 4M-pair size)."""
    import torch

    import paper_1004_3980_gb300 as Z
    res = {}
    out = torch.empty_like(hr_exact)
    p3 = params(search=3)
    for _ in range(2):
        Z.upscale(ix, lr, p3, out=out)
    ms6 = timed_steps(lambda: Z.upscale(ix, lr, p3, out=out), a.steps, st, torch, world)
    f3 = stage_profile(ctx, lambda: Z.upscale(ix, lr, p3, out=out)).get("knn_filter_kernel", 0.0)
    ach3 = nq * wl.n_pairs * 2.0 * 80 / (f3 / 1e3) / 1e12 if f3 > 0 else None
    res["exact_split_filter"] = {
        "value": world * hr_px / 1e6 / (ms6 / 1e3), "unit": UNIT, "ms_per_step": ms6,
        "identical_to_exact_form": bool(torch.equal(out, hr_exact)),
        "roofline": {"kernel": "k_knn_tc<10,16,0> (FP16 hi/lo split, K = 80)", "bound": "tensor",
                     "achieved": ach3, "peak": tc_peak, "unit": "TFLOP/s",
                     "frac": ach3 / tc_peak if ach3 else None, "kernel_ms": f3, "work": "dense pairs x 2 x 80"}}
    p2 = params(search=1)
    ms2 = timed_steps(lambda: Z.upscale(ix, lr, p2, out=out), 1, st, torch, world)
    res["fp32_simt_scan"] = {"value": world * hr_px / 1e6 / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2,
                             "identical_to_exact_form": bool(torch.equal(out, hr_exact))}
    # gradient features (Sec. 4.1): the 2 P^2 first-order gradients of each LR
    # patch as its feature, w = 8
    d_g = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, wl.scale, wl.patch,
                       wl.blur_sigma, feature=1)
    D_g = 2 * wl.patch ** 2
    a_g, b_g = S.lsh_draws(wl.proj_seed, wl.L, wl.k, D_g, GRAD_W)
    ixg = Z.Index(d_g, wl.L, wl.k, GRAD_W, a_g, b_g)
    pg = params()
    for _ in range(2):
        Z.upscale(ixg, lr, pg, out=out)
    ms4 = timed_steps(lambda: Z.upscale(ixg, lr, pg, out=out), a.steps, st, torch, world)
    fg = stage_profile(ctx, lambda: Z.upscale(ixg, lr, pg, out=out)).get("knn_filter_kernel", 0.0)
    st_g = ctx.stats()
    ach_g = nq * wl.n_pairs * 2.0 * 64 / (fg / 1e3) / 1e12 if fg > 0 else None
    res["gradient_features"] = {
        "value": world * hr_px / 1e6 / (ms4 / 1e3), "unit": UNIT, "ms_per_step": ms4,
        "feature_dim": D_g, "w": GRAD_W, "mean_bucket_sum_per_query": st_g["mean_bucket_sum"],
        "filter_fallback_queries": st_g["n_filter_fallback"],
        "roofline": {"kernel": "k_knn_tw<8,16,0> (M128 x N256 single-term FP16, K = 64)", "bound": "tensor",
                     "achieved": ach_g, "peak": tc_peak, "unit": "TFLOP/s",
                     "frac": ach_g / tc_peak if ach_g else None, "kernel_ms": fg,
                     "work": f"{nq} queries x {wl.n_pairs} entries x 2 x 64 flops (dense)"}}
    ixg.close()
    d_g.close()
    # training-crop sampling (Sec. 5.1): 25 crops of 100 x 100 per training image
    imgs_t = [torch.from_numpy(x).cuda() for x in train]
    n_draw, side = 25, 100
    u_s = np.random.default_rng(17).random((len(train), n_draw))
    for _ in range(2):
        Z.sample_crops(ctx, imgs_t, u_s, side, side)
    ms5 = timed_steps(lambda: Z.sample_crops(ctx, imgs_t, u_s, side, side), a.steps, st, torch, world)
    px = sum(x.size for x in train)
    byts = px * 4 + len(train) * n_draw * (1024 * 4 + 2 * side * side * 4)
    res["crop_sampling"] = {
        "value": world * len(train) * n_draw / (ms5 / 1e3), "unit": "crops/s", "ms_per_step": ms5,
        "images": len(train), "pixels": px, "crops_per_image": n_draw, "crop": [side, side],
        "algorithmic_bytes": byts, "GB/s": byts / (ms5 / 1e3) / 1e9, "frac_hbm": byts / (ms5 / 1e3) / 1e9 / hbm_peak}
    return res


# ---------------------------------------------------------------------------
# the batched form
# ---------------------------------------------------------------------------
def batch_launches(shapes, bp_iters: int, precision: int) -> int:
    """Kernels of one recorded batch: per image features, hash, the two
    overlap-average passes and two per back-projection step; per scale the
    search (see launches_per_step) and the LLE."""
    per_image = 4 + 2 * bp_iters
    per_scale = (9 if precision == 0 else 5) + 1
    return len(shapes) * per_image + len({s for *_, s in shapes}) * per_scale


def run_batch(a, rank, world, local, steps: int, warmup: int):
    """64 mixed images through zoom_upscale_batch (BF16 form, recorded graph),
    with the exact FP32 form batched and looped image by image beside it."""
    import torch

    import paper_1004_3980_gb300 as Z
    shapes = S.batch_shapes(64)
    ctx = Z.Context(local)
    indexes, dicts = [], []
    for s, hrs, nimg in ((2, 512, 64), (3, 768, 128)):
        wl = S.Workload(f"dict{s}x", 0, 0, s, 5, nimg, hrs, 1_000_000, L=16, k=16, K=8, bp_iters=5,
                        train_seed0=1000 if s == 2 else 5000)
        train = S.training_images(wl)
        lrs = hrs // s
        pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, 5, wl.n_pairs)
        alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, 25, wl.w)
        imgs = [torch.from_numpy(x).cuda() for x in train]
        d = Z.Dictionary(ctx, imgs, pos, s, 5)
        dicts.append(d)
        indexes.append(Z.Index(d, wl.L, wl.k, wl.w, alpha, beta))
        del imgs, train
    lr_np = [(s, S.make_image(seed, h, w)) for seed, h, w, s in shapes]
    lrs = [(s, torch.from_numpy(x).cuda()) for s, x in lr_np]
    hr_px = sum(s * s * x.shape[0] * x.shape[1] for s, x in lrs)
    nq = sum((x.shape[0] - 4) * (x.shape[1] - 4) for _, x in lrs)
    # the batched form's lists: the best 16 chunks (rerank_mult * K = 16;
    # the best-32 reading belongs to the single 3x image)
    p1 = Z.UpscaleParams(K=8, bp_iters=5, precision=1, rerank_mult=2)
    st = torch.cuda.current_stream()
    outs, _ = Z.upscale_batch(indexes, lrs, p1)            # autotune + record
    for _ in range(max(0, warmup - 1)):
        Z.upscale_batch(indexes, lrs, p1, outs=outs)
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(lambda: Z.upscale_batch(indexes, lrs, p1, outs=outs), steps, st, torch, world, "zoom_batch")
    clk = clocks.stop()
    _, lat = Z.upscale_batch(indexes, lrs, p1, outs=outs, want_latency=True)
    value = whole_job_rate(hr_px / 1e6, world, ms)
    # end to end: every step copies the 64 LR images in from pinned host
    # memory and the 64 HR images out
    hosts_in = [torch.from_numpy(x).pin_memory() for _, x in lr_np]
    hosts_out = [torch.empty(o.shape, dtype=torch.float32).pin_memory() for o in outs]

    def e2e_step():
        for hx, (_, x) in zip(hosts_in, lrs):
            x.copy_(hx, non_blocking=True)
        Z.upscale_batch(indexes, lrs, p1, outs=outs)
        for ho, o in zip(hosts_out, outs):
            ho.copy_(o, non_blocking=True)

    e2e_step()
    st.synchronize()
    n_e2e = max(2, min(steps, 5))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
        st.synchronize()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    # the exact FP32 form looped image by image, and batched
    p0 = Z.UpscaleParams(K=8, bp_iters=5)
    by = {ix.dictionary.scale: ix for ix in indexes}
    loop_outs = [torch.empty_like(o) for o in outs]

    def loop():
        for (s, x), o in zip(lrs, loop_outs):
            Z.upscale(by[s], x, p0, out=o)

    loop()
    ms_loop = timed_steps(loop, 2, st, torch, world)
    mse = float(sum(((o.double() - lo.double()) ** 2).sum() for o, lo in zip(outs, loop_outs)) / hr_px)
    outs0, _ = Z.upscale_batch(indexes, lrs, p0)
    Z.upscale_batch(indexes, lrs, p0, outs=outs0)
    ms_exact = timed_steps(lambda: Z.upscale_batch(indexes, lrs, p0, outs=outs0), min(steps, 5), st, torch, world)
    same = all(bool(torch.equal(o, lo)) for o, lo in zip(outs0, loop_outs))
    Z.batch_release(ctx)
    for ix in indexes:
        ix.close()
    for d in dicts:
        d.close()
    ctx.close()
    h2d = sum(x.numel() * 4 for x in hosts_in)
    d2h = sum(x.numel() * 4 for x in hosts_out)
    return {"value": value, "unit": UNIT, "ms_per_batch": ms, "dtype": "bf16",
            "workload": "64 LR images 96..768 x 128..1024, half 2x / half 3x, 1M-pair dictionary per scale, "
                        "K=8, 5 back-projection steps, BF16 filter + FP32 rerank of the best 16 chunks, "
                        "one zoom_upscale_batch call (recorded CUDA graph)",
            "hr_megapixels_per_batch": hr_px / 1e6, "lr_patch_queries_per_s": world * nq / (ms / 1e3),
            "per_image_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "fp32_exact_loop": {"value": world * hr_px / 1e6 / (ms_loop / 1e3), "ms_per_batch": ms_loop},
            "fp32_exact_batch": {"value": world * hr_px / 1e6 / (ms_exact / 1e3), "ms_per_batch": ms_exact,
                                 "identical_to_exact_loop": same},
            "psnr_bf16_batch_vs_fp32_exact_db": 10 * np.log10(1.0 / max(mse, 1e-30)),
            "clocks": clk, "gpu_launches": batch_launches(shapes, 5, 1) * steps,
            "e2e": {"value": world * hr_px / 1e6 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h}}


# ---------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def reference_arm(a, wl, config, rank):
    """The FP64 oracle, as it stands, timed on the host cores: every step is
    one seeded block of 16 query rows (one row per host thread) of 2 queries
    at 4M pairs, 8 below (a few seconds of oracle work on 16 threads; hash,
    candidates, top-K, LLE) plus the block's blend, with the back-projection
    cost per HR pixel from one 64-row band; extrapolated to HR megapixels/s."""
    if rank != 0:
        return
    threads = a.cpu_threads or os.cpu_count() or 1
    side, cols = BLOCK, (2 if wl.n_pairs > 1_000_000 else 8)
    train, pos, alpha, beta, lr = workload_inputs(wl)
    od, oi, setup_s = oracle_setup(wl, train, pos, alpha, beta)
    bp_px, band = oracle_bp_seconds_per_px(wl, lr)
    origins = block_origins(wl, a.warmup + a.steps, seed=41)
    vals = []
    for i, org in enumerate(origins):
        blocks, wall = oracle_block_queries(wl, lr, od, oi, [org], threads, side, cols)
        t0 = time.perf_counter()
        oracle_block_hr(wl, train, pos, blocks[0], side, cols)
        blend = (time.perf_counter() - t0) / (side * cols)
        if i >= a.warmup:
            vals.append(cpu_rate(wl, wall / (side * cols), blend, bp_px))
    v = statistics.median(vals)
    hr_px = wl.scale * wl.lr_h * wl.scale * wl.lr_w
    sample = (f"per step one seeded block of {side} x {cols} queries ({threads} threads) and its blend, plus the "
              f"back-projection cost per HR pixel of a {band}-row band; extrapolated to the {n_queries(wl)} "
              f"queries and {hr_px} HR pixels")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                      "steps": a.steps, "warmup": a.warmup, "ms_per_step": hr_px / 1e6 / v * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": config,
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                       "sample": sample, "setup_s": setup_s, "cpu_model": cpu_model()},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def single_config(wl: S.Workload, world: int) -> dict:
    return {"workload": wl.name, "lr": [wl.lr_h, wl.lr_w], "scale": wl.scale, "dict_pairs": wl.n_pairs,
            "lr_patch": wl.patch, "L": wl.L, "k": wl.k, "K": wl.K, "bp_iters": wl.bp_iters,
            "precision": "bf16 filter (fp32 accumulate) + fp32 exact rerank of the best 32 chunks; "
                         "fp32_exact: exact fp32 neighbours",
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": ("inputs larger than L2 (dictionary operands, features and HR patches: "
                   f"{(wl.n_pairs * (64 + 112 + 4 * (wl.scale * wl.patch) ** 2)) / 1e9:.1f} GB)")}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    batch_only = a.workload == "batch64_mixed"
    wl = None if batch_only else S.WORKLOADS[a.workload]
    if batch_only:
        config = {"workload": "batch64_mixed: 64 LR images 96..768 x 128..1024, half 2x / half 3x, "
                              "1M-pair dictionary per scale, K=8, 5 back-projection steps, BF16 form",
                  "parallelism": f"replicas{world}" if world > 1 else "single"}
    else:
        config = single_config(wl, world)
    if a.impl == "reference":
        if batch_only:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-image "
                                  "workloads only"}), flush=True)
            return
        reference_arm(a, wl, config, rank)
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
    if batch_only:
        b = run_batch(a, rank, world, local, a.steps, a.warmup)
        res = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": b["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": config,
               "gpu_launches": b["gpu_launches"], "clocks": b["clocks"], "e2e": b["e2e"], "batch64_mixed": b}
    else:
        res = run_single(a, wl, config, rank, world, local)
        if not a.no_batch:
            res["batch64_mixed"] = run_batch(a, rank, world, local, min(a.steps, 5), 2)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
