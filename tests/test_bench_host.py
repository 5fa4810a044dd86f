"""Host logic of bench.py on the CPU: the clock sampler (against a stand-in
nvidia-smi that prints the queried fields), the launch count of one step and
the DRAM traffic taken from an ncu summary only while the kernel's source is
the one profiled."""
import hashlib
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth_inputs as S  # noqa: E402


def _fake_smi(tmp_path, line, delay=0.2):
    p = tmp_path / "nvidia-smi"
    p.write_text(f"#!/bin/sh\nsleep {delay}\nwhile true; do echo '{line}'; sleep 0.05; done\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, "1980, 2070, 1350.5, 0x4, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    t0 = time.perf_counter()
    c.start()
    assert time.perf_counter() - t0 < 3.5        # waited for the first sample, bounded
    time.sleep(0.4)
    r = c.stop()
    assert r["samples"] >= 2
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_sampler_keeps_only_samples_after_start(tmp_path, monkeypatch):
    # stopped at once: the sample that announced the process is not counted
    d = _fake_smi(tmp_path, "2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active", 0.0)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r["samples"] <= 1


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_launches_per_step():
    wl = S.WORKLOADS["zoom3x_1920x1080_dict4m"]
    # features, hash, lookup; 9 launches of the three-stage exact search or 5
    # of the BF16 search; LLE, the two overlap-average passes; 2 per
    # back-projection step
    assert bench.launches_per_step(wl, 0) == 3 + 9 + 3 + 2 * wl.bp_iters == 25
    assert bench.launches_per_step(wl, 1) == 21
    shapes = [(1, 100, 120, 2), (2, 90, 130, 3), (3, 100, 100, 2)]
    assert bench.batch_launches(shapes, 5, 1) == 3 * 14 + 2 * 6


def test_block_rows_and_covered_window():
    wl = S.WORKLOADS["zoom3x_1920x1080_dict4m"]
    nw = wl.lr_w - wl.patch + 1
    rows = bench.block_rows(wl, 10, 20)
    assert len(rows) == bench.BLOCK ** 2 and rows[0] == 10 * nw + 20 and rows[bench.BLOCK] == 11 * nw + 20
    (fy, fx), (ly, lx) = bench.covered_window(wl, 10, 20)
    s, PH = wl.scale, wl.scale * wl.patch
    assert fy.start == s * 10 + PH - 1 and fy.stop == s * (10 + bench.BLOCK)
    assert ly.stop - ly.start == fy.stop - fy.start and lx.start == PH - 1
    for i0, j0 in bench.block_origins(wl, 5):
        assert 0 <= i0 <= wl.lr_h - wl.patch + 1 - bench.BLOCK and 0 <= j0 <= nw - bench.BLOCK


def test_oracle_blocks_equal_the_whole_image_oracle():
    # the bench's parity sample: the oracle run on a block's own sub-image
    # gives the whole image's queries of that block, and its HR estimate over
    # the covered window equals the whole image's reconstruction there
    import dataclasses

    import numpy as np

    from oracle import zoom_oracle as O
    wl = dataclasses.replace(S.WORKLOADS["zoom2x_64_dict20k"], n_pairs=3000, lr_h=24, lr_w=26)
    train = S.training_images(wl, 4)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, wl.patch ** 2, wl.w)
    lr = S.test_image(wl)
    od, oi, _ = bench.oracle_setup(wl, train, pos, alpha, beta)
    origins = [(3, 5)]
    blocks, _ = bench.oracle_block_queries(wl, lr, od, oi, origins, 2)
    full = O.build_dictionary(train, pos, wl.scale, wl.patch, wl.blur_sigma)
    qr = O.query(lr, full, oi, wl.K, wl.reg_rel)
    rows = bench.block_rows(wl, *origins[0])
    b = blocks[0]
    assert (b["nbr"][:, :wl.K] == qr.nbr[rows]).all()
    np.testing.assert_allclose(b["wgt"], qr.wgt[rows], atol=1e-12)
    x0 = O.reconstruct(qr.nbr, qr.wgt, qr.mu, full, wl.lr_h, wl.lr_w)
    xb = bench.oracle_block_hr(wl, train, pos, b)
    fw, lw = bench.covered_window(wl, *origins[0])
    np.testing.assert_allclose(xb[lw], x0[fw], atol=1e-12)
    # the comparison of a GPU-shaped result (here the oracle's own) is exact
    par = {"origins": origins, "blocks": blocks, "hr": [xb],
           "excluded": bench.block_exclusions(blocks, od, oi, 2)}
    c = bench.compare_with_oracle(wl, par, qr.nbr, qr.wgt, x0)
    assert c["identical_neighbours"] + c["excluded_tie_or_boundary"] == c["queries"] == bench.BLOCK ** 2
    assert c["recall"] == 1.0 and c["max_abs"] < 1e-12 and c["weights_max_abs"] < 1e-12


def test_profiled_traffic_follows_the_source(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    summ = tmp_path / "s.md"
    summ.write_text(f"# capture\n\nCommand: ncu ...\n\nkernel_source_sha256_16: {sha}\n"
                    "traffic_bytes_per_launch: 123456\n")
    assert bench.profiled_traffic(str(src), str(summ)) == 123456
    src.write_text("__global__ void k() { }\n")          # the kernel changed: no traffic
    assert bench.profiled_traffic(str(src), str(summ)) is None
    assert bench.profiled_traffic(str(src), str(tmp_path / "missing.md")) is None

