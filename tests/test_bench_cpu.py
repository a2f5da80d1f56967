"""Host-side pieces of bench.py that need no GPU: the committed ncu summaries it reads for the
roofline (parsed, keyed by a hash of the kernel sources, ignored once the sources change) and the
ALU roofline arithmetic."""
import os
import shutil

import pytest

import bench


def test_trace_profile_summary_is_parsed_and_keyed_by_the_sources(tmp_path):
    path = bench.TRACE_PROFILE
    assert os.path.exists(path), "the trace's ncu summary is committed under profiles/"
    text = open(path).read()
    assert "--clock-control none" in text  # the command that made it is recorded
    kv = bench.profile_summary()
    if kv is None:
        pytest.skip("the trace sources changed since the summary was captured (bench reports null)")
    for key in ("dram_bytes_per_launch", "lts_bytes_per_launch", "warp_execution_efficiency", "alu_pipe_pct",
                "issue_active_pct", "duration_ms"):
        assert bench.profiled(kv, key) is not None, key
    assert 0.0 < bench.profiled(kv, "warp_execution_efficiency") <= 1.0
    assert 0.0 < bench.profiled(kv, "alu_pipe_pct") <= 100.0
    # the same summary under another file list (other sources) is not used
    assert bench.profile_summary(path, files=("k_prep.cu",)) is None
    # a summary whose hash line is altered is not used either
    alt = tmp_path / "alt.txt"
    shutil.copy(path, alt)
    lines = alt.read_text().splitlines()
    lines = [("kernel_source_sha256_16: 0000000000000000" if ln.startswith("kernel_source_sha256_16") else ln)
             for ln in lines]
    alt.write_text("\n".join(lines) + "\n")
    assert bench.profile_summary(str(alt)) is None
    assert bench.profile_summary(str(tmp_path / "missing.txt")) is None


def test_profiled_tolerates_missing_and_malformed_values():
    assert bench.profiled(None, "x") is None
    assert bench.profiled({"x": "n/a"}, "x") is None
    assert bench.profiled({"x": "1.5"}, "y") is None
    assert bench.profiled({"x": "1.5"}, "x") == 1.5


def test_whole_job_rate_and_alu_peak_arithmetic():
    # 152 SMs x 64 ALU-pipe lanes x 2070 MHz = 20.14 T lane-ops/s, the roofline's derived ALU peak
    assert bench.alu_peak_gops(2070.0) == pytest.approx(20136.96)
    # the achieved figure reproduces from the line's fields: 29 ops x iterations + 100 x samples
    assert bench.alu_achieved_gops(320_000_000, 12_700_000, 2.5) == pytest.approx(
        (29 * 320e6 + 100 * 12.7e6) / 2.5e-3 / 1e9)
    # one rank, 23.04 M rays in 3.2 ms
    assert bench.whole_job_rate(23040000.0, 1, 3.2) == pytest.approx(7.2e9)


def test_parity_record_counts_pixels_hits_and_gradient_errors():
    """The bench's parity record: per-pixel RGB error relative to max(|oracle|_inf, 1e-3) on the
    pixels whose samples hit alike (and that no differing sample hits), hit agreement per
    sample, gradient error relative to each buffer's scale on those pixels."""
    import numpy as np
    hits = np.array([[[[1, 2], [3, 4]], [[5, 6], [7, -1]]]], np.int32)  # [V=1, H=2, W=2, spp=2]
    orc = {"final": np.ones((1, 2, 2, 3)), "hit_idx": hits,
           "grads": {"rough": np.array([[[1.0, -2.0], [0.5, 0.25]]]), "env": np.ones((2, 4, 3))}}
    fin = np.ones((1, 2, 2, 3), np.float32)
    fin[0, 0, 0, 1] = 1.0 + 3e-4   # pixel (0, 0) over 1e-4
    fin[0, 1, 1, 2] = 1.0 + 5e-5   # pixel (1, 1) within
    fin[0, 0, 1, 0] = 2.0          # pixel (0, 1): its sample hits differently, left out
    hg = hits.copy()
    hg[0, 0, 1, 0] = 0             # the GPU says pixel 0 = (0, 0), the oracle pixel 3 = (1, 1)
    gr = np.array([[[1.0, 9.0], [0.5, 0.25]]], np.float32)
    gr[0, 1, 0] = 0.502            # pixel (1, 0): 0.002 / scale 0.5 (the only pixel left in)
    gpu = {"final": fin, "hit_idx": hg, "grads": {"rough": gr, "env": np.ones((2, 4, 3), np.float32)}}
    rec = bench.parity_record(gpu, orc)
    assert rec["hit_index_match"] == 7 / 8
    # left out: the receiver (0, 1), and the pixels either side hit: (0, 0) and (1, 1)
    assert rec["pixels_with_a_differing_hit"] == 3 and rec["pixels_compared"] == 1
    assert rec["pixels_over_1e-4"] == 0 and rec["pixels_within_1e-4"] == 1.0
    assert abs(rec["grad_max_err_over_scale"]["rough"] - 0.004) < 1e-6
    assert rec["grad_max_err_over_scale"]["env"] == 0.0
