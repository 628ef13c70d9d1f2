"""Host-side logic that needs no GPU: the roofline byte counts of bench.py
against their closed forms, the autotuner's report format, and the argument
checks of the entry points that return before any CUDA call."""
import ctypes
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_algorithmic_bytes_2d_1024():
    # kept columns under the two-thirds rule: 3 |k| < 1024 -> kx = 0..341 (342 of the 513
    # half-spectrum columns); per step 8 bytes x M modes x (4 + 2 f), M = 513 x 1024
    b = _bench().algorithmic_bytes_2d(1024, 1024)
    M = 513 * 1024
    assert b["step"] == pytest.approx(8 * M * (4 + 2 * 342 / 513))
    assert b["col"] + b["row"] == pytest.approx(b["step"])
    assert round(b["step"] / 1e6, 2) == 22.41


def test_algorithmic_bytes_3d_256():
    # per field-step 8 M (6 + 2 fx fy + 2 fx), fx = 86/129 kept kx, fy = 171/256 kept ky
    b = _bench().algorithmic_bytes_3d(256, 256, 256)
    M = 129 * 256 * 256
    fx, fy = 86 / 129, 171 / 256
    assert b["step"] == pytest.approx(8 * M * (6 + 2 * fx * fy + 2 * fx))
    assert round(b["step"] / 1e6, 1) == 556.2


def test_whole_job_rate_single_rank():
    value, t = _bench().whole_job_rate(1_000_000, 250.0, 1)
    assert t == 250.0 and value == pytest.approx(4e6)


def test_kernel_source_hash_follows_code_not_comments(tmp_path):
    # the traffic record stays valid across comment edits and is dropped by a code change
    b = _bench()
    csrc = tmp_path / "paper_2405_02410_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = csrc / "k.cuh"
    old_root = b.ROOT
    try:
        b.ROOT = str(tmp_path)
        src.write_text("int f(int x) {  // one\n    return x + 1;\n}\n")
        h0 = b.kernel_source_hash()
        src.write_text("// a new header line\nint f(int x) {  // two\n\n    return x + 1; /* note */\n}\n")
        assert b.kernel_source_hash() == h0
        src.write_text("int f(int x) {\n    return x + 2;\n}\n")
        assert b.kernel_source_hash() != h0
    finally:
        b.ROOT = old_root


def test_line_summary_is_short_and_complete():
    # the JSON line ends with a summary of its main results, short enough for a tail of stdout
    import json
    line = {"ms_per_step": 0.0115, "value": 9.1e10, "roofline": {"frac": 0.285}, "e2e": {"value": 3.5e10},
            "extra": {"model_ab_256cubed": {"ms_per_step_two_fields": 0.3646, "site_steps_per_s_per_field": 9.2e10,
                                            "hbm_frac_of_measured": 0.449},
                      "ensemble_512": {"ms_per_step": 0.455, "site_steps_per_s": 9.46e10, "speedup_vs_sequential": 8.9,
                                       "S_q_mean_by_side": {"64": [0.0] * 64}},
                      "adjoint_256": {"adjoint_ms": 30.9, "forward_plain_ms": 11.0, "adjoint_over_forward": 2.8},
                      "variants": {"kpz_1024": {"ms_per_step": 0.0156, "over_model_b_step": 1.45}},
                      "cufft_step_1024": {"ms_per_step": 0.0641, "ours_over_cufft": 5.96}},
            "parity_vs_fp64_oracle": {"a": {"steps": 63, "rel_l2": 1.5e-6},
                                      "b": {"rel_l2_model_a": 2.9e-7, "rel_l2_model_b": 6.6e-6}}}
    sm = _bench().summary_of(line)
    assert sm["us_per_step"] == 11.5 and sm["roofline_frac"] == 0.285
    assert sm["model_ab_256cubed"]["hbm_frac_of_measured"] == 0.449
    assert sm["adjoint_256"]["adjoint_over_forward"] == 2.8
    assert sm["parity_max_rel_l2"] == 6.6e-6
    assert "S_q_mean_by_side" not in json.dumps(sm) and len(json.dumps(sm)) < 1000


def test_tune_report_parsing():
    from paper_2405_02410_gb300 import pss
    rep = pss.parse_tune_report("path=1 trials=25 skipped=0 initial_ms=0.015071 tuned_ms=0.0149 "
                                "col2_radix=16 row2_pairs=0 pdl=-1 graph_steps=32")
    assert rep == {"path": 1, "trials": 25, "skipped": 0, "initial_ms": 0.015071, "tuned_ms": 0.0149,
                   "col2_radix": 16, "row2_pairs": 0, "pdl": -1, "graph_steps": 32}


def test_null_handles_are_rejected_without_a_gpu():
    from paper_2405_02410_gb300 import pss
    lib = pss.lib
    buf = ctypes.create_string_buffer(64)
    assert lib.pss_autotune(None, 16, buf, len(buf)) == pss.PSS_EINVAL
    assert lib.pss_set_tuning(None, b"pdl", 1) == pss.PSS_EINVAL
    assert lib.pss_step(None, 1) == pss.PSS_EINVAL
    assert lib.pss_step_path(None) == pss.PSS_EINVAL
