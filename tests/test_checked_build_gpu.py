"""The checked build of the library (libwrs_checked.so, compiled with
WRS_CHECKED): every kernel tests the indices and bulk-copy ranges it uses
against their buffers and records a failed test in the stream's check word
instead of touching memory. The parity cases with ragged sizes, every launch
and pipeline shape, flush maps, the index ring, batches and reprojection run
against it in a child process (WRS_CHECKED=1 makes the package load it); each
case ends in wrs_check_status, which fails on any recorded bit, and still
compares with the oracle bit for bit."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_parity_gpu.py::test_tiny_workload_bit_exact",
    "tests/test_parity_gpu.py::test_k_and_ragged_sizes",
    "tests/test_parity_gpu.py::test_launch_shapes_agree",
    "tests/test_parity_gpu.py::test_pipeline_shapes_agree",
    "tests/test_parity_gpu.py::test_pipeline_many_tiles_per_cta",
    "tests/test_parity_gpu.py::test_pipeline_without_fused_resolve",
    "tests/test_parity_gpu.py::test_fp16_colour",
    "tests/test_parity_gpu.py::test_flush_map",
    "tests/test_parity_gpu.py::test_padded_pitch_and_standalone_resolve",
    "tests/test_parity_gpu.py::test_literal_rule_bit_exact",
    "tests/test_parity_gpu.py::test_literal_rule_ragged",
    "tests/test_parity_gpu.py::test_full_temporal_bias_bit_exact",
    "tests/test_index_ring_gpu.py",
    "tests/test_batch_gpu.py::test_batch_equals_individual_pushes",
    "tests/test_batch_gpu.py::test_batch_mixes_literal_and_key_streams",
    "tests/test_reproj_gpu.py::test_ragged_sizes",
    "tests/test_reproj_gpu.py::test_mixed_plain_and_reprojected_pushes",
]


def _env():
    env = dict(os.environ)
    env["WRS_CHECKED"] = "1"
    return env


def test_checked_library_is_the_one_loaded():
    r = subprocess.run([sys.executable, "-c",
                        "import paper_2510_03964_gb300 as w; import sys; "
                        "sys.exit(0 if w.load().wrs_checked_build() == 1 else 3)"],
                       cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]


def test_parity_cases_run_clean_under_the_checked_build():
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        *CASES], cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-1000:])
