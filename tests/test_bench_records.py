"""The benchmark's committed records stay tied to the sources they describe (no GPU needed).

bench.py reports the block build's DRAM traffic from profiles/block_pair_he4_traffic.txt only while
the tensor-core kernel's code is the code that was profiled; the record carries a hash of the code
tokens (comments and blank space removed).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_tokens_ignore_comments_and_layout():
    a = "int f(int x) {\n    return x + 1;  // one more\n}\n"
    b = "/* the successor */ int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b)
    assert bench.code_tokens(a) != bench.code_tokens(c)


def test_traffic_record_matches_the_kernel_source():
    """A kernel change without a new ncu capture leaves the record stale (bench reports null)."""
    assert bench.recorded_traffic() is not None
    # per launch: four one-source slabs; at least the algorithmic bytes (the sink-upper rows)
    assert bench.recorded_traffic() >= 4 * 128 * 4096 * 1152 // 4
