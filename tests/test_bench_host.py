"""Host-side pieces of bench.py (CPU only).

A stored ncu figure (DRAM bytes per launch, shared-memory pipe utilisation) is
reported only while the sources its kernels are built from are the ones it
was captured on; the key is a hash of their code with comments and layout
removed, so that editing a comment keeps the figure and editing code drops it.
"""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_hash_ignores_comments_and_layout_but_not_code():
    src = open(os.path.join(ROOT, "paper_1505_05655_gb300", "csrc", "lutc_tma.cu")).read()
    base = bench._code_only(src)
    commented = src.replace("namespace lutc {", "// a new comment line\nnamespace lutc {  /* and a block */", 1)
    reflowed = src.replace("constexpr int kConsumers = 256;", "constexpr  int   kConsumers =\n  256;", 1)
    assert bench._code_only(commented) == base
    assert bench._code_only(reflowed) == base
    assert bench._code_only(src.replace("constexpr int kConsumers = 256;", "constexpr int kConsumers = 128;", 1)) != base
    # preprocessor lines stay lines: joining a define with the next statement would change the code
    assert bench._code_only("#define A 1\nint x;") != bench._code_only("#define A 1 int x;")

