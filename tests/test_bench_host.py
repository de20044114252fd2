"""Host logic of bench.py that decides whether a roofline figure may be
printed: a committed ncu summary carries the SHA-256 of the kernel's sources
(the .cu file and its local includes, comments and blank space removed), and
bench.py reports the summary's figures only while that stamp matches the
code that is built. Checked here on a temporary source tree, without a GPU."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _tree(root, kernel, header):
    csrc = root / "paper_2609_31258_b300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    (csrc / "k.cu").write_text(kernel)
    (csrc / "k.cuh").write_text(header)
    return csrc


KERNEL = '#include "k.cuh"\n// the step\n__global__ void k(float *x) { x[0] = f(x[0]); }\n'
HEADER = '#pragma once\n/* a helper */\n__device__ float f(float v) { return v * 2.0f; }\n'


@pytest.fixture
def tree(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path, _tree(tmp_path, KERNEL, HEADER)


def test_stamp_ignores_comments_and_blank_space(tree):
    root, csrc = tree
    s0 = bench.source_stamp("k.cu")
    (csrc / "k.cu").write_text("// new comment\n\n" + KERNEL.replace("// the step", "/* changed\n comment */"))
    (csrc / "k.cuh").write_text(HEADER.replace("/* a helper */", "   \n// another\n"))
    assert bench.source_stamp("k.cu") == s0


def test_stamp_follows_code_and_includes(tree):
    root, csrc = tree
    s0 = bench.source_stamp("k.cu")
    (csrc / "k.cuh").write_text(HEADER.replace("2.0f", "3.0f"))  # a change in an included file
    s1 = bench.source_stamp("k.cu")
    assert s1 != s0
    (csrc / "k.cuh").write_text(HEADER)
    (csrc / "k.cu").write_text(KERNEL.replace("x[0] = f(x[0])", "x[0] = f(x[1])"))
    assert bench.source_stamp("k.cu") not in (s0, s1)


def test_profile_fields_fresh_stale_and_missing(tree):
    root, csrc = tree
    prof = root / "profiles" / "k.txt"
    prof.write_text(f"# summary\nsources_sha256: {bench.source_stamp('k.cu')} (k.cu)\ninst_per_pack_step: 552.5\n")
    out, stale = bench._profile_fields("k.txt", "k.cu")
    assert stale is None and out["inst_per_pack_step"] == "552.5"
    (csrc / "k.cu").write_text(KERNEL.replace("f(x[0])", "f(x[0]) + 1.0f"))
    out, stale = bench._profile_fields("k.txt", "k.cu")
    assert stale is not None and "re-profile" in stale and out["inst_per_pack_step"] == "552.5"
    out, stale = bench._profile_fields("absent.txt", "k.cu")
    assert out == {} and stale == "no profile summary"
