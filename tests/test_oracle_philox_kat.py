"""Known answers for the oracle's Philox4x32-10 (Salmon et al., SC'11; the
counter-based generator of the collision and source draws, Eq. 6 and Eq. 5
sampling).

The statistical pins of test_oracle_rng.py cannot tell a correct Philox from
one with a swapped output word, a wrong Weyl constant or a transposed
multiplier. This test compares the oracle block by block with PyTorch's
independent open-source implementation (ATen's philox_engine, compiled from
the header that ships with the installed torch), on random counters and keys
and on the edge words (all zeros, all ones, carries)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_include():
    import torch
    return os.path.join(os.path.dirname(torch.__file__), "include")


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    inc = _torch_include()
    if shutil.which("g++") is None or not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("g++ or ATen headers unavailable")
    exe = str(tmp_path_factory.mktemp("kat") / "aten_philox_kat")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, os.path.join(HERE, "aten_philox_kat.cpp"), "-o", exe],
                   check=True, capture_output=True)

    def run(rows):
        txt = "\n".join(" ".join(str(int(x)) for x in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout
        return np.array([[int(x) for x in ln.split()] for ln in out.strip().splitlines()], dtype=np.uint64)

    return run


def _oracle_blocks(orc, rows):
    return np.array([orc.philox(list(r[:4]), list(r[4:])) for r in rows], dtype=np.uint64)


def test_philox_matches_aten_on_random_blocks(orc, aten_philox):
    rng = np.random.default_rng(20260931)
    rows = rng.integers(0, 2 ** 32, size=(1500, 6), dtype=np.uint64)
    ref = aten_philox(rows)
    got = _oracle_blocks(orc, rows)
    assert ref.shape == (1500, 4)
    bad = np.nonzero((ref != got).any(axis=1))[0]
    assert bad.size == 0, (bad[:5], rows[bad[:1]], ref[bad[:1]], got[bad[:1]])


def test_philox_matches_aten_on_edge_words(orc, aten_philox):
    m = 2 ** 32 - 1
    rows = [[0, 0, 0, 0, 0, 0], [m, m, m, m, m, m], [m, 0, 0, 0, 0, 0], [0, m, 0, 0, 0, 0], [0, 0, m, 0, 0, 0],
            [0, 0, 0, m, 0, 0], [0, 0, 0, 0, m, 0], [0, 0, 0, 0, 0, m], [1, 2, 3, 4, 5, 6],
            [2 ** 31, 2 ** 31, 2 ** 31, 2 ** 31, 2 ** 31, 2 ** 31]]
    # the counters the step itself uses: (pack id, step, draw block, purpose), key (seed lo, seed hi)
    for pack in (0, 1, 99_999, 999_999):
        for step in (0, 1, 79_999):
            for block in (0, 1, 2, 63, 128):
                rows.append([pack, step, block, 0, 1, 0])
    rows = np.array(rows, dtype=np.uint64)
    ref = aten_philox(rows)
    got = _oracle_blocks(orc, rows)
    assert (ref == got).all()
