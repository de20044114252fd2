"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/*.h; the Python binding names the same
set."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mucite_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2609_31258_b300 import build, mucite
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(mucite.EXPORTS) == declared


def test_state_layout_without_gpu():
    from paper_2609_31258_b300 import mucite
    for prec, pb in ((mucite.FP32, 4), (mucite.FP64, 8)):
        L = mucite.state_layout(prec, 1000)
        offs = [L.off_x, L.off_y, L.off_z, L.off_vx, L.off_vy, L.off_vz, L.off_eint, L.off_status, L.off_t_term,
                L.off_lnsy, L.off_tau]
        assert all(o % 256 == 0 for o in offs)
        assert offs == sorted(offs) and L.pos_bytes == pb
        assert L.total_bytes >= offs[-1] + 1000 * pb
        # arrays do not overlap: each gap holds its array (status 1 byte, t_term 4)
        sizes = [pb] * 7 + [1, 4, pb, pb]
        assert all(offs[i] + 1000 * sizes[i] <= offs[i + 1] for i in range(len(offs) - 1))


def test_binding_fails_loudly_without_device():
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2609_31258_b300 import mucite
    with pytest.raises(RuntimeError):
        mucite.Context(0)
