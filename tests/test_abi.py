"""The C-ABI library builds, loads and exports every declared entry point.
CPU only: no compute call is made (there is no GPU here)."""
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    text = (ROOT / "include" / "sympix.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sympix_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_04653_gb300._build import build_library
    build_library()
    from paper_1504_04653_gb300 import sympix
    return sympix.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_1504_04653_gb300 import sympix
    bound = {s[0] for s in sympix.SIGNATURES}
    assert set(_declared()) == bound


def test_argument_errors_need_no_device(lib):
    import ctypes
    from paper_1504_04653_gb300 import sympix as S
    h = ctypes.c_void_p()
    assert lib.sympix_grid(0, 1, 0, -1.0, ctypes.byref(h)) == S.EINVAL
    assert b"lmax" in lib.sympix_last_error()
    assert lib.sympix_grid(64, 2, S.LAYOUT_GREEDY, -1.0, ctypes.byref(h)) == S.EINVAL
    assert lib.sympix_grid(64, 1, 7, -1.0, ctypes.byref(h)) == S.EINVAL
    assert lib.sympix_support(None, 1, None, 0, 1, ctypes.byref(h)) == S.EINVAL
    assert lib.sympix_sample_blocks(None, None, 0, 0, None, None) == S.EINVAL
    assert lib.sympix_factor_blocks(None, 0, 0, None, None, None) == S.EINVAL
    assert lib.sympix_version().startswith(b"sympix")


def test_no_device_fails_loudly(lib):
    """Without a usable GPU the grid call reports an error instead of computing
    anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1504_04653_gb300 import sympix as S
    with pytest.raises(S.SympixError):
        S.Grid(16)


def test_package_does_not_import_oracle():
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle|#include.*oracle)", re.M)
    for f in (ROOT / "paper_1504_04653_gb300").rglob("*"):
        if f.suffix in (".py", ".cu", ".cuh", ".h"):
            assert not pat.search(f.read_text()), f
