"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/gs.h declares (no GPU needed: nothing is called)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "gs.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    from paper_2412_00578_gb300 import build, raster

    lib_path = build.build()
    lib = ctypes.CDLL(str(lib_path))
    names = declared_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(raster.EXPORTS) == set(names)


def test_frame_sizes_without_gpu():
    from paper_2412_00578_gb300 import raster

    sz = raster.frame_sizes(1000, 320, 240, 16, 5000)
    assert sz.proj == 3 * 1000 * 16 and sz.keys == 2 * 5000 * 8 and sz.vals == 2 * 5000 * 4
    assert sz.ranges == 20 * 15 * 8 and sz.image == 3 * 320 * 240 * 4
    import pytest

    for bad in [(1000, 320, 240, 12, 10), (1000, 0, 240, 16, 10), (1000, 320, 240, 16, 1 << 31)]:
        with pytest.raises(raster.GsError):
            raster.frame_sizes(*bad)


def test_missing_library_fails_loudly(tmp_path):
    """Without the compiled library the binding raises: there is no CPU path
    to fall back on."""
    import pytest

    from paper_2412_00578_gb300 import raster

    with pytest.raises(RuntimeError, match="no CPU fallback"):
        raster.load(tmp_path / "libgs.so")
