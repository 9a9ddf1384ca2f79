"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|size_t)\s*\*?\s*(\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ea_init_disorder", "muca_run_sweeps", "muca_update_weights", "get_histograms",
                     "get_roundtrips", "pt_run"):
        assert required in names, required


def test_library_exports_every_declared_symbol():
    from paper_2011_08560_gb300 import build
    build.build()
    lib = ctypes.CDLL(str(build.LIB))
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2011_08560_gb300 import eamc
    assert set(eamc.SIGNATURES) == _declared()


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """The binding raises instead of computing anything when the library is absent."""
    from paper_2011_08560_gb300 import eamc
    monkeypatch.setattr(eamc, "LIB", tmp_path / "missing.so")
    monkeypatch.setattr(eamc, "_lib", None)
    with pytest.raises(ImportError):
        eamc.lib()


def test_tile_width_options_per_order():
    """Host-side width queries (no GPU): the lexicographic kernel has tiles of 16 at L = 7, 8; the
    colour-order kernel has 16 at L = 4..8, 8 at L = 4..10 and 4 at L = 11, 12 (3D), and the
    autotuner tries every one of them beside full tiles (in stages when the combinations are
    many)."""
    from paper_2011_08560_gb300 import autotune, build, eamc
    build.build()
    assert eamc.narrow_widths(3, 8, 0) == [16] and eamc.narrow_widths(3, 8, 1) == [8, 16]
    assert eamc.narrow_widths(3, 6, 0) == [] and eamc.narrow_widths(3, 6, 1) == [8, 16]
    assert eamc.narrow_widths(2, 8, 1) == [] and eamc.narrow_widths(3, 3, 1) == []
    assert [eamc.narrow_width(3, L, 1) for L in range(4, 13)] == [8, 8, 8, 8, 8, 8, 8, 4, 4]
    assert autotune.width_options([(3, 8, 1024)], 0) == [{}, {"8": 16}]
    assert autotune.width_options([(3, 8, 1024)], 1) == [{}, {"8": 8}, {"8": 16}]
    assert len(autotune.width_options([(3, L, 10) for L in (4, 6, 8, 10, 12)], 1)) == 3 * 3 * 3 * 2 * 2
    assert len(autotune.width_options([(3, L, 10) for L in (4, 6, 8, 10, 12)], 0)) == 2
