"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every entry point its header declares."""
import os
import re

from paper_1908_03565_gb300 import binding
from paper_1908_03565_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(jxl_recon_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib_path = B.build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert {"jxl_recon_create", "jxl_recon_submit", "jxl_recon_poll",
            "jxl_recon_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) == names


def test_filter_defaults_without_gpu():
    """jxl_recon_filter_defaults is pure host code: C.10 / L.2 defaults."""
    B.build()
    p = binding.filter_defaults()
    assert p.epf == 0 and p.gab == 0
    assert abs(p.epf_scale[0] - 899.676941) < 1e-3 and p.epf_sigma_max == 170
    assert abs(p.gab_w1[1] - 0.115169525) < 1e-7 and abs(p.epf_sharp_lut[7] - 1.0) < 1e-7
    assert p.target_nits_div50 == 5 and abs(p.inv_opsin[0] - 2542.568359375) < 1e-3
