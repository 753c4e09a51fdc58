"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/*.h."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(mrg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("mrg_create_streams", "mrg_generate", "mrg_skip", "mrg_get_state", "mrg_set_state",
              "mrg_fused_pi_normsum", "mrg_substream_next", "mrg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2201_06604_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu():
    from paper_2201_06604_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.mrg_seed_check.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    good = (ctypes.c_uint32 * 6)(12345, 12345, 12345, 12345, 12345, 12345)
    assert lib.mrg_seed_check(good) == 0
    for bad in ([0, 0, 0, 1, 2, 3], [1, 2, 3, 0, 0, 0], [4294967087, 1, 1, 1, 1, 1],
                [1, 1, 1, 4294944443, 1, 1]):
        assert lib.mrg_seed_check((ctypes.c_uint32 * 6)(*bad)) == -1
    lib.mrg_version.restype = ctypes.c_char_p
    assert b"mrg32k3a" in lib.mrg_version()
