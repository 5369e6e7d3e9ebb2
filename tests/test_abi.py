"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("cc_graph_create", "cc_graph_destroy", "cc_cluster", "cc_cluster_ex", "cc_disagreements",
              "cc_permutation", "cc_batch_run", "cc_status_string"):
        assert f in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1507_05086_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, f"libcc.so lacks {missing}"


def test_status_strings_without_gpu():
    from paper_1507_05086_gb300 import native
    lib = native.load()
    for code, text in native.STATUS.items():
        assert lib.cc_status_string(code).decode() == text


def test_graph_create_rejects_unknown_flags_without_gpu():
    """Argument checks of cc_graph_create come before any device work: an
    unknown flag bit (or a negative n) is CC_ERR_INVALID_ARG on any machine,
    and CC_VALIDATE is a known bit."""
    import ctypes
    import numpy as np
    from paper_1507_05086_gb300 import native
    lib = native.load()
    flags = dict((k, int(v, 16) if v.startswith("0x") else int(v))
                 for k, v in re.findall(r"#define\s+CC_(VALIDATE|DEVICE_PTRS|OFFSETS_I32|VALIDATE_EXACT)\s+(\w+?)u",
                                        open(HEADER).read()))
    assert flags == {"VALIDATE": 1, "DEVICE_PTRS": 2, "OFFSETS_I32": 4, "VALIDATE_EXACT": 8}
    off = np.zeros(2, np.int64)
    h = ctypes.c_void_p()
    p = off.ctypes.data_as(ctypes.c_void_p)
    assert lib.cc_graph_create(ctypes.c_int64(1), p, None, ctypes.c_uint32(16), None, ctypes.byref(h)) == -1
    assert lib.cc_graph_create(ctypes.c_int64(-1), p, None, ctypes.c_uint32(1), None, ctypes.byref(h)) == -1
    assert not h.value


def test_binding_matches_header_stats_layout():
    from paper_1507_05086_gb300 import native
    text = open(HEADER).read()
    body = text[text.index("typedef struct cc_round_stats"):text.index("} cc_round_stats;")]
    fields = re.findall(r"int64_t\s+(\w+);", body)
    assert tuple(fields) == native.ROUND_STAT_FIELDS


def test_binding_matches_header_algorithm_ids():
    from paper_1507_05086_gb300 import native
    ids = dict((k, int(v)) for k, v in re.findall(r"#define\s+CC_ALGO_(\w+)\s+(\d+)", open(HEADER).read()))
    assert ids == {"C4": native.C4, "CLUSTERWILD": native.CLUSTERWILD, "C4_EST": native.C4_EST,
                   "CLUSTERWILD_EST": native.CLUSTERWILD_EST, "C4_ASYNC": native.C4_ASYNC}
    assert native.ALGOS["c4-async"] == native.C4_ASYNC


def test_product_and_oracle_are_independent():
    """The oracle never imports the CUDA package and the package never
    imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1507_05086_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f), errors="replace").read()
                assert "oracle" not in re.sub(r"(#|//).*", "", src).lower(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1507_05086_gb300" not in src and "graphgen" not in src


def test_cuda_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1507_05086_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        native.load(build_if_missing=False)
