"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute call: these run without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

from paper_1505_00914_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ch_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ch_reduce", "ch_chain", "ch_hull", "ch_convex_hull", "ch_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_and_binds_without_gpu(lib_path):
    from paper_1505_00914_gb300 import ch
    lib = ch.lib()
    assert lib.ch_version() >> 16 == 1
    for name in _declared():
        assert hasattr(lib, name)
    assert ch.strerror(ch.CH_ERR_RANGE)
    assert ch.strerror(0) == "ok"


def test_objects_target_sm_103a(lib_path):
    """The build passes one -gencode, for sm_103a only."""
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_sparse_workspace_holds_the_tree_of_bit_words():
    """The persistent part of the sparse path's workspace is L (8 bytes a
    column) and the 32-bit words of every level of the w = 32 tree, each
    region rounded up to 256 bytes (no GPU needed for the size query)."""
    import oracle
    from paper_1505_00914_gb300 import ch
    r = lambda b: (b + 255) // 256 * 256
    for p in (1, 31, 32, 33, 1024, 1025, 65536, 1 << 24, (1 << 30) - 7, 1 << 30):
        expect = r(8 * p) + sum(r(4 * k) for k in oracle.tree_words(p, 32))
        assert ch.ch_sparse_workspace_size(1000, p)[1] == expect, p
        assert len(oracle.tree_words(p, 32)) <= 7


def test_product_path_never_reaches_the_oracle():
    """The package and the C ABI neither import, include nor link the CPU
    oracle (test infrastructure only), and the binding has no CPU fallback:
    it raises when libch.so cannot be loaded."""
    import ast
    pkg = os.path.join(ROOT, "paper_1505_00914_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(a.name.split(".")[0] != "oracle" for a in node.names), path
            if isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*")):
        text = open(path).read()
        assert "oracle" not in re.findall(r'#include\s*[<"]([^>"]+)', text).__str__(), path
        assert "liboracle" not in text, path


def test_binding_raises_without_the_library(tmp_path, monkeypatch):
    """No fallback: a library that cannot be loaded is an error."""
    from paper_1505_00914_gb300 import ch
    bad = tmp_path / "libch.so"
    bad.write_bytes(b"not a shared object")
    monkeypatch.setattr(ch, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(bad))
    with pytest.raises(RuntimeError, match="could not be loaded"):
        ch.lib()


def test_oracle_uses_only_the_generators_of_the_package():
    """The oracle shares no code with the CUDA path: from the package it may
    import the seeded input generators (synth) and nothing else."""
    import ast
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.ImportFrom) and (node.module or "").startswith("paper_1505_00914_gb300"):
                assert node.module == "paper_1505_00914_gb300" and [a.name for a in node.names] == ["synth"], path
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("paper_1505_00914_gb300") for a in node.names), path
    text = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert re.findall(r'#include\s*[<"]([^>"]+)', text) and "ch.h" not in text


def test_binding_rejects_host_point_arrays():
    """Device entry points refuse CPU tensors before any call into the
    library (a host pointer must never reach a kernel)."""
    import torch
    from paper_1505_00914_gb300 import ch
    host = torch.ones((4, 2), dtype=torch.int32)
    for call in (lambda: ch.ch_reduce(host, 4), lambda: ch.ch_convex_hull(host, 4),
                 lambda: ch.ch_reduce_u16(torch.zeros(4, dtype=torch.int32), 4),
                 lambda: ch.ch_hull_batched(host, None, torch.ones(1, dtype=torch.int32), None, None,
                                            None, None),
                 lambda: ch.ch_reduce_batched(host, None, torch.ones(1, dtype=torch.int32), None,
                                              None, None)):
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
    # any device argument, not only the points: the pointer helper refuses host memory
    with pytest.raises(ValueError, match="CUDA tensors"):
        ch._ptr(torch.zeros(3, dtype=torch.int32))
    assert ch._ptr(None) is None


def test_python_constants_match_the_header():
    """The binding's copies of the header's #define values agree with it."""
    from paper_1505_00914_gb300 import ch
    text = open(os.path.join(ROOT, "include", "ch.h")).read()
    defs = {m.group(1): m.group(2) for m in re.finditer(r"#define\s+(CH_[A-Z0-9_]+)\s+(.+)", text)}

    def value(expr):
        expr = re.sub(r"/\*.*?\*/", "", expr).strip()
        return eval(expr, {}, {})

    names = ["CH_CHAIN_NOALLOC_MAX_P", "CH_OK", "CH_ERR_ARG", "CH_ERR_RANGE", "CH_ERR_CAPACITY",
             "CH_ERR_TIMEOUT", "CH_ERR_CUDA", "CH_ERR_WORKSPACE", "CH_MLP_IN", "CH_MLP_HID",
             "CH_MLP_K", "CH_MLP_PARAMS", "CH_BATCH_FOLD_DEFAULT"]
    for n in names:
        if hasattr(ch, n):
            assert getattr(ch, n) == value(defs[n]), n
    assert ch.CH_CHAIN_NOALLOC_MAX_P == value(defs["CH_CHAIN_NOALLOC_MAX_P"])


def test_chain_binding_checks_array_sizes():
    """The chain bindings refuse arrays too small for p, or of the wrong type,
    before the library is called (CPU tensors fail the CUDA check first)."""
    import torch
    from paper_1505_00914_gb300 import ch
    L = torch.empty((4, 2), dtype=torch.int32)
    lo = torch.empty((4, 2), dtype=torch.int32)
    cnt = torch.empty(2, dtype=torch.int32)
    with pytest.raises(ValueError):
        ch.ch_chain_noalloc(L, 4, lo, lo, cnt)  # host tensors
    with pytest.raises(ValueError):
        ch._check_chain_args(L, 4, lo, lo, cnt, None)


def test_misaligned_workspace_is_refused_before_any_launch(lib_path):
    """A workspace that does not start on a 256-byte boundary is an argument
    error, returned before any CUDA call (the pointers are never touched, so
    no GPU is needed)."""
    import ctypes
    lib = ctypes.CDLL(lib_path)
    P = ctypes.c_void_p
    dev = P(1 << 20)              # 8-byte-aligned stand-ins for device arrays
    bad = P((1 << 21) + 16)       # 16-byte but not 256-byte aligned
    lib.ch_chain.argtypes = [P, ctypes.c_int32, P, P, P, P, P, ctypes.c_size_t, P]
    lib.ch_hull.argtypes = [P, P, P, ctypes.c_int32, P, P, P, ctypes.c_size_t, P]
    lib.ch_polyline.argtypes = [P, ctypes.c_int32, P, P, P, ctypes.c_size_t, P]
    big = 1 << 30
    assert lib.ch_chain(dev, 4096, dev, dev, dev, None, bad, big, None) == -1
    assert lib.ch_hull(dev, dev, dev, 4096, dev, dev, bad, big, None) == -1
    assert lib.ch_polyline(dev, 4096, dev, dev, bad, big, None) == -1
