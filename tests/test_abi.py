"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = ""
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        with open(h) as f:
            src += f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2503_12749_gb300 import buildlib
    return buildlib.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gbs_make_network", "gbs_sample", "gbs_binned_counts", "gbs_free_network",
                     "gbs_last_error", "gbs_debug_samples", "gbs_mlp_create", "gbs_mlp_train",
                     "gbs_mlp_gradients", "gbs_surrogate_encode", "gbs_surrogate_decode"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (gbs_[a-z0-9_]+)\b", out.stdout))
    assert set(_declared()) <= exported


def test_binding_mirrors_abi_names():
    import paper_2503_12749_gb300 as g
    for name in _declared():
        assert hasattr(g, name), name


def test_last_error_is_callable_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gbs_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.gbs_last_error(), bytes)
    # argument validation runs before any device call
    lib.gbs_make_network.restype = ctypes.c_int
    out = ctypes.c_void_p()
    code = lib.gbs_make_network(0, 0, None, None, 0, None, ctypes.byref(out))
    assert code == -1


def _prototypes():
    """{name: parameter count} of every function include/*.h declares."""
    src = ""
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        with open(h) as f:
            src += f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for name, params in re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", src):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(libpath):
    """Every argtypes list the binding sets has as many entries as the C
    prototype has parameters (a changed signature must change both)."""
    import paper_2503_12749_gb300 as g
    L = g.lib()
    protos = _prototypes()
    assert set(protos) == set(_declared())
    checked = 0
    for name, n in protos.items():
        argtypes = getattr(L, name).argtypes
        if argtypes is None:
            continue
        assert len(argtypes) == n, (name, len(argtypes), n)
        checked += 1
    assert checked >= 40


def test_binding_constants_match_the_header():
    """Status codes, precisions and sizes: every numeric #define of
    include/*.h that the binding also names has the same value there."""
    import paper_2503_12749_gb300 as g
    src = ""
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        with open(h) as f:
            src += f.read()
    defs = {k: int(v) for k, v in
            re.findall(r"^#define\s+(GBS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src, flags=re.M)}
    shared = [k for k in defs if hasattr(g, k)]
    for k in shared:
        assert getattr(g, k) == defs[k], (k, getattr(g, k), defs[k])
    for k in ("GBS_OK", "GBS_EINVAL", "GBS_ETIMEOUT", "GBS_FP64", "GBS_FP32", "GBS_BF16X3",
              "GBS_BF16X6", "GBS_NPHASES", "GBS_SUR_OUT"):
        assert k in shared, k
    assert g.PRECISIONS == {"fp64": defs["GBS_FP64"], "fp32": defs["GBS_FP32"],
                            "bf16x3": defs["GBS_BF16X3"], "bf16x6": defs["GBS_BF16X6"]}
