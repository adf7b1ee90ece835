"""The C-ABI library loads and exports every entry point include/fbn.h declares.

Runs without a GPU: no compute call is made, except fbn_create's refusal when
no device is present (it must fail loudly, never fall back to the CPU).
"""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fbn_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2212_04259_gb300 import build
    return build.build()


def test_header_declares_expected_calls():
    names = _declared()
    for want in ("fbn_create", "fbn_learn_skeleton", "fbn_ci_test"):
        assert want in names


def test_header_has_no_torch_types():
    for h in HEADERS:
        src = open(h).read()
        assert "torch" not in src.lower() and "at::" not in src and "Tensor" not in src


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (fbn_[a-z0-9_]+)", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declared_symbol(built):
    import paper_2212_04259_gb300 as f
    lib = f.lib()
    for name in _declared():
        assert name in f.EXPORTS
        assert hasattr(lib, name)


def test_create_rejects_bad_arguments_before_touching_a_device(built):
    import paper_2212_04259_gb300 as f
    with pytest.raises(f.FbnError) as e:
        f.fbn_create(np.zeros((1, 10), np.uint8), [2])       # n_vars < 2
    assert e.value.code == -1
    with pytest.raises(f.FbnError) as e:
        f.fbn_create(np.zeros((2, 10), np.uint8), [2, 1])    # arity < 2
    assert e.value.code == -1
    with pytest.raises(f.FbnError) as e:                     # the depth-1 tensor path takes arities <= 8
        f.fbn_create(np.zeros((2, 10), np.uint8), [2, 9], depth1="tensor")
    assert e.value.code == -1 and "arities <= 8" in str(e.value)
    with pytest.raises(f.FbnError) as e:
        f.fbn_create(np.zeros((2, 10), np.uint8), [2, 2], depth0="gram", form="pool", group_threads=48)
    assert e.value.code == -1
    o = f.fbn.Options(device=-1, loop=2)                     # neither loop driver
    out = f.fbn.C.c_void_p()
    data = np.zeros((2, 10), np.uint8)
    ar = np.array([2, 2], np.uint8)
    rc = f.fbn.lib().fbn_create(f.fbn._ptr(data), 2, 10, f.fbn._ptr(ar), f.fbn.C.byref(o), f.fbn.C.byref(out))
    assert rc == -1 and "bad loop" in f.fbn_last_error(None)
    o = f.fbn.Options(device=-1, count=3)                    # no such counting strategy
    rc = f.fbn.lib().fbn_create(f.fbn._ptr(data), 2, 10, f.fbn._ptr(ar), f.fbn.C.byref(o), f.fbn.C.byref(out))
    assert rc == -1 and "bad count" in f.fbn_last_error(None)


def test_no_cpu_fallback_without_gpu(built):
    import torch
    import paper_2212_04259_gb300 as f
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(f.FbnError) as e:
        f.fbn_create(np.zeros((3, 10), np.uint8), [2, 2, 2])
    assert e.value.code == -4
