"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every entry point include/trplk.h declares; the binding's structs
match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_1711_10128_gb300 import build
    build.build()
    from paper_1711_10128_gb300 import binding as b
    return b


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(trplk_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(binding):
    declared = declared_entry_points()
    assert "trplk_solve" in declared and len(declared) >= 12
    for name in declared:
        assert hasattr(binding.LIB, name), name


def test_binding_structs_match_header(binding):
    # field counts of the three structs, read from the header
    text = open(os.path.join(ROOT, "include", "trplk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for struct, pyname in (("trplk_csr", "trplk_csr"), ("trplk_params", "trplk_params"), ("trplk_info", "trplk_info")):
        m = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", text)
        assert m, struct
        body = m.group(1)
        decls = [d.strip() for d in body.split(";") if d.strip()]
        nfields = sum(len(d.split(",")) for d in decls)
        assert nfields == len(getattr(binding, pyname)._fields_), struct
    assert ctypes.sizeof(binding.trplk_csr) == 48
    assert binding.LIB.trplk_abi_version() == binding.ABI_VERSION == 2


def test_create_without_gpu_fails_cleanly(binding):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.TrplkError) as e:
        binding.Handle(0)
    assert e.value.code == binding.EINVAL


def test_mlp_init_starts_from_jacobi(binding):
    """Host-only initialiser: W3 = 0 and softplus(b3[c]) = 1, so the learned
    G starts at D^-1/2; He-normal hidden weights; same seed, same weights."""
    import numpy as np
    w = binding.trplk_fsai_mlp_init(7)
    p = binding.unpack_mlp(w)
    assert np.all(p["W3"] == 0) and np.all(p["b1"] == 0) and np.all(p["b2"] == 0)
    assert abs(np.logaddexp(0.0, p["b3"][3]) - 1.0) < 1e-6
    assert np.count_nonzero(p["b3"]) == 1
    assert abs(p["W1"].std() - np.sqrt(2 / 8)) < 0.1 * np.sqrt(2 / 8)
    assert abs(p["W2"].std() - np.sqrt(2 / 64)) < 0.05 * np.sqrt(2 / 64)
    assert abs(p["W2"].mean()) < 0.01
    assert np.array_equal(w, binding.trplk_fsai_mlp_init(7))
    assert not np.array_equal(w, binding.trplk_fsai_mlp_init(8))
