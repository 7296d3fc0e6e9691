"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: this runs without a GPU); the binding's launch-shape cache
file."""
import ctypes
import os
import re

import pytest

from paper_2102_00514_gb300 import build, pes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(pes_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pes_linearize", "pes_filter_scan", "pes_smooth_scan", "pes_ieks_run", "pes_init_forward",
                     "pes_init_train_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build_cuda()
    lib = ctypes.CDLL(pes.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(pes.EXPORTED) == declared_symbols()


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        pes.Smoother(16)


def test_tuning_cache_file(tmp_path):
    """The launch-shape cache of Smoother.autotune: keys by GPU, method,
    precision and size class (N and B rounded up to powers of two); an absent
    file is an empty cache; an update keeps the other entries."""
    k = pes.tune_cache_key("GPU X", pes.CUBATURE, pes.FP32, 1048577, 1)
    assert k == "GPU X|cubature|fp32|N<=2097152|B<=1"
    assert pes.tune_cache_key("GPU X", pes.CUBATURE, pes.REFINED, 1 << 20, 3) == "GPU X|cubature|fp32|N<=1048576|B<=4"
    assert pes.tune_cache_key("GPU X", pes.IEKS, pes.FP64, 1000, 4096).endswith("|ieks|fp64|N<=1024|B<=4096")
    path = str(tmp_path / "tune.json")
    assert pes.read_tune_cache(path) == {}
    pes.update_tune_cache(path, k, {"threads": 256, "min_steps": 4, "ms_per_run": 0.5})
    pes.update_tune_cache(path, "other", {"threads": 128, "min_steps": 8, "ms_per_run": 0.7})
    pes.update_tune_cache(path, k, {"threads": 128, "min_steps": 16, "ms_per_run": 0.4})
    data = pes.read_tune_cache(path)
    assert data == {k: {"threads": 128, "min_steps": 16, "ms_per_run": 0.4},
                    "other": {"threads": 128, "min_steps": 8, "ms_per_run": 0.7}}
