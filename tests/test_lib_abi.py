"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/nnc.h declares.  No device work is done here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nnc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_build_and_exports():
    from paper_2509_22462_gb300 import build as b
    lib_path = b.build()
    assert os.path.exists(lib_path)
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "nnc_hessian_lag" in names and "nnc_load_weights" in names
    for name in names:
        assert hasattr(lib, name), name
    from paper_2509_22462_gb300 import nnc
    assert sorted(nnc.EXPORTS) == sorted(names)


def test_ipm_option_defaults_match_oracle():
    """The C driver's defaults are the constants of the oracle's reading of Eq. 2."""
    from paper_2509_22462_gb300 import nnc
    from oracle import ipm
    o = nnc.ipm_options()
    ref = ipm.Options()
    for name, _ in nnc.IpmOptions._fields_:
        if name in ("verbose", "kkt_on_device"):    # not part of the method: output, placement
            continue
        assert getattr(o, name) == getattr(ref, name), name
    assert o.kkt_on_device == 0


def test_status_codes_match_header():
    src = open(os.path.join(ROOT, "include", "nnc.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"(NNC_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    from paper_2509_22462_gb300 import nnc
    for code, name in nnc.STATUS.items():
        assert codes[name] == code
    assert codes["NNC_FP64"] == nnc.FP64 and codes["NNC_BF16X3"] == nnc.BF16X3
    assert codes["NNC_TANH"] == nnc.ACTS["tanh"] and codes["NNC_GELU"] == nnc.ACTS["gelu"]


def test_argument_errors_need_no_device():
    from paper_2509_22462_gb300 import nnc
    lib = nnc.load_library()
    h = ctypes.c_void_p()
    # n_layers = 0 is rejected before any CUDA call
    assert lib.nnc_load_weights(ctypes.byref(h), 0, None, None, None, None, 0, None) == -1
    assert b"bad layer" in lib.nnc_last_error()
    assert lib.nnc_eval(None, None, None, 0) == -1


@pytest.mark.skipif(os.environ.get("NNC_HAS_GPU") == "1", reason="GPU present")
def test_no_device_fails_loudly():
    """Without a GPU, building a net returns NNC_ERR_CUDA: there is no CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    from paper_2509_22462_gb300 import nnc
    with pytest.raises(nnc.NNCError) as e:
        nnc.Net([2, 2], ["tanh"], [np.eye(2)], precision="fp64")
    assert e.value.code == -2
