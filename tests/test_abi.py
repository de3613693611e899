"""The C-ABI library loads and exports every entry point include/kamd.h declares.

No compute: on a machine without a GPU only argument validation runs (it
precedes any CUDA call), and a valid md_create reports a CUDA/unsupported
error instead of crashing.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2001_07089_gb300 import build as kbuild
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "kamd.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = kbuild.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(kamd.EXPORTED) == names


def _create(**over):
    args = dict(n=100, types=np.zeros(100, np.uint8), ntypes=2, L=10.0, eps=wl.KA_EPS, sigma=wl.KA_SIG,
                rc=wl.KA_RC, mass=1.0, skin=0.3, prec=kamd.MD_PREC_MIXED)
    args.update(over)
    return kamd.md_create(args["n"], args["types"], args["ntypes"], args["L"], args["eps"], args["sigma"],
                          args["rc"], args["mass"], args["skin"], args["prec"])


@pytest.mark.parametrize("over,needle", [
    (dict(L=4.0), "L/2"),
    (dict(ntypes=5, eps=np.ones((5, 5)), sigma=np.ones((5, 5)), rc=np.ones((5, 5))), "ntypes"),
    (dict(eps=np.array([[1.0, 1.5], [1.4, 0.5]])), "symmetric"),
    (dict(sigma=np.array([[1.0, -0.8], [-0.8, 0.88]])), "> 0"),
    (dict(types=np.full(100, 3, np.uint8)), "type index"),
    (dict(mass=0.0), "mass"),
    (dict(n=1, types=np.zeros(1, np.uint8)), "n >= 2"),
    (dict(skin=-0.1), "skin"),
])
def test_invalid_arguments_rejected_before_any_cuda_call(over, needle):
    with pytest.raises(kamd.KamdError) as ei:
        _create(**over)
    assert ei.value.status == kamd.MD_ERR_INVALID_ARG
    assert needle in str(ei.value)


def test_valid_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kamd.KamdError) as ei:
        _create()
    assert ei.value.status in (kamd.MD_ERR_CUDA, kamd.MD_ERR_NOT_SUPPORTED)
