"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/gp.h declares; the Python binding refuses to run without one."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> list[str]:
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not path.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", path)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(gp_\w+)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith("typedef"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gp_coarsen", "gp_contract", "gp_sparsify", "gp_partition", "gp_create",
                     "gp_destroy", "gp_partition_host", "gp_refine", "gp_initial_partition"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2504_17615_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a_only():
    from paper_2504_17615_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_defaults_match_the_paper():
    import paper_2504_17615_gb300 as gp
    c = gp.default_config()
    assert (c.tau_e_num, c.tau_e_den, c.tau_d_num, c.tau_d_den, c.rho_num, c.rho_den) == (1, 2, 1, 2, 4, 1)
    assert (c.cluster_factor, c.coarsest_factor, c.shrink_num, c.shrink_den) == (160, 160, 5, 2)
    assert c.sparsifier == gp.GP_SPARSIFY_TWEIGHT


def test_binding_fails_loudly_without_gpu():
    import torch
    import paper_2504_17615_gb300 as gp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        gp.Context(0)
    with pytest.raises(RuntimeError):
        gp.Server(0, workers=2)


def test_no_cpu_fallback_in_the_package():
    pkg = os.path.join(ROOT, "paper_2504_17615_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gp_oracle" not in text, f
