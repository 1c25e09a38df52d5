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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes records of the binding have the C layout of include/gp.h (sizes and the offsets
    of the fields the batched form and the partition statistics hand back)."""
    import shutil
    import subprocess
    import paper_2504_17615_gb300 as gp
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    checks = {
        "gp_graph": ["n", "m2", "adjwgt"],
        "gp_config": ["tau_e_num", "small_lp_nodes"],
        "gp_level_stats": ["m_hat", "threshold", "clusters_final"],
        "gp_partition_stats": ["lv", "U", "n_coarsest", "ms_total"],
        "gp_batch_item": ["g", "eps", "blocks", "cut", "status", "engine", "stats"],
        "gp_batch_tuning": ["threads", "max_entries", "arena_bytes", "class_entries", "class_items",
                            "class_threads", "class_engine_gps", "class_path_gps", "tune_ms"],
        "gp_request": ["n", "k", "blocks"],
        "gp_response": ["status", "estimate_bytes", "peak_used_bytes"],
    }
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gp.h"', "int main(void) {"]
    for s, fields in checks.items():
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'  printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    c = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, fields in checks.items():
        t = getattr(gp, s)
        assert int(c[s]) == ctypes.sizeof(t), s
        for f in fields:
            assert int(c[f"{s}.{f}"]) == getattr(t, f).offset, f"{s}.{f}"
