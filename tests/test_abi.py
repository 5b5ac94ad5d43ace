"""The C-ABI library loads, exports every entry point include/smpc.h declares, and
rejects malformed input on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1604_01074_gb300 as smpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(smpc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(smpc.LIB_PATH):
        pytest.skip("library not built")
    return smpc.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "smpc_solve" in names and "smpc_factor" in names and "smpc_tree_create" in names
    raw = ctypes.CDLL(smpc.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
    assert set(names) <= set(smpc.SIGNATURES)


def test_status_strings(lib):
    assert smpc.smpc_status_string(smpc.SMPC_OK) == "ok"
    assert "invalid" in smpc.smpc_status_string(smpc.SMPC_EINVAL)
    assert smpc.smpc_version() >= 1


@pytest.mark.parametrize("parent,prob,msg", [
    ([0, 0, 0], None, "root"),                         # parent[0] must be -1
    ([-1, 0, 2], None, "precede"),                     # parent after child
    ([-1, 0, 0, 1, 2, 1], None, "non-decreasing"),     # children not contiguous
    ([-1, 0, 0, 1], None, "last stage"),               # leaf at a shallower stage
    ([-1, 0, 0], [1.0, 0.3, 0.3], "probability"),      # children do not add up
    ([-1, 0, 0], [1.0, 0.5, -0.5], "positive"),
    ([-1, 0, 0], [0.9, 0.45, 0.45], "root"),
    ([], None, "n_nodes"),
    ([-1, -1, 0, 1, -1], None, "precede"),              # forest: a root after the first non-root
    ([-1, -1, 0, 0, 1, 2], None, "last stage"),         # forest: tree 0 has leaves at stages 1 and 2
    ([-1, -1, 0, 1], [1.0, 0.5, 1.0, 1.0], "root"),     # forest: every root has probability 1
])
def test_tree_validation(lib, parent, prob, msg):
    with pytest.raises(smpc.SmpcError) as ei:
        smpc.smpc_tree_create(np.asarray(parent, np.int32), prob)
    assert ei.value.code == smpc.SMPC_EINVAL
    assert msg in str(ei.value)


def test_valid_tree_without_device_is_a_cuda_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(smpc.SmpcError) as ei:
        smpc.smpc_tree_create(np.asarray([-1, 0, 0], np.int32))
    assert ei.value.code == smpc.SMPC_ECUDA


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a struct in include/smpc.h has the C compiler's size and field
    offsets (a field added, dropped or reordered on one side only fails here), and the
    binding's status codes and iteration limit are the header's."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [smpc.smpc_network, smpc.smpc_cost, smpc.smpc_factor_opts, smpc.smpc_step_data,
               smpc.smpc_solve_opts, smpc.smpc_result, smpc.smpc_tree_info]
    cname = {"lambda_": "lambda"}  # Python keyword
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "smpc.h"', "int main(void) {"]
    for s in structs:
        t = s.__name__
        lines.append(f'  printf("{t} sizeof %zu\\n", sizeof({t}));')
        for name, _ in s._fields_:
            c = cname.get(name, name)
            lines.append(f'  printf("{t} {name} %zu\\n", offsetof({t}, {c}));')
    lines.append('  printf("const SMPC_MAX_ITERS %d\\n", (int)SMPC_MAX_ITERS);')
    for code in ("SMPC_OK", "SMPC_EINVAL", "SMPC_ENOMEM", "SMPC_ECUDA", "SMPC_EBUSY", "SMPC_ETIMEOUT",
                 "SMPC_EDIVERGED", "SMPC_ENOTSUP", "SMPC_FP64", "SMPC_FP32", "SMPC_BF16"):
        lines.append(f'  printf("const {code} %d\\n", (int){code});')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        t, field, val = line.split()
        got[(t, field)] = int(val)
    for (t, name), val in got.items():  # the binding's constants are the header's
        if t == "const":
            assert getattr(smpc, name) == val, name
    for s in structs:
        t = s.__name__
        assert got[(t, "sizeof")] == ctypes.sizeof(s), t
        for name, _ in s._fields_:
            assert got[(t, name)] == getattr(s, name).offset, (t, name)
