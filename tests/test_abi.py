"""The C-ABI library builds, loads and exports every entry point its header declares (CPU only:
no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^SPC_API[^(]*?\b(spc_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2204_11757_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("spc_context_create", "spc_coarsen", "spc_coarsen_batched", "spc_score",
                 "spc_sort_fitness", "spc_select_merges", "spc_contract",
                 "spc_contract_backward", "spc_status_string", "spc_context_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (spc_\w+)", out))
    assert _declared() <= exported, _declared() - exported
    # nothing but the ABI is exported
    assert exported == _declared()


def test_binding_covers_header_and_loads(built):
    from paper_2204_11757_gb300 import native as N
    assert set(N.SIGNATURES) == _declared()
    L = N.lib()
    for name in _declared():
        assert getattr(L, name) is not None
    # pure host functions are safe without a GPU
    assert L.spc_status_string(-2) == b"SPC_ERR_NOT_SYMMETRIC"
    o = L.spc_default_options()
    assert (o.levels, o.validate, o.use_graph, o.schedule) == (1, 1, 1, 0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2204_11757_gb300 import native as N
    monkeypatch.setattr(N, "_lib", None)
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        N.lib()


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2204_11757_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower() or f == "inputs.py", f


def _close(s, i):
    """Index just past the parenthesis that closes the one at s[i]."""
    depth = 0
    while True:
        depth += {"(": 1, ")": -1}.get(s[i], 0)
        i += 1
        if depth == 0:
            return i


def _kernels():
    """(file, name, body) of every __global__ function defined in the library's sources."""
    csrc = os.path.join(ROOT, "paper_2204_11757_gb300", "csrc")
    out = []
    for f in sorted(os.listdir(csrc)):
        if not f.endswith((".cu", ".cuh")):
            continue
        s = open(os.path.join(csrc, f)).read()
        for mm in re.finditer(r"__global__\s+void\b", s):
            rest = s[mm.end():].lstrip()
            if rest.startswith("__launch_bounds__"):  # skip the attribute and its arguments
                rest = rest[_close(rest, rest.index("(")):].lstrip()
            name = re.match(r"(\w+)\s*\(", rest).group(1)
            i = _close(rest, rest.index("("))  # past the parameter list
            body_start = rest.index("{", i)
            assert ";" not in rest[i:body_start], (f, name)  # a definition, not a declaration
            out.append((f, name, rest[body_start + 1:]))
    return out


def test_every_kernel_waits_for_its_predecessor_first():
    """Kernels are launched with programmatic stream serialization: each may start while the
    kernel before it on the stream is still running, so before its first memory access each
    must wait for it (spc::pdl_wait()).  Only compile-time statements may precede the wait."""
    ks = _kernels()
    assert len(ks) > 100
    for f, name, body in ks:
        for stmt in body.split(";"):
            st = stmt.strip()
            if st.startswith(("static_assert", "constexpr")):
                continue
            assert re.fullmatch(r"(spc::)?pdl_wait\(\)", st), (f, name, st[:80])
            break
