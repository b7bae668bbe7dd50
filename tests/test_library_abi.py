"""CPU checks of the C ABI: the library builds, loads and exports every
function include/dgmg.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os

import pytest

from paper_1805_11930_gb300 import build, dgmg


def _lib_or_skip():
    if not build.up_to_date():
        try:
            build.build()
        except RuntimeError as e:       # no nvcc in this environment
            pytest.skip(str(e))
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = dgmg.exported_symbols()
    for required in ("dgmg_create", "dgmg_destroy", "dgmg_set_mesh", "dgmg_set_coefficients",
                     "dgmg_assemble_rhs", "dgmg_apply", "dgmg_block_apply", "dgmg_block_smooth",
                     "dgmg_restrict", "dgmg_prolong_add", "dgmg_coarse_cycle", "dgmg_vcycle",
                     "dgmg_solve", "dgmg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib_or_skip()
    for name in dgmg.exported_symbols():
        assert hasattr(lib, name), name
    assert set(dgmg.exported_symbols()) == set(dgmg._SIG), "binding and header disagree"


def test_default_opts_without_gpu():
    _lib_or_skip()
    o = dgmg.default_opts()
    assert o.rtol == 1e-8 and o.restart == 30 and o.eps_inner == 1e-2 and o.npre == 1 and o.npost == 1


def test_create_fails_cleanly_without_device():
    lib = dgmg.load()
    h = ctypes.c_void_p()
    st = lib.dgmg_create(ctypes.byref(h), 10_000, None)
    assert st == 1 and not h.value


def _header_struct(name):
    """(type, field) pairs of `typedef struct {...} name;` in include/dgmg.h."""
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "dgmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    out = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z_ ]*?)\s+([A-Za-z_][A-Za-z0-9_]*(?:\s*,\s*[A-Za-z_][A-Za-z0-9_]*)*)\s*;",
                         body):
        out += [(" ".join(m.group(1).split()), n.strip()) for n in m.group(2).split(",")]
    return out


@pytest.mark.parametrize("cname, pyname", [("dgmg_solve_opts", "SolveOpts"), ("dgmg_solve_stats", "SolveStats")])
def test_binding_structs_match_header(cname, pyname):
    """The ctypes mirrors of the option and statistics structs list the
    header's fields in the same order with the same C types."""
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong}
    fields = getattr(dgmg, pyname)._fields_
    decl = _header_struct(cname)
    assert [n for n, _ in fields] == [n for _, n in decl]
    for (n, t), (ct, _) in zip(fields, decl):
        assert t is ctype[ct], n


def test_null_context_is_an_argument_error():
    lib = dgmg.load()
    assert lib.dgmg_set_penalty(None, 2.0) == 1
    assert lib.dgmg_destroy(None) == 1


def test_every_declaration_is_documented():
    """Each function the header declares sits under a comment block (a pair
    of declarations may share one), so its argument layout, ownership and
    errors are stated where the boundary is defined."""
    import re
    lines = open(os.path.join(os.path.dirname(__file__), "..", "include", "dgmg.h")).read().splitlines()
    for i, line in enumerate(lines):
        m = re.match(r"^(?:dgmg_status|const char\*|void)\s+(dgmg_[a-z0-9_]+)\(", line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
            j -= 1                      # continuation lines of the neighbouring declaration
        assert j >= 0 and lines[j].rstrip().endswith("*/"), m.group(1)


def _header_prototypes():
    """{name: (return type, [parameter types])} of the functions the header declares."""
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "dgmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"(dgmg_status|const char\s*\*|void)\s+(dgmg_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = []
        for prm in m.group(3).split(","):
            prm = " ".join(prm.split())
            if prm in ("", "void"):
                continue
            prm = re.sub(r"\s*\[\d*\]$", "*", re.sub(r"\s+[A-Za-z_][A-Za-z0-9_]*(\s*\[\d*\])?$",
                                                   lambda q: "*" if q.group(1) else "", prm))
            params.append(prm.replace(" *", "*"))
        out[m.group(2)] = (" ".join(m.group(1).split()), params)
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes signature in the binding has the header's arity and, per
    argument, a ctypes type of the same kind (pointer, int/enum, double,
    long long pointer), so no argument is passed with the wrong width."""
    protos = _header_prototypes()
    assert set(protos) == set(dgmg._SIG)
    ints = {"int", "dgmg_prec", "dgmg_status"}
    for name, (res, args) in dgmg._SIG.items():
        ret, params = protos[name]
        assert len(params) == len(args), name
        if ret == "dgmg_status":
            assert res is ctypes.c_int, name
        elif ret == "void":
            assert res is None, name
        else:
            assert res is ctypes.c_char_p, name
        for c, a in zip(params, args):
            base = c.replace("const ", "")
            if base.endswith("*"):
                assert a is ctypes.c_void_p or issubclass(a, ctypes._Pointer), (name, c)
                if base == "long long*":
                    assert a._type_ is ctypes.c_longlong, (name, c)
                if base == "int*" and a is not ctypes.c_void_p:
                    assert a._type_ is ctypes.c_int, (name, c)
            elif base in ints:
                assert a is ctypes.c_int, (name, c)
            elif base == "double":
                assert a is ctypes.c_double, (name, c)
            else:
                raise AssertionError((name, c))


def test_binding_fails_loudly_without_the_library_or_a_gpu_tensor(monkeypatch, tmp_path):
    """No CPU fallback: a missing library raises instead of computing
    anything, and host tensors are refused where device pointers are due."""
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(dgmg, "_lib", None)
    monkeypatch.setattr(dgmg._build, "LIB", str(tmp_path / "missing" / "libdgmg.so"))
    with pytest.raises(dgmg.DgmgError):
        dgmg.load(build_if_missing=False)
    with pytest.raises(dgmg.DgmgError, match="CUDA tensor"):
        dgmg._ptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(dgmg.DgmgError, match="dtype"):
        dgmg._prec(torch.zeros(4, dtype=torch.int32))
