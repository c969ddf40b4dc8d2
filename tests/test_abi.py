"""The C-ABI library builds, loads and exports every entry point that
include/sgm.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sgm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["sgm_create", "sgm_destroy", "sgm_graph_load_csr", "sgm_graph_free", "sgm_query_register",
                 "sgm_query_set_order", "sgm_query_order_greedy", "sgm_count", "sgm_enumerate",
                 "sgm_count_root_range", "sgm_filter", "sgm_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2604_10601_gb300 import sgm
    lib = ctypes.CDLL(sgm.library_path() if os.path.exists(sgm.library_path()) else sgm.lib()._name)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared entry points
    assert sorted(sgm.declared_symbols()) == _declared()


def test_host_only_calls_work_without_gpu():
    from paper_2604_10601_gb300 import sgm
    o = sgm.sgm_opts_default()
    assert o.struct_size == ctypes.sizeof(sgm.sgm_opts)
    assert o.tau == 10 ** 6 and o.use_filter == 1
    assert o.exec_model == sgm.SGM_EXEC_FINE_BATCH and o.unroll == 1  # the fine-grained batched model
    assert isinstance(sgm.sgm_last_error(), str)


def test_options_are_checked_by_name():
    from paper_2604_10601_gb300 import sgm
    o = sgm.Engine.opts(None, refine_rounds=3, split_min=64)
    assert o.refine_rounds == 3 and o.split_min == 64 and o.struct_size == ctypes.sizeof(sgm.sgm_opts)
    assert sgm.sgm_opts_default().refine_rounds == 0  # refinement is off by default
    for bad in ("refine_round", "reserved", "struct_size"):
        with pytest.raises(TypeError):
            sgm.Engine.opts(None, **{bad: 1})


@pytest.mark.parametrize("struct", ["sgm_opts", "sgm_stats", "sgm_graph_stats"])
def test_struct_layouts_match_the_header(struct, tmp_path):
    """Every field of the binding's ctypes structures sits at the offset
    the C compiler gives it in include/sgm.h, with the same total size."""
    import subprocess
    from paper_2604_10601_gb300 import sgm
    cls = getattr(sgm, struct)
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {name}));' for name, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"sgm.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, name).offset for name, _ in cls._fields_]
    assert got == want


def _header_prototypes():
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sgm.h")).read(), flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(sgm_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        ret, name, args = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        protos[name] = (ret, [] if args in ("", "void") else [a.strip() for a in args.split(",")])
    return protos


def _ctype_of(decl):
    if "*" in decl:
        return ctypes.c_void_p
    words = decl.replace("const", "").split()
    base = words[0] if len(words) == 1 or words[0] not in ("unsigned", "signed") else " ".join(words[:2])
    return {"int32_t": ctypes.c_int32, "sgm_status": ctypes.c_int32, "int64_t": ctypes.c_int64,
            "uint32_t": ctypes.c_uint32, "uint64_t": ctypes.c_uint64, "double": ctypes.c_double,
            "float": ctypes.c_float}[base]


def test_binding_signatures_match_the_header():
    """Each entry point's ctypes argument and return types agree with its C
    prototype (pointers as void pointers)."""
    from paper_2604_10601_gb300 import sgm
    protos = _header_prototypes()
    assert sorted(protos) == sorted(sgm._SIGS)
    for name, (ret, args) in protos.items():
        res, argtypes = sgm._SIGS[name]
        want_ret = None if ret == "void" else (ctypes.c_char_p if ret == "const char*" or ret == "const char *"
                                               else _ctype_of(ret))
        assert res == want_ret, (name, ret)
        assert [_ctype_of(a) for a in args] == list(argtypes), (name, args)


def test_binding_constants_match_the_header():
    """Status codes, flags, modes and sizes: the binding's values are the header's."""
    from paper_2604_10601_gb300 import sgm
    src = open(os.path.join(ROOT, "include", "sgm.h")).read()
    defs = {}
    for name, val in re.findall(r"#define\s+(SGM_[A-Z0-9_]+)\s+([^/\n]+)", src):
        val = val.strip()
        if name == "SGM_H" or not val:
            continue
        parts = val.replace("(", "").replace(")", "").replace("u", "").split("<<")
        defs[name] = int(parts[0]) << (int(parts[1]) if len(parts) > 1 else 0)
    checked = [n for n in defs if hasattr(sgm, n)]
    assert len(checked) >= 26, checked
    for n in checked:
        assert getattr(sgm, n) == defs[n], n
    # every status code of the header has a name in the binding
    for n, v in defs.items():
        if n.startswith(("SGM_E_", "SGM_W_")) or n == "SGM_OK":
            assert sgm.STATUS_NAMES[v] == n
