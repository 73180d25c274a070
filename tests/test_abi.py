"""The C ABI library builds, loads and exports every entry point that
include/mgr_gb300.h declares (no GPU needed: nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "mgr_gb300.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mgr_setup", "mgr_apply", "fgmres_solve", "mgr_destroy"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1904_05960_gb300 import mgr
    L = mgr.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(mgr.EXPORTED) == declared_functions()


def test_loaded_library_was_built_from_the_current_sources():
    """The build id compiled into the library equals the hash of the sources
    and flags in this tree (a stale library would be rebuilt by build())."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1904_05960_gb300 import build, mgr
    assert mgr.mgr_build_id() == build.source_hash() == build.built_hash()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1904_05960_gb300 import mgr
    monkeypatch.setattr(mgr, "_lib", None)
    monkeypatch.setattr(mgr, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mgr.lib()


def test_error_strings_without_gpu():
    from paper_1904_05960_gb300 import mgr
    assert mgr.lib().mgr_error_string(-4).decode().startswith("zero pivot")
    o = mgr.mgr_options_default(True)
    assert o.num_levels == 2 and o.nmax_drop[0] == 4 and o.nmax_drop[1] == -1
    assert o.global_sweeps[1] == 3 and abs(o.amg_theta - 0.25) < 1e-15


def _header_src():
    with open(os.path.join(ROOT, "include", "mgr_gb300.h")) as f:
        return re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)


def _struct_fields(src, name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    m = re.search(r"typedef struct\s*\{((?:(?!typedef struct).)*?)\}\s*" + name + r"\s*;", src,
                  flags=re.S)
    assert m, name
    return re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*(?:\[[^\]]*\])?\s*;", m.group(1))


def test_binding_structs_and_constants_match_the_header():
    """The ctypes mirrors of the option and info structs list the header's
    fields in the header's order, and every MGR_* constant the binding
    defines has the header's value (a field added on one side only would
    shift every later field of the other)."""
    from paper_1904_05960_gb300 import mgr
    src = _header_src()
    for cname, pyname in (("mgr_options_t", "MgrOptions"), ("fgmres_options_t", "FgmresOptions"),
                          ("fgmres_info_t", "FgmresInfo"), ("mgr_matrix_t", "MgrMatrix")):
        fields = [f[0] for f in getattr(mgr, pyname)._fields_]
        assert fields == _struct_fields(src, cname), cname
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(MGR_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)}
    shared = [k for k in defines if hasattr(mgr, k)]
    assert len(shared) >= 10
    for k in shared:
        assert getattr(mgr, k) == defines[k], k
    fo = mgr.fgmres_options_default()
    assert fo.ortho == mgr.MGR_ORTHO_AUTO and fo.restart == 50
