"""The C-ABI library builds, loads and exports every entry point include/dtt.h declares
(no GPU needed: nothing is computed)."""
import os
import re
import subprocess


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    """Entry points declared by one header of include/ (all headers when None)."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)) if header is None else [header]:
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(dtt_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dtt_grid_create", "dtt_set_material", "dtt_set_constraints", "dtt_set_indenter",
                 "dtt_solve_step", "dtt_get_fields", "dtt_get_reactions", "dtt_get_contact",
                 "dtt_apply_green", "dtt_apply_residual", "dtt_transform"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2607_26082_b300 import build, dtt
    build.build()
    L = dtt.lib()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", dtt.LIB_PATH], capture_output=True, text=True).stdout
    for name in _declared():
        assert re.search(r"\bT %s\b" % name, out), name
    assert dtt.version().startswith("libdtt")


def test_binding_names_match_header():
    from paper_2607_26082_b300 import dtt, net
    assert sorted(dtt.EXPORTS) == _declared("dtt.h")
    assert sorted(net.EXPORTS) == _declared("dtt_net.h")


def test_package_import_is_lazy():
    import importlib
    import paper_2607_26082_b300
    importlib.reload(paper_2607_26082_b300)
    assert "dtt" in paper_2607_26082_b300.__all__
