"""The C-ABI library builds, loads and exports every symbol include/bddc.h declares.

No compute call is made (the CPU suite runs without a GPU).
"""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bddc_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2501_01676_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("bddc_setup", "bddc_apply", "bddc_gmres_solve", "bddc_schur_apply", "bddc_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    L = ct.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2501_01676_gb300 import bddc
    assert set(declared_functions()) <= set(bddc.EXPORTED)


def test_host_only_calls(libpath):
    from paper_2501_01676_gb300 import bddc
    o = bddc.default_opts()
    assert o.theta_E == 10.0 and o.tau == 0.7 and o.max_iter == 300 and o.rtol == 1e-8
    assert bddc.lib().bddc_strerror(-1).decode() == "invalid argument"
    # invalid arguments are rejected before any device work
    assert bddc.lib().bddc_setup(None, None, None, 0.0, None, None, None) == -1


def test_precision_modes_match_the_header():
    """The binding's precision constants equal the header's; the defaults are the FP64
    path, tensor-core trailing updates for the mixed path, and the small-coarse route."""
    from paper_2501_01676_gb300 import bddc
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (BDDC_PREC_\w+)\s+(\d+)", txt)}
    assert consts == {"BDDC_PREC_FP64": bddc.PREC_FP64, "BDDC_PREC_MIXED": bddc.PREC_MIXED,
                      "BDDC_PREC_BF16": bddc.PREC_BF16}
    o = bddc.default_opts()
    assert o.precision == bddc.PREC_FP64 and o.tensor_cores == 1 and o.coarse_elim == 0


def _struct_fields(txt, name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    body = re.search(r"typedef struct \{((?:(?!typedef).)*?)\}\s*" + name + r";", txt, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)              # array extents
        for part in decl.split(","):
            tok = re.findall(r"[A-Za-z_]\w*", part)
            if tok:
                names.append(tok[-1])
    return names


@pytest.mark.parametrize("cname,pyname", [("bddc_opts", "Opts"), ("bddc_stats", "Stats"),
                                          ("bddc_coeffs", "Coeffs")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes structures list the header's fields in the header's order."""
    from paper_2501_01676_gb300 import bddc
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    assert [f for f, _ in getattr(bddc, pyname)._fields_] == _struct_fields(txt, cname)


def test_edge_modes_and_new_option_defaults():
    from paper_2501_01676_gb300 import bddc
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (BDDC_EDGE_\w+)\s+(\d+)", txt)}
    assert consts == {"BDDC_EDGE_NONE": bddc.EDGE_NONE, "BDDC_EDGE_NEW": bddc.EDGE_NEW,
                      "BDDC_EDGE_OLD": bddc.EDGE_OLD}
    o = bddc.default_opts()
    assert o.edge_gep == bddc.EDGE_NEW and o.apply_launch == 0 and o.cond_est == 1


def test_element_constants_last_error_and_local_nd_default():
    """The element constants equal the header's; the defaults are Q1 bricks and the
    dense interior elimination; a rejected setup leaves its reason in
    bddc_last_error (host-only: the null arguments are refused before device work)."""
    from paper_2501_01676_gb300 import bddc
    txt = open(os.path.join(ROOT, "include", "bddc.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (BDDC_ELEM_\w+)\s+(\d+)", txt)}
    assert consts == {"BDDC_ELEM_Q1": bddc.ELEM_Q1, "BDDC_ELEM_P1": bddc.ELEM_P1}
    o = bddc.default_opts()
    assert o.element == bddc.ELEM_Q1 and o.local_nd == 0
    assert bddc.lib().bddc_setup(None, None, None, 0.0, None, None, None) == -1
    assert isinstance(bddc.lib().bddc_last_error().decode(), str)
