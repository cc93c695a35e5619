"""CPU-side checks of the library: it builds, loads and exports every declared symbol."""
import os
import re

import paper_1908_10169_gb300 as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bilu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:bilu_status|void|const char \*)\s*\**\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(B.EXPORTED)


def test_library_builds_and_exports_every_symbol():
    from paper_1908_10169_gb300 import build
    build.build()
    L = B.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_params_default_matches_paper_constants():
    p = B.bilu_params_default()
    assert p.pert_tau == 1e-2 and p.pert_rho == 1e-1  # Sec. 3.6
    assert p.perturb == 1 and p.max_block == 64 and p.precision == B.BILU_PREC_FP64


def test_no_device_gives_error_not_crash():
    import torch
    if torch.cuda.is_available():
        return
    try:
        B.bilu_create(0)
    except B.BiluError as e:
        assert e.status == B.BILU_ERR_ARG
    else:
        raise AssertionError("bilu_create succeeded without a device")
