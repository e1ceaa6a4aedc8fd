"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/rt.h (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    return sorted(set(re.findall(r"RT_API\s+[\w\s\*]+?\b(rt_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for n in ["rt_create", "rt_inverse", "rt_propagator", "rt_step", "rt_observables", "rt_destroy"]:
        assert n in names


def test_library_builds_loads_and_exports_every_symbol():
    import paper_1404_5776_gb300 as rt
    path = rt.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rt.EXPORTED) == set(declared_symbols())


def test_default_params_without_gpu():
    import paper_1404_5776_gb300 as rt
    p = rt.rt_default_params()
    assert p.taylor_terms == 6 and p.prop == rt.RT_PROP_EM and p.dt == 0.05
    assert p.r_U == 8.0 and p.precision == rt.RT_FP64


def test_library_has_no_cpu_fallback_symbols():
    """The product library contains no host implementation of the products:
    its only exported names are the C ABI."""
    import subprocess
    import paper_1404_5776_gb300 as rt
    out = subprocess.run(["nm", "-D", "--defined-only", rt.build()], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(declared_symbols())
