"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/msmg.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as pkg
    return pkg.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "msmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msmg_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    assert "msmg_setup" in names and "msmg_solve" in names and len(names) >= 10


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_2403_19342_gb300 as pkg
    assert sorted(pkg.exported_symbols()) == declared_functions()


def test_status_strings_and_validation(lib):
    import paper_2403_19342_gb300 as pkg
    assert lib.msmg_status_string(-2).decode().startswith("element sizes")
    # validation runs on the host without a device
    g = pkg.make_grid((8, 8, 8))
    o = pkg.Options(n_levels=3, block=(3, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4]).to_c()
    with pytest.raises(pkg.MsmgError) as e:
        pkg.msmg_workspace_size(g, o)
    assert e.value.status == -2
    o = pkg.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4]).to_c()
    with pytest.raises(pkg.MsmgError) as e:          # E_2 would be one element
        pkg.msmg_workspace_size(g, o)
    assert e.value.status == -4
    o = pkg.Options(n_levels=3, block=(2, 2, 2), ratio=[(2, 2, 2)], n_eig=[9, 4]).to_c()
    with pytest.raises(pkg.MsmgError) as e:          # more eigenvectors than cells
        pkg.msmg_workspace_size(g, o)
    assert e.value.status == -1
    o = pkg.Options(n_levels=3, block=(2, 2, 2), ratio=[(2, 2, 2)], n_eig=[4, 4]).to_c()
    assert pkg.msmg_workspace_size(g, o) > 8 * 512 * 10


def test_new_entry_points_reject_bad_arguments_on_the_host(lib):
    # every check below returns before any device work, so it runs without a GPU
    import paper_2403_19342_gb300 as pkg
    bad = -1                                               # MSMG_ERR_INVALID_ARG
    dummy = ctypes.c_void_p(256)                           # non-null, never dereferenced
    out = ctypes.c_double()
    assert lib.msmg_velocity(None, dummy, dummy, dummy, ctypes.byref(out), None) == bad
    ok_fluid = pkg.msmg_fluid(0.3, 3.0, 0.2, 0.2)
    # empty problem, missing fluid, residual saturations summing to one, non-positive viscosity
    assert lib.msmg_impes_pressure_terms(0, ctypes.byref(ok_fluid), dummy, dummy, dummy, dummy, 4000.0,
                                         dummy, dummy, dummy, None) == bad
    assert lib.msmg_impes_pressure_terms(8, None, dummy, dummy, dummy, dummy, 4000.0, dummy, dummy, dummy,
                                         None) == bad
    for f in (pkg.msmg_fluid(0.3, 3.0, 0.5, 0.5), pkg.msmg_fluid(0.0, 3.0, 0.2, 0.2)):
        assert lib.msmg_impes_pressure_terms(8, ctypes.byref(f), dummy, dummy, dummy, dummy, 4000.0, dummy,
                                             dummy, dummy, None) == bad
    # transport: no context, negative sub-step count, non-positive saturation step
    assert lib.msmg_impes_transport(None, ctypes.byref(ok_fluid), dummy, dummy, dummy, 4000.0, dummy, dummy,
                                    dummy, 1, 1e-3, ctypes.byref(out), None) == bad
    assert lib.msmg_impes_transport(dummy, ctypes.byref(ok_fluid), dummy, dummy, dummy, 4000.0, dummy, dummy,
                                    dummy, -1, 1e-3, ctypes.byref(out), None) == bad
    assert lib.msmg_impes_transport(dummy, ctypes.byref(ok_fluid), dummy, dummy, dummy, 4000.0, dummy, dummy,
                                    dummy, 1, 0.0, ctypes.byref(out), None) == bad
    ms = (ctypes.c_double * 3)()
    assert lib.msmg_net_forward(None, dummy, dummy, 4, None) == bad
    assert lib.msmg_net_time_products(None, dummy, 4, ms, None) == bad
