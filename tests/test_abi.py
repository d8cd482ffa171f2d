"""The C ABI library loads and exports every entry point its header declares.

No call here launches GPU work: only argument checks that return before
any CUDA call are exercised.
"""
import ctypes
import os
import re

import pytest

from paper_2609_37058_b300 import rgf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rgf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2609_37058_b300 import build
    build.build()
    return rgf.lib()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("rgf_plan_create", "rgf_set_device_blocks", "rgf_set_leads", "rgf_transmission",
              "rgf_submit", "rgf_poll", "rgf_plan_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    for n in declared_functions():
        assert hasattr(L, n), n
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_defaults_and_version(L):
    o = rgf.rgf_options_default()
    assert o.precision == rgf.RGF_FP64 and o.eta == 1e-6 and o.dec_tol == 1e-14
    assert o.dec_max_iter == 100 and o.ns_steps == 6 and o.energy_wave == 0
    assert "sm_103a" in rgf.rgf_version()


def test_invalid_arguments_fail_before_cuda(L):
    h = ctypes.c_void_p()
    assert L.rgf_plan_create(ctypes.byref(h), 0, 8, None, None) == rgf.RGF_E_INVALID
    assert "n_layers" in rgf.rgf_last_error()
    assert L.rgf_plan_create(ctypes.byref(h), 4, 0, None, None) == rgf.RGF_E_INVALID
    assert L.rgf_plan_create(ctypes.byref(h), 4, 1024, None, None) == rgf.RGF_E_INVALID
    o = rgf.rgf_options_default()
    o.precision = 7
    assert L.rgf_plan_create(ctypes.byref(h), 4, 8, ctypes.byref(o), None) == rgf.RGF_E_INVALID
    o = rgf.rgf_options_default()
    o.dec_max_iter = 0
    assert L.rgf_plan_create(ctypes.byref(h), 4, 8, ctypes.byref(o), None) == rgf.RGF_E_INVALID
    assert L.rgf_transmission(None, None, 0, None, None, None, 0) == rgf.RGF_E_INVALID
    assert L.rgf_set_leads(None, 0, None, None, None, None, None, None, 0) == rgf.RGF_E_INVALID
    assert L.rgf_poll(ctypes.c_uint64(123456789), None, None, None, 0) == rgf.RGF_E_INVALID
    assert L.rgf_plan_destroy(None) == rgf.RGF_OK


def test_server_defaults_and_invalid_arguments(L):
    o = rgf.rgf_server_options_default()
    assert (o.slots, o.class_step, o.capacity_bytes, o.ns_steps, o.dec_max_iter) == (148, 32, 0, 6, 100)
    assert o.dec_tol == 1e-14
    t = ctypes.c_uint64()
    req = rgf.rgf_request()
    assert L.rgf_server_submit(None, ctypes.byref(req), ctypes.byref(t)) == rgf.RGF_E_INVALID
    assert L.rgf_server_create(None, None) == rgf.RGF_E_INVALID
    bad = rgf.rgf_server_options_default()
    bad.slots = 0
    h = ctypes.c_void_p()
    assert L.rgf_server_create(ctypes.byref(h), ctypes.byref(bad)) == rgf.RGF_E_INVALID
    assert L.rgf_server_poll(None, 1, None, None, None, None, 0) == rgf.RGF_E_INVALID
    assert L.rgf_server_destroy(None) == rgf.RGF_OK


def test_library_has_no_unresolved_internal_symbols(L):
    # Every symbol of the library's own namespace must be defined in it.
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--undefined-only", rgf.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    bad = [ln for ln in out.splitlines() if "rgf" in ln]
    assert not bad, bad
