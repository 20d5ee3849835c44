"""The C ABI of libsve on the CPU (no GPU, no compute): the library builds for
sm_103a, loads, exports every symbol include/sve.h declares, and its host-side
argument checks answer without touching a device."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1307_0491_gb300 import build as B
from paper_1307_0491_gb300 import sve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sve.load()


def declared_functions() -> set[str]:
    text = open(os.path.join(ROOT, "include", "sve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(sve_\w+)\s*\(", text))


def test_header_matches_binding():
    assert declared_functions() == set(sve.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_config_struct_layout(lib):
    c = sve.sve_config()
    assert sve.sve_config_default(c) == 0
    assert c.g == 9.81 and c.cfl == 0.9 and c.kappa_a == 1.1 and c.beta_min == 0.01 and c.gamma_z == 2.0
    assert c.newton_maxit == 30 and c.newton_tol == 1e-9 and c.m_g == 3.0
    assert list(c.bc) == [sve.SVE_BC_PERIODIC, sve.SVE_BC_PERIODIC, sve.SVE_BC_FREE, sve.SVE_BC_FREE]


@pytest.mark.parametrize("field,value", [("dim", 3), ("nx", 0), ("cfl", -1.0), ("kappa_a", 1.0), ("m_g", 5.0),
                                         ("precision", 7), ("newton_maxit", 0)])
def test_invalid_config_rejected_on_host(lib, field, value):
    c = sve.sve_config()
    sve.sve_config_default(c)
    c.nx, c.ny = 8, 4
    setattr(c, field, value)
    rc, h = sve.sve_create(c)
    assert rc == sve.SVE_ERR_ARG and not h.value


def test_mismatched_periodic_rejected(lib):
    c = sve.sve_config()
    sve.sve_config_default(c)
    c.nx, c.ny = 8, 4
    c.bc = (ctypes.c_int * 4)(sve.SVE_BC_PERIODIC, sve.SVE_BC_FREE, sve.SVE_BC_FREE, sve.SVE_BC_FREE)
    rc, _ = sve.sve_create(c)
    assert rc == sve.SVE_ERR_ARG


def test_mpm_needs_friction(lib):
    c = sve.sve_config()
    sve.sve_config_default(c)
    c.nx, c.ny = 8, 4
    c.bedload = sve.SVE_MPM
    rc, _ = sve.sve_create(c)
    assert rc == sve.SVE_ERR_ARG


def test_null_handles(lib):
    assert lib.sve_step(None, 1, None) == sve.SVE_ERR_ARG
    assert lib.sve_get_state(None, None, None, None, None, 0) == sve.SVE_ERR_ARG
    assert lib.sve_set_stream(None, None) == sve.SVE_ERR_ARG
    lib.sve_destroy(None)


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert sve.sve_strerror(code)
    assert sve.sve_strerror(-99) == "unknown error"


def test_config_mapping_from_workload(lib):
    from paper_1307_0491_gb300 import workloads as W

    w = W.antidune2d(nx=16, ny=8)
    c = sve.config_from_params(w["params"], "fp32")
    assert c.bedload == sve.SVE_MPM and c.friction == sve.SVE_FRIC_DARCY and c.precision == sve.SVE_FP32
    assert list(c.bc) == [sve.SVE_BC_INFLOW_QH, sve.SVE_BC_FREE, sve.SVE_BC_FREE, sve.SVE_BC_FREE]
    assert c.h_in == 0.5 and c.f_dw == 0.02 and c.nx == 16 and c.ny == 8


def test_null_handle_checks_of_later_calls(lib):
    """The host-to-host call, the persistent-step switch, its bounded-wait
    check and the recording query answer SVE_ERR_ARG for a NULL handle on
    the host, before any device call."""
    null = ctypes.c_void_p(None)
    z = [None, None, None, None]
    rc, _ = sve.sve_advance(null, 1, z, z, sve.SVE_HOST)
    assert rc == sve.SVE_ERR_ARG
    assert lib.sve_set_persistent(null, 1) == sve.SVE_ERR_ARG
    assert lib.sve_get_persistent(null) == sve.SVE_ERR_ARG
    assert lib.sve_check_sync_timeout(null, 100) == sve.SVE_ERR_ARG
    assert lib.sve_get_checkpoint_every(null) == sve.SVE_ERR_ARG
    assert lib.sve_set_adjoint_budget(null, 0) == sve.SVE_ERR_ARG
    assert lib.sve_get_adjoint_kept_steps(null) == sve.SVE_ERR_ARG
    assert lib.sve_set_scheme(null, sve.SVE_SCHEME_SPLIT) == sve.SVE_ERR_ARG
    assert lib.sve_get_scheme(null) == sve.SVE_ERR_ARG
    assert lib.sve_set_history(null, 4) == sve.SVE_ERR_ARG
    assert lib.sve_get_history(null, None, 0) == sve.SVE_ERR_ARG
    rc, _, _, _ = sve.sve_get_safeguards(null)
    assert rc == sve.SVE_ERR_ARG
    assert lib.sve_block_get_edge(null, 0, None, sve.SVE_HOST) == sve.SVE_ERR_ARG
    assert lib.sve_block_set_ghosts(null, 0, None, sve.SVE_HOST) == sve.SVE_ERR_ARG
    rc, _, _ = sve.sve_block_speeds(null)
    assert rc == sve.SVE_ERR_ARG
    assert lib.sve_block_advance(null, 1.0, 1.0) == sve.SVE_ERR_ARG
    assert lib.sve_batch_autotune_trials(null, 0, None, None, None, None) == sve.SVE_ERR_ARG
    assert lib.sve_batch_set_rows(null, 32) == sve.SVE_ERR_ARG
    assert lib.sve_batch_get_rows(null) == sve.SVE_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libsve.so the binding raises instead of
    computing anything."""
    monkeypatch.setattr(sve, "_LIB", None)
    monkeypatch.setattr(sve, "lib_path", lambda: str(tmp_path / "libsve.so"))
    with pytest.raises(RuntimeError, match="libsve.so not found"):
        sve.load()
