"""The C-ABI library builds, loads and exports every function include/lbnlm.h declares; argument
validation that happens before any CUDA call is exercised on the CPU."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_7450_gb300 import build, lbnlm
    build.build()
    return lbnlm.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbnlm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["lb_create", "lb_step", "lb_get_fields", "lb_residual", "lb_destroy"]:
        assert want in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror(lib):
    from paper_1310_7450_gb300 import lbnlm
    assert lbnlm.lb_strerror(lbnlm.LB_OK) == "ok"
    assert "unstable" in lbnlm.lb_strerror(lbnlm.LB_EUNSTABLE)


@pytest.mark.parametrize("bad", [
    dict(ny=2), dict(nx=0), dict(tau_lb=0.5), dict(tau_lb=float("nan")), dict(gamma_c=0.0),
    dict(rho0=0.0), dict(rho_pert_amp=1.0), dict(G_inf=-1.0), dict(precision=7), dict(stress_mode=3),
])
def test_invalid_arguments_rejected_before_any_device_work(lib, bad):
    from paper_1310_7450_gb300 import lbnlm
    p = dict(tau_lb=0.9, g_x=1e-6, G_inf=1e-3, tau0=1.0, theta=10.0, gamma_c=0.1, rho0=1.0)
    kw = dict(nx=4, ny=16, precision=0, stress_mode=0)
    for k, v in bad.items():
        if k in kw:
            kw[k] = v
        else:
            p[k] = v
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_create(kw["nx"], kw["ny"], p, kw["precision"], kw["stress_mode"])
    assert e.value.status == lbnlm.LB_EINVAL
    assert lbnlm.lb_last_error()


def test_null_handle_calls_fail_cleanly(lib):
    from paper_1310_7450_gb300 import lbnlm
    assert lib.lb_step(None, 1) == lbnlm.LB_EINVAL
    assert lib.lb_step_count(None) == -1
    assert lib.lb_num_nodes(None) == 0
    lib.lb_destroy(None)


@pytest.mark.parametrize("bnd", [dict(x_mode=0), dict(x_mode=3), dict(walls=0), dict(walls=5)])
def test_invalid_boundary_rejected_before_any_device_work(lib, bnd):
    from paper_1310_7450_gb300 import lbnlm
    p = dict(tau_lb=0.9, g_x=1e-6, G_inf=1e-3, tau0=1.0, theta=10.0, gamma_c=0.1, rho0=1.0)
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_create(4, 16, p, 0, 0, **bnd)
    assert e.value.status == lbnlm.LB_EINVAL


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built library every call raises."""
    from paper_1310_7450_gb300 import lbnlm
    monkeypatch.setattr(lbnlm, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "liblbnlm.so"))
    monkeypatch.setattr(lbnlm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        lbnlm.load()
    with pytest.raises(RuntimeError, match="not built"):
        lbnlm.lb_strerror(0)


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_gpu_present(), reason="checks the behaviour on a machine without a GPU")
def test_no_cpu_fallback_without_a_gpu(lib):
    """A valid configuration on a machine without a usable GPU fails with LB_ECUDA and a message;
    nothing is computed on the host."""
    from paper_1310_7450_gb300 import lbnlm
    p = dict(tau_lb=0.9, g_x=1e-6, G_inf=1e-3, tau0=1.0, theta=10.0, gamma_c=0.1, rho0=1.0)
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_create(4, 16, p, 0, 0)
    assert e.value.status == lbnlm.LB_ECUDA
    assert "lb_create" in lbnlm.lb_last_error()


def test_wait_limit_validation_before_device_work(lib):
    """lb_set_wait_limit rejects a null handle before touching the device."""
    from paper_1310_7450_gb300 import lbnlm
    assert lib.lb_set_wait_limit(None, 1.0) == lbnlm.LB_EINVAL


def test_monitor_mode_validation_before_device_work(lib):
    from paper_1310_7450_gb300 import lbnlm
    assert lib.lb_set_monitor_mode(None, lbnlm.LB_MONITOR_FLUX_MAX) == lbnlm.LB_EINVAL


@pytest.mark.parametrize("flags,stress_mode,x_mode,walls", [
    (16 | 32, 0, 1, 1),   # both comparison schemes
    (16, 1, 1, 1),        # generalized Newtonian with the time-stepped stress
    (32, 0, 2, 1),        # stress divergence with pressure-driven ends
    (16, 0, 1, 2),        # generalized Newtonian with a moving wall
])
def test_comparison_scheme_combinations_rejected_before_device_work(lib, flags, stress_mode, x_mode, walls):
    from paper_1310_7450_gb300 import lbnlm
    p = dict(tau_lb=0.9, g_x=1e-6, G_inf=1e-3, tau0=1.0, theta=10.0, gamma_c=0.1, rho0=1.0)
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_create(4, 16, p, 0, stress_mode, flags, None, x_mode, walls)
    assert e.value.status == lbnlm.LB_EINVAL
    assert "scheme" in lbnlm.lb_last_error()


@pytest.mark.parametrize("flags,precision", [(16 | 64, 0), (32 | 64, 1), (64, 3), (64, 4)])
def test_relaxation_model_combinations_rejected_before_device_work(lib, flags, precision):
    """LB_GRID_RELAXATION_MODEL with a comparison scheme, or with a mixed diagnostic precision."""
    from paper_1310_7450_gb300 import lbnlm
    p = dict(tau_lb=0.9, g_x=1e-6, G_inf=1e-3, tau0=1.0, theta=10.0, gamma_c=0.1, rho0=1.0)
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_create(4, 16, p, precision, 0, flags)
    assert e.value.status == lbnlm.LB_EINVAL
