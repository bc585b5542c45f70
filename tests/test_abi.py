"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function declared in include/swdg.h (no compute call is made here, except
by the gpu-marked probe test at the end)."""
import ctypes
import os
import re
import pytest

from paper_2505_18743_gb300 import build as B
from paper_2505_18743_gb300 import swdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "swdg.h")).read()
    return sorted(set(re.findall(r"\b(swdg_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib_path = B.build()
    assert os.path.exists(lib_path)
    lib = ctypes.CDLL(lib_path)
    names = declared()
    assert "swdg_step" in names and "swdg_residual" in names
    for name in names:
        assert hasattr(lib, name), name
    # the binding covers the same names
    assert set(names) <= set(swdg.SIGNATURES)


def test_invalid_config_is_rejected_without_touching_the_gpu():
    lib = swdg.load()
    cfg = swdg.swdg_config(7, 0, 0, 0, 9.81, 0.01, 0.01, 1e-6, 0.1, 20, 1e-12, None)
    h = ctypes.c_void_p()
    assert lib.swdg_create(ctypes.byref(cfg), ctypes.byref(h)) == swdg.SWDG_EINVAL
    assert not h.value


@pytest.mark.gpu
def test_fma_probe_measures_the_pipes():
    """swdg_probe_fma: FP64 and FP32 FMA-chain rates of the device, positive
    and in the order the hardware fixes (FP32 well above FP64)"""
    import torch
    assert torch.cuda.is_available()
    B.build()
    f64, ms64 = swdg.probe_fma(swdg.SWDG_PIX_F64)
    f32, ms32 = swdg.probe_fma(swdg.SWDG_PIX_F32)
    assert f64 > 0.1 and ms64 > 0.0 and f32 > 10 * f64
    with pytest.raises(swdg.SwdgError):
        swdg.probe_fma(7)


def test_noalloc_refuses_an_empty_mesh_before_any_device_call():
    """swdg_residual_noalloc checks its sizes before it touches a pointer or
    the device: n = 0 (and n above its scratch) come back SWDG_EINVAL"""
    cfg = swdg.swdg_config(1, 0, 0, 0, 9.81, 0.01, 0.01, 1e-6, 0.1, 20, 1e-12, None)
    for n in (0, -1, 1048577):
        with pytest.raises(swdg.SwdgError) as e:
            swdg.residual_noalloc(cfg, n, None, None, None, 8, swdg.SWDG_PIX_F64, None, None, 0.0,
                                  None, None)
        assert e.value.code == swdg.SWDG_EINVAL and "n_cells" in str(e.value)


@pytest.mark.gpu
def test_manning_root_within_a_few_ulp():
    """the kernels' own z = h^(-1/3) (FP32 seed, two Newton-Raphson steps for
    z^-3 = h) against the exact root, and z^3 against 1/h, over depths from
    1e-9 m to 1e5 m and beyond the FP32 range (the 1/cbrt branch)"""
    import numpy as np
    import torch
    assert torch.cuda.is_available()
    B.build()
    rng = np.random.default_rng(11)
    h = np.concatenate([np.logspace(-9, 5, 40001), rng.uniform(1e-3, 50.0, 20000),
                        [1e-35, 3e-31, 7e30, 1e35, 1.0, 8.0, 27.0]])
    z, r = swdg.probe_roots(h)
    # exact checks in rational arithmetic (a libm cbrt can itself be a few ulp
    # off): z within 2 ulp brackets the root, (z -+ 2 ulp)^3 h <= 1 <= ...,
    # and z^3 is within 6 ulp of 1/h
    from fractions import Fraction as Fr
    for hi, zi, ri in zip(h.tolist(), z.tolist(), r.tolist()):
        hf, du = Fr(hi), 2 * np.spacing(zi)
        assert Fr(zi - du) ** 3 * hf <= 1 <= Fr(zi + du) ** 3 * hf, (hi, zi)
        assert abs(Fr(ri) - 1 / hf) <= 6 * Fr(float(np.spacing(1.0 / hi))), (hi, ri)
    with pytest.raises(swdg.SwdgError):
        swdg.probe_roots(np.zeros(0))
