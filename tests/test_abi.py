"""The C ABI library loads, exports every entry point include/fga.h declares, and
rejects bad configurations on the host (no GPU needed for any of this)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(fga_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = F.load()
    names = declared_functions()
    assert "fga_plan" in names and "fga_reconstruct" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = F.load()
    for code in range(8):
        assert lib.fga_status_string(code)
    assert lib.fga_status_string(1) == b"invalid argument"


def _plan(**kw):
    args = dict(dim=2, n=(16, 16), h=(0.1, 0.1), origin=(0.0, 0.0), periodic=(False, False),
                velocity=np.ones(256), eps=[0.01], T=1.0, dt=0.1, kappa=6.0, tau=1e-3)
    args.update(kw)
    return F.Plan(**args)


@pytest.mark.parametrize("kw, msg", [
    (dict(dt=0.3), "T/dt"),
    (dict(dim=0, n=(), h=(), origin=(), periodic=(), velocity=np.ones(1)), "dim"),
    (dict(dim=3, n=(8, 8, 8), h=(1, 1, 1), origin=(0, 0, 0), periodic=(0, 0, 0),
          velocity=np.ones(512), box=[[66, 8, 8]]), "3D"),
    (dict(dim=3, n=(8, 8, 8), h=(1, 1, 1), origin=(0, 0, 0), periodic=(0, 0, 0),
          velocity=np.ones(512), precision=F.FGA_MIXED_TF32X3), "2D"),
    (dict(eps=[-1.0]), "eps"),
    (dict(eps=[float("nan")]), "eps"),
    (dict(kappa=0.0), "kappa"),
    (dict(keep_n=-1), "keep_n"),
    (dict(z_method=2), "z_method"),
    (dict(z_method=F.FGA_Z_DIVIDED), "dz_eta"),
    (dict(z_method=F.FGA_Z_DIVIDED, dz_eta=1.0), "dz_eta"),
    (dict(z_method=F.FGA_Z_DIVIDED, dz_eta=float("nan")), "dz_eta"),
    (dict(dim=3, n=(8, 8, 8), h=(1, 1, 1), origin=(0, 0, 0), periodic=(0, 0, 0),
          velocity=np.ones(512), z_method=F.FGA_Z_DIVIDED, dz_eta=0.5), "1D and 2D"),
    (dict(tau=-1.0), "tau"),
    (dict(h=(0.0, 0.1)), "spacing"),
    (dict(n=(2, 16), velocity=np.ones(32)), "grid size"),
    (dict(box=[[7, 8]]), "box"),
    (dict(periodic=(True, False), box=[[8, 32]], q_stride=[[2, 2]]), "periodic"),
    (dict(precision=F.FGA_MIXED_BF16X3), "precision"),
    (dict(precision=F.FGA_MIXED_TF32X3, periodic=(True, False), box=[[16, 32]], q_stride=[[2, 2]]),
     "open"),
    (dict(precision=F.FGA_MIXED_TF32X3, dim=1, n=(16,), h=(0.1,), origin=(0.0,), periodic=(False,),
          velocity=np.ones(16)), "2D"),
])
def test_invalid_configurations_are_rejected_on_the_host(kw, msg):
    with pytest.raises(F.FGAError) as ei:
        _plan(**kw)
    assert ei.value.status == 1  # FGA_ERR_INVALID
    assert msg in str(ei.value)


def test_null_arguments():
    lib = F.load()
    out = ctypes.c_void_p()
    assert lib.fga_plan(None, None, None, ctypes.byref(out)) == 1
    assert lib.fga_plan(None, None, None, None) == 1
    assert lib.fga_destroy(None) == 0
    assert lib.fga_count(None, 0) == -1
    assert lib.fga_decompose(None, None, None, None) == 1


def test_wrong_dtype_and_size_rejected_in_binding():
    with pytest.raises(TypeError):
        _plan(velocity=np.ones(256, dtype=np.float32))
    with pytest.raises(ValueError):
        _plan(velocity=np.ones(255))


def test_grid_receivers_cover_the_grid_inside_its_bounds():
    import math

    from paper_1304_3542_gb300 import autograd as FA
    from paper_1304_3542_gb300 import workloads as WL

    prob = WL.lens_2d(N=64, eps=1.0 / 400, T=0.1, dt=2e-3, s=2, box=32, tau=1e-2, kappa=8.0,
                      k0=24 * math.pi, width2=0.004)
    xr = FA.grid_receivers(prob)
    assert xr.shape == (64 * 64, 2) and xr.flags["C_CONTIGUOUS"]
    for k in range(2):
        hi = prob.origin[k] + (prob.n[k] - 1) * prob.h[k]
        assert xr[:, k].min() == prob.origin[k]
        assert hi - 4 * np.spacing(hi) <= xr[:, k].max() < hi
    # C order: the last axis runs fastest
    assert xr[1, 1] - xr[0, 1] == prob.h[1] and xr[1, 0] == xr[0, 0]
