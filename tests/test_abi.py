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
          velocity=np.ones(512), box=[[8, 8, 7]]), "box"),
    (dict(dim=3, n=(8, 8, 8), h=(1, 1, 1), origin=(0, 0, 0), periodic=(0, 0, 0),
          velocity=np.ones(512), precision=F.FGA_MIXED_TF32X3), "2D"),
    (dict(eps=[-1.0]), "eps"),
    (dict(eps=[float("nan")]), "eps"),
    (dict(kappa=0.0), "kappa"),
    (dict(keep_n=-1), "keep_n"),
    (dict(z_method=2), "z_method"),
    (dict(interp=2), "interp"),
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


@pytest.mark.parametrize("shape, periodic", [((9,), (False,)), ((8,), (True,)),
                                             ((13, 11), (False, False)), ((12, 7), (True, False)),
                                             ((6, 5, 7), (False, True, False))])
def test_spline_prefilter_matches_the_oracle_and_is_symmetric(shape, periodic):
    import oracle as O

    rng = np.random.default_rng(31)
    c = 1.0 + rng.uniform(0.0, 1.0, shape)
    g = O.Grid(shape, (1.0,) * len(shape), (0.0,) * len(shape), periodic)
    got = F.spline_prefilter(c, periodic)
    np.testing.assert_allclose(got, O.interp_coefficients(g, c), rtol=0, atol=1e-12)
    # the map is symmetric (fga_grad applies it as its own adjoint)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    lhs = float(np.sum(F.spline_prefilter(x, periodic) * y))
    rhs = float(np.sum(x * F.spline_prefilter(y, periodic)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_spline_prefilter_in_place_and_errors():
    L = F.load()
    c = np.random.default_rng(32).uniform(1.0, 2.0, (10, 9))
    ref = F.spline_prefilter(c, (False, False))
    n = np.ascontiguousarray(c.shape, dtype=np.int64)
    per = np.zeros(2, dtype=np.int32)
    a = c.copy()
    assert L.fga_spline_prefilter(2, n.ctypes.data, per.ctypes.data, a.ctypes.data, a.ctypes.data) == 0
    np.testing.assert_array_equal(a, ref)
    with pytest.raises(F.FGAError) as ei:
        F.spline_prefilter(np.ones(3), (False,))
    assert ei.value.status == 1 and "grid size" in str(ei.value)
    assert L.fga_spline_prefilter(4, n.ctypes.data, per.ctypes.data, a.ctypes.data, a.ctypes.data) == 1


def test_config_layout_matches_the_header(tmp_path):
    # the ctypes mirror of fga_config must have the C compiler's offsets and size
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = [f[0] for f in F.Config._fields_]
    src = tmp_path / "layout.c"
    body = "".join('  printf("%%s %%zu\\n", "%s", offsetof(fga_config, %s));\n' % (n, n) for n in names)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "fga.h"\nint main(void) {\n'
                   + body + '  printf("sizeof %zu\\n", sizeof(fga_config));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for n in names:
        assert int(got[n]) == getattr(F.Config, n).offset, n
    assert int(got["sizeof"]) == ctypes.sizeof(F.Config)
