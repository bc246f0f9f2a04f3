"""The C-ABI library builds, loads and exports every symbol include/tensorctl.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tensorctl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tctl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tctl_setup", "tctl_apply_op", "tctl_apply_precond", "tctl_pcg_solve",
                     "tctl_truncate", "tctl_fullgrid_solve", "tctl_destroy", "tctl_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2006_09314_gb300 import tensorctl as T
    lib = T.load(build_if_missing=True)
    missing = [s for s in _declared() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(T.EXPORTED) <= set(_declared())


def test_default_opts_and_error_paths_without_gpu():
    from paper_2006_09314_gb300 import tensorctl as T
    o = T.tctl_default_opts()
    assert o.pcg_rtol == 1e-7 and o.max_iter == 100 and o.basis == 1 and o.r_pre == 24
    assert o.range_tol == 0.03 and o.seed == 1
    lib = T.load()
    # argument validation happens before any device work
    import ctypes
    import numpy as np
    ctx = ctypes.c_void_p()
    coeffs = np.ones((3, 9))
    assert lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, 8, 1.5, 1e-2, 1e-6, None, None) == -1
    assert lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, 1, 0.5, 1e-2, 1e-6, None, None) == -1
    coeffs[2, 4] = 0.0
    assert lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, 8, 0.5, 1e-2, 1e-6, None, None) == -2
    assert "positive" in T.tctl_last_error(None)
    coeffs[2, 4] = 1.0
    bad = T.tctl_default_opts(range_tol=2.0)
    assert lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, 8, 0.5, 1e-2, 1e-6,
                          ctypes.byref(bad), None) == -1
    assert "range_tol" in T.tctl_last_error(None)
    for bad in (T.tctl_default_opts(tc_digits=5), T.tctl_default_opts(refine=9),
                T.tctl_default_opts(refine=-1)):
        assert lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, 8, 0.5, 1e-2, 1e-6,
                              ctypes.byref(bad), None) == -1
    assert "refine" in T.tctl_last_error(None)
    o = T.tctl_default_opts()
    assert o.tc_digits == 6 and o.refine == 0
    # the GEMM entry points refuse a missing context before touching the device
    assert lib.tctl_gemm(None, 6, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == -1
    assert lib.tctl_gemm_kr(None, 6, 4, 2, 2, 4, 1.0, None, 4, None, 4, None, 4, 0.0, None, 4) == -1


def test_inputs_generator_is_seeded():
    import numpy as np
    from paper_2006_09314_gb300.inputs import make_problem
    a = make_problem(16, 0.5, 1e-2, 3, 5)
    b = make_problem(16, 0.5, 1e-2, 3, 5)
    assert np.array_equal(a.coeffs, b.coeffs) and all(np.array_equal(x, y) for x, y in zip(a.yU, b.yU))
    assert a.coeffs.min() >= 0.5 - 1e-15 and a.coeffs.max() <= 1.5 + 1e-15


def test_uneven_batch_generator():
    """The uneven batch: seeded, n from the choices, design rank 1..8,
    alpha in [0.2, 0.8], log10 beta in [-4, 0]."""
    import numpy as np
    from paper_2006_09314_gb300.inputs import batch_problems
    a = batch_problems(40, 11)
    b = batch_problems(40, 11)
    assert [p.n for p in a] == [p.n for p in b]
    assert all(np.array_equal(x.coeffs, y.coeffs) for x, y in zip(a, b))
    assert {p.n for p in a} <= set(range(64, 513, 32)) and len({p.n for p in a}) > 5
    assert all(1 <= len(p.yw) <= 8 for p in a)
    assert all(0.2 <= p.alpha <= 0.8 and 1e-4 <= p.beta <= 1.0 for p in a)
    assert batch_problems(3, 12)[0].n != a[0].n or not np.array_equal(batch_problems(3, 12)[0].coeffs,
                                                                       a[0].coeffs)


def test_map_constants_without_gpu():
    """(beta_p, gamma) of Section 3.1 -> beta = gamma / beta_p^2, u_paper = u / beta_p."""
    from paper_2006_09314_gb300 import tensorctl as T
    b, sc = T.tctl_map_constants(2.0, 0.5)
    assert b == 0.125 and sc == 0.5
    b, sc = T.tctl_map_constants(1.0, 1e-2)
    assert b == 1e-2 and sc == 1.0
    import pytest
    with pytest.raises(T.TctlError):
        T.tctl_map_constants(0.0, 1.0)
