"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol declared in include/bie.h, and rejects invalid input before touching a
GPU.  No compute call is made."""
import os
import re

import numpy as np
import pytest

from paper_1912_04501_gb300 import _build, bie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return bie.library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bie_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(bie.exported_symbols()) == names


def test_default_opts(lib):
    o = bie.bie_default_opts()
    assert o.precision == bie.BIE_MIXED and o.n_proxy == 48 and o.n_coll == 24
    assert o.gmres_tol == 1e-10 and o.lam_rel == 1e-8
    # bit-reproducible by default: the fixed tile shape, direct launches, no preconditioner
    assert o.autotune == 0 and o.graph == 0 and o.precond == 0
    assert o.close_capacity == 0 and o.residual == bie.BIE_DF64
    assert o.n_images == 9
    assert o.close_rule == 0


@pytest.mark.parametrize("mutate", [
    lambda c: c["bodies"][0].update(n=7),
    lambda c: c["bodies"][0].update(n=4),
    lambda c: c["bodies"][0].update(a=-0.1),
    lambda c: c.update(e2=[2.0, 0.0]),
    lambda c: c.update(mu=0.0),
    lambda c: c.update(gamma=float("nan")),
    lambda c: c["bodies"][0].update(n=16386),
    lambda c: c["bodies"][0].update(xc=[float("inf"), 0.5]),
    lambda c: c.update(bodies=[]),
])
def test_invalid_input_rejected_without_gpu(lib, mutate):
    from paper_1912_04501_gb300 import workloads
    cell = workloads.config1()
    mutate(cell)
    with pytest.raises(bie.BieError) as e:
        bie.Context(cell)
    assert e.value.code == bie.BIE_EINVAL


def test_null_arguments(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.bie_init(ctypes.byref(h), None, 1.0, 1.0, 1, None, None) == bie.BIE_EINVAL
    assert lib.bie_apply(None, None, None, 0, 0) == bie.BIE_EINVAL
    assert lib.bie_size(None, None, None) == bie.BIE_EINVAL


@pytest.mark.parametrize("opt", [dict(n_proxy=2), dict(n_proxy=300), dict(n_coll=1), dict(gmres_max=0),
                                 dict(gmres_max=5000), dict(warm_start=4), dict(residual=1),
                                 dict(close_factor=-1.0), dict(precision=3), dict(gmres_tol=0.0),
                                 dict(autotune=2), dict(graph=-1), dict(precond=2), dict(n_images=5),
                                 dict(n_images=4, n_proxy=50), dict(n_images=4, autotune=1), dict(close_rule=2)])
def test_invalid_options_rejected_without_gpu(lib, opt):
    from paper_1912_04501_gb300 import workloads
    with pytest.raises(bie.BieError) as e:
        bie.Context(workloads.config1(), **{k: v for k, v in opt.items() if k != "precision"},
                    **({"precision": opt["precision"]} if "precision" in opt else {}))
    assert e.value.code == bie.BIE_EINVAL


def test_invalid_batches_rejected_without_gpu(lib):
    from paper_1912_04501_gb300 import workloads
    good = workloads.config1()
    empty = dict(good, bodies=[])
    with pytest.raises(bie.BieError) as e:
        bie.Context([good, empty])
    assert e.value.code == bie.BIE_EINVAL
    import ctypes
    h = ctypes.c_void_p()
    assert lib.bie_init_batch(ctypes.byref(h), 0, None, None, None) == bie.BIE_EINVAL
    assert lib.bie_init_batch(ctypes.byref(h), 5000, None, None, None) == bie.BIE_EINVAL


def test_network_arguments_rejected_without_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.bie_net_init(ctypes.byref(h), 0, 0) == bie.BIE_EINVAL
    assert lib.bie_net_init(ctypes.byref(h), 17, 0) == bie.BIE_EINVAL
    assert lib.bie_net_forward(None, None, 0, None) == bie.BIE_EINVAL
    assert lib.bie_features(None, None, 0) == bie.BIE_EINVAL


def test_precond_needs_single_cell_without_gpu(lib):
    from paper_1912_04501_gb300 import workloads
    with pytest.raises(bie.BieError) as e:
        bie.Context([workloads.config1(), workloads.config1()], precond=1)
    assert e.value.code == bie.BIE_EINVAL


def test_unknown_option_is_an_error(lib):
    from paper_1912_04501_gb300 import workloads
    with pytest.raises(TypeError):
        bie.Context(workloads.config1(), precnod=1)
