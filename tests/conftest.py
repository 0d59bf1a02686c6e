import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only oracle runs")


def oracle_suspension(cell):
    """Oracle Suspension from a workload dict."""
    from oracle import geometry
    return geometry.Suspension(cell["e1"], cell["e2"], cell["centre"], cell["mu"], cell["gamma"],
                               cell["bodies"])


def oracle_operator(cell, **kw):
    from oracle import bie
    sv = cell["solver"]
    args = dict(n_proxy=sv["n_proxy"], proxy_radius=sv["proxy_radius"], n_coll=sv["n_coll"])
    args.update(kw)
    return bie.Operator(oracle_suspension(cell), **args)
