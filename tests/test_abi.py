"""The C ABI library builds, loads and exports every entry point of
include/fbs.h; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1705_06284_gb300 as fbs
from paper_1705_06284_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fbs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fbs_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libfbs():
    _build.build()
    return fbs.lib()


def test_every_declared_symbol_is_exported(libfbs):
    names = _declared()
    assert "fbs_bispectrum" in names and "fbs_plan_create" in names
    for n in names:
        assert hasattr(libfbs, n), n
    # and the binding knows all of them (same names, argument marshalling only)
    bound = {s[0] for s in fbs._SIGS}
    assert set(names) == bound


def test_version_and_errors(libfbs):
    assert libfbs.fbs_version() == 100
    assert isinstance(libfbs.fbs_last_error(), bytes)
    assert len(fbs.kernel_class_names()) == libfbs.fbs_num_kernel_classes()


@pytest.mark.parametrize("N", [7, 10, 20, 1024, 4, 15])
def test_unsupported_N_rejected_on_host(libfbs, N):
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(N, 100.0, [0.1, 0.2])
    assert e.value.status == -2


def test_bad_edges_rejected_on_host(libfbs):
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(32, 100.0, [0.3, 0.2])
    assert e.value.status == -1
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(32, -1.0, [0.1, 0.2])
    assert e.value.status == -1
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(32, 100.0, [0.1, float("nan")])
    assert e.value.status == -1
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(32, 100.0, [0.1, 0.2], precision=7)
    assert e.value.status == -1


def test_null_arguments(libfbs):
    assert libfbs.fbs_bispectrum(None, None, None, None) == -1
    assert libfbs.fbs_plan_num_triplets(None) == -1
    libfbs.fbs_plan_free(None)  # no-op


def test_no_cpu_fallback_without_device(libfbs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_plan_create(16, 100.0, [0.1, 0.5, 1.0])
    assert e.value.status == -4


def test_device_budget_arguments(libfbs):
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_set_device_budget(-1)
    assert e.value.status == -1
    fbs.fbs_set_device_budget(0)
    assert fbs.fbs_device_bytes_in_use() >= 0
    assert libfbs.fbs_plan_check(None) == -1


def test_enum_values_match_the_binding():
    """Every FBS_OPT_* and FBS_PREC_* value of include/fbs.h is the binding's
    constant of the same name (the options are passed as plain ints), and the
    autotuner's options are among them."""
    txt = open(os.path.join(ROOT, "include", "fbs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    found = dict((k, int(v)) for k, v in re.findall(r"\b(FBS_(?:OPT|PREC)_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    assert "FBS_OPT_TC_STACK" in found and "FBS_OPT_TC_BSTAGES" in found
    for name, value in found.items():
        if hasattr(fbs, name):
            assert getattr(fbs, name) == value, name
    opts = {v for k, v in found.items() if k.startswith("FBS_OPT_")}
    for fbs_name in [k for k in found if k.startswith("FBS_OPT_")]:
        assert hasattr(fbs, fbs_name), fbs_name
    from paper_1705_06284_gb300 import batch
    assert {opt for _, opt, _ in batch.TUNABLE} <= opts
