"""CPU checks of the C ABI: the library loads, exports every symbol that
include/hyb.h declares, and validates descriptors on the host (no GPU call)."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hyb():
    from paper_1502_01376_gb300 import build
    build.build()
    from paper_1502_01376_gb300 import hyb as h
    return h


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hyb.h")).read()
    return sorted(set(re.findall(r"HYB_API\s+[\w\s\*]+?\b(hyb_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("hyb_create_grid", "hyb_deposit", "hyb_correct_current", "hyb_filter", "hyb_advance",
                     "hyb_diag", "hyb_destroy_grid", "hyb_bind_fields", "hyb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(hyb):
    L = hyb.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_courant_limit_on_host(hyb):
    d = hyb.make_desc(n1=64, n2=32, dx1=0.2, dx2=0.2, dt=0.1)
    assert hyb.hyb_courant_limit(d) == pytest.approx(2 / math.sqrt(math.pi ** 2 / 0.04 + 4 / 0.04), rel=1e-15)
    d3 = hyb.make_desc(dims=3, n1=64, n2=32, n3=16, dx1=0.2, dx2=0.2, dx3=0.2, dt=0.08)
    assert hyb.hyb_courant_limit(d3) == pytest.approx(2 / math.sqrt(math.pi ** 2 / 0.04 + 8 / 0.04), rel=1e-15)


def test_descriptor_validation_without_gpu(hyb):
    bad_dt = hyb.make_desc(n1=64, n2=32, dx1=0.2, dx2=0.2, dt=0.2)
    with pytest.raises(hyb.HybError) as e:
        hyb.hyb_create_grid(bad_dt)
    assert e.value.status == hyb.HYB_ECOURANT
    for kw in (dict(n1=100), dict(n1=4), dict(precision=16), dict(dims=4), dict(n2=1)):
        d = hyb.make_desc(**{**dict(n1=64, n2=32, dx1=0.2, dx2=0.2, dt=0.05), **kw})
        with pytest.raises(hyb.HybError) as e:
            hyb.hyb_create_grid(d)
        assert e.value.status == hyb.HYB_EINVAL
    assert "n1" in hyb.hyb_last_error() or "dims" in hyb.hyb_last_error() or "n2" in hyb.hyb_last_error()


def test_fused_path_request_validated(hyb):
    d = hyb.make_desc(n1=64, n2=32, dx1=0.2, dx2=0.2, dt=0.05, precision=64, path=2)
    with pytest.raises(hyb.HybError) as e:
        hyb.hyb_create_grid(d)
    assert e.value.status == hyb.HYB_EINVAL


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1502_01376_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liborc" not in txt and "hyb_oracle" not in txt, f
