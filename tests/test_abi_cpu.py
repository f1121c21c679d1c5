"""CPU-side checks of the C ABI: the library loads, exports every function
include/amy.h declares, and rejects invalid problems before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "amy.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(amy_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2005_06191_gb300 import build
    build.build()
    from paper_2005_06191_gb300 import _abi
    return _abi.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["amy_build", "amy_synthesize", "amy_backup_step", "amy_query_rows", "amy_info",
                 "amy_destroy", "amy_last_error", "amy_grid_count", "amy_server_create", "amy_submit",
                 "amy_poll", "amy_wait", "amy_cancel", "amy_server_destroy", "amy_result_free"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_grid_count_matches_paper_sizes(lib):
    import paper_2005_06191_gb300 as amy
    assert amy.amy_grid_count(-10, 10, 0.5) == 41
    assert amy.amy_grid_count(0, 10, 0.37) == 28
    assert amy.amy_grid_count(-0.04, 0.04, 0.02) == 5
    assert amy.amy_grid_count(-0.3, 0.3, 0.1) == 7


def _expect_invalid(amy, problem, **kw):
    with pytest.raises(amy.AmyError) as e:
        amy.amy_build(problem, **kw)
    return str(e.value)


def test_invalid_problems_rejected(lib):
    import paper_2005_06191_gb300 as amy
    rng = np.random.default_rng(0)
    base = W.random_affine(rng, 2, [9, 9], 3).problem
    # even explicit window
    p = W.random_affine(rng, 2, [9, 9], 3, window=[3, 4]).problem
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # gamma at or above the peak density
    p = W.random_affine(rng, 2, [9, 9], 3).problem
    p.gamma = 100.0
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # wrong number of affine parameters
    p = W.random_affine(rng, 2, [9, 9], 3).problem
    p.params = p.params[:-1]
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # more than 8 dims
    p = W.random_affine(rng, 9, [2] * 9, 2, window=[1] * 9).problem
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # more than 65535 inputs
    p = W.random_affine(rng, 1, [5], 2).problem
    p.u_count = [70000]
    p.params = np.zeros(70000 * 2)
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # dense rows on a periodic dim
    p = W.random_affine(rng, 2, [9, 9], 3, periodic=[0, 1]).problem
    p.gamma = 0.0
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # non-positive sigma
    p = W.random_affine(rng, 2, [9, 9], 3).problem
    p.sigma = [0.2, 0.0]
    assert "INVALID_ARG" in _expect_invalid(amy, p)
    # 16-bit V storage with FP64
    assert "INVALID_ARG" in _expect_invalid(amy, base, prec="fp64", v_store="bf16")


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2005_06191_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower().replace("oracle/", ""), f
