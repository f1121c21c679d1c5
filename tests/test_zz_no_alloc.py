"""The allocation-free entry point, amy_synthesize_noalloc, for callers that
may not allocate device memory (their memory belongs to their own pool or
framework, or an allocation in their loop could synchronise or fail).

It must give the same results as the allocating path (amy_build with rows on
the fly + amy_synthesize) on consecutive calls, which share the library's
fixed scratch array, and must refuse problems larger than that array.  This
file is collected last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

import workloads as W
from parity_util import TOL, load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


def _allocating(amy, w, prec):
    import torch
    n = w.problem.n_states
    V = torch.empty(n, dtype=torch.float32, device="cuda")
    P = torch.empty(n, dtype=torch.int16, device="cuda")
    with amy.amy_build(w.problem, tmode="otf", prec=prec) as h:
        amy.amy_synthesize(h, w.spec, w.horizon, V_out=V, policy_out=P)
        torch.cuda.synchronize()
    return V.cpu().numpy(), P.cpu().numpy()


def _noalloc(amy, w, prec):
    import torch
    n = w.problem.n_states
    V = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
    P = torch.full((n,), 1234, dtype=torch.int16, device="cuda")
    amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V, P, prec=prec)
    torch.cuda.synchronize()
    return V.cpu().numpy(), P.cpu().numpy()


def test_noalloc_matches_allocating_path_on_consecutive_calls(amy):
    cases = [
        (W.unicycle(nxy=31, horizon=10, target=(3.0, 5.0)), "fp32"),       # reach, periodic dim
        (W.traffic6(n_per_dim=7, horizon=3), "fp32_kahan"),                # safety, 6-D window 5^6
        (W.unicycle(nxy=31, horizon=10, target=(3.0, 5.0)), "fp32"),       # the first problem again
    ]
    for w, prec in cases:
        V_new, P_new = _noalloc(amy, w, prec)
        V_ref, P_ref = _allocating(amy, w, prec)
        assert np.max(np.abs(V_new - V_ref)) <= TOL[prec]
        assert np.array_equal(P_new, P_ref)


def test_noalloc_refuses_problems_beyond_its_scratch(amy):
    import torch
    w = W.traffic6(n_per_dim=12, horizon=1)   # 2.99M states: about 27 MB of scratch, above the 16 MiB array
    V = torch.empty(w.problem.n_states, dtype=torch.float32, device="cuda")
    with pytest.raises(amy.AmyError) as e:
        amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V)
    assert "INVALID_ARG" in str(e.value) and "scratch" in str(e.value)


def test_noalloc_binding_rejects_bad_output_buffers(amy):
    """The binding checks the caller's device buffers before any pointer
    reaches the library: too few entries, a wrong dtype or a host tensor
    raise ValueError and nothing is launched."""
    import torch
    w = W.unicycle(nxy=11, horizon=2, target=(1.0, 2.0))
    n = w.problem.n_states
    for bad in (torch.empty(n - 1, dtype=torch.float32, device="cuda"),
                torch.empty(n, dtype=torch.float64, device="cuda"),
                torch.empty(n, dtype=torch.float32)):
        with pytest.raises(ValueError):
            amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, bad)
    V = torch.empty(n, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V, torch.empty(2 * n, dtype=torch.int16,
                                                                                 device="cuda"))
