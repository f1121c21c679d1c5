"""Serving (continuous batching) on the GPU: results in the mix equal results
alone and the single-problem path, admission by memory, cancellation,
timeouts and queue limits."""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import TOL, load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


def _stream(n, cap_h=14, seed=W.SEED):
    reqs = W.served_stream(n, seed=seed)
    for w in reqs:
        w.horizon = min(w.horizon, cap_h)
    return reqs


def _alone(amy, w):
    with amy.amy_build(w.problem, tmode="stored_separable", prec=w.precision, v_store=w.v_store) as h:
        return amy.amy_synthesize(h, w.spec, w.horizon)


@pytest.mark.parametrize("batched", [True, False])
def test_mix_equals_single_problem_path(amy, batched):
    reqs = _stream(24)
    with amy.amy_server_create(batched=batched, max_slots=16) as srv:
        tickets = [amy.amy_submit(srv, w) for w in reqs]
        results = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in tickets]
        st = amy.amy_server_stats(srv)
    assert st["completed"] == len(reqs)
    for w, r in zip(reqs, results):
        assert r["status"] == 0
        V, pi = _alone(amy, w)
        assert np.array_equal(r["V"], V), w.problem.name
        assert np.array_equal(r["policy"], pi), w.problem.name


def test_mix_matches_oracle(amy):
    reqs = _stream(10, cap_h=8, seed=W.SEED + 3)
    with amy.amy_server_create(batched=True) as srv:
        tickets = [amy.amy_submit(srv, w) for w in reqs]
        results = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in tickets]
    for w, r in zip(reqs, results):
        ref = oracle.synthesize(w.problem, w.spec, w.horizon)
        assert np.max(np.abs(r["V"] - ref["V"])) <= TOL["fp32"]
        sure = ref["gap"][0] > 1e-5 if w.horizon else np.ones(w.problem.n_states, bool)
        if w.horizon:
            assert np.all(r["policy"][sure] == ref["pi"][0][sure])


def test_alone_vs_mix_same_result(amy):
    reqs = _stream(16, seed=W.SEED + 7)
    probe = reqs[5]
    with amy.amy_server_create(batched=True) as srv:
        alone = amy.amy_wait(srv, amy.amy_submit(srv, probe), timeout_us=60_000_000)
    with amy.amy_server_create(batched=True, max_slots=8) as srv:
        tickets = [amy.amy_submit(srv, w) for w in reqs]   # probe arrives in the middle of the mix
        mixed = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in tickets]
    assert np.array_equal(alone["V"], mixed[5]["V"])
    assert np.array_equal(alone["policy"], mixed[5]["policy"])


def test_16bit_storage_requests(amy):
    reqs = _stream(6, seed=W.SEED + 11)
    for w in reqs:
        w.v_store = "u16"
    with amy.amy_server_create(batched=True) as srv:
        results = [amy.amy_wait(srv, amy.amy_submit(srv, w), timeout_us=60_000_000) for w in reqs]
    for w, r in zip(reqs, results):
        V, _ = _alone(amy, w)
        assert np.array_equal(r["V"], V)
        ref = oracle.synthesize(w.problem, w.spec, w.horizon)
        assert np.max(np.abs(r["V"] - ref["V"])) <= TOL["u16"]


def test_memory_budget_serialises_admission(amy):
    reqs = _stream(6, seed=W.SEED + 13)
    with amy.amy_server_create(batched=True, device_mem_budget=3 << 20) as srv:
        tickets = [amy.amy_submit(srv, w) for w in reqs]
        results = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in tickets]
    for w, r in zip(reqs, results):
        assert r["status"] == 0
        V, _ = _alone(amy, w)
        assert np.array_equal(r["V"], V)
    # a request that can never fit is rejected, not queued forever
    big = W.traffic6(n_per_dim=12, horizon=2)
    with amy.amy_server_create(batched=True, device_mem_budget=1 << 20) as srv:
        r = amy.amy_wait(srv, amy.amy_submit(srv, big), timeout_us=60_000_000)
    assert r["status"] == 2  # AMY_E_OUT_OF_MEMORY


def test_cancel_queued_and_running(amy):
    long = W.traffic6(n_per_dim=11, horizon=8)
    quick = _stream(3, seed=W.SEED + 17)
    with amy.amy_server_create(batched=True, max_slots=1) as srv:
        t_long = amy.amy_submit(srv, long)
        t_q = [amy.amy_submit(srv, w) for w in quick]
        amy.amy_cancel(srv, t_q[1])          # still queued behind the long one
        time.sleep(0.05)
        amy.amy_cancel(srv, t_long)          # resident (or about to be)
        r_long = amy.amy_wait(srv, t_long, timeout_us=120_000_000)
        rq = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in t_q]
    assert r_long["status"] in (0, 7)        # finished before the cancel, or cancelled
    assert rq[1]["status"] == 7              # AMY_E_CANCELLED
    for i in (0, 2):
        assert rq[i]["status"] == 0
        V, _ = _alone(amy, quick[i])
        assert np.array_equal(rq[i]["V"], V)


def test_timeout_not_found_and_queue_full(amy):
    long = W.traffic6(n_per_dim=11, horizon=8)
    with amy.amy_server_create(batched=True, max_queue=2) as srv:
        t1 = amy.amy_submit(srv, long)
        t2 = amy.amy_submit(srv, long)
        with pytest.raises(amy.AmyError) as e:
            amy.amy_submit(srv, long)
        assert "QUEUE_FULL" in str(e.value)
        with pytest.raises(amy.AmyError) as e:
            amy.amy_wait(srv, t2, timeout_us=0)
        assert "TIMEOUT" in str(e.value)
        for t in (t1, t2):
            assert amy.amy_wait(srv, t, timeout_us=120_000_000)["status"] == 0
        with pytest.raises(amy.AmyError) as e:
            amy.amy_poll(srv, t1)          # retired
        assert "NOT_FOUND" in str(e.value)


def test_invalid_request_rejected_at_submit(amy):
    w = _stream(1)[0]
    w.problem.window = [4] * w.problem.n
    with amy.amy_server_create() as srv:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_submit(srv, w)
    assert "INVALID_ARG" in str(e.value)


@pytest.mark.parametrize("batched", [True, False])
def test_tick_graphs_match_direct_launches(amy, batched):
    """Ticks replayed from captured CUDA graphs (a layout captured at its
    second occurrence) give the results of directly launched ticks bit for
    bit, for the same mix of requests; the graphs are actually replayed."""
    reqs = _stream(20, cap_h=24, seed=W.SEED + 23)
    out = {}
    for graphs in (False, True):
        with amy.amy_server_create(batched=batched, max_slots=6, use_graphs=graphs) as srv:
            tickets = [amy.amy_submit(srv, w) for w in reqs]
            out[graphs] = [amy.amy_wait(srv, t, timeout_us=120_000_000) for t in tickets]
            gs = amy.amy_server_graph_stats(srv)
        if graphs:
            assert gs["captures"] > 0 and gs["replays"] > gs["captures"], gs
        else:
            assert gs["captures"] == 0 and gs["replays"] == 0
    for w, a, b in zip(reqs, out[False], out[True]):
        assert a["status"] == 0 and b["status"] == 0
        assert np.array_equal(a["V"], b["V"]), w.problem.name
        assert np.array_equal(a["policy"], b["policy"]), w.problem.name


def test_bf16_storage_requests(amy):
    """Folded-bfloat16 V through the server (batched ticks, graphs on) equals
    the single-problem path bit for bit, within 2e-3 of the oracle."""
    reqs = _stream(6, seed=W.SEED + 29)
    for w in reqs:
        w.v_store = "bf16"
    with amy.amy_server_create(batched=True) as srv:
        results = [amy.amy_wait(srv, amy.amy_submit(srv, w), timeout_us=60_000_000) for w in reqs]
    for w, r in zip(reqs, results):
        V, _ = _alone(amy, w)
        assert np.array_equal(r["V"], V)
        ref = oracle.synthesize(w.problem, w.spec, w.horizon)
        assert np.max(np.abs(r["V"] - ref["V"])) <= TOL["bf16"]
