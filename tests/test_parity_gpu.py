"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (all five workloads, reduced and full sizes, every T mode
and precision, ragged shapes and edge cases)."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import GAP, TOL, compare_one_step, compare_rows, compare_steps, compare_synthesis, load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


# ---- robot_lin: dense 41x41 rows, reach-avoid, horizon 8 -------------------
@pytest.fixture(scope="module")
def robot_ref():
    w = W.robot_lin()
    return w, oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)


@pytest.mark.parametrize("tmode", ["stored_full", "otf", "stored_factored"])
def test_robot_lin_fp64(amy, robot_ref, tmode):
    w, ref = robot_ref
    compare_synthesis(amy, w, tmode, "fp64", ref=ref)


@pytest.mark.parametrize("tmode", ["stored_full", "otf", "stored_factored"])
@pytest.mark.parametrize("prec", ["fp32", "fp32_kahan"])
def test_robot_lin_fp32(amy, robot_ref, tmode, prec):
    w, ref = robot_ref
    compare_synthesis(amy, w, tmode, prec, ref=ref)


@pytest.mark.parametrize("tmode", ["stored_full", "stored_factored", "otf"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_wide_row_split(amy, robot_ref, tmode, prec):
    """Wide rows (the robot's dense 41 x 41 windows; stored, or on the fly with
    each pair's masses computed once per block into shared memory) are summed by
    groups of window rows, their pair sums reduced per state by a second
    kernel (backup kernel 6); without room in the budget for the pair sums
    one thread takes each pair (kernel 0).  Both match the oracle; they
    agree with each other to rounding (the row groups only reassociate the
    sum) and their policies agree wherever the top-two gap is clear."""
    w, ref = robot_ref
    out, kernels = [], []
    with amy.amy_build(w.problem, tmode=tmode, prec=prec) as h:
        info = amy.amy_info(h)
        kernels.append(info["backup_kernel"])
        assert info["backup_launch_kernels"] == 2
        full_bytes = info["device_bytes"]
        out.append(amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True))
    with amy.amy_build(w.problem, tmode=tmode, prec=prec, device_mem_budget=full_bytes - 1) as h:
        info = amy.amy_info(h)
        kernels.append(info["backup_kernel"])
        assert info["backup_launch_kernels"] == 1
        out.append(amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True))
    assert kernels == [6, 0]
    tol = TOL[prec]
    for V, pi in out:
        assert float(np.max(np.abs(V.astype(np.float64) - ref["V"]))) <= tol
        sure = ref["gap"] > GAP[prec]
        assert not ((pi != ref["pi"]) & sure).any()
    assert float(np.max(np.abs(out[0][0].astype(np.float64) - out[1][0]))) <= (1e-14 if prec == "fp64" else 2e-6)
    compare_synthesis(amy, w, tmode, prec, ref=ref)


def test_robot_lin_rows(amy):
    w = W.robot_lin()
    for tmode, prec, tol in [("stored_full", "fp64", 1e-14), ("otf", "fp32", 2e-6)]:
        mism, worst = compare_rows(amy, w, tmode, prec)
        assert mism == 0
        assert worst <= tol, (tmode, prec, worst)


# ---- unicycle: full size (51x51x30, 45 inputs, gamma 1e-6, horizon 32) -----
@pytest.fixture(scope="module")
def unicycle_ref():
    w = W.unicycle()
    return w, oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)


@pytest.mark.parametrize("tmode,prec", [("stored_factored", "fp32"), ("stored_full", "fp32_kahan"),
                                        ("otf", "fp32"), ("otf", "fp64")])
def test_unicycle_full(amy, unicycle_ref, tmode, prec):
    w, ref = unicycle_ref
    compare_synthesis(amy, w, tmode, prec, ref=ref)


@pytest.mark.parametrize("v_store", ["u16", "bf16"])
def test_unicycle_16bit_v(amy, unicycle_ref, v_store):
    """16-bit V over the unicycle's 32 backups against the stated 2e-3.
    unorm16 meets it.  Folded bfloat16 (2^-10 per backup at worst) is
    expected to end near 3e-3 after 32 backups (about 2.8e-3 in a CPU
    emulation of its rounding): the test then reports the measured number
    as an expected failure rather than widening the bound."""
    w, ref = unicycle_ref
    st = compare_synthesis(amy, w, "stored_factored", "fp32", v_store=v_store, ref=ref, bf16_over_ok=True)
    if "bf16_over" in st:
        assert st["bf16_over"] < 1e-2
        pytest.xfail(f"folded bf16 V: max|dV| = {st['bf16_over']:.2e} > 2e-3 after {w.horizon} backups")


def test_unicycle_rows_origins_exact(amy):
    w = W.unicycle()
    mism, worst = compare_rows(amy, w, "otf", "fp64", n_pairs=4096)
    # cos/sin of CUDA and of the host libm may differ in the last bit; an origin
    # can then differ only if the mean sits within an ulp of a slot boundary.
    assert mism == 0
    assert worst <= 1e-13


# ---- rooms7: reduced to 5 points per dim, horizon 3; full size one step ----
def test_rooms7_reduced(amy):
    w = W.rooms7(n_per_dim=5, horizon=3)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for tmode, prec in [("otf", "fp32_kahan"), ("stored_factored", "fp32"), ("otf", "fp32")]:
        compare_synthesis(amy, w, tmode, prec, ref=ref)


def test_rooms7_full_one_step(amy):
    w = W.rooms7()
    rng = np.random.default_rng(W.SEED)
    V_next = rng.uniform(0.0, 1.0, size=w.problem.n_states)
    states = rng.choice(w.problem.n_states, size=3000, replace=False)
    compare_one_step(amy, w, "otf", "fp32_kahan", "native", states, V_next)


@pytest.mark.parametrize("tmode", ["stored_separable", "otf"])
def test_rooms7_full_every_step(amy, tmode):
    """9^7 states, all 10 backups from V_N on the GPU; at each step the oracle
    recomputes 10^5 seeded states (10^6 at the first) from the GPU's own
    V_{k+1}: the tables path the benchmark times and the on-the-fly path."""
    w = W.rooms7()
    worst, checked = compare_steps(amy, w, tmode, "fp32_kahan", 100_000, W.SEED + 31, first_sample=1_000_000)
    assert checked > 0


# ---- traffic6: reduced to 6 points per dim, horizon 2; full size one step ---
def test_traffic6_reduced(amy):
    w = W.traffic6(n_per_dim=6, horizon=2)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    compare_synthesis(amy, w, "otf", "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32", v_store="u16", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32", v_store="bf16", ref=ref)


@pytest.mark.parametrize("tmode", ["stored_separable", "otf"])
def test_traffic6_full_one_step(amy, tmode):
    w = W.traffic6()
    rng = np.random.default_rng(W.SEED + 5)
    V_next = rng.uniform(0.0, 1.0, size=w.problem.n_states)
    states = rng.choice(w.problem.n_states, size=20_000, replace=False)
    compare_one_step(amy, w, tmode, "fp32_kahan", "native", states, V_next)


@pytest.mark.parametrize("tmode,v_store", [("stored_separable", "native"), ("otf", "native"),
                                           ("stored_separable", "bf16")])
def test_traffic6_full_every_step(amy, tmode, v_store):
    """21^6 states (85.8 M), all 8 backups from V_N on the GPU in the
    benchmark's precision; at each step the oracle recomputes 2 x 10^4
    seeded states (2 x 10^5 at the first) from the GPU's own V_{k+1}.  This
    covers every kind of tile at full size, interior ones included."""
    w = W.traffic6()
    first = 200_000 if v_store == "native" and tmode == "stored_separable" else 0
    worst, checked = compare_steps(amy, w, tmode, "fp32_kahan", 20_000, W.SEED + 41, v_store=v_store,
                                   first_sample=first)
    assert checked > 0


# ---- served-stream problems, one by one through amy_synthesize ---------------
def test_served_requests_individually(amy):
    reqs = W.served_stream(12)
    for w in reqs:
        w.horizon = min(w.horizon, 12)
        compare_synthesis(amy, w, "otf", "fp32")


def _served_cost(w):
    Wd, _ = oracle.window_shape(w.problem)
    return w.problem.n_states * w.problem.n_inputs * int(np.prod(Wd)) * w.horizon


def test_served_requests_full_horizons(amy):
    """Requests of the 256-request stream at their own horizons (the longest
    ones whose oracle run takes a few seconds), FP32 on the fly and with
    tables, and folded-bfloat16 V."""
    pool = [w for w in W.served_stream(256) if w.horizon >= 30 and _served_cost(w) <= 3e9]
    reqs = []
    for n in (2, 3, 4):   # the two longest horizons of each dimension count
        reqs += sorted([w for w in pool if w.problem.n == n], key=lambda w: -w.horizon)[:2]
    assert len(reqs) == 6
    over = []
    for w in reqs:
        ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
        compare_synthesis(amy, w, "otf", "fp32", ref=ref)
        compare_synthesis(amy, w, "stored_separable", "fp32", ref=ref)
        st = compare_synthesis(amy, w, "otf", "fp32", v_store="bf16", ref=ref, bf16_over_ok=True)
        if "bf16_over" in st:
            over.append((w.problem.name, w.horizon, st["bf16_over"]))
    if over:
        pytest.xfail("folded bf16 V above 2e-3 on " + ", ".join(f"{n} (horizon {h}): {d:.2e}" for n, h, d in over))


@pytest.mark.parametrize("tmode", ["otf", "stored_separable"])
def test_served_stream_origins_exact(amy, tmode):
    """Every request of the 256-request stream: window origins of sampled
    (state, input) pairs bit-exact against the oracle, masses within FP32
    rounding."""
    for i, w in enumerate(W.served_stream(256)):
        mism, worst = compare_rows(amy, w, tmode, "fp32", n_pairs=24, seed=i)
        assert mism == 0, (w.problem.name, mism)
        assert worst <= 2e-6, (w.problem.name, worst)


@pytest.mark.parametrize("tmode", ["stored_separable", "otf"])
def test_high_d_full_origins_exact(amy, tmode):
    """The 7-room (9^7) and 6-D traffic (21^6) workloads at full size: window
    origins bit-exact, masses within FP32 rounding, on seeded pairs."""
    for w, n_pairs in [(W.rooms7(), 2048), (W.traffic6(), 384)]:
        mism, worst = compare_rows(amy, w, tmode, "fp32", n_pairs=n_pairs, seed=7)
        assert mism == 0, (w.problem.name, mism)
        assert worst <= 2e-6, (w.problem.name, worst)


# ---- ragged shapes, every dimension count, periodic dims, all specs ---------
@pytest.mark.parametrize("n,per_dim,window,gamma,periodic", [
    (1, [37], None, 5e-2, None),
    (2, [13, 29], [3, 5], 0.0, [0, 1]),
    (3, [7, 9, 11], None, 1e-2, [1, 0, 0]),
    (4, [5, 6, 7, 5], [3, 3, 3, 3], 0.0, None),
    (5, [4, 5, 4, 5, 3], None, 0.2, None),
    (6, [3, 4, 3, 4, 3, 4], [3, 1, 3, 1, 3, 1], 0.0, None),
    (7, [3, 3, 3, 3, 3, 3, 4], None, 0.3, None),
    (8, [3, 3, 3, 3, 3, 3, 3, 3], [3] * 8, 0.0, None),
])
@pytest.mark.parametrize("kind", [W.SAFETY, W.REACH, W.REACH_AVOID])
def test_random_shapes(amy, n, per_dim, window, gamma, periodic, kind):
    rng = np.random.default_rng(100 + n)
    w = W.random_affine(rng, n, per_dim, 3, gamma=gamma, window=window, periodic=periodic,
                        kind=kind, horizon=3)
    if window is None and gamma == 0.0:
        w.problem.gamma = 0.0
    for tmode in ["otf", "stored_factored", "stored_full"]:
        compare_synthesis(amy, w, tmode, "fp32_kahan")
    compare_synthesis(amy, w, "otf", "fp64")
    # window origins bit-exact in every row mode
    for tmode, prec, tol in [("otf", "fp64", 1e-13), ("stored_full", "fp64", 1e-13), ("stored_factored", "fp32", 2e-6),
                             ("stored_separable", "fp32", 2e-6)]:
        mism, worst = compare_rows(amy, w, tmode, prec, n_pairs=96, seed=n)
        assert mism == 0 and worst <= tol, (tmode, mism, worst)


def test_horizon_zero_and_single_input(amy):
    rng = np.random.default_rng(9)
    w = W.random_affine(rng, 2, [9, 7], 1, gamma=1e-2, horizon=0)
    compare_synthesis(amy, w, "otf", "fp32")
    w.horizon = 4
    compare_synthesis(amy, w, "stored_full", "fp32")


def test_single_state_grid(amy):
    rng = np.random.default_rng(4)
    w = W.random_affine(rng, 2, [1, 1], 3, window=[3, 3], kind=W.SAFETY, horizon=3)
    w.problem.x_eta = [1.0, 1.0]
    w.spec = W.Spec(W.SAFETY, safe=([-10.0, -10.0], [10.0, 10.0]))
    compare_synthesis(amy, w, "otf", "fp32")


def test_backup_step_matches_synthesize(amy):
    w = W.unicycle(nxy=21, horizon=1, target=(2.0, 3.0))
    with amy.amy_build(w.problem, tmode="stored_factored", prec="fp32") as h:
        V1, pi1 = amy.amy_synthesize(h, w.spec, 1)
        mask = oracle.spec_mask(w.problem, w.spec)
        VN = ((mask & 1) != 0).astype(np.float32)
        V2, pi2 = amy.amy_backup_step(h, w.spec, VN)
    assert np.array_equal(V1, V2) and np.array_equal(pi1, pi2)


def test_deterministic_reruns(amy):
    w = W.rooms7(n_per_dim=4, horizon=3)
    with amy.amy_build(w.problem, tmode="otf", prec="fp32_kahan") as h:
        a = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        b = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_device_outputs(amy):
    import torch
    w = W.unicycle(nxy=21, horizon=6, target=(2.0, 3.0))
    ref = oracle.synthesize(w.problem, w.spec, w.horizon)
    with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
        V = torch.empty(w.problem.n_states, dtype=torch.float32, device="cuda")
        pi = torch.empty(w.problem.n_states, dtype=torch.int16, device="cuda")
        amy.amy_synthesize(h, w.spec, w.horizon, V_out=V, policy_out=pi)
        torch.cuda.synchronize()
    assert np.max(np.abs(V.cpu().numpy() - ref["V"])) <= TOL["fp32"]


@pytest.mark.parametrize("tmode,prec", [("stored_separable", "fp32"), ("otf", "fp32_kahan"), ("stored_full", "fp64")])
def test_host_outputs_pinned_pageable_device_agree(amy, tmode, prec):
    """Host outputs in page-locked memory are written by the kernels in place,
    pageable ones go through the handle's staging buffer, device outputs stay
    on the device: all three give the same V_0 and policies, bit for bit, on
    repeated calls (the staging buffer is reused) and for horizon 0."""
    import torch
    w = W.unicycle(nxy=21, horizon=6, target=(2.0, 3.0))
    n, N = w.problem.n_states, w.horizon
    fdt = torch.float64 if prec == "fp64" else torch.float32
    with amy.amy_build(w.problem, tmode=tmode, prec=prec) as h:
        Vd = torch.empty(n, dtype=fdt, device="cuda")
        Pd = torch.empty((N, n), dtype=torch.int16, device="cuda")
        amy.amy_synthesize(h, w.spec, N, V_out=Vd, policy_out=Pd, policy_all_steps=True)
        torch.cuda.synchronize()
        Vd, Pd = Vd.cpu().numpy(), Pd.cpu().numpy().view(np.uint16)
        for _ in range(2):
            Vp = torch.full((n,), -1.0, dtype=fdt, pin_memory=True).numpy()
            Pp = torch.full((N, n), 7, dtype=torch.int16, pin_memory=True).numpy()
            amy.amy_synthesize(h, w.spec, N, V_out=Vp, policy_out=Pp, policy_all_steps=True)
            Vq, Pq = amy.amy_synthesize(h, w.spec, N, policy_all_steps=True)   # pageable
            assert np.array_equal(Vp, Vd) and np.array_equal(Pp.view(np.uint16), Pd)
            assert np.array_equal(Vq, Vd) and np.array_equal(Pq, Pd)
        V0p = torch.full((n,), -1.0, dtype=fdt, pin_memory=True).numpy()
        amy.amy_synthesize(h, w.spec, 0, V_out=V0p)
        V0q, _ = amy.amy_synthesize(h, w.spec, 0)
        assert np.array_equal(V0p, V0q) and set(np.unique(V0q)) <= {0.0, 1.0}


def test_memory_budget_rejected(amy):
    w = W.unicycle()
    with pytest.raises(amy.AmyError) as e:
        amy.amy_build(w.problem, tmode="stored_full", prec="fp32", device_mem_budget=1 << 20)
    assert "OUT_OF_MEMORY" in str(e.value)


# ---- separable per-dimension tables ------------------------------------------
@pytest.mark.parametrize("prec,v_store", [("fp32", "native"), ("fp32_kahan", "native"), ("fp32", "u16")])
def test_unicycle_separable(amy, unicycle_ref, prec, v_store):
    w, ref = unicycle_ref
    compare_synthesis(amy, w, "stored_separable", prec, v_store=v_store, ref=ref)


def test_separable_tables_match_factored_bitwise(amy):
    """Tabulating each component over its dependencies changes no value: with
    the per-state kernel the tables give the factored rows' results bit for
    bit.  (The unicycle's inputs come in runs sharing the x and y rows, where
    the tables' kernel contracts those rows once per run, and the banded
    rings run the plane kernel: different summation orders, compared within
    FP32 rounding instead -- and bit for bit once the plane kernel is off.)"""
    for w in [W.unicycle(nxy=31, horizon=6, target=(3.0, 5.0)), W.rooms7(n_per_dim=4, horizon=3),
              W.traffic6(n_per_dim=5, horizon=2), W.served_stream(3)[2]]:
        out, grouped, plane = {}, False, False
        for tmode in ["stored_factored", "stored_separable"]:
            with amy.amy_build(w.problem, tmode=tmode, prec="fp32") as h:
                grouped = grouped or amy.amy_info(h)["grouped_inputs"] == 1
                if amy.amy_info(h)["backup_kernel"] == 7:
                    plane = True
                    Vp, _ = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
                    amy.amy_set_plane(h, 0)
                out[tmode] = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        if plane:
            assert np.max(np.abs(out["stored_factored"][0] - Vp)) <= 2e-6
        if grouped:
            assert w.problem.name.startswith("unicycle")
            assert np.max(np.abs(out["stored_factored"][0] - out["stored_separable"][0])) <= 2e-6
            continue
        assert np.array_equal(out["stored_factored"][0], out["stored_separable"][0])
        assert np.array_equal(out["stored_factored"][1], out["stored_separable"][1])


def _steer_problem():
    """2-D affine system whose second input only moves the inner dim (runs of 5
    inputs share the outer row) and whose outer dim spreads its windows over
    the whole grid, so that every row tile's box overflows shared memory."""
    p = W.Problem(name="steer2", x_lb=[-3.0, -3.0], x_eta=[6.0 / 63, 6.0 / 29], x_count=[64, 30],
                  x_periodic=[0, 0], u_lb=[-1.0, -1.0], u_eta=[1.0, 0.5], u_count=[3, 5],
                  sys_kind=W.AFFINE, params=np.zeros(0), sigma=[0.3, 0.25], gamma=0.0, window=[3, 3])
    A = np.array([[3.0, 0.0], [0.0, 1.0]])
    B = np.array([[0.5, 0.0], [0.0, 0.1]])
    p.params = W.linear_system_params(A, B, W.input_centres(p))
    spec = W.Spec(W.REACH_AVOID, targets=[([0.2, 1.0], [0.6, 2.5])], avoids=[([-0.5, -1.0], [0.0, 0.0])])
    return W.Workload(p, spec, 6, precision="fp32")


def test_grouped_inputs_box_and_global_paths(amy):
    """The per-run outer contraction: staged (unicycle) and from global memory
    when the window box overflows (steer2) both match the oracle."""
    for w in [W.unicycle(nxy=31, horizon=6, target=(3.0, 5.0)), _steer_problem()]:
        with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32") as h:
            info = amy.amy_info(h)
            # the default shape takes row tiles: the per-run kernel k_backup_runs,
            # or its persistent form when every block of the grid can be resident
            assert info["grouped_inputs"] == 1 and info["backup_kernel"] in (4, 5)
            if w.problem.name.startswith("unicycle"):
                # 5 speeds x 9 turn rates; heading windows start at most 1 slot apart
                assert (info["input_runs"], info["inner_span"]) == (5, 4)
            else:
                assert info["input_runs"] == 3 and 3 <= info["inner_span"] <= 6
        compare_synthesis(amy, w, "stored_separable", "fp32")
        compare_synthesis(amy, w, "stored_separable", "fp32_kahan")
        compare_synthesis(amy, w, "stored_separable", "fp32", v_store="u16")


def test_launch_shapes_agree_bitwise(amy):
    """Any launch shape (input lanes per state; staged tiles of whole rows or of
    consecutive states; boxes too wide for shared memory falling back to the
    register-resident body) gives the same values and policies."""
    rng = np.random.default_rng(5)
    cases = [
        W.unicycle(nxy=31, horizon=6, target=(3.0, 5.0)),                          # rows of 30, periodic
        W.random_affine(rng, 2, [37, 30], 6, window=[3, 3], horizon=5),             # 2-D rows of 30
        W.random_affine(rng, 3, [6, 7, 60], 5, window=[5, 5, 5], horizon=3),        # rows of 60: 2 chunks
        W.random_affine(rng, 3, [5, 6, 29], 3, window=[3, 3, 3], periodic=[0, 0, 1], horizon=4),
    ]
    # fixed shapes: (input lanes, states per block, rows 1 / consecutive 2, box floats);
    # a 256-float box overflows for most tiles and takes the global-memory path
    # (5th entry: values of dim 0 per row tile of the per-run kernels; 3 does
    # not divide the 5 rows of (1, 160, 1, 0, 3), which then take the staged kernel)
    fixed = [(1, 256, 2, 0), (5, 32, 1, 0), (2, 64, 1, 256), (3, 64, 2, 0), (8, 32, 0, 1024), (5, 96, 1, 0),
             (1, 512, 2, 0), (4, 128, 1, 0), (1, 288, 1, 0, 3), (2, 192, 1, 0, 2), (1, 160, 1, 0, 3),
             (1, 384, 1, 0, 4)]
    for i, w in enumerate(cases):
        out, shapes, kernels = [], [], set()
        runs = [dict(autotune=False), dict(autotune=True)] + [dict(launch_shape=f) for f in fixed]
        for kw in runs:
            with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32", **kw) as h:
                info = amy.amy_info(h)
                shapes.append((info["input_lanes"], info["block_states"], info["row_tiles"]))
                kernels.add(info["backup_kernel"])
                out.append(amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True))
        for k in range(1, len(runs)):
            assert np.array_equal(out[0][0], out[k][0]), (i, shapes[k])
            assert np.array_equal(out[0][1], out[k][1]), (i, shapes[k])
        if i == 0:
            assert shapes[0][2] == 1   # the default shape of the unicycle uses row tiles
            # the per-step kernels (staged per-run pass, per-run kernel) and the
            # persistent horizon kernel all took part, and agree bitwise
            assert {3, 4, 5} <= kernels, kernels
        compare_synthesis(amy, w, "stored_separable", "fp32")
    for bad in [(9, 0, 0, 0), (0, 48, 0, 0), (4, 256, 0, 0), (0, 544, 0, 0), (0, 0, 3, 0), (0, 0, 0, 100),
                (0, 0, 0, 0, 9)]:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_build(cases[0].problem, tmode="stored_separable", prec="fp32", launch_shape=bad)
        assert "INVALID_ARG" in str(e.value)


def test_separable_rows_and_other_workloads(amy, robot_ref):
    w, ref = robot_ref
    compare_synthesis(amy, w, "stored_separable", "fp32", ref=ref)   # 41-wide rows: generic kernel
    mism, worst = compare_rows(amy, W.unicycle(), "stored_separable", "fp32", n_pairs=2048)
    assert mism == 0 and worst <= 2e-6
    w3 = W.rooms7(n_per_dim=5, horizon=3)
    compare_synthesis(amy, w3, "stored_separable", "fp32_kahan")
    w5 = W.traffic6(n_per_dim=6, horizon=2)
    compare_synthesis(amy, w5, "stored_separable", "fp32_kahan")
    for w4 in W.served_stream(6):
        w4.horizon = min(w4.horizon, 10)
        compare_synthesis(amy, w4, "stored_separable", "fp32")


@pytest.mark.parametrize("tmode", ["stored_full", "stored_factored", "stored_separable", "otf"])
def test_rebuild_with_new_parameters(amy, tmode):
    rng = np.random.default_rng(21)
    w = W.random_affine(rng, 3, [9, 8, 7], 4, gamma=2e-2, horizon=4)
    w2 = W.random_affine(np.random.default_rng(22), 3, [9, 8, 7], 4, gamma=2e-2, horizon=4)
    w2.problem.sigma = w.problem.sigma
    ref2 = oracle.synthesize(w2.problem, w.spec, w.horizon)
    with amy.amy_build(w.problem, tmode=tmode, prec="fp32") as h:
        amy.amy_synthesize(h, w.spec, w.horizon)
        amy.amy_rebuild(h, w2.problem.params)
        V, _ = amy.amy_synthesize(h, w.spec, w.horizon)
    assert np.max(np.abs(V - ref2["V"])) <= TOL["fp32"]


def test_random_shapes_separable(amy):
    for n, per_dim, window, gamma in [(1, [37], None, 5e-2), (4, [5, 6, 7, 5], [3, 3, 3, 3], 0.0),
                                      (5, [4, 5, 4, 5, 3], None, 0.2), (8, [3] * 8, [3] * 8, 0.0),
                                      (2, [11, 13], [7, 5], 0.0)]:
        for kind in [W.SAFETY, W.REACH_AVOID]:
            w = W.random_affine(np.random.default_rng(300 + n), n, per_dim, 3, gamma=gamma, window=window,
                                kind=kind, horizon=3)
            compare_synthesis(amy, w, "stored_separable", "fp32")
            compare_synthesis(amy, w, "otf", "fp32_kahan", v_store="u16")


def test_graph_replay_matches_direct_launches(amy):
    import torch
    w = W.unicycle(nxy=31, horizon=9, target=(3.0, 5.0))
    w2 = W.unicycle(nxy=31, horizon=9, target=(1.0, 2.0))
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32", use_graphs=True) as h:
        Vh, pih = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)   # host path, no graph
        V = torch.empty(w.problem.n_states, dtype=torch.float32, device="cuda")
        PI = torch.empty((w.horizon, w.problem.n_states), dtype=torch.int16, device="cuda")
        for _ in range(3):   # capture once, replay twice
            amy.amy_synthesize(h, w.spec, w.horizon, V_out=V, policy_out=PI, policy_all_steps=True)
            torch.cuda.synchronize()
            assert np.array_equal(V.cpu().numpy(), Vh)
            assert np.array_equal(PI.cpu().numpy().view(np.uint16), pih)
        # a different spec must not replay the cached graph
        V2h, _ = amy.amy_synthesize(h, w2.spec, w2.horizon)
        amy.amy_synthesize(h, w2.spec, w2.horizon, V_out=V, policy_out=PI, policy_all_steps=True)
        torch.cuda.synchronize()
        assert np.array_equal(V.cpu().numpy(), V2h)


@pytest.mark.parametrize("step_wait", [0, 1])
def test_persistent_barrier_wait_is_bounded(amy, step_wait):
    """The persistent horizon kernel's waits between backups (neighbour tiles,
    or the grid barrier) have a poll limit: with a limit of zero every wait
    gives up at once, the blocks leave the kernel and the synthesis reports
    AMY_E_TIMEOUT (no fault, no hang); with the default limit restored the
    same handle gives the same values and policies as before."""
    w = W.unicycle(nxy=31, horizon=6, target=(3.0, 5.0))
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32", launch_shape=(4, 128, 1, 0)) as h:
        assert amy.amy_info(h)["backup_kernel"] == 5
        amy.amy_set_step_wait(h, step_wait)
        ref = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        amy.amy_set_wait_limit(h, 0)
        with pytest.raises(amy.AmyError) as e:
            amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        assert "TIMEOUT" in str(e.value)
        amy.amy_set_wait_limit(h, -1)
        again = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        assert np.array_equal(ref[0], again[0]) and np.array_equal(ref[1], again[1])
        with pytest.raises(amy.AmyError) as e:
            amy.amy_set_step_wait(h, 2)
        assert "INVALID_ARG" in str(e.value)
    compare_synthesis(amy, w, "stored_separable", "fp32")


def _periodic_x(w, nxy):
    """The unicycle with its x coordinate periodic as well (a wrapping tile
    extent for the persistent kernel's neighbour wait)."""
    import dataclasses
    p = dataclasses.replace(w.problem, x_periodic=[1, 0, 1], name=f"unicycle_px{nxy}")
    return W.with_sizes(w, problem=p)


def test_persistent_step_waits_agree(amy):
    """Waiting between backups only for the neighbour tiles (the tiles a
    block's window box reads, and those whose boxes read it) gives the same
    values and policies, bit for bit, as the grid-wide barrier: on plain
    tiles, on tiles that wrap around a periodic dim in whole tiles (27 x
    values in tiles of 3), on a periodic dim the tiles do not divide (28 x
    values: the whole extent is waited for), and with one x value per tile.
    Both agree with the oracle."""
    cases = [
        (W.unicycle(nxy=31, horizon=7, target=(3.0, 5.0)), (1, 288, 1, 0, 3)),
        (_periodic_x(W.unicycle(nxy=27, horizon=7, target=(3.0, 5.0)), 27), (1, 288, 1, 0, 3)),
        (_periodic_x(W.unicycle(nxy=28, horizon=7, target=(3.0, 5.0)), 28), (1, 288, 1, 0, 3)),
        (_periodic_x(W.unicycle(nxy=27, horizon=7, target=(3.0, 5.0)), 27), (2, 96, 1, 0, 1)),
    ]
    for w, shape in cases:
        out = []
        with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32", launch_shape=shape) as h:
            assert amy.amy_info(h)["backup_kernel"] == 5, w.problem.name
            assert amy.amy_info(h)["step_wait"] == 1   # the default without autotuning
            for mode in (0, 1, 0):
                amy.amy_set_step_wait(h, mode)
                assert amy.amy_info(h)["step_wait"] == mode
                out.append(amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True))
        for k in (1, 2):
            assert np.array_equal(out[0][0], out[k][0]), (w.problem.name, shape, k)
            assert np.array_equal(out[0][1], out[k][1]), (w.problem.name, shape, k)
        ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
        dV = float(np.max(np.abs(out[0][0].astype(np.float64) - ref["V"])))
        assert dV <= TOL["fp32"], (w.problem.name, dV)
        sure = ref["gap"] > GAP["fp32"]
        assert not ((out[0][1] != ref["pi"]) & sure).any(), w.problem.name


def test_profiling_counts_kernels(amy):
    w = W.unicycle(nxy=21, horizon=5, target=(2.0, 3.0))
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32") as h:
        amy.amy_set_profiling(h, True)
        amy.amy_rebuild(h)
        amy.amy_synthesize(h, w.spec, w.horizon)
        kt = amy.amy_kernel_times(h)
    # five backups: one per launch, or all five in one persistent launch
    assert kt["backup_steps"] == 5 and kt["backup_launches"] in (1, 5) and kt["build_launches"] == 1
    assert kt["backup_ms"] > 0 and kt["build_ms"] > 0


def test_auto_mode_picks_and_matches(amy):
    """AMY_T_AUTO: tables for few dependencies, factored rows for dense systems."""
    picks = {}
    for w in W.served_stream(8, seed=W.SEED + 21):
        w.horizon = min(w.horizon, 8)
        with amy.amy_build(w.problem, tmode="auto", prec="fp32", device_mem_budget=4 << 30) as h:
            picks[w.problem.name] = amy.amy_info(h)["tmode"]
        compare_synthesis(amy, w, "auto", "fp32")
    assert set(picks.values()) <= {0, 2, 3}
    with amy.amy_build(W.unicycle().problem, tmode="auto", prec="fp32") as h:
        assert amy.amy_info(h)["tmode"] == 3


def test_backup_kernel_reported_and_lane_load_ceilings(amy):
    expect = [(W.rooms7(n_per_dim=4, horizon=1), "stored_separable", 7),   # 7-D ring: the plane kernel
              (W.rooms7(n_per_dim=4, horizon=1), "stored_factored", 1),    # 7-D: register-resident
              (W.random_affine(np.random.default_rng(3), 2, [37, 30], 6, window=[3, 3]), "stored_separable", 2),
              (W.robot_lin(), "stored_full", 6),     # dense 41-wide stored rows: split over window rows
              (W.robot_lin(), "otf", 6)]             # 41-wide rows on the fly: the same split
    for w, tmode, kern in expect:
        with amy.amy_build(w.problem, tmode=tmode, prec="fp32") as h:
            assert amy.amy_info(h)["backup_kernel"] == kern, (w.problem.name, tmode)
    peaks = amy.amy_measure_lane_loads()
    # 152 SMs x 32 lanes x ~2 GHz is about 1e13 lane-loads/s for either path
    for k in ("shared", "global_l1"):
        assert 1e12 < peaks[k] < 3e13, peaks
    # FP32: 152 SMs x 128 lanes x ~2 GHz is about 4e13 FMA/s; FP64 far below it
    fma = amy.amy_measure_fma()
    assert 1e13 < fma["fp32"] < 1e14 and 1e10 < fma["fp64"] < fma["fp32"], fma
    # erfc: tens of instructions per evaluation, so well below the FMA rates
    erfc = amy.amy_measure_erfc()
    assert 1e10 < erfc["fp32"] < fma["fp32"] and 1e8 < erfc["fp64"] < min(erfc["fp32"], fma["fp64"]), erfc
