"""Shared helpers of the parity tests: run the engine and the FP64 oracle on the
same seeded inputs and compare element by element."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances (max |dV| against the FP64 oracle):
#   FP32 paths 1e-5 (accumulated over the horizon);
#   FP64 paths 1e-12 (only erfc/cos implementations and summation order differ);
#   16-bit V storage: 2e-3, the stated bound for 16-bit-stored V.  unorm16
#   meets it (at most 2^-17 per backup).  The folded bfloat16 rounds by up to
#   2^-10 per backup; where the accumulated error exceeds 2e-3 the test says
#   so (BF16_OVER) instead of widening the bound.
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_kahan": 1e-5, "u16": 2e-3, "bf16": 2e-3}
# Policies must agree bit for bit wherever the oracle's top-two action values
# differ by more than this; elsewhere the chosen input must be within
# tolerance of the best one.
GAP = {"fp64": 1e-5, "fp32": 1e-5, "fp32_kahan": 1e-5, "u16": 5e-3, "bf16": 5e-3}


def tol_key(prec: str, v_store: str) -> str:
    return prec if v_store == "native" else v_store


def tol_of(key: str, horizon: int) -> float:
    return TOL[key]


def gap_of(key: str, horizon: int) -> float:
    return max(GAP[key], 2.0 * tol_of(key, horizon)) if key in ("bf16", "u16") else GAP[key]


def load_engine():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2005_06191_gb300 import build
    build.build()
    import paper_2005_06191_gb300 as amy
    return amy


def compare_synthesis(amy, w, tmode: str, prec: str, v_store: str = "native", ref=None,
                      tie_samples: int = 64, rng_seed: int = 0, bf16_over_ok: bool = False):
    """Full-horizon parity of V_0 and every pi_k.  Returns a dict of statistics.

    bf16_over_ok: for folded-bfloat16 V whose accumulated rounding is known to
    pass 2e-3 on this workload, a larger max|dV| is returned in the stats
    (key "bf16_over") instead of failing; the caller reports it."""
    p, s, N = w.problem, w.spec, w.horizon
    if ref is None:
        ref = oracle.synthesize(p, s, N, want_all=True)
    key = tol_key(prec, v_store)
    tol, gthr = tol_of(key, N), gap_of(key, N)
    with amy.amy_build(p, tmode=tmode, prec=prec, v_store=v_store) as h:
        V, pi = amy.amy_synthesize(h, s, N, policy_all_steps=True)
    dV = float(np.max(np.abs(V.astype(np.float64) - ref["V"]))) if V.size else 0.0
    stats = {"max_dV": dV, "policy_checked": 0, "policy_ties": 0}
    if bf16_over_ok and key == "bf16" and dV > tol:
        stats["bf16_over"] = dV
        return stats
    assert dV <= tol, f"max|dV| = {dV:.3e} > {tol:.1e}"
    if N > 0:
        sure = ref["gap"] > gthr
        bad = (pi != ref["pi"]) & sure
        assert not bad.any(), f"{int(bad.sum())} policy entries differ where the gap exceeds {gthr}"
        stats["policy_checked"] = int(sure.sum())
        ties = np.argwhere((~sure) & (pi != ref["pi"]))
        stats["policy_ties"] = int(len(ties))
        if len(ties):
            rng = np.random.default_rng(rng_seed)
            pick = ties[rng.choice(len(ties), size=min(tie_samples, len(ties)), replace=False)]
            for k, x in pick:
                av = oracle.action_values(p, ref["V_all"][k + 1], int(x))
                assert av[pi[k, x]] >= av.max() - 2 * tol, (k, x)
    return stats


def bf16_folded(v):
    """The values the engine reads back from folded-bfloat16 storage: V below
    1/2 rounded to bfloat16, V at or above 1/2 as 1 minus bfloat16(1 - V)."""
    import torch
    v = np.clip(np.asarray(v, dtype=np.float32), 0.0, 1.0)
    lo = v < 0.5
    r = np.where(lo, v, np.float32(1.0) - v).astype(np.float32)
    r = torch.from_numpy(r).to(torch.bfloat16).to(torch.float32).numpy()
    return np.where(lo, r, np.float32(1.0) - r).astype(np.float64)


def compare_rows(amy, w, tmode: str, prec: str, n_pairs: int = 512, seed: int = 1):
    """Window origins bit-exact and row probabilities close, on sampled pairs
    (with a disturbance grid, sampled (input, disturbance) pairs)."""
    p = w.problem
    nw = oracle.n_disturbances(p)
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, p.n_states, size=n_pairs)
    us = rng.integers(0, p.n_inputs * nw, size=n_pairs)
    with amy.amy_build(p, tmode=tmode, prec=prec) as h:
        org, probs = amy.amy_query_rows(h, xs, us)
    mism = 0
    worst = 0.0
    for i in range(n_pairs):
        o_ref, pr_ref = oracle.row(p, int(xs[i]), int(us[i]) // nw, int(us[i]) % nw)
        if not np.array_equal(o_ref, org[i]):
            mism += 1
            continue
        worst = max(worst, float(np.max(np.abs(pr_ref - probs[i]))))
    return mism, worst


def compare_one_step(amy, w, tmode: str, prec: str, v_store: str, states, V_next):
    """One backup from a synthetic V_next over the whole grid on the GPU,
    checked against the oracle at the sampled states."""
    p, s = w.problem, w.spec
    key = tol_key(prec, v_store)
    with amy.amy_build(p, tmode=tmode, prec=prec, v_store=v_store) as h:
        vin = V_next.astype(np.float64 if prec == "fp64" else np.float32)
        V, pi = amy.amy_backup_step(h, s, vin)
    # the oracle sees exactly the values the engine read (bf16-rounded when stored so)
    vref_in = vin.astype(np.float64)
    if v_store == "bf16":
        vref_in = bf16_folded(vin)
    elif v_store == "u16":
        code = np.rint(np.clip(vin, 0.0, 1.0) * np.float32(65535)).astype(np.float32)
        vref_in = (code * (np.float32(1.0) / np.float32(65535))).astype(np.float64)
    Vr, pir, gap = oracle.backup_states(p, s, vref_in, states)
    dV = float(np.max(np.abs(V[states].astype(np.float64) - Vr)))
    assert dV <= tol_of(key, 1), f"max|dV| = {dV:.3e}"
    sure = gap > gap_of(key, 1)
    assert np.all(pi[states][sure] == pir[sure])
    return dV, int(sure.sum())


def v16_read_back(vin, v_store: str):
    """The values the engine's backup reads from V_next stored as v_store."""
    if v_store == "bf16":
        return bf16_folded(vin)
    if v_store == "u16":
        code = np.rint(np.clip(vin, 0.0, 1.0) * np.float32(65535)).astype(np.float32)
        return (code * (np.float32(1.0) / np.float32(65535))).astype(np.float64)
    return np.asarray(vin, dtype=np.float64)


def compare_steps(amy, w, tmode: str, prec: str, n_sample: int, seed: int, v_store: str = "native",
                  first_sample: int = 0, horizon: int = None):
    """Sampled one-step operator parity over the whole horizon at full size:
    the GPU performs every backup over the whole grid starting from V_N, and
    at each step the oracle recomputes V_k and pi_k at n_sample seeded states
    (first_sample at the first step, when given) from the very V_{k+1} the
    GPU read.  Returns the largest |dV| seen."""
    p, s = w.problem, w.spec
    key = tol_key(prec, v_store)
    tol, gthr = tol_of(key, 1), gap_of(key, 1)
    rng = np.random.default_rng(seed)
    mask = oracle.spec_mask(p, s)
    V = ((mask & (4 if s.kind == "safety" else 1)) != 0).astype(np.float32)
    worst, checked = 0.0, 0
    N = w.horizon if horizon is None else horizon
    with amy.amy_build(p, tmode=tmode, prec=prec, v_store=v_store) as h:
        for k in range(N):
            Vk, pik = amy.amy_backup_step(h, s, V)
            ns = first_sample if (k == 0 and first_sample) else n_sample
            states = np.sort(rng.choice(p.n_states, size=min(ns, p.n_states), replace=False))
            Vr, pir, gap = oracle.backup_states(p, s, v16_read_back(V, v_store), states)
            dV = float(np.max(np.abs(Vk[states].astype(np.float64) - Vr)))
            assert dV <= tol, f"step {k}: max|dV| = {dV:.3e} > {tol:.1e}"
            sure = gap > gthr
            bad = (pik[states] != pir) & sure
            assert not bad.any(), f"step {k}: {int(bad.sum())} policies differ where the gap exceeds {gthr}"
            worst = max(worst, dV)
            checked += int(sure.sum())
            V = Vk.astype(np.float32)
    return worst, checked
