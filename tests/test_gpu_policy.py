"""GPU BF16 policy kernels (inference, gradient, Adam) against the FP64 CPU
oracle.  The network is not in the paper: these pins are finite differences
(CPU, test_oracle_pins) and this comparison."""
import os

import numpy as np
import pytest

import qpgen
from oracle import mlp

pytestmark = pytest.mark.gpu

SHAPES = mlp.PARAM_SHAPES
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding


def make_params(seed):
    rng = np.random.default_rng(seed)
    flat = np.zeros(4622, np.float32)
    flat[0:4] = rng.standard_normal(4)            # feature means
    flat[4:8] = 0.5 + rng.uniform(size=4)          # feature std devs
    off = 8
    d = {}
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        scale = np.sqrt(2.0 / SHAPES[k][-1]) if k.startswith("W") else 0.1
        v = (rng.standard_normal(n) * scale).astype(np.float32)
        flat[off:off + n] = v
        d[k] = v.astype(np.float64).reshape(SHAPES[k])
        off += n
    flat[off:off + 4] = [np.log(10.0), 0.01, 0.5, 0.0]
    return flat, d


def unpack_grad(flat):
    out, off = {}, 8
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = flat[off:off + n].astype(np.float64).reshape(SHAPES[k])
        off += n
    return out


def normalised(flat, feats):
    f = feats.astype(np.float32)
    return ((f - flat[0:4]) / flat[4:8]).astype(np.float32).astype(np.float64)


def test_policy_forward_matches_oracle(gb):
    flat, d = make_params(0)
    feats = np.random.default_rng(1).standard_normal((300, 4)).astype(np.float32) * 3
    got = gb.gbosqp_policy_forward(flat, feats)
    ref = mlp.forward_bf16(d, normalised(flat, feats))
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [16, 37, 500])
def test_mlp_gradient_matches_oracle(gb, n):
    flat, d = make_params(2)
    rng = np.random.default_rng(3)
    feats = (rng.standard_normal((n, 4)) * 2).astype(np.float32)
    tgt = rng.standard_normal((n, 2)).astype(np.float32)
    wgt = np.ones((n, 2), np.float32)
    wgt[::4, 1] = 0.0
    g, loss = gb.gbosqp_mlp_grad(flat, feats, tgt, wgt)
    gg = unpack_grad(g)
    X = normalised(flat, feats)
    # same rounding points: the FP32-accumulated GPU result agrees closely
    lref, gref, _ = mlp.grads_bf16(d, X, tgt.astype(np.float64), wgt.astype(np.float64))
    assert abs(loss - lref) <= 1e-4 * max(lref, 1e-6)
    for k in ORDER:
        num = np.linalg.norm(gg[k] - gref[k])
        assert num <= 2e-2 * np.linalg.norm(gref[k]) + 1e-7, k
    # against the exact FP64 gradient: BF16 operands cost about 1e-2
    lex, gex = mlp.grads(d, X, tgt.astype(np.float64), wgt.astype(np.float64))
    for k in ORDER:
        a, b = gg[k].ravel(), gex[k].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert cos >= 0.999, (k, cos)
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-7, k


def test_mlp_train_follows_adam_and_reduces_loss(gb):
    flat, d = make_params(4)
    rng = np.random.default_rng(5)
    n = 2000
    feats = (rng.standard_normal((n, 4)) * 2).astype(np.float32)
    # regression target: a fixed smooth function of the features
    tgt = np.stack([np.tanh(feats[:, 0] - 0.5 * feats[:, 1]), 0.3 * feats[:, 2]], axis=1).astype(np.float32)
    wgt = np.ones((n, 2), np.float32)
    # one step equals the oracle's Adam step on the oracle's BF16 gradient
    batches = rng.integers(0, n, size=(1, 256)).astype(np.int32)
    new, hist = gb.gbosqp_mlp_train(flat, feats, tgt, wgt, batches, 1e-3)
    sel = batches[0]
    _, gref, _ = mlp.grads_bf16(d, normalised(flat, feats[sel]), tgt[sel].astype(np.float64),
                                wgt[sel].astype(np.float64))
    ref = mlp.adam_step({k: v.copy() for k, v in d.items()}, gref, {}, 1, lr=1e-3)
    got = unpack_grad(new)
    agree = 0
    total = 0
    for k in ORDER:
        big = np.abs(gref[k]) > 1e-3 * np.max(np.abs(gref[k]))
        agree += np.sum(np.abs(got[k] - ref[k])[big] <= 1e-5)
        total += np.sum(big)
    assert agree >= 0.98 * total
    # many steps reduce the loss
    batches = rng.integers(0, n, size=(400, 256)).astype(np.int32)
    _, hist = gb.gbosqp_mlp_train(flat, feats, tgt, wgt, batches, 3e-3)
    assert np.mean(hist[-20:]) <= 0.3 * np.mean(hist[:20])


def _constant_policy(log_mult):
    """A network whose output is constant: zero weights, output bias."""
    p = np.zeros(4622, np.float32)
    p[4:8] = 1.0
    off_b3 = 8 + 64 * 4 + 64 + 64 * 64 + 64 + 2 * 64
    p[off_b3] = log_mult
    p[off_b3 + 2:off_b3 + 6] = [np.log(10.0), 0.05, 0.5, 0.0]
    return p


def test_stalled_policy_falls_back_to_ratio_rule(gb):
    """A policy that always sets 10x the ratio rule's rho stalls; the
    stall rule hands rho back to the residual-ratio rule and the solve still
    reaches the tolerance."""
    import qpgen
    from oracle import checks
    qp = qpgen.random_qp(300, 3000, 0)
    with gb.Solver(qp, rho_policy=gb.RHO_LEARNED, policy_params=_constant_policy(np.log(10.0))) as s:
        st = s.solve()
        info = s.info()
        x, y, z = s.solution()
    assert st == gb.SOLVED, info
    assert info["policy_fallbacks"] > 0
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) and v.dual <= info["eps_dual"] * (1 + 1e-6)


def test_zero_correction_reproduces_the_ratio_rule(gb):
    """A policy whose log correction is zero sets exactly the ratio rule's
    rho at every decision: the solve is bitwise the ratio-rule solve."""
    import qpgen
    qp = qpgen.random_qp(100, 1000, 1)
    out = []
    for kw in ({}, dict(rho_policy=gb.RHO_LEARNED, policy_params=_constant_policy(0.0))):
        with gb.Solver(qp, **kw) as s:
            assert s.solve() == gb.SOLVED
            out.append((s.info()["iters"], s.info()["rho"], s.solution()[0]))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


POLICY = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.dirname(
    __import__("os").path.abspath(__file__))), "paper_1912_04263_gb300", "policy", "rho_policy.bin")


@pytest.mark.parametrize("seed", [200500, 200501, 200502])
def test_trained_policy_solutions_judged_by_oracle(gb, seed):
    """Held-out random QPs (seeds disjoint from training): the learned-rho
    FP32 solve meets the tolerances on the unscaled data and its objective
    lies within the convexity bound of the tight FP64 oracle optimum."""
    import qpgen
    from oracle import admm, checks
    params = gb.load_policy(POLICY)
    qp = qpgen.random_qp(1000, 10000, seed)
    with gb.Solver(qp, rho_policy=gb.RHO_LEARNED, policy_params=params) as s:
        assert s.solve() == gb.SOLVED
        x, y, z = s.solution()
        info = s.info()
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) and v.dual <= info["eps_dual"] * (1 + 1e-6)
    ref = admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=100000))
    f = admm.objective(qp.P, qp.q, x)
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, ref.x, ref.y)
    assert abs(f - ref.obj) <= 1.001 * bound + 1e-9
    assert abs(f - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj))


def test_trained_policy_gain_over_ratio_rule(gb):
    """What the trained network gains over the residual-ratio rule (Section
    3.4) on held-out QPs of the training family at n = 3000, m = 30000:
    fewer ADMM iterations and less device time, FP32 both ways; and the
    learned FP32 form is faster than the plain FP64 form."""
    import qpgen
    params = gb.load_policy(POLICY)
    tot = {"ratio": 0.0, "learned": 0.0, "fp64": 0.0}
    its = {"ratio": 0, "learned": 0}
    for seed in (200600, 200601):
        qp = qpgen.random_qp(3000, 30000, seed)
        for tag, kw in [("ratio", {}), ("learned", dict(rho_policy=gb.RHO_LEARNED, policy_params=params)),
                        ("fp64", dict(precision=gb.FP64))]:
            with gb.Solver(qp, **kw) as s:
                s.solve()
                assert s.solve() == gb.SOLVED
                info = s.info()
            tot[tag] += info["solve_ms"]
            if tag in its:
                its[tag] += info["iters"]
    print(f"\nlearned/ratio device time {tot['learned'] / tot['ratio']:.3f}, iterations "
          f"{its['learned']}/{its['ratio']}, learned FP32 / plain FP64 time {tot['learned'] / tot['fp64']:.3f}")
    assert its["learned"] <= its["ratio"]
    assert tot["learned"] <= 1.02 * tot["ratio"]
    assert tot["learned"] < tot["fp64"]


# ------------------------------------------------ on-device decisions replayed --

def _replay_decisions(gb, qp, flat, decisions):
    """Run a learned-policy FP32 solve with the host-driven loop, ten
    iterations (one rho decision) at a time, and replay every decision
    through the oracle's restatement (oracle.policy.decide) with the check
    values of the same state.  Returns the compared (device, oracle) pairs."""
    from oracle import admm, policy
    st = policy.PolicyState()
    pairs = []
    with gb.Solver(qp, precision=gb.FP32, loop_mode=gb.LOOP_HOST, rho_policy=gb.RHO_LEARNED,
                   policy_params=flat) as s:
        gb.gbosqp_set_iterates(s.h, np.zeros(qp.n), np.zeros(qp.m), np.zeros(qp.m), np.zeros(qp.n), 0.1)
        rho, lam = 0.1, 0.15
        for _ in range(decisions):
            status, per = gb.gbosqp_admm_iterations(s.h, 10)
            if status != 0:
                break
            c = gb.gbosqp_check(s.h)  # the residuals the decision read (iterates unchanged since)
            rho_dev = gb.gbosqp_get_iterates(s.h)[4]
            scaled = admm.Residuals(c["r_prim_s"], c["r_dual_s"], 0.0, 0.0, c["norm_Ax_s"], c["norm_z_s"],
                                    c["norm_Px_s"], c["norm_Aty_s"], c["norm_q_s"])
            rho_ref, lam_ref, used = policy.decide(flat, st, scaled, c["r_prim"], c["r_dual"], c["eps_prim"],
                                                   c["eps_dual"], rho, int(np.sum(per)), 10)
            lam = lam_ref if lam_ref is not None else lam
            dev = {"rho": rho_dev, "lambda": c["lambda"], "stalls": int(c["stall_count"]),
                   "fallbacks": int(c["fallbacks"])}
            ref = {"rho": rho_ref, "lambda": lam,
                   "stalls": st.stall_count, "fallbacks": st.fallbacks, "used": used}
            pairs.append((dev, ref))
            rho = rho_dev
    return pairs


def test_device_decisions_match_oracle_restatement(gb):
    """Every rho decision of a learned-policy solve (committed weights) equals
    the oracle's restatement of readings S11 and S12 on the same check: the
    new rho to 1e-6 relative (the device forms the features in FP32, the
    oracle in FP64, before the same BF16 rounding), lambda likewise, and the
    stall and fallback counters exactly."""
    import os
    flat = gb.load_policy(os.path.join(os.path.dirname(gb.__file__), "policy", "rho_policy.bin"))
    pairs = []
    for name in ["random_300x3000", "lasso_50x2000", "portfolio_3000x30"]:
        pairs += _replay_decisions(gb, qpgen.by_name(name, 0), flat, 12)
    assert len(pairs) >= 8
    assert any(r["used"] for _, r in pairs), "the network decided nowhere"
    for dev, ref in pairs:
        assert abs(dev["rho"] - ref["rho"]) <= 1e-6 * ref["rho"], (dev, ref)
        assert abs(dev["lambda"] - ref["lambda"]) <= 1e-6 * ref["lambda"], (dev, ref)
        assert dev["stalls"] == ref["stalls"] and dev["fallbacks"] == ref["fallbacks"], (dev, ref)


def test_overflowing_network_is_a_stall(gb):
    """Finite parameters (1e30) that overflow inside the network give a
    non-finite output: every decision the network would take counts as a
    stall and falls back to the ratio rule (reading S12), on the device as in
    the oracle, with the same stall and fallback counts at every decision."""
    flat = np.zeros(4622, np.float32)
    flat[4:8] = 1.0                                  # std
    off = 8 + 256                                    # W1 = 0
    flat[off:off + 64] = 1e30                        # b1: every hidden unit of layer 1 is 1e30
    off += 64
    flat[off:off + 4096] = 1e30                      # W2: layer 2 sums 64 x 1e60, past the FP32 range
    off += 4096 + 64
    flat[off:off + 128] = 1.0                        # W3
    off += 128 + 2
    flat[off:off + 4] = [np.log(10.0), 0.05, 0.5, 1.0]
    assert np.all(np.isfinite(flat))
    pairs = _replay_decisions(gb, qpgen.by_name("random_300x3000", 0), flat, 8)
    assert len(pairs) >= 4
    assert not any(r["used"] for _, r in pairs)
    for dev, ref in pairs:
        assert abs(dev["rho"] - ref["rho"]) <= 1e-12 * ref["rho"], (dev, ref)
        assert dev["stalls"] == ref["stalls"] and dev["fallbacks"] == ref["fallbacks"], (dev, ref)
    assert pairs[-1][0]["stalls"] >= 1 and pairs[-1][0]["fallbacks"] == len(pairs)


# -------------------------------------------- held-out learned-policy workload --

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_optima.json")


@pytest.mark.parametrize("seed", [200000, 200001, 200002])
def test_learned_policy_on_held_out_random_5000x50000(gb, seed):
    """The first seeds of the held-out evaluation (n = 5000, m = 50000): the
    learned FP32 solve reaches the eps = 1e-3 rule on the unscaled data, and
    its objective is judged against the FP64 oracle's optimum (committed by
    tests/golden/make_full_size_optima.py): within the convexity bound, and
    within 1e-3 relative where the oracle's own 1e-3 solve is."""
    import json
    from oracle import admm, checks
    key = f"random_5000x50000@{seed}"
    with open(GOLDEN) as f:
        gold = json.load(f).get(key)
    if gold is None:
        pytest.skip(f"no oracle optimum committed for {key}")
    qp = qpgen.by_name("random_5000x50000", seed)
    flat = gb.load_policy(os.path.join(os.path.dirname(gb.__file__), "policy", "rho_policy.bin"))
    with gb.Solver(qp, precision=gb.FP32, rho_policy=gb.RHO_LEARNED, policy_params=flat) as s:
        st = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert st == gb.SOLVED, info
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) + 1e-12 and v.dual <= info["eps_dual"] * (1 + 1e-6) + 1e-12
    t = gold["tight"]
    f = admm.objective(qp.P, qp.q, x)
    # ||x - x*||_1 from the committed x* (FP32: its rounding adds 2^-24 ||x*||_1),
    # else bounded by ||x||_1 + ||x*||_1
    dx = float(np.sum(np.abs(x))) + t["x_norm1"]
    xpath = os.path.join(os.path.dirname(GOLDEN), "full_size_xstar.npz")
    if os.path.exists(xpath):
        with np.load(xpath) as zf:
            if key in zf.files:
                dx = float(np.sum(np.abs(x - zf[key].astype(np.float64)))) + 2.0 ** -24 * t["x_norm1"]
    bound = max(float(np.sum(np.abs(y))), t["y_norm1"]) * v.prim + v.dual * dx
    assert abs(f - t["obj"]) <= 1.001 * bound + 1e-9 * max(1.0, abs(t["obj"])), (f, t["obj"], bound)
    if abs(gold["eps_1e-3"]["obj"] - t["obj"]) <= 1e-3 * max(1.0, abs(t["obj"])):
        assert abs(f - t["obj"]) <= 1e-3 * max(1.0, abs(t["obj"])), (f, t["obj"])
