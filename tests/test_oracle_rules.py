"""Pins of the oracle's step-size and tolerance rules (no GPU).  These
functions steer the iteration but not its limit, so the solution pins cannot
catch a mistake in them; each is pinned here by a value worked out by hand,
an invariant the rule must have, or an inequality checked at random points."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import admm, checks, mlp


def _res(rp, rd, nAx=1.0, nz=1.0, nPx=1.0, nAty=1.0, nq=1.0):
    return admm.Residuals(rp, rd, 0.0, 0.0, nAx, nz, nPx, nAty, nq)


# ------------------------------------------------ residuals (Section 3.1) --

def test_residuals_hand_worked_example():
    """P = [2], q = [1], A = [1; 2], x = 1, z = (1, 5), y = (2, -3):
    Ax - z = (0, -3), Px + q + A'y = 2 + 1 - 4 = -1; norms ||Ax|| = 2,
    ||z|| = 5, ||Px|| = 2, ||A'y|| = 4, ||q|| = 1, so with eps_abs = 1e-3 and
    eps_rel = 1e-2: eps_prim = 1e-3 + 5e-2, eps_dual = 1e-3 + 4e-2."""
    P = sp.csr_matrix([[2.0]])
    A = sp.csr_matrix([[1.0], [2.0]])
    r = admm.residuals(P, np.array([1.0]), A, np.array([1.0]), np.array([1.0, 5.0]),
                       np.array([2.0, -3.0]), eps_abs=1e-3, eps_rel=1e-2)
    assert (r.r_prim, r.r_dual) == (3.0, 1.0)
    assert (r.norm_Ax, r.norm_z, r.norm_Px, r.norm_Aty, r.norm_q) == (2.0, 5.0, 2.0, 4.0, 1.0)
    assert r.eps_prim == pytest.approx(0.051, rel=1e-15)
    assert r.eps_dual == pytest.approx(0.041, rel=1e-15)
    assert not r.converged()


# -------------------------------------------- residual-ratio rule (Sec. 3.4) --

def test_rho_rule_keeps_rho_when_relative_residuals_balance():
    for rho in (1e-3, 0.1, 7.0):
        assert admm.rho_ratio_rule(rho, _res(2e-3, 5e-4, nAx=4.0, nz=1.0, nPx=0.5, nq=1.0)) == pytest.approx(rho)


def test_rho_rule_direction_and_square_root():
    """A primal residual that is 4x (relatively) the dual one doubles rho; the
    reverse halves it (rho grows when primal infeasibility dominates)."""
    assert admm.rho_ratio_rule(0.1, _res(4e-3, 1e-3)) == pytest.approx(0.2, rel=1e-14)
    assert admm.rho_ratio_rule(0.1, _res(1e-3, 4e-3)) == pytest.approx(0.05, rel=1e-14)


def test_rho_rule_normalises_by_the_largest_norm_of_each_side():
    # prim normaliser max(||Ax||, ||z||) = 8 whichever holds it; dual max = 2
    for kw in (dict(nAx=8.0, nz=0.5), dict(nAx=0.5, nz=8.0)):
        for kd in (dict(nPx=2.0, nAty=0.1, nq=0.1), dict(nPx=0.1, nAty=2.0, nq=0.1),
                   dict(nPx=0.1, nAty=0.1, nq=2.0)):
            # (rp / 8) / (rd / 2) = 4  ->  factor 2
            assert admm.rho_ratio_rule(1.0, _res(16.0, 1.0, **kw, **kd)) == pytest.approx(2.0, rel=1e-14)


def test_rho_rule_is_scale_invariant_per_side():
    base = admm.rho_ratio_rule(0.3, _res(3e-2, 2e-3, nAx=5.0, nz=2.0, nPx=1.0, nAty=4.0, nq=3.0))
    for s in (1e-3, 10.0, 1e5):
        assert admm.rho_ratio_rule(0.3, _res(3e-2 * s, 2e-3, nAx=5.0 * s, nz=2.0 * s, nPx=1.0, nAty=4.0,
                                             nq=3.0)) == pytest.approx(base, rel=1e-13)
        assert admm.rho_ratio_rule(0.3, _res(3e-2, 2e-3 * s, nAx=5.0, nz=2.0, nPx=1.0 * s, nAty=4.0 * s,
                                             nq=3.0 * s)) == pytest.approx(base, rel=1e-13)


def test_rho_rule_clamps_and_degenerate_cases():
    assert admm.rho_ratio_rule(1e5, _res(1e6, 1e-6)) == admm.RHO_MAX
    assert admm.rho_ratio_rule(1e-5, _res(1e-6, 1e6)) == admm.RHO_MIN
    # zero dual residual or zero normaliser: no information, rho unchanged
    assert admm.rho_ratio_rule(0.4, _res(1.0, 0.0)) == 0.4
    assert admm.rho_ratio_rule(0.4, _res(1.0, 1.0, nAx=0.0, nz=0.0)) == 0.4
    assert admm.rho_ratio_rule(0.4, _res(1.0, 1.0, nPx=0.0, nAty=0.0, nq=0.0)) == 0.4


# ------------------------------------------- PCG tolerance (Section 5.3.4) --

def test_pcg_tolerance_is_a_floored_geometric_mean():
    assert admm.pcg_tolerance(4.0, 1.0) == pytest.approx(0.3, rel=1e-15)   # 0.15 * sqrt(4)
    assert admm.pcg_tolerance(1.0, 4.0) == pytest.approx(0.3, rel=1e-15)
    assert admm.pcg_tolerance(2e-3, 2e-3) == pytest.approx(3e-4, rel=1e-14)
    # the geometric mean is unchanged when one residual grows as the other shrinks
    assert admm.pcg_tolerance(8e-2 * 9, 2e-4 / 9) == pytest.approx(admm.pcg_tolerance(8e-2, 2e-4), rel=1e-14)
    # floor
    assert admm.pcg_tolerance(1e-12, 1e-12) == 1e-7
    assert admm.pcg_tolerance(1e-12, 1e-12, eps_min=1e-9) == 1e-9
    assert admm.pcg_tolerance(4.0, 1.0, lam=0.5) == pytest.approx(1.0, rel=1e-15)


# ------------------------------------------- Ruiz limits (Algorithm 2, S4) --

def test_limit_scaling_special_values():
    v = admm.limit_scaling([0.0, 5e-5, 1e-4, 0.5, 1.0, 1e4, 3e6])
    assert v.tolist() == [1.0, 1.0, 1e-4, 0.5, 1.0, 1e4, 1e4]


def test_row_and_column_norms_on_a_hand_matrix():
    M = sp.csr_matrix(np.array([[0.0, -3.0, 1.0], [0.0, 0.0, 0.0], [2.0, 0.5, -4.0]]))
    assert admm.row_inf_norms(M).tolist() == [3.0, 0.0, 4.0]
    assert admm.col_inf_norms(M).tolist() == [2.0, 3.0, 4.0]
    assert admm.norm_inf(np.array([])) == 0.0
    assert admm.norm_inf(np.array([1.0, -2.5])) == 2.5


# --------------------------------------------------------- Adam (policy) --

def test_adam_steps_with_a_constant_gradient_are_lr_times_sign():
    """With bias correction the moment estimates of a constant gradient g are
    exactly g and g^2 at every step t, so every step moves a parameter by
    -lr g / (|g| + eps) (Kingma and Ba, Algorithm 1)."""
    g = {"W": np.array([[0.3, -2.0], [1e-4, -7e-3]]), "b": np.array([5.0, -0.25])}
    p = {k: np.zeros_like(v) for k, v in g.items()}
    state = {}
    for t in range(1, 6):
        prev = {k: v.copy() for k, v in p.items()}
        p = mlp.adam_step(p, g, state, t, lr=1e-2)
        for k in g:
            np.testing.assert_allclose(p[k] - prev[k], -1e-2 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-10)


def test_adam_second_step_after_the_gradient_vanishes():
    """Gradient g at step 1, then 0 at step 2: m2 = b1 (1 - b1) g and
    v2 = b2 (1 - b2) g^2, so after bias correction the second step is
    -lr (b1 / (1 + b1)) g / (sqrt(b2 / (1 + b2)) |g| + eps)."""
    b1, b2, lr, eps = 0.9, 0.999, 1e-3, 1e-8
    g = {"w": np.array([0.7, -3.0, 2e-2])}
    p = {"w": np.zeros(3)}
    state = {}
    p = mlp.adam_step(p, g, state, 1, lr=lr, b1=b1, b2=b2, eps=eps)
    before = p["w"].copy()
    p = mlp.adam_step(p, {"w": np.zeros(3)}, state, 2, lr=lr, b1=b1, b2=b2, eps=eps)
    gw = g["w"]
    want = -lr * (b1 / (1 + b1)) * gw / (math.sqrt(b2 / (1 + b2)) * np.abs(gw) + eps)
    np.testing.assert_allclose(p["w"] - before, want, rtol=1e-10)


# ---------------------------------------- objective error bound (checker) --

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_objective_error_bound_holds_at_random_points(seed):
    """For any x and any (z, y) with z in [l, u] and y in the normal cone of
    [l, u] at z, |f(x) - f*| is within the convexity bound.  Checked at random
    x with (z, y) = (z*, y*) and with (z, y) = (proj(Ax), 0); the dual term
    of the bound is needed (it alone exceeds the error at some points)."""
    qp = qpgen.tiny_qp(4, 7, seed, n_eq=1, n_inf=2)
    xs, ys = checks.brute_force(qp)
    zs = qp.A @ xs
    fs = admm.objective(qp.P, qp.q, xs)
    rng = np.random.default_rng(seed)
    dual_needed = False
    for _ in range(200):
        x = xs + rng.standard_normal(qp.n) * 10.0 ** rng.uniform(-4, 0)
        for z, y in ((zs, ys), (np.clip(qp.A @ x, qp.l, qp.u), np.zeros(qp.m))):
            rp = float(np.max(np.abs(qp.A @ x - z)))
            rd = float(np.max(np.abs(qp.P @ x + qp.q + qp.A.T @ y)))
            err = abs(admm.objective(qp.P, qp.q, x) - fs)
            bound = checks.objective_error_bound(x, y, rp, rd, xs, ys)
            assert err <= bound * (1 + 1e-9) + 1e-12
            prim_only = max(np.sum(np.abs(ys)), np.sum(np.abs(y))) * rp
            dual_needed |= err > prim_only * (1 + 1e-6) + 1e-12
    assert dual_needed
    assert checks.objective_error_bound(xs, ys, 0.0, 0.0, xs, ys) == 0.0


# ------------------------------------------------ MLP forward (policy) --

def _hand_network():
    """Layer 1 copies the 4 inputs into units 0-3; layer 2 rotates them
    (unit i takes unit (i + 1) mod 4); layer 3 weighs them.  With input
    x, h1 = relu(x) and h2_i = relu(x_{(i+1) mod 4}) on units 0-3, so
    o0 = 1 h2_0 - 1 h2_1 + 2 h2_2 + 0.5 h2_3 + 0.25 and
    o1 = h2_3 - 1."""
    p = {k: np.zeros(s) for k, s in mlp.PARAM_SHAPES.items()}
    for i in range(4):
        p["W1"][i, i] = 1.0
        p["W2"][i, (i + 1) % 4] = 1.0
    p["W3"][0, :4] = [1.0, -1.0, 2.0, 0.5]
    p["W3"][1, 3] = 1.0
    p["b3"][:] = [0.25, -1.0]
    return p


@pytest.mark.parametrize("x,o", [
    ([1.0, 2.0, -3.0, 4.0], [2.0 - 0.0 + 2.0 * 4.0 + 0.5 * 1.0 + 0.25, 1.0 - 1.0]),   # h2 = (2, 0, 4, 1)
    ([-1.0, -2.0, 0.5, 0.25], [0.0 - 0.5 + 0.5 + 0.0 + 0.25, 0.0 - 1.0]),             # h2 = (0, .5, .25, 0)
    ([3.0, 0.0, 0.0, -8.0], [0.0 - 0.0 + 0.0 + 0.5 * 3.0 + 0.25, 3.0 - 1.0]),          # h2 = (0, 0, 0, 3)
])
def test_mlp_forward_on_a_hand_built_network(x, o):
    p = _hand_network()
    out, _ = mlp.forward(p, np.array([x]))
    assert out[0].tolist() == o
    # every value here is exact in BF16, so the BF16 forward gives the same numbers
    assert mlp.forward_bf16(p, np.array([x]))[0].tolist() == o


def test_masked_mse_loss_by_hand():
    """loss = sum_k w_k (o_k - t_k)^2 / (2B) with B = 2 samples:
    (1 * 1^2 + 0.5 * 2^2 + 0 * 3^2 + 2 * (-1)^2) / 4 = 5 / 4; dL/do = w (o - t) / B."""
    out = np.array([[1.0, 2.0], [3.0, -1.0]])
    tgt = np.zeros((2, 2))
    w = np.array([[1.0, 0.5], [0.0, 2.0]])
    loss, g = mlp.loss_and_grad_out(out, tgt, w)
    assert loss == 1.25
    assert g.tolist() == [[0.5, 0.5], [0.0, -1.0]]
