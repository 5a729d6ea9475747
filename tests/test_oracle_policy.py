"""Pins of the oracle's restatement of the learned rho decision and its stall
rule (readings S11 and S12; no GPU), by hand-built networks whose decisions
are worked out by hand and by a hand-traced sequence of stalls."""
import math

import numpy as np
import pytest

from oracle import admm, policy


def _flat(b3=(0.0, 0.0), W1=0.0, W2=0.0, use_lambda=1.0):
    p = np.zeros(policy.N_PARAMS)
    p[4:8] = 1.0                                   # feature std
    p[8:8 + 256] = W1
    p[8 + 256 + 64:8 + 256 + 64 + 4096] = W2
    p[-6:-4] = b3
    p[-4:] = [math.log(10.0), 0.05, 0.5, use_lambda]
    return p


def _scaled(rp=4e-3, rd=1e-3):
    # the ratio rule proposes rho * sqrt(rp / rd) with unit normalisers: x2 here
    return admm.Residuals(rp, rd, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0)


def _decide(flat, st, merit, rho=0.1, scaled=None):
    # merit = max(r_prim / eps_prim, r_dual / eps_dual) with eps = 1
    return policy.decide(flat, st, scaled or _scaled(), merit, 0.0, 1.0, 1.0, rho, 7, 10)


def test_unpack_follows_the_documented_order():
    v = np.arange(policy.N_PARAMS, dtype=np.float64)
    p = policy.unpack(v)
    assert p["mean"].tolist() == [0, 1, 2, 3] and p["std"].tolist() == [4, 5, 6, 7]
    assert p["W1"][0, 0] == 8 and p["W1"][63, 3] == 8 + 255 and p["W1"][1, 0] == 12  # row major
    assert p["b1"][0] == 264 and p["W2"][0, 0] == 328 and p["b2"][0] == 328 + 4096
    assert p["W3"][1, 63] == 4488 + 127 and p["b3"].tolist() == [4616, 4617]
    assert (p["clamp"], p["lambda_min"], p["lambda_max"], p["use_lambda"]) == (4618, 4619, 4620, 4621)


def test_features_by_hand():
    f = policy.features(math.exp(-3.0), math.exp(-5.0), math.exp(0.5), 0)
    np.testing.assert_allclose(f, [-3.0, -5.0, 0.5, 0.0], rtol=0, atol=1e-15)
    assert policy.features(0.0, 1.0, 1.0, math.e - 1)[0] == math.log(1e-30)


def test_a_zero_network_is_the_ratio_rule():
    st = policy.PolicyState()
    rho, lam, used = _decide(_flat(), st, merit=100.0)
    assert used and rho == pytest.approx(0.2, rel=1e-14) and lam == pytest.approx(0.15, rel=1e-15)
    assert st.fallbacks == 0


def test_output_biases_scale_rho_and_lambda():
    st = policy.PolicyState()
    rho, lam, used = _decide(_flat(b3=(math.log(2.0), math.log(2.0))), st, merit=100.0)
    # biases are not rounded to BF16, so exp(b3) is exactly the factor
    assert used and rho == pytest.approx(0.4, rel=1e-12) and lam == pytest.approx(0.3, rel=1e-12)
    st = policy.PolicyState()
    rho, lam, _ = _decide(_flat(b3=(5.0, 5.0)), st, merit=100.0)
    assert rho == pytest.approx(2.0, rel=1e-12)        # clamped to x10 the ratio rule's 0.2
    assert lam == 0.5                                   # 0.15 e^5 clamped to lambda_max
    _, lam, _ = _decide(_flat(use_lambda=0.0), policy.PolicyState(), merit=100.0)
    assert lam is None


def test_rho_is_clamped_to_its_range():
    st = policy.PolicyState()
    rho, _, _ = policy.decide(_flat(b3=(5.0, 0.0)), st, _scaled(), 1.0, 0.0, 1.0, 1.0, 0.9e6, 0, 10)
    assert rho == admm.RHO_MAX


def test_stall_sequence_by_hand():
    """rho_every = 10.  Decision 1 has no previous merit; decision 2 improves
    by 20%; decision 3 by ~1%: stall 1, the ratio rule decides for the next
    50 iterations (decisions 3-8, counting the stalled one); decision 9
    uses the network again; two more stalls disable it for good."""
    flat, st = _flat(b3=(math.log(2.0), 0.0)), policy.PolicyState()
    used = [_decide(flat, st, m)[2] for m in [100.0, 80.0, 79.0]]
    assert used == [True, True, False] and st.stall_count == 1 and st.stall_left == 50
    used = [_decide(flat, st, m)[2] for m in [70.0, 60.0, 50.0, 40.0, 30.0]]
    assert used == [False] * 5 and st.stall_left == 0 and st.fallbacks == 6
    assert _decide(flat, st, 20.0)[2]                  # 20 <= 0.9 * 30: the network decides
    assert not _decide(flat, st, 19.0)[2]              # stall 2
    assert st.stall_count == 2 and st.stall_left == 50 and not st.disabled
    for m in [18.0, 17.0, 16.0, 15.0, 14.0]:
        _decide(flat, st, m)
    assert not _decide(flat, st, 13.9)[2]              # stall 3: 13.9 > 0.9 * 14
    assert st.disabled and st.stall_count == 3
    rho, _, used = _decide(flat, st, 1.0)              # big progress no longer matters
    assert not used and rho == pytest.approx(0.2, rel=1e-14)


@pytest.mark.filterwarnings("ignore:overflow encountered:RuntimeWarning",
                            "ignore:invalid value encountered:RuntimeWarning")
def test_a_non_finite_output_is_a_stall():
    """Finite weights near the FP32 limit overflow inside the network: the
    standardised features here (log 4e-3, log 1e-3, log 0.1, log 8) sum to
    about -12.6, so W1 = -3e38 gives pre-activations near +3.8e39, infinite
    once rounded through FP32 to BF16, and 0 * inf in the last layer is NaN.
    The output is not finite, the ratio rule decides and a stall is counted."""
    flat = _flat(W1=-3.0e38, W2=1.0)
    st = policy.PolicyState()
    rho, lam, used = _decide(flat, st, merit=100.0)
    assert not used and lam is None and rho == pytest.approx(0.2, rel=1e-14)
    assert st.stall_count == 1 and st.stall_left == 50 and st.fallbacks == 1
