"""The policy weight file (no GPU): round trip, the committed weights load
and are well formed (finite, positive feature scales, the clamp and lambda
range the device code expects), and a corrupted file is refused."""
import os

import numpy as np
import pytest

from paper_1912_04263_gb300 import binding as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMITTED = os.path.join(ROOT, "paper_1912_04263_gb300", "policy", "rho_policy.bin")


def test_round_trip(tmp_path):
    p = np.random.default_rng(0).standard_normal(gb.POLICY_PARAMS).astype(np.float32)
    path = str(tmp_path / "w.bin")
    gb.save_policy(path, p)
    assert np.array_equal(gb.load_policy(path), p)


def test_corrupt_or_foreign_files_are_refused(tmp_path):
    p = np.ones(gb.POLICY_PARAMS, np.float32)
    path = str(tmp_path / "w.bin")
    gb.save_policy(path, p)
    raw = bytearray((tmp_path / "w.bin").read_bytes())
    raw[100] ^= 0x40  # flip a payload bit: the CRC no longer matches
    bad = str(tmp_path / "bad.bin")
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        gb.load_policy(bad)
    other = str(tmp_path / "other.bin")
    (tmp_path / "other.bin").write_bytes(b"NOTAPOLICYFILE" + bytes(16))
    with pytest.raises(ValueError):
        gb.load_policy(other)


def test_committed_weights_are_well_formed():
    p = gb.load_policy(COMMITTED)
    assert p.shape == (gb.POLICY_PARAMS,) and np.all(np.isfinite(p))
    assert np.all(p[4:8] > 0.0)                      # feature scales
    clamp, lam_min, lam_max, use_lambda = p[-4:]
    assert clamp == pytest.approx(np.log(10.0))      # log-multiplier clamp
    assert 0.0 < lam_min < 0.15 < lam_max < 1.0      # lambda range around 0.15
    assert use_lambda in (0.0, 1.0)


def _layout():
    """The parameter order documented for GBOSQP_POLICY_PARAMS: feature mean
    (4), std (4), W1 (64 x 4), b1 (64), W2 (64 x 64), b2 (64), W3 (2 x 64),
    b3 (2), then clamp, lambda_min, lambda_max, use_lambda."""
    sizes = [("mean", 4), ("std", 4), ("W1", 256), ("b1", 64), ("W2", 4096), ("b2", 64), ("W3", 128), ("b3", 2),
             ("extra", 4)]
    out, off = {}, 0
    for name, k in sizes:
        out[name] = slice(off, off + k)
        off += k
    assert off == gb.POLICY_PARAMS
    return out


def test_trainer_initialisation_fills_the_documented_slots():
    """The trainer writes the flat vector in the order the device code reads:
    standardisation from the data, He-scaled weights, zero biases, and the
    clamp log 10, lambda in [0.05, 0.5] with the lambda output on."""
    from paper_1912_04263_gb300 import policy_train
    rng = np.random.default_rng(4)
    feats = rng.standard_normal((500, 4)) * [1.0, 2.0, 0.5, 3.0] + [-3.0, -5.0, -1.0, 2.0]
    p = policy_train.init_params(feats.astype(np.float32), seed=7)
    L = _layout()
    np.testing.assert_allclose(p[L["mean"]], feats.mean(axis=0), rtol=1e-5)
    np.testing.assert_allclose(p[L["std"]], feats.std(axis=0), rtol=1e-5)
    for b in ("b1", "b2", "b3"):
        assert not np.any(p[L[b]])
    for w, fan_in in (("W1", 4), ("W2", 64), ("W3", 64)):
        v = p[L[w]]
        assert np.all(v != 0.0)
        assert 0.8 < np.std(v) / np.sqrt(2.0 / fan_in) < 1.25  # He initialisation
    np.testing.assert_allclose(p[L["extra"]], [np.log(10.0), 0.05, 0.5, 1.0], rtol=1e-6)


def test_committed_weights_follow_the_layout():
    p = gb.load_policy(COMMITTED)
    L = _layout()
    assert np.all(p[L["std"]] > 0.0)
    np.testing.assert_allclose(p[L["extra"]][:3], [np.log(10.0), 0.05, 0.5], rtol=1e-6)
    assert p[L["extra"]][3] in (0.0, 1.0)
    # trained weights moved away from zero in every layer
    for w in ("W1", "W2", "W3"):
        assert np.count_nonzero(p[L[w]]) > 0.9 * (L[w].stop - L[w].start)
