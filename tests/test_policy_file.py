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
