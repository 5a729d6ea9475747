"""FP64 restatement of the learned rho decision and its stall rule.
TEST INFRASTRUCTURE.

The paper has no learned component (parity unpinned against the paper); this
module restates the decision as the solver's readings define it, so that the
device decisions can be compared with an independent implementation:

* Reading S11.  At a rho decision the network sees the standardised
  features (log ||r_prim||, log ||r_dual|| of the scaled problem, log rho,
  log(1 + PCG steps since the last decision)) with BF16 operands.  Output 0,
  clamped to [-clamp, clamp], is a log factor on the residual-ratio rule's
  proposal: rho_new = rho_ratio * exp(o0), clamped to [rho_min, rho_max].
  When the last parameter (use_lambda) is 1, output 1 sets the PCG
  tolerance weight lambda = 0.15 exp(o1), clamped to [lambda_min,
  lambda_max].
* Reading S12.  The merit is max(r_prim / eps_prim, r_dual / eps_dual) of
  the check.  If the network was to decide and the merit is not at most 0.9
  times the merit of the previous decision, or the network's output is not
  finite, that is a stall: the ratio rule decides for the next 50
  iterations, and after 3 stalls for the rest of the solve.  Every decision
  the ratio rule takes counts as a fallback.

The caller invokes ``decide`` at every check where the solve continues and
the iteration count is a multiple of rho_every.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import admm, mlp

N_PARAMS = 4622
LAMBDA0 = 0.15
STALL_ITERS = 50
STALL_LIMIT = 3
PROGRESS = 0.9


@dataclass
class PolicyState:
    stall_left: int = 0      # iterations for which the ratio rule still decides
    stall_count: int = 0
    disabled: bool = False
    prev_merit: float = 0.0  # merit at the previous decision (0: none yet)
    fallbacks: int = 0


def unpack(flat) -> dict:
    """The flat FP32 parameter vector in its documented order: feature mean
    (4), std (4), W1 (64 x 4), b1 (64), W2 (64 x 64), b2 (64), W3 (2 x 64),
    b3 (2), clamp, lambda_min, lambda_max, use_lambda."""
    v = np.asarray(flat, dtype=np.float64)
    if v.size != N_PARAMS:
        raise ValueError(f"expected {N_PARAMS} parameters, got {v.size}")
    out, off = {}, 0
    for name, shape in [("mean", (4,)), ("std", (4,)), ("W1", (64, 4)), ("b1", (64,)), ("W2", (64, 64)),
                        ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]:
        k = int(np.prod(shape))
        out[name] = v[off:off + k].reshape(shape)
        off += k
    out["clamp"], out["lambda_min"], out["lambda_max"], out["use_lambda"] = (float(t) for t in v[off:off + 4])
    return out


def features(r_prim_s: float, r_dual_s: float, rho: float, pcg_steps: int) -> np.ndarray:
    return np.array([math.log(max(r_prim_s, 1e-30)), math.log(max(r_dual_s, 1e-30)), math.log(rho),
                     math.log1p(pcg_steps)])


def decide(flat, st: PolicyState, scaled: "admm.Residuals", r_prim: float, r_dual: float, eps_prim: float,
           eps_dual: float, rho: float, pcg_steps: int, rho_every: int, rho_min: float = admm.RHO_MIN,
           rho_max: float = admm.RHO_MAX):
    """One decision.  ``scaled`` holds the scaled residuals and norms of the
    check (those the ratio rule reads); r_prim, r_dual, eps_prim, eps_dual
    are the unscaled ones of the termination test.  Updates ``st`` and
    returns (rho_new, lambda_new or None, used_network)."""
    p = unpack(flat)
    merit = max(r_prim / eps_prim, r_dual / eps_dual)
    use = (not st.disabled) and st.stall_left <= 0
    if st.stall_left > 0:
        st.stall_left -= rho_every
    if use and st.prev_merit > 0.0 and not (merit <= PROGRESS * st.prev_merit):
        _stall(st)
        use = False
    st.prev_merit = merit
    ratio = min(max(admm.rho_ratio_rule(rho, scaled), rho_min), rho_max)
    if use:
        x = mlp.bf16_round((features(scaled.r_prim, scaled.r_dual, rho, pcg_steps) - p["mean"]) / p["std"])
        o = mlp.forward_bf16(p, x[None, :])[0]
        if np.all(np.isfinite(o)):
            lm = min(max(o[0], -p["clamp"]), p["clamp"])
            rho_new = min(max(ratio * math.exp(lm), rho_min), rho_max)
            lam = None
            if p["use_lambda"] != 0.0:
                lam = min(max(LAMBDA0 * math.exp(o[1]), p["lambda_min"]), p["lambda_max"])
            return rho_new, lam, True
        _stall(st)
    st.fallbacks += 1
    return ratio, None, False


def _stall(st: PolicyState) -> None:
    st.stall_count += 1
    if st.stall_count >= STALL_LIMIT:
        st.disabled = True
    else:
        st.stall_left = STALL_ITERS
