"""Per-result tolerances of the integration parity tests (fp32 on the GPU against
the fp64 oracle on the same points).

Estimates:  |I32 - I64| <= 1e-6 |I64| + 1e-12 W, W = sum_c |w_c| (1 for the other
            integrands): the floor covers estimates that underflow in fp32.
Gradient means J (theta order w, mu, nu, sigma per component):
            |J32 - J64| <= tau (|J64| + [mu, nu] S64) + 3e-12 k
  where S = the oracle's grad_scale, the mean of the summed absolute values of
  the terms of df/dtheta: the mu and nu means cancel twice -- over the samples and
  inside each sample's sum of differences x_d - mu -- and each fp32 term carries
  rounding relative to the size of its parts, so their bound is relative to S;
  k = the component's constant factor (1, w/sigma^2, w/sigma^2, w/sigma^3) times
  the floor for means that underflow in fp32; tau = 1e-6 by default."""
import numpy as np


def est_tol(ref, W):
    return 1e-6 * np.abs(ref) + 1e-12 * W


def grad_tol(theta, J64, S64, tau=1e-6):
    theta = np.asarray(theta, np.float64).reshape(-1, 16)
    w, sg = theta[:, 0::4], theta[:, 3::4]
    scale = np.stack([np.ones_like(w), w / sg**2, w / sg**2, w / sg**3], axis=2).reshape(-1, 16)
    cancel = np.tile(np.array([0.0, 1.0, 1.0, 0.0]), 4)[None, :]
    return tau * (np.abs(J64) + cancel * S64) + 3e-12 * np.abs(scale)


def tau_needed(theta, J32, J64, S64):
    """The smallest tau for which every |J32 - J64| meets grad_tol, per parameter kind."""
    floor = grad_tol(theta, J64, S64, tau=0.0)
    cancel = np.tile(np.array([0.0, 1.0, 1.0, 0.0]), 4)[None, :]
    need = np.maximum(np.abs(J32 - J64) - floor, 0.0) / np.maximum(np.abs(J64) + cancel * S64, 1e-300)
    return {k: float(need[:, v::4].max()) for k, v in (("w", 0), ("mu", 1), ("nu", 2), ("sigma", 3))}
