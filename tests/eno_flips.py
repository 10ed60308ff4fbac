"""Stencil-choice flips of second-order ENO between the float32 kernel and
the FP64 oracle, and the bound they put on one time step.

ENO2 (paper Section 3.1.4) picks, on each side of a node, the second
difference of smaller magnitude.  That choice is a discontinuous function of
the data: where the two candidates are equal in magnitude up to float32
rounding, the float32 kernel and the FP64 oracle may pick different ones
from the same input window.  Both picks are valid ENO choices; they give
one-sided derivatives that differ by |s_a - s_b| / (2 h), s the candidate
second differences in value units.

For one stage of the Lax-Friedrichs update the right-hand side L is
Lipschitz in each one-sided derivative of axis d with constant alpha_d (the
dissipation bound of the axis bounds |f_d|), so a flip moves the node's
stage value by at most dt * alpha_d * |s_a - s_b| / (2 h_d).  `stage_flips`
finds the flips of one stage and this bound per node; `step_bound` combines
the two stages of TVD-RK2 (a stage-1 flip reaches the nodes within two cells
along each axis through stage 2's stencil).

Decisions are compared on the same window:

* the kernel's decision, in float32 with the kernel's differences
  (a = f0 - fm1, b = fp1 - f0; left a - (fm1 - fm2), centre b - a,
  right (fp2 - fp1) - b) and its float32 ghost nodes;
* the oracle's decision, the reading of the paper it implements (R10): the
  one-sided candidate wins only when its magnitude is smaller by more than
  2^-40 times the sum of the window's magnitudes.

A decision also counts as a flip when its two candidates are within `band`
(relative to the window's magnitudes) of a tie, so that rounding of the
stage input that the test cannot see (the kernel's own stage-1 values) is
covered.
"""
from __future__ import annotations

import numpy as np

TIE = 2.0 ** -40      # the oracle's tie margin (reading R10)
BAND_EXACT = 2.0 ** -21   # the stage input is the kernel's own float32 values
BAND_STAGE2 = 2.0 ** -17  # the stage input is the oracle's stand-in for them


def _shift(phi, axis, k):
    """phi at offset k along axis (periodic wrap), as np.roll does it."""
    return np.roll(phi, -k, axis=axis)


def windows(phi, axis, periodic):
    """The five-node window (i-2 .. i+2) of every node along `axis`, in the
    dtype of `phi`; ghost nodes on a non-periodic axis keep the sign of the
    boundary node (Section 3.1.1): g_k = phi_b + k sign(phi_b) |phi_b - phi_in|."""
    if periodic:
        return tuple(_shift(phi, axis, k) for k in (-2, -1, 0, 1, 2))
    n = phi.shape[axis]
    dt = phi.dtype.type
    take = lambda i: np.take(phi, [i], axis=axis)
    lo_b, lo_in = take(0), take(1 if n > 1 else 0)
    hi_b, hi_in = take(n - 1), take(n - 2 if n > 1 else 0)

    def ghost(pb, pin, k):
        sgn = np.where(pb >= 0, dt(1), dt(-1))
        return pb + (dt(k) * sgn) * np.abs(pb - pin)

    ext = np.concatenate([ghost(lo_b, lo_in, 2), ghost(lo_b, lo_in, 1), phi,
                          ghost(hi_b, hi_in, 1), ghost(hi_b, hi_in, 2)], axis=axis)
    sl = lambda a, b: np.take(ext, np.arange(a, b), axis=axis)
    return tuple(sl(k, k + n) for k in range(5))


def _kernel_picks(w):
    fm2, fm1, f0, fp1, fp2 = w
    a = f0 - fm1
    b = fp1 - f0
    left = a - (fm1 - fm2)
    mid = b - a
    right = (fp2 - fp1) - b
    return np.abs(left) < np.abs(mid), np.abs(right) < np.abs(mid)


def stage_flips(phi32, periodic, dz, alpha, dt, band):
    """Flips of one stage whose input is `phi32` (the kernel's float32
    values).  Returns (count, E): the number of flipped decisions and, per
    node, the bound on how far they move the node's stage value."""
    phi32 = np.ascontiguousarray(phi32, dtype=np.float32)
    phi64 = phi32.astype(np.float64)
    E = np.zeros(phi32.shape)
    count = 0
    for d in range(phi32.ndim):
        kl, kr = _kernel_picks(windows(phi32, d, periodic[d]))
        fm2, fm1, f0, fp1, fp2 = windows(phi64, d, periodic[d])
        s_l = f0 - 2.0 * fm1 + fm2
        s_m = fp1 - 2.0 * f0 + fm1
        s_r = fp2 - 2.0 * fp1 + f0
        mag = np.abs(fm2) + np.abs(fm1) + np.abs(f0) + np.abs(fp1) + np.abs(fp2)
        ol = np.abs(s_l) < np.abs(s_m) - TIE * mag
        orr = np.abs(s_r) < np.abs(s_m) - TIE * mag
        near_l = np.abs(np.abs(s_l) - np.abs(s_m)) <= band * mag
        near_r = np.abs(np.abs(s_r) - np.abs(s_m)) <= band * mag
        fl = ((kl != ol) | near_l) & (s_l != s_m)
        fr = ((kr != orr) | near_r) & (s_r != s_m)
        count += int(((kl != ol) & (s_l != s_m)).sum() + ((kr != orr) & (s_r != s_m)).sum())
        coef = dt * float(alpha[d]) / (2.0 * float(dz[d]))
        E += coef * (np.where(fl, np.abs(s_l - s_m), 0.0) + np.where(fr, np.abs(s_r - s_m), 0.0))
    return count, E


def dilate(E, periodic, radius=2):
    """max of E over the axis-aligned cross of `radius` cells around every
    node (the stencil of one ENO2 stage)."""
    out = E.copy()
    for d in range(E.ndim):
        for k in range(1, radius + 1):
            for s in (k, -k):
                if periodic[d]:
                    sh = np.roll(E, s, axis=d)
                else:
                    sh = np.zeros_like(E)
                    n = E.shape[d]
                    if k < n:
                        src = [slice(None)] * E.ndim
                        dst = [slice(None)] * E.ndim
                        if s > 0:
                            src[d], dst[d] = slice(0, n - k), slice(k, n)
                        else:
                            src[d], dst[d] = slice(k, n), slice(0, n - k)
                        sh[tuple(dst)] = E[tuple(src)]
                out = np.maximum(out, sh)
    return out


def step_bound(phi32, stage1_out, periodic, dz, alpha, dt, time_order):
    """Per-node bound on what ENO2 stencil-choice flips can change in one
    full step from the kernel's state `phi32`.  `stage1_out` is the oracle's
    first stage from that state (used for TVD-RK2's second stage).
    Returns (flips of stage 1, flips of stage 2, bound array)."""
    c1, E1 = stage_flips(phi32, periodic, dz, alpha, dt, BAND_EXACT)
    if time_order == 1:
        return c1, 0, E1
    c2, E2 = stage_flips(np.asarray(stage1_out, dtype=np.float32), periodic, dz, alpha, dt, BAND_STAGE2)
    return c1, c2, dilate(E1, periodic) + E2
