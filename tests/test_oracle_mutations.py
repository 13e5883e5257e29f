"""Planted mistakes in the oracle must fail at least one pin.

Each case patches one oracle function with a plausible slip (a dropped factor,
a flipped sign, a wrong update order) and runs the pins that should catch it.
This shows the pins in test_oracle_pins.py are strong enough to notice the
mistakes they are meant to notice.  Everything here runs on the CPU.
"""
import math

import numpy as np

import pytest

import oracle
import oracle.cac_mfz as om
import test_oracle_pins as pins


def _fails(check, *args):
    try:
        check(*args)
    except AssertionError:
        return True
    return False


def _inj_eta_half(j, e, R, h, eta, tau):
    return j * e * (R * h - (eta * eta / 2.0) * math.sqrt(tau))


def _inj_no_R(j, e, R, h, eta, tau):
    return j * e * (h - (eta * eta / 4.0) * math.sqrt(tau))


def _cn_sign(Goff, R, c, hz, tau):
    st = math.sqrt(tau)
    return +Goff @ (R * (c + st) / 4.0) + (st / 2.0) * hz[:, None]


def _cn_half(Goff, R, c, hz, tau):
    st = math.sqrt(tau)
    return -Goff @ (R * (c + st) / 2.0) + (st / 2.0) * hz[:, None]


def _bn_geq(Goff, R, c, hz, tau):
    st = math.sqrt(tau)
    return -(st / 2.0) * (Goff @ (R * (c >= 0.0)) - hz[:, None])


def _euler_sequential(c, e, p, inj, prm):
    c1 = c + prm.dt * ((-1.0 + p - c * c) * c + prm.K * inj)
    e1 = e + prm.dt * (-prm.beta * (c1 * c1 - prm.tau) * e)
    return c1, e1


def _brute_force_pin():
    # the correct oracle hits 8 of the 12 seeds of brute_force_hits()
    assert pins.brute_force_hits() >= 7


@pytest.mark.parametrize("name,target,fake,checks", [
    ("eta^2/2 threshold", "injection", _inj_eta_half, ["separable_cn"]),
    ("R_r dropped from injection", "injection", _inj_no_R, ["separable_cn", "brute"]),
    ("coupling sign flipped", "local_field_cn", _cn_sign, ["J", "brute"]),
    ("coupling halved 1/4 -> 1/2", "local_field_cn", _cn_half, ["J", "three"]),
    ("H(0) = 1 in the binarised field", "local_field_bn", _bn_geq, ["three"]),
    ("e updated from the new c", "euler_step", _euler_sequential, ["three"]),
])
def test_planted_mistake_is_caught(monkeypatch, name, target, fake, checks):
    monkeypatch.setattr(om, target, fake)
    monkeypatch.setattr(oracle, target, fake)
    table = {
        "separable_cn": (pins.test_separable_case_is_hard_threshold, "cn"),
        "brute": (_brute_force_pin,),
        "J": (pins.test_coupling_J_symmetric_zero_diagonal,),
        "three": (pins.test_three_spin_hand_worked_step,),
    }
    caught = [c for c in checks if _fails(*table[c])]
    assert caught, f"planted mistake '{name}' passed every pin in {checks}"


def test_planted_refit_mistake_is_caught(monkeypatch):
    orig = om.refit_exact

    def wrong(G, hz, g, sigma):
        R, s = orig(G, hz, g, sigma)
        off = sigma == 0
        R = R.copy()
        R[off] = hz[off] / g[off]  # forgets the coupling to the support
        return R, s

    monkeypatch.setattr(om, "refit_exact", wrong)
    monkeypatch.setattr(oracle, "refit_exact", wrong)
    assert _fails(pins.test_refit_matches_lstsq_and_is_jacobi_fixed_point)


def _jacobi_undamped(Goff, hz, g, sigma, R, dtc, iters):
    s = sigma.astype(float)
    for _ in range(iters):
        R = (hz - Goff @ (s * R)) / g
    return R


def _jacobi_complement_step(Goff, hz, g, sigma, R, dtc, iters):
    s = sigma.astype(float)
    for _ in range(iters):
        R = R + (1.0 - dtc) * ((hz - Goff @ (s * R)) / g - R)
    return R


def _jacobi_ignores_sigma(Goff, hz, g, sigma, R, dtc, iters):
    for _ in range(iters):
        R = R + dtc * ((hz - Goff @ R) / g - R)
    return R


def _jacobi_gauss_seidel(Goff, hz, g, sigma, R, dtc, iters):
    s = sigma.astype(float)
    R = R.copy()
    for _ in range(iters):
        for r in range(R.size):
            R[r] = R[r] + dtc * ((hz[r] - Goff[r] @ (s * R)) / g[r] - R[r])
    return R


def _jacobi_extra_sweep(Goff, hz, g, sigma, R, dtc, iters):
    s = sigma.astype(float)
    for _ in range(iters + 1):
        R = R + dtc * ((hz - Goff @ (s * R)) / g - R)
    return R


@pytest.mark.parametrize("fake", [_jacobi_undamped, _jacobi_complement_step, _jacobi_ignores_sigma,
                                  _jacobi_gauss_seidel, _jacobi_extra_sweep])
def test_planted_jacobi_mistake_is_caught(monkeypatch, fake):
    """An undamped sweep, the step applied as (1 - dtc), the support ignored, an
    in-place (Gauss-Seidel) sweep and one sweep too many each fail the hand-worked
    two-sweep pin."""
    monkeypatch.setattr(om, "refit_jacobi", fake)
    monkeypatch.setattr(oracle, "refit_jacobi", fake)
    assert _fails(pins.test_damped_jacobi_two_sweeps_hand_worked)


def _corr_half(g, R, tau):
    return (math.sqrt(tau) / 2.0) * g[:, None] * R * R


def _readout_no_diagonal(Goff, g, hz, R, sigma, lam):
    x = sigma * R
    return 0.5 * np.sum(x * (Goff @ x), axis=0) - hz @ x + lam * np.sum(sigma, axis=0)


def test_planted_self_term_mistake_is_caught(monkeypatch):
    """The correction with 1/2 in place of 1/4 fails the hand-worked step and the
    separable case of the corrected mode."""
    monkeypatch.setattr(om, "self_term_correction", _corr_half)
    monkeypatch.setattr(oracle, "self_term_correction", _corr_half)
    assert _fails(pins.test_three_spin_hand_worked_step)
    assert _fails(pins.test_separable_case_corrected_mode_is_the_objective_threshold, "cn")


def test_planted_readout_mistake_is_caught(monkeypatch):
    """A readout energy without the diagonal term fails the trajectory pin."""
    monkeypatch.setattr(om, "readout_energy", _readout_no_diagonal)
    monkeypatch.setattr(oracle, "readout_energy", _readout_no_diagonal)
    assert _fails(pins.test_best_readout_is_the_first_lowest_objective_on_the_trajectory, "bn")


def _cg_beta_inverted(G, hz, g, sigma, R, iters, tol):
    S = np.flatnonzero(sigma)
    R = np.array(R, dtype=float)
    Gss, b, x = G[np.ix_(S, S)], hz[S], R[S].copy()
    r = b - Gss @ x
    p, rr = r.copy(), float(r @ r)
    for _ in range(iters):
        q = Gss @ p
        a = rr / float(p @ q)
        x, r = x + a * p, r - a * q
        rn = float(r @ r)
        p, rr = r + (rr / rn) * p, rn
    R[S] = x
    off = sigma == 0
    R[off] = (hz[off] - G[np.ix_(off, S)] @ x) / g[off]
    return R


def _cg_cold_start(G, hz, g, sigma, R, iters, tol):
    return om_refit_cg_orig(G, hz, g, sigma, np.zeros_like(R), iters, tol)


om_refit_cg_orig = om.refit_cg


@pytest.mark.parametrize("fake", [_cg_beta_inverted, _cg_cold_start])
def test_planted_cg_mistake_is_caught(monkeypatch, fake):
    """An inverted beta and a start from zero instead of the trial's R fail the
    hand-worked two-step pin."""
    monkeypatch.setattr(om, "refit_cg", fake)
    monkeypatch.setattr(oracle, "refit_cg", fake)
    assert _fails(pins.test_cg_refit_two_steps_hand_worked)


def _fista_no_momentum(G, hz, lam1, iters):
    L = float(np.max(np.sum(np.abs(G), axis=1)))
    x = np.zeros_like(hz)
    for _ in range(iters):
        v = x - (G @ x - hz) / L
        x = np.sign(v) * np.maximum(np.abs(v) - lam1 / L, 0.0)
    return x


def _fista_threshold_unscaled(G, hz, lam1, iters):
    L = float(np.max(np.sum(np.abs(G), axis=1)))
    x = np.zeros_like(hz)
    z, t = x.copy(), 1.0
    for _ in range(iters):
        v = z - (G @ z - hz) / L
        xn = np.sign(v) * np.maximum(np.abs(v) - lam1, 0.0)
        tn = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z, x, t = xn + ((t - 1.0) / tn) * (xn - x), xn, tn
    return x


@pytest.mark.parametrize("fake", [_fista_no_momentum, _fista_threshold_unscaled])
def test_planted_fista_mistake_is_caught(monkeypatch, fake):
    """Plain ISTA (no momentum) and a threshold not divided by L fail the three-step pin."""
    monkeypatch.setattr(om, "lasso_fista", fake)
    monkeypatch.setattr(oracle, "lasso_fista", fake)
    assert _fails(pins.test_fista_three_steps_hand_worked)
