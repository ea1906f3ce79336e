"""Pins of the oracle's three time solvers (paper, section "Code G-MHD3D" and Table I: Adams-Bashforth,
Runge-Kutta 4 and predictor-corrector, "checked to provide identical results").

* discrete pin: on a small sound wave the oracle follows, step by step, each method's recursion for
  the linear system y' = A y (RK4: the degree-4 Taylor polynomial of exp(dt A); predictor-corrector:
  AB2 predictor, trapezoidal corrector), for fixed and CFL-variable dt;
* order pin: on a nonlinear state the error falls by 16 (RK4) and 4 (PC, AB2) per halving of dt;
* the paper's agreement statement: the three methods agree to their truncation error, which falls
  as dt^2.
"""
import numpy as np
import pytest

import test_oracle_invariants as inv
import test_oracle_linear_waves as lw
from paper_1810_12707_gb300.inputs import grid

AB2, RK4, PC = 0, 1, 2


def linear_run(A, y0, dts, method):
    y = np.array(y0, dtype=np.complex128)
    f_prev = dt_prev = None
    I = np.eye(len(y0))
    for dt in dts:
        f = A @ y
        if method == RK4:
            hA = dt * A
            P = I + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
            y = P @ y
        else:
            if f_prev is None:
                ystar = y + dt * f
            else:
                r = dt / dt_prev
                ystar = y + dt * ((1 + 0.5 * r) * f - 0.5 * r * f_prev)
            y = ystar if method == AB2 else y + 0.5 * dt * (f + A @ ystar)
        f_prev, dt_prev = f, dt
    return y


@pytest.mark.parametrize("method", [RK4, PC])
@pytest.mark.parametrize("fixed_dt", [True, False])
def test_sound_wave_follows_the_linear_recursion(oracle_mod, method, fixed_dt):
    n, k, cs, nu = 16, 2, 1.3, 0.02
    X = grid(n)[1]
    o = oracle_mod.Oracle(n, nu, 0.01, cs, dt=0.01 if fixed_dt else 0.0, integrator=method)
    o.set_state(1.0 + lw.EPS * np.cos(k * X), np.zeros((3, n, n, n)), np.zeros((3, n, n, n)))
    dts = lw.run_oracle(o, 60, fixed_dt)
    A = np.array([[0, -1j * k], [-1j * k * cs ** 2, -nu * k * k]])
    y = linear_run(A, [lw.EPS / 2, 0.0], dts, method)
    i = lw.idx(n, 1, k)
    got = np.array([o.spectrum(0)[i], o.spectrum(2)[i]])
    assert np.max(np.abs(got - y)) <= 1e-5 * np.max(np.abs(y)), (got, y)
    # the recursions of the three methods are really different at this dt
    other = linear_run(A, [lw.EPS / 2, 0.0], dts, AB2)
    assert np.max(np.abs(other - y)) > 1e-4 * np.max(np.abs(y))


def _solution(oracle_mod, method, dt, t_end=0.08):
    n = 16
    state = inv.smooth_state(n, 5)
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0, dt=dt, integrator=method)
    o.set_state(*state)
    o.step(int(round(t_end / dt)))
    return np.concatenate([np.ravel(a) for a in o.get_state()])


@pytest.mark.parametrize("method,order", [(RK4, 4), (PC, 2)])
def test_convergence_order(oracle_mod, method, order):
    dts = (0.008, 0.004, 0.002, 0.001) if method == RK4 else (0.004, 0.002, 0.001, 0.0005)
    sols = [_solution(oracle_mod, method, dt) for dt in dts]
    d = [np.linalg.norm(a - c) for a, c in zip(sols, sols[1:])]
    ratios = [d0 / d1 for d0, d1 in zip(d, d[1:])]
    want = 2.0 ** order
    assert all(0.85 * want < r < 1.15 * want for r in ratios), ratios


def test_three_solvers_agree_to_their_truncation_error(oracle_mod):
    """The paper reports identical results from its Adams-Bashforth, RK4 and predictor-corrector
    solvers; in exact terms they agree up to O(dt^2), which this checks by halving dt."""
    gaps = []
    for dt in (0.002, 0.001):
        a, r, p = (_solution(oracle_mod, m, dt) for m in (AB2, RK4, PC))
        scale = np.linalg.norm(r)
        gaps.append((np.linalg.norm(a - r) / scale, np.linalg.norm(p - r) / scale))
        assert gaps[-1][0] < 1e-4 and gaps[-1][1] < 1e-4
    assert 3.0 < gaps[0][0] / gaps[1][0] < 5.0
    assert 3.0 < gaps[0][1] / gaps[1][1] < 5.0
