"""Pins of the oracle's tracer particles (paper, section "Tracer Particles": cloud-in-cell
interpolation, Eq. tracer_eq; Boris push with q = M = 1 and no electric field, Eq. boris; position
update, Eq. euler; periodic box).

* interpolation: exact at grid points and for constant fields; for a field that depends on x only
  it is numpy's periodic linear interpolation; for a product g1(x) g2(y) g3(z) it is the product of
  the three 1D linear interpolants (the tensor-product property that fixes every corner weight);
* the initial velocity is the interpolated grid velocity;
* push: in uniform u and B (a steady state of the equations) the velocity turns about B by exactly
  2 atan(|B| dt / 2) per step (the Boris rotation), so after n steps it is a Rodrigues rotation of
  the initial velocity, and the position is the wrapped sum of dt v_k;
* with B = 0 tracers move in straight lines through the periodic boundaries;
* in a turbulent field the speed of every tracer is conserved (a pure rotation per step).
"""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

L = 2 * np.pi


def uniform_state(om, n, U, B, dt, lib=None):
    o = om.Oracle(n, 0.01, 0.01, 1.0, dt=dt, lib=lib)
    o.set_state(np.ones((n, n, n)), np.broadcast_to(np.asarray(U)[:, None, None, None], (3, n, n, n)).copy(),
                np.broadcast_to(np.asarray(B)[:, None, None, None], (3, n, n, n)).copy())
    return o


def rotation(axis, angle):
    a = np.asarray(axis, dtype=float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def interp_periodic(xs, vals, x):
    return np.interp(np.mod(x, L), np.append(xs, L), np.append(vals, vals[0]))


def interpolation_failures(om, lib=None):
    failed = []
    n = 16
    X, Y, Z = inputs.grid(n)
    xs = 2 * np.pi * np.arange(n) / n
    rng = np.random.default_rng(4)
    pos = rng.uniform(-1.0, L + 1.0, (40, 3))  # some outside the box: wrapped
    # constant field
    o = uniform_state(om, n, [0.1, 0.2, 0.3], [0.7, -0.4, 1.1], 0.01, lib)
    if np.max(np.abs(o.tracer_field("B", pos) - [0.7, -0.4, 1.1])) > 1e-14:
        failed.append("constant")
    # B_z = sin(3x) + 0.2 cos(x): numpy's linear interpolation along x
    b = np.zeros((3, n, n, n))
    b[2] = np.sin(3 * X) + 0.2 * np.cos(X)
    o = om.Oracle(n, 0.01, 0.01, 1.0, lib=lib)
    o.set_state(np.ones((n, n, n)), np.zeros((3, n, n, n)), b)
    got = o.tracer_field("B", pos)[:, 2]
    want = interp_periodic(xs, np.sin(3 * xs) + 0.2 * np.cos(xs), pos[:, 0])
    if np.max(np.abs(got - want)) > 1e-13:
        failed.append("linear in x")
    # u_x = g1(x) g2(y) g3(z): product of the 1D interpolants; also the tracers' initial velocity
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(X) * np.cos(2 * Y) * np.sin(Z + 0.3)
    u[1] = np.cos(3 * Z) * (1.0 + 0.5 * np.sin(Y))
    o = om.Oracle(n, 0.01, 0.01, 1.0, lib=lib)
    o.set_state(np.ones((n, n, n)), u, np.zeros((3, n, n, n)))
    got = o.tracer_field("u", pos)
    wx = (interp_periodic(xs, np.sin(xs), pos[:, 0]) * interp_periodic(xs, np.cos(2 * xs), pos[:, 1]) *
          interp_periodic(xs, np.sin(xs + 0.3), pos[:, 2]))
    wy = interp_periodic(xs, np.cos(3 * xs), pos[:, 2]) * interp_periodic(xs, 1.0 + 0.5 * np.sin(xs), pos[:, 1])
    if np.max(np.abs(got[:, 0] - wx)) > 1e-13 or np.max(np.abs(got[:, 1] - wy)) > 1e-13:
        failed.append("tensor product")
    o.tracers_set(pos)
    p0, v0 = o.tracers_get()
    if np.max(np.abs(v0 - got)) > 0 or np.max(np.abs(p0 - np.mod(pos, L))) > 1e-15:
        failed.append("initial velocity")
    # exact at grid points
    gp = np.stack([xs[rng.integers(0, n, 20)] for _ in range(3)], axis=1)
    idx = np.rint(gp / (L / n)).astype(int)
    want = np.stack([u[a][idx[:, 2], idx[:, 1], idx[:, 0]] for a in range(3)], axis=1)
    if np.max(np.abs(o.tracer_field("u", gp) - want)) > 1e-14:
        failed.append("grid points")
    return failed


def push_failures(om, lib=None):
    failed = []
    n, dt, steps = 16, 0.013, 40
    U = np.array([0.3, -0.2, 0.45])
    B = np.array([0.8, -1.1, 1.7])
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, L, (6, 3))
    o = uniform_state(om, n, U, B, dt, lib)
    o.tracers_set(pos)
    o.step(steps)
    p, v = o.tracers_get()
    # dv/dt = v x B turns v about B in the negative sense
    theta = 2 * np.arctan(np.linalg.norm(B) * dt / 2)
    vk = [rotation(B, -theta * k) @ U for k in range(1, steps + 1)]
    want_v = vk[-1]
    want_p = np.mod(pos + dt * np.sum(vk, axis=0), L)
    dp = np.abs(p - want_p)
    dp = np.minimum(dp, L - dp)
    if np.max(np.abs(v - want_v)) > 1e-13 or np.max(dp) > 1e-12:
        failed.append("boris rotation")
    # B = 0: straight lines through the periodic boundaries
    o = uniform_state(om, n, [1.3, -0.7, 2.9], [0, 0, 0], 0.05, lib)
    o.tracers_set(pos)
    o.step(60)
    p, _ = o.tracers_get()
    want = np.mod(pos + 60 * 0.05 * np.array([1.3, -0.7, 2.9]), L)
    d = np.abs(p - want)
    if np.max(np.minimum(d, L - d)) > 1e-12 or p.min() < 0 or p.max() >= L:
        failed.append("periodic drift")
    return failed


def test_interpolation(oracle_mod):
    assert interpolation_failures(oracle_mod) == []


def test_push(oracle_mod):
    assert push_failures(oracle_mod) == []


def test_speed_is_conserved_in_a_turbulent_field(oracle_mod):
    n = 16
    rng = np.random.default_rng(2)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0)
    o.set_state(np.ones((n, n, n)), u / inputs.rms(u), b / inputs.rms(b))
    pos = rng.uniform(0, L, (50, 3))
    o.tracers_set(pos)
    _, v0 = o.tracers_get()
    o.step(30)
    p, v = o.tracers_get()
    assert np.allclose(np.linalg.norm(v, axis=1), np.linalg.norm(v0, axis=1), rtol=1e-13)
    assert np.all((p >= 0) & (p < L))
    assert np.max(np.abs(v - v0)) > 1e-3  # the field did turn them


def test_removing_tracers(oracle_mod):
    o = uniform_state(oracle_mod, 16, [0.1, 0, 0], [0, 0, 1], 0.01)
    o.tracers_set(np.zeros((3, 3)))
    o.tracers_set(np.zeros((0, 3)))
    o.step(2)
    p, v = o.tracers_get()
    assert p.shape == (0, 3)
