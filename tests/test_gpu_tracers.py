"""Tracer particles through the C ABI (paper, section "Tracer Particles"), against the oracle:
initial velocities, trajectories under each time solver and in both precisions, the exact Boris
rotation in uniform fields, a large particle count, passivity (the flow is bitwise the same with
and without tracers), CUDA-graph replay, and argument checks.
"""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu
L = 2 * np.pi


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


def mhd_state(n, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.2 * np.cos(X + 2 * Y) * np.sin(Z - 0.3)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    b *= 1.5 / inputs.rms(b)
    return rho, u, b


def periodic_diff(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b))
    return np.minimum(d, L - d)


def positions(count, seed):
    return np.random.default_rng(seed).uniform(-0.5, L + 0.5, (count, 3))


@pytest.mark.parametrize("precision,integrator", [(0, 0), (0, 1), (0, 2), (1, 0), (2, 0)])
def test_trajectories_match_oracle(lib, oracle_mod, precision, integrator):
    n, count, steps = 32, 300, 40
    rho, u, b = mhd_state(n, 3)
    ctx = lib.mhd_init(n, [(0.01, 0.01, 2.0)], precision=precision, integrator=integrator)
    lib.mhd_set_state(ctx, 0, rho, u, b)
    pos = positions(count, 5)
    lib.mhd_tracers_set(ctx, 0, pos)
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0, integrator=integrator)
    o.set_state(rho, u, b)
    o.tracers_set(pos)
    p0, v0 = lib.mhd_tracers_get(ctx, 0)
    q0, w0 = o.tracers_get()
    assert np.max(np.abs(p0 - q0)) == 0.0  # wrapping is exact arithmetic on both sides
    assert np.max(np.abs(v0 - w0)) <= 1e-13
    lib.mhd_step(ctx, steps)
    o.step(steps)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    p, v = lib.mhd_tracers_get(ctx, 0)
    q, w = o.tracers_get()
    tol = 2e-5 if precision == 1 else 1e-10  # the mixed mode's FP32 field; FP64 and double-float
    assert np.max(periodic_diff(p, q)) <= tol
    assert np.max(np.abs(v - w)) <= tol
    assert np.all((p >= 0) & (p < L))
    # the field turned them, and each push kept the speed (a rotation)
    assert np.max(np.abs(v - v0)) > 1e-2
    assert np.allclose(np.linalg.norm(v, axis=1), np.linalg.norm(v0, axis=1), rtol=1e-12)


def rotation(axis, angle):
    a = np.asarray(axis, dtype=float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def test_uniform_field_gives_the_boris_rotation(lib):
    n, dt, steps = 16, 0.013, 40
    U = np.array([0.3, -0.2, 0.45])
    B = np.array([0.8, -1.1, 1.7])
    ctx = lib.mhd_init(n, [(0.01, 0.01, 1.0)], dt=dt)
    one = np.ones((n, n, n))
    lib.mhd_set_state(ctx, 0, one, U[:, None, None, None] * one, B[:, None, None, None] * one)
    pos = positions(8, 1)
    lib.mhd_tracers_set(ctx, 0, pos)
    lib.mhd_step(ctx, steps)
    p, v = lib.mhd_tracers_get(ctx, 0)
    theta = 2 * np.arctan(np.linalg.norm(B) * dt / 2)
    vk = [rotation(B, -theta * k) @ U for k in range(1, steps + 1)]
    assert np.max(np.abs(v - vk[-1])) <= 1e-13
    assert np.max(periodic_diff(p, np.mod(pos + dt * np.sum(vk, axis=0), L))) <= 1e-12


def test_many_tracers_match_oracle(lib, oracle_mod):
    n, count, steps = 64, 200_000, 5
    rho, u, b = mhd_state(n, 8)
    ctx = lib.mhd_init(n, [(0.01, 0.01, 2.0)])
    lib.mhd_set_state(ctx, 0, rho, u, b)
    pos = positions(count, 6)
    lib.mhd_tracers_set(ctx, 0, pos)
    assert lib.load_library().mhd_tracers_count(ctx.handle, 0) == count
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0)
    o.set_state(rho, u, b)
    o.tracers_set(pos)
    lib.mhd_step(ctx, steps)
    o.step(steps)
    p, v = lib.mhd_tracers_get(ctx, 0)
    q, w = o.tracers_get()
    assert np.max(periodic_diff(p, q)) <= 1e-11
    assert np.max(np.abs(v - w)) <= 1e-11


def test_tracers_are_passive_and_graph_replay_matches(lib):
    """Two instances, tracers on the second only: both flows are bitwise those of a run without
    tracers, and graph replay gives bitwise the tracers of direct launches."""
    n = 32
    s0, s1 = mhd_state(n, 1), mhd_state(n, 2)
    phys = [(0.01, 0.02, 2.0), (0.015, 0.01, 1.5)]
    out = []
    for tracers, graph in ((False, True), (True, True), (True, False)):
        ctx = lib.mhd_init(n, phys)
        if not graph:
            lib.mhd_set_option(ctx, lib.MHD_OPT_CUDA_GRAPH, 0)
        lib.mhd_set_state(ctx, 0, *s0)
        lib.mhd_set_state(ctx, 1, *s1)
        if tracers:
            lib.mhd_tracers_set(ctx, 1, positions(100, 3))
        lib.mhd_step(ctx, 25)
        states = [np.concatenate([np.ravel(a) for a in lib.mhd_get_state(ctx, i)]) for i in range(2)]
        out.append((states, lib.mhd_tracers_get(ctx, 1) if tracers else None, lib.mhd_tracers_get(ctx, 0)))
    for i in range(2):
        assert np.array_equal(out[0][0][i], out[1][0][i])
        assert np.array_equal(out[1][0][i], out[2][0][i])
    assert np.array_equal(out[1][1][0], out[2][1][0]) and np.array_equal(out[1][1][1], out[2][1][1])
    assert out[1][2][0].shape == (0, 3)  # instance 0 has none


def test_tracer_arguments(lib):
    n = 16
    ctx = lib.mhd_init(n, [(0.01, 0.01, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_tracers_set(ctx, 0, positions(4, 0))  # no state yet
    lib.mhd_set_state(ctx, 0, *mhd_state(n, 4))
    bad = positions(4, 0)
    bad[2, 1] = np.nan
    with pytest.raises(lib.MhdError):
        lib.mhd_tracers_set(ctx, 0, bad)
    with pytest.raises(lib.MhdError):
        lib.mhd_tracers_set(ctx, 3, positions(4, 0))
    lib.mhd_tracers_set(ctx, 0, positions(4, 0))
    lib.mhd_step(ctx, 3)
    lib.mhd_tracers_set(ctx, 0, np.zeros((0, 3)))  # removal
    lib.mhd_step(ctx, 3)
    assert lib.mhd_tracers_get(ctx, 0)[0].shape == (0, 3)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
