"""The oracle's fixed-step setter (used to replay on a coarser grid a step-size sequence decided on
a finer one) changes only which dt the next steps take: replaying the oracle's own CFL sequence
as fixed steps reproduces its run bitwise, and switching a CFL instance to a fixed dt equals an
instance created with that dt."""
import numpy as np

from paper_1810_12707_gb300 import inputs


def test_replayed_cfl_sequence_is_bitwise_the_cfl_run(oracle_mod):
    ic = inputs.orszag_tang(16, seed=3, mach=0.2)
    a = oracle_mod.Oracle(16, ic.nu, ic.eta, ic.cs)
    a.set_state(ic.rho, ic.u, ic.b)
    dts = []
    for _ in range(4):
        a.step(1)
        dts.append(a.diagnostics()["dt"])
    assert len(set(dts)) > 1  # the CFL step really varies
    b = oracle_mod.Oracle(16, ic.nu, ic.eta, ic.cs)
    b.set_state(ic.rho, ic.u, ic.b)
    for dt in dts:
        b.set_fixed_dt(dt)
        b.step(1)
    for f in range(7):
        assert np.array_equal(a.spectrum(f), b.spectrum(f))
    assert a.diagnostics()["t"] == b.diagnostics()["t"]


def test_switch_to_fixed_dt_equals_fixed_instance(oracle_mod):
    ic = inputs.abc_dynamo(16, seed=1, b_energy=1e-2)
    a = oracle_mod.Oracle(16, ic.nu, ic.eta, ic.cs, dt=2e-3)
    b = oracle_mod.Oracle(16, ic.nu, ic.eta, ic.cs)
    b.set_fixed_dt(2e-3)
    for o in (a, b):
        o.set_state(ic.rho, ic.u, ic.b)
        o.step(3)
    for f in range(7):
        assert np.array_equal(a.spectrum(f), b.spectrum(f))
