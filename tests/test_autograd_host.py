"""Host logic of the differentiable multi-step run (paper_1412_0934_gb300/autograd.py) on the CPU:
the library calls it makes are replaced by the oracle's steps on CPU tensors, so the checkpoint
schedule, the recorded time steps, the segment-by-segment recomputation and the order of the
adjoint steps are checked without a GPU.  The gradient must equal the oracle's own chain of
adjoint steps bit for bit (the recomputed states are the forward's, the same calls in the same
order), for segment lengths that divide the run, do not, exceed it, or are 1."""
import types

import numpy as np
import pytest
import torch

import oracle
import workloads

import paper_1412_0934_gb300.autograd as ag


class FakeLibrary:
    """The five library calls of the run, done by the oracle on CPU tensors, with call counts."""

    def __init__(self, dx):
        self.dx = dx
        self.cfg = oracle.config()
        self.steps = 0
        self.adjoints = 0
        self.calls = []

    def patch(self, t, ng, dx):
        assert ng == 0 and dx == self.dx
        return types.SimpleNamespace(t=t)

    def prim_to_cons(self, ctx, pW, pU):
        pU.t.copy_(torch.from_numpy(oracle.prim_to_cons(pW.t.numpy(), self.cfg)))

    def cfl_dt(self, ctx, pU, d):
        d[0] = oracle.cfl_periodic(pU.t.numpy(), self.dx, self.cfg)

    def step(self, ctx, pa, pb, dt, dt_next=None):
        assert dt.numel() == 1 and (dt_next is None or dt_next.numel() == 1)
        self.steps += 1
        self.calls.append(("step", float(dt.item())))
        pb.t.copy_(torch.from_numpy(oracle.step_periodic(pa.t.numpy(), self.dx, dt.item(), self.cfg)))
        if dt_next is not None:
            dt_next[0] = oracle.cfl_periodic(pb.t.numpy(), self.dx, self.cfg)

    def adjoint_step(self, ctx, pU, dt, plam, pout):
        self.adjoints += 1
        self.calls.append(("adjoint", float(dt.item())))
        pout.t.copy_(torch.from_numpy(
            oracle.step_periodic_adjoint(pU.t.numpy(), plam.t.numpy(), self.dx, dt.item(), self.cfg)))

    def prim_to_cons_adjoint(self, ctx, pW, plam, pg):
        pg.t.copy_(torch.from_numpy(oracle.prim_to_cons_adjoint(pW.t.numpy(), plam.t.numpy(), self.cfg)))


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLibrary(dx=1.0 / 8)
    monkeypatch.setattr(ag, "patch", lib.patch)
    monkeypatch.setattr(ag, "hydro_prim_to_cons", lib.prim_to_cons)
    monkeypatch.setattr(ag, "hydro_cfl_dt", lib.cfl_dt)
    monkeypatch.setattr(ag, "hydro_step", lib.step)
    monkeypatch.setattr(ag, "hydro_adjoint_step", lib.adjoint_step)
    monkeypatch.setattr(ag, "hydro_prim_to_cons_adjoint", lib.prim_to_cons_adjoint)
    return lib


def initial_state():
    U, _ = workloads.sound_wave((4, 6, 8), amp=1e-2, kvec=(1, 1, 1), phase=0.3)
    q = oracle.recover(U.numpy())
    return torch.from_numpy(q[0].copy()), torch.from_numpy(q[1:4].copy()), torch.from_numpy(q[4].copy())


def oracle_chain(rho0, vel0, p0, g, nsteps, dx):
    """The gradient of sum(g * rho_final) by the oracle alone: forward with the CFL dt of each
    state, then the adjoint steps in reverse and the transpose of the primitive map."""
    cfg = oracle.config()
    W = np.stack([rho0.numpy(), *vel0.numpy(), p0.numpy()])
    U = oracle.prim_to_cons(W, cfg)
    states, dts = [], []
    for _ in range(nsteps):
        dts.append(oracle.cfl_periodic(U, dx, cfg))
        states.append(U)
        U = oracle.step_periodic(U, dx, dts[-1], cfg)
    lam = np.zeros_like(U)
    lam[0] = g
    for n in range(nsteps - 1, -1, -1):
        lam = oracle.step_periodic_adjoint(states[n], lam, dx, dts[n], cfg)
    return oracle.prim_to_cons_adjoint(W, lam, cfg), U, dts


@pytest.mark.parametrize("nsteps,every", [(7, 3), (6, 3), (4, 8), (5, 1)])
def test_checkpointed_gradient_equals_the_oracle_chain(fake, nsteps, every):
    rho0, vel0, p0 = initial_state()
    ctx = types.SimpleNamespace(dtype=torch.float64)
    sim = ag.Simulation(ctx, rho0.shape, fake.dx, nsteps, checkpoint_every=every)
    rho0.requires_grad_(True)
    vel0.requires_grad_(True)
    p0.requires_grad_(True)
    out = sim(rho0, vel0, p0)
    g = np.random.default_rng(5).standard_normal(out.shape)
    want, U_final, dts = oracle_chain(rho0.detach(), vel0.detach(), p0.detach(), g, nsteps, fake.dx)
    # forward: the final density and the recorded time steps (dt[n+1] from step n's fused CFL)
    np.testing.assert_array_equal(out.detach().numpy(), U_final[0])
    np.testing.assert_array_equal(sim.last_dts[:nsteps].numpy(), np.array(dts))
    assert fake.steps == nsteps and fake.adjoints == 0
    (out * torch.from_numpy(g)).sum().backward()
    np.testing.assert_array_equal(rho0.grad.numpy(), want[0])
    np.testing.assert_array_equal(vel0.grad.numpy(), want[1:4])
    np.testing.assert_array_equal(p0.grad.numpy(), want[4])
    # backward: every step recomputed once from its segment's checkpoint, one adjoint step each,
    # the segments taken last to first and each segment's adjoints in reverse step order
    assert fake.steps == 2 * nsteps and fake.adjoints == nsteps
    back = fake.calls[nsteps:]
    segs = [(s, min(s + every, nsteps)) for s in range(0, nsteps, every)][::-1]
    expect = []
    for s, e in segs:
        expect += [("step", dts[n]) for n in range(s, e)]
        expect += [("adjoint", dts[n]) for n in range(e - 1, s - 1, -1)]
    assert back == expect


def test_forward_only_reuses_a_recorded_dt_sequence(fake):
    rho0, vel0, p0 = initial_state()
    ctx = types.SimpleNamespace(dtype=torch.float64)
    sim = ag.Simulation(ctx, rho0.shape, fake.dx, 5, checkpoint_every=2)
    r1 = sim.forward_only(rho0, vel0, p0)
    dts = sim.last_dts.clone()
    r2 = sim.forward_only(rho0 * 1.0, vel0, p0, dts=dts)
    np.testing.assert_array_equal(r1.numpy(), r2.numpy())
    np.testing.assert_array_equal(sim.last_dts.numpy(), dts.numpy())  # a given sequence is not rewritten
