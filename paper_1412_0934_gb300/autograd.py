"""Gradients of a final-state loss with respect to the initial density and velocity, through the
library's hand-written adjoint (hydro_adjoint_step) behind a torch.autograd.Function.

Forward: W = (rho, u, v, w, p) -> U^0 (hydro_prim_to_cons), then nsteps periodic steps, each with
the CFL dt of its own input computed on the device (fused into the previous step) and recorded;
every `checkpoint_every` steps the state is kept.  Backward: segment by segment in reverse, the
states inside a segment are recomputed from its checkpoint with the recorded dts, then
hydro_adjoint_step carries lambda back one step at a time, and hydro_prim_to_cons_adjoint maps
lambda^0 to (d/d rho, d/du, d/dv, d/dw, d/dp).  The time steps are treated as constants (the
gradient does not flow through the CFL minimum).  Memory: nsteps/checkpoint_every + checkpoint_every
states instead of nsteps.  All arithmetic runs in the library's kernels; torch only holds memory.
"""
import torch

from . import hydro_adjoint_step, hydro_cfl_dt, hydro_prim_to_cons, hydro_prim_to_cons_adjoint, hydro_step, patch


class Simulation:
    """nsteps periodic steps of a (nz, ny, nx) box with cell size dx, as a differentiable map
    (rho0, vel0, p0) -> rho_final."""

    def __init__(self, ctx, shape, dx, nsteps, checkpoint_every=8):
        self.ctx = ctx
        self.shape = tuple(shape)
        self.dx = float(dx)
        self.nsteps = int(nsteps)
        self.every = int(checkpoint_every)
        self.dtype = ctx.dtype
        self.last_dts = None
        self.recording = False

    def _p(self, t):
        return patch(t, 0, self.dx)

    def _prim(self, rho0, vel0, p0):
        return torch.stack([rho0, vel0[0], vel0[1], vel0[2], p0]).to(self.dtype).contiguous()

    def run(self, U, dts, n0, n1, keep=None):
        """Advance U (in place, returns the result) from step n0 to n1 with dts[n] (device);
        if dts is being recorded, dt[n+1] is written by step n's fused CFL.  keep(n, U) is called
        with the state before each step."""
        a, b = U, torch.empty_like(U)
        for n in range(n0, n1):
            if keep is not None:
                keep(n, a)
            hydro_step(self.ctx, self._p(a), self._p(b), dts[n:n + 1], dts[n + 1:n + 2] if self.recording else None)
            a, b = b, a
        return a

    def forward_only(self, rho0, vel0, p0, dts=None):
        """rho after nsteps (no graph); dts: reuse a recorded dt sequence (device, nsteps + 1)."""
        W = self._prim(rho0, vel0, p0)
        U = torch.empty_like(W)
        hydro_prim_to_cons(self.ctx, self._p(W), self._p(U))
        self.recording = dts is None
        if dts is None:
            dts = torch.empty(self.nsteps + 1, dtype=torch.float64, device=U.device)
            hydro_cfl_dt(self.ctx, self._p(U), dts[0:1])
        U = self.run(U, dts, 0, self.nsteps)
        self.recording = False
        self.last_dts = dts
        return U[0].clone()

    def __call__(self, rho0, vel0, p0):
        return _Run.apply(rho0, vel0, p0, self)


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(fctx, rho0, vel0, p0, sim):
        W = sim._prim(rho0, vel0, p0)
        U = torch.empty_like(W)
        hydro_prim_to_cons(sim.ctx, sim._p(W), sim._p(U))
        dts = torch.empty(sim.nsteps + 1, dtype=torch.float64, device=U.device)
        hydro_cfl_dt(sim.ctx, sim._p(U), dts[0:1])
        ckpt = {}

        def keep(n, X):
            if n % sim.every == 0:
                ckpt[n] = X.clone()

        sim.recording = True
        UN = sim.run(U, dts, 0, sim.nsteps, keep)
        sim.recording = False
        sim.last_dts = dts
        fctx.sim = sim
        fctx.ckpt = ckpt
        fctx.dtypes = (rho0.dtype, vel0.dtype, p0.dtype)
        fctx.save_for_backward(W, dts)
        return UN[0].clone()

    @staticmethod
    def backward(fctx, grad_rho):
        sim = fctx.sim
        W, dts = fctx.saved_tensors
        lam = torch.zeros_like(W)
        lam[0] = grad_rho.to(W.dtype)
        other = torch.empty_like(W)
        starts = sorted(fctx.ckpt.keys(), reverse=True)
        for s in starts:
            e = min(s + sim.every, sim.nsteps)
            states = {}

            def keep(n, X):
                states[n] = X.clone()

            sim.run(fctx.ckpt[s].clone(), dts, s, e, keep)
            for n in range(e - 1, s - 1, -1):
                hydro_adjoint_step(sim.ctx, sim._p(states[n]), dts[n:n + 1], sim._p(lam), sim._p(other))
                lam, other = other, lam
            del states
        gW = torch.empty_like(W)
        hydro_prim_to_cons_adjoint(sim.ctx, sim._p(W), sim._p(lam), sim._p(gW))
        dr, dv, dp = fctx.dtypes
        return gW[0].to(dr), gW[1:4].to(dv), gW[4].to(dp), None
