"""Plain GPU baseline: the same pseudo-spectral MHD step built the conventional way.

Every field is a full half-complex spectrum (N, N, N/2+1); each RHS evaluation runs one cuFFT
inverse real transform per state field (7), the products as separate elementwise tensor
operations, one cuFFT forward real transform per product (12), then the assembly, the 2/3 mask and
the AB2 update as elementwise operations.  cuFFT is reached through torch.fft; nothing is fused and
no spectrum is truncated.  This is what the hand-written path is timed against; it follows the same
readings (conservative fluxes, spectral pressure, cubic 2/3 truncation, variable-step AB2 with a
forward-Euler first step, the same CFL formula) so both compute the same thing.
"""
from __future__ import annotations

import math

import torch


class PlainMHD:
    def __init__(self, n: int, nu: float, eta: float, cs: float, dt: float = 0.0, cfl_adv: float = 0.2,
                 cfl_visc: float = 0.5, dtype=torch.float64, device="cuda"):
        self.n, self.nu, self.eta, self.cs = n, nu, eta, cs
        self.dt_fixed, self.cfl_adv, self.cfl_visc = dt, cfl_adv, cfl_visc
        self.rdt = dtype
        self.dev = torch.device(device)
        k = torch.fft.fftfreq(n, 1.0 / n, dtype=dtype, device=self.dev)
        kh = torch.fft.rfftfreq(n, 1.0 / n, dtype=dtype, device=self.dev)
        k[n // 2] = 0.0  # derivative of the Nyquist index
        self.kz = k.view(n, 1, 1)
        self.ky = k.view(1, n, 1)
        self.kx = kh.view(1, 1, n // 2 + 1)
        self.k2 = self.kx ** 2 + self.ky ** 2 + self.kz ** 2
        ai = torch.fft.fftfreq(n, 1.0 / n, device=self.dev).abs()
        aih = torch.fft.rfftfreq(n, 1.0 / n, device=self.dev)
        self.mask = ((3 * ai.view(n, 1, 1) < n) & (3 * ai.view(1, n, 1) < n) & (3 * aih.view(1, 1, -1) < n)).to(dtype)
        self.kmax = (n - 1) // 3
        self.state = None
        self.hist = None
        self.dt_prev = None
        self.step_count = 0

    def fwd(self, f):
        return torch.fft.rfftn(f, norm="forward")

    def inv(self, fh):
        return torch.fft.irfftn(fh, s=(self.n,) * 3, norm="forward")

    def set_state(self, rho, u, b):
        t = lambda a: torch.as_tensor(a, dtype=self.rdt, device=self.dev)
        rho, u, b = t(rho), t(u), t(b)
        fields = [rho] + [rho * u[i] for i in range(3)] + [b[i] for i in range(3)]
        self.state = torch.stack([self.fwd(f) * self.mask for f in fields])
        self.hist = torch.zeros_like(self.state)
        self.dt_prev = None
        self.step_count = 0

    def rhs(self):
        n = self.n
        r = [self.inv(self.state[i]) for i in range(7)]
        rho, m, B = r[0], r[1:4], r[4:7]
        u = [mi / rho for mi in m]
        b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        hb = 0.5 * b2
        T = {(0, 0): m[0] * u[0] + hb - B[0] * B[0], (1, 1): m[1] * u[1] + hb - B[1] * B[1],
             (2, 2): m[2] * u[2] + hb - B[2] * B[2], (0, 1): m[0] * u[1] - B[0] * B[1],
             (0, 2): m[0] * u[2] - B[0] * B[2], (1, 2): m[1] * u[2] - B[1] * B[2]}
        E = [u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]]
        smax = (torch.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2) + torch.sqrt(self.cs ** 2 + b2 / rho)).max()
        Th = {key: self.fwd(v) for key, v in T.items()}
        Eh = [self.fwd(e) for e in E]
        uh = [self.fwd(v) for v in u]
        kk = (self.kx, self.ky, self.kz)
        Tm = lambda i, j: Th[(min(i, j), max(i, j))]
        s = self.state
        out = torch.empty_like(s)
        out[0] = -1j * (self.kx * s[1] + self.ky * s[2] + self.kz * s[3])
        for a in range(3):
            div = kk[0] * Tm(a, 0) + kk[1] * Tm(a, 1) + kk[2] * Tm(a, 2)
            out[1 + a] = -1j * div - 1j * kk[a] * self.cs ** 2 * s[0] - self.nu * self.k2 * uh[a]
        curl = [1j * (self.ky * Eh[2] - self.kz * Eh[1]), 1j * (self.kz * Eh[0] - self.kx * Eh[2]),
                1j * (self.kx * Eh[1] - self.ky * Eh[0])]
        for a in range(3):
            out[4 + a] = curl[a] - self.eta * self.k2 * s[4 + a]
        return out * self.mask, smax

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            f, smax = self.rhs()
            if self.dt_fixed > 0:
                dt = torch.as_tensor(self.dt_fixed, dtype=self.rdt, device=self.dev)
            else:
                dt = self.cfl_adv * (2 * math.pi / self.n) / smax
                diff = max(self.nu, self.eta)
                if diff > 0:
                    dt = torch.minimum(dt, torch.as_tensor(self.cfl_visc / (diff * self.kmax ** 2), dtype=self.rdt,
                                                           device=self.dev))
            if self.dt_prev is None:
                self.state = self.state + dt * f
            else:
                r = dt / self.dt_prev
                self.state = self.state + dt * ((1 + 0.5 * r) * f - 0.5 * r * self.hist)
            self.hist = f
            self.dt_prev = dt
            self.step_count += 1

    def get_state(self):
        return [self.inv(self.state[i]).cpu().numpy() for i in range(7)]
