"""torch.autograd.Function around ls_pac_grad: the PAC log-likelihood as a differentiable function
of log mu and of per-group log-scales of rho.

    rho_m = rho0_m * exp(delta[interval_of[m]]),   mu = exp(log_mu)

PacLogLik.apply(log_mu, delta, ctx, rho0, interval_of) sets the parameters on the library
context, runs the adjoint on the GPU and returns the PAC log-likelihood (float64 scalar); its
backward returns grad * dPAC/dlog_mu and grad * dPAC/ddelta from the same call.  All arithmetic is
in libls; this module only marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ls


class PacLogLik(torch.autograd.Function):
    @staticmethod
    def forward(actx, log_mu, delta, ctx, rho0, interval_of, t_from=0, t_to=None):
        io = np.ascontiguousarray(interval_of, dtype=np.int32)
        K = int(delta.numel())
        d = delta.detach().to("cpu", torch.float64).numpy()
        rho = np.asarray(rho0, dtype=np.float64) * np.exp(d[io])
        mu = float(np.exp(float(log_mu.detach().cpu())))
        ls.ls_set_params(ctx, rho, mu)
        _, pac, gmu, grho = ls.ls_pac_grad(ctx, io, K, t_from, t_to)
        actx.save_for_backward(torch.tensor(gmu, dtype=torch.float64), torch.from_numpy(grho))
        actx.devices = (log_mu.device, delta.device)
        return torch.tensor(pac, dtype=torch.float64, device=log_mu.device)

    @staticmethod
    def backward(actx, g):
        gmu, grho = actx.saved_tensors
        dm, dd = actx.devices
        g = g.to(torch.float64)
        return (g.to(dm) * gmu.to(dm)).reshape(()), g.to(dd) * grho.to(dd), None, None, None, None, None


def pac_loglik(log_mu, delta, ctx, rho0, interval_of, t_from=0, t_to=None):
    """Differentiable PAC log-likelihood (see PacLogLik)."""
    return PacLogLik.apply(log_mu, delta, ctx, rho0, interval_of, t_from, t_to)
