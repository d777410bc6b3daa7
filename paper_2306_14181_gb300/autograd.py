"""torch.autograd.Function over the discrete adjoint of the C ABI (bte_adjoint).

``probe_temperature(Q, log_tau, problem)`` returns J = sum_i p_i T_L,i after
``problem["steps"]`` steps of the explicit DOM scheme (T_L of Eq. BTE_get_e0) for the
per-cell heat source Q (W/m^3, shape (nz, ny, nx)) and the per-band log relaxation times.
The forward pass runs the library's forward sweep and its adjoint sweep together (the adjoint
needs the whole trajectory, recomputed from checkpoints), keeps dJ/dQ and dJ/dlog tau, and
the backward pass scales them by the incoming gradient.  Every step runs in the CUDA library;
this module only marshals arguments.
"""
import numpy as np
import torch

from . import bte


def _context(problem, tau):
    cfg = problem
    return bte.bte_create(cfg["dim"], cfg["n"], cfg["h"], cfg["C"], cfg["v"], tau, cfg["quad"], cfg["bc"], cfg["Tw"],
                          cfg["dt"], storage=cfg.get("storage", bte.BTE_STORE_F32),
                          limiter=cfg.get("limiter", bte.BTE_LIM_VANALBADA), T_scale=cfg.get("T_scale", 1.0),
                          rounding=cfg.get("rounding", bte.BTE_ROUND_NEAREST), seed=cfg.get("seed", 0),
                          kernel=cfg.get("kernel", bte.BTE_KERNEL_AUTO))


class ProbeTemperature(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, log_tau, problem):
        tau = torch.exp(log_tau.detach().to(torch.float64)).cpu().numpy()
        h = _context(problem, tau)
        bte.bte_init_temperature(h, problem.get("dT0"))
        Qd = Q.detach().to(device="cuda", dtype=torch.float32).contiguous().reshape(-1)
        bte.bte_set_source(h, Qd, problem.get("amps"))
        torch.cuda.current_stream().synchronize()
        J, gQ, gt = bte.bte_adjoint(h, problem["steps"], problem["probe"], problem.get("ckpt", 0))
        ctx.save_for_backward(torch.from_numpy(gQ).to(Q.device, Q.dtype).reshape(Q.shape),
                              torch.from_numpy(gt).to(log_tau.device, log_tau.dtype))
        return torch.tensor(J, dtype=torch.float64, device=Q.device)

    @staticmethod
    def backward(ctx, gJ):
        gQ, gt = ctx.saved_tensors
        return (gJ.to(device=gQ.device, dtype=gQ.dtype) * gQ, gJ.to(device=gt.device, dtype=gt.dtype) * gt, None)


def probe_temperature(Q, log_tau, problem):
    """J(Q, log tau) with gradients through the discrete adjoint (see the module docstring).
    ``problem``: a workload dict (``inputs``) plus ``probe`` ((nz, ny, nx) weights), ``steps``
    and optionally ``amps``, ``dT0``, ``ckpt``, ``storage``, ``limiter``, ``kernel``."""
    return ProbeTemperature.apply(Q, log_tau, problem)
