"""torch.autograd integration of the QMC integrals (argument marshalling only).

QMCIntegrate.apply(theta, integrator) returns the fp64 estimates I_p(theta);
its backward calls the hand-written adjoint kernel (qmc_integrate_backward),
which regenerates the deterministic points instead of storing them, so the
forward keeps only theta and the counts alive.  GaussMixIntegrator bundles the
device-side inputs of the 4-Gaussian mixture problem (generator matrices,
per-integral scramble seeds, counts, workspace); with index_bits and
partition_log2 = q, integral p draws its samples from element p mod 2^q of the
Sobol' sequence partitioned by the matrices' dimension 0 (Sec. 2.5.1).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class GaussMixIntegrator:
    """Integrals of the 6-D four-Gaussian mixture over scrambled Sobol' points,
    one per row of theta [n][16]."""

    def __init__(self, matrices, counts, seeds=None, scramble=B.SCRAMBLE_NESTED, chunk=0, block=0,
                 device="cuda", index_bits=0, partition_log2=0):
        self.device = torch.device(device)
        C = np.ascontiguousarray(matrices, dtype=np.uint32)
        want = (6 + (1 if partition_log2 else 0), index_bits or 32)
        if C.shape != want:
            raise ValueError(f"the mixture needs generator matrices of shape {want} here")
        self.counts_host = np.ascontiguousarray(counts, dtype=np.uint32).reshape(-1)
        self.n = int(self.counts_host.size)
        self.matrices = B.u32_tensor(C, self.device)
        self.counts = B.u32_tensor(self.counts_host, self.device)
        self.seeds = None if seeds is None else B.u32_tensor(np.asarray(seeds, np.uint32).reshape(self.n, 6),
                                                            self.device)
        self.problem = B.make_problem(B.SOURCE_SOBOL, B.F_GAUSSMIX4_6D, 6, scramble if seeds is not None else 0,
                                      matrices=self.matrices, seeds=self.seeds,
                                      seeds_per_integral=seeds is not None, chunk=chunk, block=block,
                                      max_count=int(self.counts_host.max(initial=0)), with_gradient=True,
                                      index_bits=index_bits, partition_log2=partition_log2)
        self.workspace = B.alloc_workspace(self.problem, self.n, self.counts_host, self.device)

    def __call__(self, theta: torch.Tensor) -> torch.Tensor:
        return QMCIntegrate.apply(theta, self)


class QMCIntegrate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, integrator):
        if theta.dtype != torch.float32 or theta.shape != (integrator.n, 16):
            raise ValueError("theta must be float32 [n][16]")
        theta = theta.contiguous()
        est = torch.empty(integrator.n, dtype=torch.float64, device=theta.device)
        B.qmc_integrate(integrator.problem, integrator.n, integrator.counts, theta, est, integrator.workspace)
        ctx.integrator = integrator
        ctx.save_for_backward(theta)
        return est

    @staticmethod
    def backward(ctx, grad_est):
        (theta,) = ctx.saved_tensors
        it = ctx.integrator
        g = torch.empty_like(theta)
        B.qmc_integrate_backward(it.problem, it.n, it.counts, theta,
                                 grad_est.to(torch.float64).contiguous(), g, it.workspace)
        return g, None
