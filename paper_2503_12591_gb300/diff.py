"""Differentiable EPI energy and thermal-derivative estimator.

Argument marshalling only: the pair counts, energies, gradients and FP64
fluctuation sums run in the CUDA library (smcx_pair_counts_batch,
smcx_epi_energy_batch, smcx_epi_grad_batch, smcx_fluct_accumulate,
smcx_fluct_gradient).  PyTorch provides the device buffers, the stream and
the autograd graph.

Energy model (Method, Eq. Total_EPI, pair form): E = 1/2 sum_i V_i C_i with
C the ordered pair counts, so dE/dV = C/2.  Thermal derivative (Supplementary
"Statistical mechanics"): d<A>/dV_i = -beta (<A C_i/2> - <A><C_i/2>).
"""
import torch

from . import smcx


def _stream():
    return torch.cuda.current_stream().cuda_stream


def pair_counts(configs: torch.Tensor, kind: int, dims, M: int, K: int) -> torch.Tensor:
    """Ordered pair counts int64 [B, K, M, M] of int8 configurations [B, N]
    (a configuration holding an id outside 0..M-1 comes back as all -1)."""
    assert configs.is_cuda and configs.dtype == torch.int8 and configs.is_contiguous()
    B = configs.shape[0]
    out = torch.empty((B, K, M, M), dtype=torch.int64, device=configs.device)
    smcx.pair_counts_batch(kind, dims, M, K, configs.data_ptr(), B, out.data_ptr(), _stream())
    return out


class EPIEnergy(torch.autograd.Function):
    """E[b] = 1/2 sum V * C[b] for V float32 [K, M, M] and counts int64
    [B, K, M, M]; backward returns 1/2 sum_b g[b] C[b]."""

    @staticmethod
    def forward(ctx, V, counts):
        assert V.is_cuda and V.dtype == torch.float32
        Vc = V.contiguous()
        B = counts.shape[0]
        KMM = Vc.numel()
        E = torch.empty(B, dtype=torch.float32, device=V.device)
        smcx.epi_energy_batch(Vc.data_ptr(), counts.data_ptr(), B, KMM, E.data_ptr(), _stream())
        ctx.save_for_backward(counts)
        ctx.shape = Vc.shape
        return E

    @staticmethod
    def backward(ctx, g):
        (counts,) = ctx.saved_tensors
        g = g.contiguous().to(torch.float32)
        KMM = 1
        for d in ctx.shape:
            KMM *= d
        grad = torch.empty(KMM, dtype=torch.float32, device=g.device)
        smcx.epi_grad_batch(g.data_ptr(), counts.data_ptr(), counts.shape[0], KMM, grad.data_ptr(), _stream())
        return grad.view(ctx.shape), None


def epi_energy(V: torch.Tensor, counts: torch.Tensor) -> torch.Tensor:
    return EPIEnergy.apply(V, counts)


class FluctuationEstimator:
    """FP64 device sums of (1, A, C, A C^T) for A = Warren-Cowley alpha of one
    shell; gradient(T) gives d<A>/dV in 1/meV as [M*M, K, M, M]."""

    def __init__(self, kind: int, K: int, M: int, shell: int, n_sites: int, device="cuda"):
        self.kind, self.K, self.M, self.shell, self.n_sites = kind, K, M, shell, n_sites
        MM, KMM = M * M, K * M * M
        self.acc = torch.zeros(1 + MM + KMM + MM * KMM, dtype=torch.float64, device=device)

    def add_lattice(self, lat: "smcx.Lattice"):
        lat.fluct_accumulate(self.shell, self.acc.data_ptr())

    def add_counts(self, counts: torch.Tensor, weights: torch.Tensor = None):
        assert counts.dtype == torch.int64 and counts.is_contiguous()
        w = 0
        if weights is not None:
            assert weights.dtype == torch.float64 and weights.is_contiguous()
            w = weights.data_ptr()
        smcx.fluct_accumulate(counts.data_ptr(), counts.shape[0], w, self.kind, self.K, self.M, self.shell,
                              self.n_sites, self.acc.data_ptr(), _stream())

    def gradient(self, T: float) -> torch.Tensor:
        MM, KMM = self.M * self.M, self.K * self.M * self.M
        g = torch.empty(MM * KMM, dtype=torch.float64, device=self.acc.device)
        smcx.fluct_gradient(self.acc.data_ptr(), self.K, self.M, T, g.data_ptr(), _stream())
        return g.view(MM, self.K, self.M, self.M)

    def mean_A(self) -> torch.Tensor:
        MM = self.M * self.M
        return (self.acc[1:1 + MM] / self.acc[0]).view(self.M, self.M)


class BatchFluctuationEstimator:
    """FluctuationEstimator for every replica of a smcx.Batch at once
    (smcx_batch_fluct_accumulate): one accumulator row per replica."""

    def __init__(self, batch: "smcx.Batch", K: int, M: int, shell: int, device="cuda"):
        self.batch, self.K, self.M, self.shell = batch, K, M, shell
        MM, KMM = M * M, K * M * M
        R = len(batch.lattices)
        self.acc = torch.zeros(R, 1 + MM + KMM + MM * KMM, dtype=torch.float64, device=device)

    def add(self):
        self.batch.fluct_accumulate(self.shell, self.acc.data_ptr())

    def gradients(self, T: float) -> torch.Tensor:
        """d<A>/dV per replica, [R, M*M, K, M, M] in 1/meV."""
        MM, KMM = self.M * self.M, self.K * self.M * self.M
        out = torch.empty(self.acc.shape[0], MM * KMM, dtype=torch.float64, device=self.acc.device)
        for r in range(self.acc.shape[0]):
            smcx.fluct_gradient(self.acc[r].data_ptr(), self.K, self.M, T, out[r].data_ptr(), _stream())
        return out.view(-1, MM, self.K, self.M, self.M)
