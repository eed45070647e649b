"""Helpers for the GPU tests: run the C-ABI transforms on numpy inputs."""
import numpy as np

from paper_1308_5706_gb300 import binding as B


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def run_analysis(plan: B.Plan, flm: np.ndarray):
    torch = torch_cuda()
    cd, rd = plan.torch_dtypes()
    f = torch.from_numpy(flm.astype(np.complex128)).to(cd).cuda()
    W, Wphi = plan.alloc_w()
    plan.analysis(f, W, Wphi)
    torch.cuda.synchronize()
    return W.double().cpu().numpy(), Wphi.double().cpu().numpy()


def run_synthesis(plan: B.Plan, W: np.ndarray, Wphi: np.ndarray):
    torch = torch_cuda()
    cd, rd = plan.torch_dtypes()
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(rd).cuda()
    Wp = torch.from_numpy(np.ascontiguousarray(Wphi)).to(rd).cuda()
    f = plan.alloc_flm()
    plan.synthesis(Wd, Wp, f)
    torch.cuda.synchronize()
    return f.to(torch.complex128).cpu().numpy()


def relerr(x, ref):
    """Normwise max relative error: max|x - ref| / max|ref|."""
    den = np.abs(ref).max()
    return float(np.abs(x - ref).max() / (den if den > 0 else 1.0))
