"""Batched launches (s2dw_analysis_batch / s2dw_synthesis_batch): jobs of
mixed L, N, lambda and J0 in one set of launches give exactly the results of
the same jobs run alone (the kernels are deterministic: no atomics, fixed
reduction order)."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu

SPECS = [(64, 3, 2.0, 0), (33, 1, 2.0, 1), (48, 5, 3.0, 0), (64, 3, 2.0, 0), (20, 2, 2.0, 0),
         (128, 5, 2.0, 2), (40, 8, 2.0, 1)]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_equals_single(prec):
    import torch
    plans = [B.Plan(L, N, lam, J0, prec) for (L, N, lam, J0) in SPECS]
    cd, rd = plans[0].torch_dtypes()
    fs = [torch.from_numpy(flm_gaussian(p.L, 40 + i, "cl")).to(cd).cuda() for i, p in enumerate(plans)]
    Wb = [p.alloc_w() for p in plans]
    Ws = [p.alloc_w() for p in plans]
    B.s2dw_analysis_batch([p.handle for p in plans], fs, [w[0] for w in Wb], [w[1] for w in Wb])
    for p, f, w in zip(plans, fs, Ws):
        p.analysis(f, w[0], w[1])
    torch.cuda.synchronize()
    for wb, ws in zip(Wb, Ws):
        assert torch.equal(wb[0], ws[0]) and torch.equal(wb[1], ws[1])
    fb = [p.alloc_flm() for p in plans]
    fsn = [p.alloc_flm() for p in plans]
    B.s2dw_synthesis_batch([p.handle for p in plans], [w[0] for w in Wb], [w[1] for w in Wb], fb)
    for p, w, f in zip(plans, Ws, fsn):
        p.synthesis(w[0], w[1], f)
    torch.cuda.synchronize()
    for a, b in zip(fb, fsn):
        assert torch.equal(a, b)
    # one member against the oracle, and every round trip
    L, N, lam, J0 = SPECS[1]
    Wo, Wpo = O.analysis(flm_gaussian(L, 41, "cl"), L, N, lam, J0)
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert relerr(Wb[1][0].double().cpu().numpy(), Wo) < tol
    for i, (p, f) in enumerate(zip(plans, fb)):
        ref = flm_gaussian(p.L, 40 + i, "cl")
        eps = np.abs(f.to(torch.complex128).cpu().numpy() - ref).max()
        assert eps < (1e-12 if prec == "fp64" else 1e-5)
    for p in plans:
        p.close()


def test_batch_argument_errors():
    a = B.Plan(16, 3, 2.0, 0, "mixed")
    b = B.Plan(16, 3, 2.0, 0, "fp64")
    W, Wp = a.alloc_w()
    f = a.alloc_flm()
    with pytest.raises(B.S2dwError) as ei:
        B.s2dw_analysis_batch([a.handle, a.handle], [f, f], [W, W], [Wp, Wp])
    assert ei.value.status == B.S2DW_EINVAL
    with pytest.raises(B.S2dwError) as ei:
        B.s2dw_analysis_batch([a.handle, b.handle], [f, f], [W, W], [Wp, Wp])
    assert ei.value.status == B.S2DW_ENOTSUP
    a.close()
    b.close()


def test_batch_in_cuda_graph_then_destroy():
    """Batched calls captured in a CUDA graph replay to the eager result, and
    the plans are destroyed cleanly afterwards (the library records none of
    its own events into the caller's graph)."""
    import torch
    plans = [B.Plan(L, N, lam, J0, "mixed") for (L, N, lam, J0) in SPECS[:4]]
    fs = [torch.from_numpy(flm_gaussian(p.L, 70 + i, "cl")).to(torch.complex64).cuda() for i, p in enumerate(plans)]
    Wg = [p.alloc_w() for p in plans]
    fg = [p.alloc_flm() for p in plans]
    hs = [p.handle for p in plans]
    s = torch.cuda.Stream()

    def step():
        B.s2dw_analysis_batch(hs, fs, [w[0] for w in Wg], [w[1] for w in Wg], s)
        B.s2dw_synthesis_batch(hs, [w[0] for w in Wg], [w[1] for w in Wg], fg, s)

    with torch.cuda.stream(s):
        step()  # warm-up outside capture (builds the cached launch lists)
    torch.cuda.synchronize()
    for f in fg:
        f.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    g.replay()
    torch.cuda.synchronize()
    for p, f, out in zip(plans, fs, fg):
        W, Wp = p.alloc_w()
        ref = p.alloc_flm()
        p.analysis(f, W, Wp)
        p.synthesis(W, Wp, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    del g
    torch.cuda.synchronize()
    for p in plans:
        p.close()  # raises on a non-zero status


def test_batch_cache_eviction():
    """More distinct plan sets than the launch-list cache holds (64): every
    batch, including ones whose lists were evicted and rebuilt, equals the
    single runs."""
    import itertools
    import torch
    specs = [(16, 1 + i % 4, 2.0, 0) for i in range(12)]
    plans = [B.Plan(*s, "mixed") for s in specs]
    cd, _ = plans[0].torch_dtypes()
    fs = [torch.from_numpy(flm_gaussian(p.L, 60 + i, "cl")).to(cd).cuda() for i, p in enumerate(plans)]
    ref = []
    for p, f in zip(plans, fs):
        W, Wp = p.alloc_w()
        p.analysis(f, W, Wp)
        ref.append(W)
    pairs = list(itertools.combinations(range(12), 2))   # 66 distinct sets
    for pair in pairs + pairs[:3]:                       # the first three again, after eviction
        Wb = [plans[i].alloc_w() for i in pair]
        B.s2dw_analysis_batch([plans[i].handle for i in pair], [fs[i] for i in pair],
                              [w[0] for w in Wb], [w[1] for w in Wb])
        torch.cuda.synchronize()
        for i, w in zip(pair, Wb):
            assert torch.equal(w[0], ref[i]), pair
    for p in plans:
        p.close()


def test_batch_mixes_grids_and_plan_kinds():
    """DH, MW (odd and even row counts N L) and multi-resolution plans in one
    batched launch set: the same bits as each plan alone, exact round trips.
    The odd-row alpha variants then serve the DH jobs too."""
    import torch
    specs = [((64, 3, 2.0, 0), {}), ((33, 5, 2.0, 0), {"mw": True}), ((32, 4, 2.0, 1), {"mw": True}),
             ((64, 3, 2.0, 0), {"multires": True}), ((33, 1, 2.0, 1), {})]
    for prec in ("mixed", "fp64"):
        plans = [B.Plan(*s, prec, **kw) for s, kw in specs]
        try:
            cd, _ = plans[0].torch_dtypes()
            fs = [torch.from_numpy(flm_gaussian(p.L, 60 + i, "cl")).to(cd).cuda() for i, p in enumerate(plans)]
            Wb = [p.alloc_w() for p in plans]
            Ws = [p.alloc_w() for p in plans]
            B.s2dw_analysis_batch([p.handle for p in plans], fs, [w[0] for w in Wb], [w[1] for w in Wb])
            for p, f, w in zip(plans, fs, Ws):
                p.analysis(f, w[0], w[1])
            torch.cuda.synchronize()
            for wb, ws in zip(Wb, Ws):
                assert torch.equal(wb[0], ws[0]) and torch.equal(wb[1], ws[1])
            fb = [p.alloc_flm() for p in plans]
            fsn = [p.alloc_flm() for p in plans]
            B.s2dw_synthesis_batch([p.handle for p in plans], [w[0] for w in Wb], [w[1] for w in Wb], fb)
            for p, w, f in zip(plans, Ws, fsn):
                p.synthesis(w[0], w[1], f)
            torch.cuda.synchronize()
            for i, (a, b, f0) in enumerate(zip(fb, fsn, fs)):
                assert torch.equal(a, b), i
                eps = (a.to(torch.complex128) - f0.to(torch.complex128)).abs().max().item()
                assert eps < (1e-12 if prec == "fp64" else 1e-5) * f0.abs().max().item(), (prec, i, eps)
        finally:
            for p in plans:
                p.close()
    assert B.s2dw_wait_timeouts() == 0
