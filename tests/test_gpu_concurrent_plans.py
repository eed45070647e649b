"""Plans created concurrently from several host threads, with transforms
running meanwhile on the main thread, all succeed and give the same
coefficients as plans created alone (the serving path creates plans in
worker threads)."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian

pytestmark = pytest.mark.gpu


def test_concurrent_plan_creation_with_transforms_running():
    import torch
    # band-limits whose chirp-z lengths differ (2^9 .. 2^13), so that the
    # plan-time kernels of different threads use different shared-memory sizes
    cfgs = [(L, N) for L in (100, 250, 700, 1500, 1942, 64, 300, 1030) for N in (1, 4)]
    main = B.Plan(512, 3, 2.0, 0, "mixed")
    f = torch.from_numpy(flm_gaussian(512, 5, "cl")).to(torch.complex64).cuda()
    W, Wp = main.alloc_w()
    fr = main.alloc_flm()
    with cf.ThreadPoolExecutor(max_workers=4) as pool:
        futs = [pool.submit(B.Plan, L, N, 2.0, 0, "mixed") for L, N in cfgs]
        while not all(fu.done() for fu in futs):
            main.analysis(f, W, Wp)
            main.synthesis(W, Wp, fr)
        plans = [fu.result() for fu in futs]  # raises if a creation failed
    torch.cuda.synchronize()
    f0 = f.to(torch.complex128)
    assert float((fr.to(torch.complex128) - f0).abs().max() / f0.abs().max()) < 1e-5
    # two of the concurrently created plans against plans created alone
    for p in (plans[5], plans[8]):
        q = B.Plan(p.L, p.N, 2.0, 0, "mixed")
        g = torch.from_numpy(flm_gaussian(p.L, 7, "cl")).to(torch.complex64).cuda()
        Wa, Wpa = p.alloc_w()
        Wb, Wpb = q.alloc_w()
        p.analysis(g, Wa, Wpa)
        q.analysis(g, Wb, Wpb)
        torch.cuda.synchronize()
        assert torch.equal(Wa, Wb) and torch.equal(Wpa, Wpb)
        q.close()
    for p in plans:
        p.close()
    main.close()
