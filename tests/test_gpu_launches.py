"""The launch counts a plan reports match the kernels one call really runs
(counted by the CUDA profiler), and every launched kernel is one of ours."""
import pytest

from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian

pytestmark = pytest.mark.gpu


def _kernels_of(fn):
    """Names of the kernels `fn` launches.  The first profiler session of a
    process can come back empty while the CUDA activity tracing starts up, so
    an empty record is taken once more."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    names = []
    for _ in range(2):
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA
                 and "memcpy" not in e.name.lower() and "memset" not in e.name.lower()]
        if names:
            break
    return names


@pytest.mark.parametrize("L,N,prec", [(16, 3, "mixed"), (96, 4, "fp64"), (256, 5, "mixed")])
def test_launch_counts(L, N, prec):
    import torch
    p = B.Plan(L, N, 2.0, 0, prec)
    cd = torch.complex64 if prec == "mixed" else torch.complex128
    f = torch.from_numpy(flm_gaussian(L, 1, "cl")).to(cd).cuda()
    W, Wp = p.alloc_w()
    g = p.alloc_flm()
    p.analysis(f, W, Wp)
    p.synthesis(W, Wp, g)
    na, ns = p.launch_counts()
    ka = _kernels_of(lambda: p.analysis(f, W, Wp))
    ks = _kernels_of(lambda: p.synthesis(W, Wp, g))
    if not ka:
        pytest.skip("profiler recorded no CUDA kernels")
    assert len(ka) == na and len(ks) == ns
    assert all(k.startswith("void s2dw::") or "s2dw" in k for k in ka + ks), ka + ks
    p.close()


def test_stage_profile_covers_the_calls():
    """Stage events bracket every launch: two calls of each direction are
    counted, every stage is timed, and the stages add up to the calls."""
    import torch
    p = B.Plan(64, 3, 2.0, 0, "mixed")
    f = torch.from_numpy(flm_gaussian(64, 2, "cl")).to(torch.complex64).cuda()
    W, Wp = p.alloc_w()
    g = p.alloc_flm()
    p.analysis(f, W, Wp)
    p.synthesis(W, Wp, g)
    torch.cuda.synchronize()
    p.profile(True)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(2):
        p.analysis(f, W, Wp)
        p.synthesis(W, Wp, g)
    e.record()
    torch.cuda.synchronize()
    ms, na, ns = p.profile_read()
    p.profile(False)
    assert (na, ns) == (2, 2)
    assert list(ms) == B.STAGES and all(v >= 0 for v in ms.values())
    total = s.elapsed_time(e)
    assert 0 < sum(ms.values()) <= total * 1.05 + 0.05
    p.close()
