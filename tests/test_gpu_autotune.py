"""Launch methods and the autotuner: every available method of the beta and
alpha sums gives the oracle's coefficients (FP64 within 1e-11, mixed within
1e-5), invalid choices are refused, and a tuned plan agrees with the default
plan and is not slower than it."""
import numpy as np
import pytest

import oracle as O
from paper_1308_5706_gb300 import binding as B
from paper_1308_5706_gb300.inputs import flm_gaussian

pytestmark = pytest.mark.gpu


def _run(p, f):
    import torch
    W, Wp = p.alloc_w()
    p.analysis(f, W, Wp)
    fr = p.alloc_flm()
    p.synthesis(W, Wp, fr)
    torch.cuda.synchronize()
    return W, Wp, fr


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_every_method_matches_the_oracle(prec, tol):
    import torch
    L, N, lam, J0 = 64, 3, 2.0, 1
    f = flm_gaussian(L, 21, "cl")
    Wo, Wpo = O.analysis(f, L, N, lam, J0)
    p = B.Plan(L, N, lam, J0, prec)
    cd, _ = p.torch_dtypes()
    fd = torch.from_numpy(f).to(cd).cuda()
    base = p.choices()
    nsc = (len(base) - 3) // 2
    # every alternative of each choice, one at a time
    trials = []
    for i in range(2):
        trials.append((i, 1 - base[i]))
    for j in range(nsc):
        for d in range(2):
            for v in (0, 1, 2):
                if v != base[2 + 2 * j + d]:
                    trials.append((2 + 2 * j + d, v))
    for v in (0, 1, 2):  # the contraction's CTA shapes
        if v != base[-1]:
            trials.append((len(base) - 1, v))
    tried = 0
    for idx, v in trials:
        ch = list(base)
        ch[idx] = v
        try:
            p.set_choices(ch)
        except B.S2dwError as e:
            assert e.status == B.S2DW_EINVAL   # method not available for that scale
            continue
        tried += 1
        W, Wp, fr = _run(p, fd)
        assert p.choices() == ch
        Wn = W.double().cpu().numpy()
        assert _rel(Wn, Wo) < tol, (idx, v)
        assert _rel(Wp.double().cpu().numpy(), Wpo) < tol or np.abs(Wpo).max() == 0
        assert _rel(fr.to(torch.complex128).cpu().numpy(), f) < tol, (idx, v)
    assert tried >= 4
    p.close()


def test_invalid_choices_are_refused():
    p = B.Plan(64, 3, 2.0, 0, "mixed")
    ch = p.choices()
    assert ch[-1] == 1  # L = 64: one tile per CTA by default (too few pairs for the SMs)
    big = B.Plan(1024, 5, 2.0, 0, "mixed")  # 528 pairs, N >= 4: both tiles of a pair per CTA
    assert big.choices()[-1] == 0
    big.close()
    big = B.Plan(1024, 3, 2.0, 0, "mixed")  # N <= 3: one tile at two CTAs per SM
    assert big.choices()[-1] == 2
    big.close()
    bad = list(ch)
    bad[-1] = 3
    with pytest.raises(B.S2dwError):
        p.set_choices(bad)
    for v in (0, 2):  # N <= 5: all three shapes available
        ok = list(ch)
        ok[-1] = v
        p.set_choices(ok)
        assert p.choices()[-1] == v
    p.set_choices(ch)
    q = B.Plan(64, 7, 2.0, 0, "mixed")  # N > 5: one tile per CTA only
    chq = q.choices()
    assert chq[-1] == 1
    for v in (0, 2):
        chq[-1] = v
        with pytest.raises(B.S2dwError):
            q.set_choices(chq)
    q.close()
    r = B.Plan(64, 3, 2.0, 0, "fp64")  # the FP64 contraction has one shape
    chr_ = r.choices()
    assert chr_[-1] == 0
    chr_[-1] = 1
    with pytest.raises(B.S2dwError):
        r.set_choices(chr_)
    r.close()
    with pytest.raises(B.S2dwError) as ei:
        p.set_choices(ch[:-1])
    assert ei.value.status == B.S2DW_EINVAL
    bad = list(ch)
    bad[0] = 7
    with pytest.raises(B.S2dwError):
        p.set_choices(bad)
    # direct sums are sized for bands up to 32: not available for the largest scale
    bad = list(ch)
    bad[2] = 0
    with pytest.raises(B.S2dwError):
        p.set_choices(bad)
    assert p.choices() == ch
    p.close()


def test_tuned_plan_agrees_with_default_and_is_not_slower(tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("S2DW_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    L, N = 512, 5
    f = torch.from_numpy(flm_gaussian(L, 2, "cl")).to(torch.complex64).cuda()
    pd = B.Plan(L, N, 2.0, 0, "mixed")
    pt = B.Plan(L, N, 2.0, 0, "mixed", autotune=True)
    assert pt.tuned[1] == "tuned"
    Wd, Wpd, frd = _run(pd, f)
    Wt, Wpt, frt = _run(pt, f)
    for j in range(pd.nscale):
        ref = Wd[j].abs().max()
        if float(ref) > 0:
            assert float((Wt[j] - Wd[j]).abs().max() / ref) < 1e-5
    f0 = f.to(torch.complex128)
    assert float((frt.to(torch.complex128) - f0).abs().max() / f0.abs().max()) < 1e-5

    def timed(p):
        W, Wp = p.alloc_w()
        fr = p.alloc_flm()
        for _ in range(3):
            p.analysis(f, W, Wp)
            p.synthesis(W, Wp, fr)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                p.analysis(f, W, Wp)
                p.synthesis(W, Wp, fr)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    td, tt = timed(pd), timed(pt)
    assert tt <= 1.05 * td, (tt, td)
    # a second plan of the configuration takes the cached choices
    pc = B.Plan(L, N, 2.0, 0, "mixed", autotune=True)
    assert pc.tuned == (pt.choices(), "cache")
    for p in (pd, pt, pc):
        p.close()


@pytest.mark.parametrize("L,N", [(300, 5), (300, 3), (1030, 2)])
def test_contraction_shapes_give_identical_results(L, N):
    """The three CTA shapes of the FP32 contraction sum the same terms in the
    same l order per output: W and the synthesis are bit-identical."""
    import torch
    p = B.Plan(L, N, 2.0, 0, "mixed")
    f = torch.from_numpy(flm_gaussian(L, 13, "cl")).to(torch.complex64).cuda()
    ch = p.choices()
    outs = []
    for shape in (0, 1, 2):
        c = list(ch)
        c[-1] = shape
        p.set_choices(c)
        W, Wp, fr = _run(p, f)
        outs.append((W.clone(), Wp.clone(), fr.clone()))
    for W, Wp, fr in outs[1:]:
        assert torch.equal(W, outs[0][0]) and torch.equal(Wp, outs[0][1]) and torch.equal(fr, outs[0][2])
    f0 = f.to(torch.complex128)
    assert float((outs[0][2].to(torch.complex128) - f0).abs().max() / f0.abs().max()) < 1e-5
    p.close()
