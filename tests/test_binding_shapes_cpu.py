"""Host-side logic of the binding's Plan: default output shapes, checked on
the CPU with a plan object that holds only its sizes and a recorder in place
of the library call (no device work)."""
import numpy as np
import torch

from paper_1308_5706_gb300 import binding as B


def _fake_plan(L, N, J, mw=False, multires=False, w_elems=0):
    p = object.__new__(B.Plan)
    p.L, p.N, p.J, p.nscale = L, N, J, J + 1
    p.nb = L if mw else 2 * L
    p.multires = multires
    p.handle = 0
    # (band-limit, offset, elements) per scale; the last entry is the scaling part
    per = w_elems // (J + 1)
    p.grids = [(L, j * per, per) for j in range(J + 1)] + [(L, 0, 0)]
    return p


def test_steer_default_shape_follows_the_beta_grid(monkeypatch):
    calls = []
    monkeypatch.setattr(B, "s2dw_steer", lambda h, W, g, out, st: calls.append(tuple(out.shape)))
    W = torch.zeros(1)
    for mw, nb in ((False, 2 * 16), (True, 16)):
        p = _fake_plan(16, 3, 4, mw=mw)
        out = p.steer(W, np.array([0.1, 0.7]))
        assert tuple(out.shape) == (5, 2, nb, 31) == calls[-1]
    p = _fake_plan(16, 3, 4, multires=True, w_elems=5 * 3 * 200)
    out = p.steer(W, np.array([0.1, 0.7, 1.3]))
    assert tuple(out.shape) == (5 * 3 * 200 // 3 * 3,)  # W holds N = 3 orientations, out the 3 requested
