"""The Delta-table entry point that allocates nothing (s2dw_delta_table_noalloc).

Some callers cannot let the library call cudaMalloc (their device memory
belongs to another allocator, or allocating is not allowed where they run);
this entry point writes the table into buffers the caller owns and keeps its
own scratch in a fixed array inside the library.  Its table must equal the
one the plans build (read back with s2dw_delta_slab) and, on sampled entries
at every l, the CPU oracle's d^l_{m'm}(pi/2), within the 1e-13 used by the
other Delta-table tests, on two calls in a row that share the scratch; the
second call must leave the device's free memory unchanged.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest

from paper_1308_5706_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _slab(table, l):
    """Expand slab l of the padded layout (documented in include/s2dw.h)."""
    C, r = l >> 2, l & 3
    c = C + 1
    base = (32 * C * (C + 1) * (C + 2)) // 3 + r * 8 * c * (c + 1)
    mp = np.arange(l + 1)[:, None]
    m = np.arange(l + 1)[None, :]
    direct = m >= 4 * (mp >> 2)
    a = np.where(direct, mp, m)
    b = np.where(direct, m, mp)
    q, rr = a >> 2, a & 3
    idx = 16 * q * c - 8 * q * (q - 1) + 4 * rr * (c - q) + (b - 4 * q)
    sign = np.where(direct | ((mp - m) % 2 == 0), 1.0, -1.0)
    return sign * table[base + idx]


def _entries(table, l, mp, m):
    """Delta^l_{m'm} read from the layout at arrays (l, m', m), 0 <= m', m <= l."""
    C, r = l >> 2, l & 3
    c = C + 1
    base = (32 * C * (C + 1) * (C + 2)) // 3 + r * 8 * c * (c + 1)
    direct = m >= 4 * (mp >> 2)
    a = np.where(direct, mp, m)
    b = np.where(direct, m, mp)
    q, rr = a >> 2, a & 3
    idx = 16 * q * c - 8 * q * (q - 1) + 4 * rr * (c - q) + (b - 4 * q)
    sign = np.where(direct | ((mp - m) % 2 == 0), 1.0, -1.0)
    return sign * table[base + idx]


def test_noalloc_delta_table_matches_plan_table_and_oracle():
    import torch
    import oracle as O
    plan = B.Plan(1024, 1, 2.0, 0, "fp64")
    stream = torch.cuda.current_stream()
    with pytest.raises(B.S2dwError) as ei:
        B.s2dw_delta_table_noalloc(1025)
    assert ei.value.status == B.S2DW_ENOTSUP
    # the binding refuses buffers of the wrong type or size before the C call
    n300 = B.s2dw_delta_table_noalloc(300)
    with pytest.raises(ValueError):
        B.s2dw_delta_table_noalloc(300, torch.zeros(n300, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        B.s2dw_delta_table_noalloc(300, torch.zeros(n300 - 1, dtype=torch.float64, device="cuda"))
    rng = np.random.default_rng(3)
    for call, Lmax in enumerate((1024, 300)):   # two calls in a row sharing the scratch array
        n = B.s2dw_delta_table_noalloc(Lmax)
        t64 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        t32 = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert B.s2dw_delta_table_noalloc(Lmax, t64, t32, stream) == n
        torch.cuda.synchronize()
        if call > 0:   # after a first call (module loading, symbol look-up) nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0
        h64 = t64.cpu().numpy()
        h32 = t32.cpu().numpy()
        assert np.isfinite(h64).all() and np.isfinite(h32).all()
        assert np.array_equal(h32, h64.astype(np.float32))
        for l in sorted({0, 1, 2, 3, 5, 63, 64, 65, Lmax // 2, Lmax - 2, Lmax - 1}):
            got = _slab(h64, l)
            ref = plan.delta_slab(l)
            assert np.abs(got - ref).max() <= 1e-13, (Lmax, l)
        # sampled entries at every l against the CPU oracle's d^l_{m'm}(pi/2)
        mp = rng.integers(0, Lmax, 160)
        m = rng.integers(0, Lmax, 160)
        ref = O.delta(Lmax, mp, m)                      # [l][pair]
        for l in range(Lmax):
            ok = (mp <= l) & (m <= l)
            if ok.any():
                got = _entries(h64, l, mp[ok], m[ok])
                assert np.abs(got - ref[l][ok]).max() <= 1e-13, (Lmax, l)
    plan.close()
