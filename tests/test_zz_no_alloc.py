"""phmm_forward_noalloc: the FP32 forward pass for callers that cannot allocate device
memory at call time (a host framework that owns the device heap, a process that reserved
all device memory up front).  Its scratch lives in fixed arrays inside the library.

Checked through the C ABI against the regular entry point (phmm_submit_batch), within
the FP32 tolerance, on two calls in a row (the scratch keeps the previous call's
contents, so the second call must not depend on it).  This file is collected last.
"""
import numpy as np
import pytest

import oracle  # noqa: F401  (same test infrastructure as the other GPU tests)
from paper_2606_25738_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-3


@pytest.fixture(scope="module")
def phmm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_25738_gb300 import phmm as P
    return P


def _regular(phmm, b):
    with phmm.Context(precision="fp32") as ctx:
        out, flags, rc, st = ctx.run(b)
    return out


def test_noalloc_matches_regular_twice(phmm):
    import torch
    batches = [W.plain_pairs(64, seed=0), W.plain_pairs(40, seed=9, k_range=(1, 1024), l_range=(1, 300))]
    for b in batches:
        ref = _regular(phmm, b)
        d = phmm.to_device(b)
        n = len(b["pair_read"])
        for _call in range(2):
            out = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
            fl = torch.full((n,), 0xFF, dtype=torch.uint8, device="cuda")
            rc = phmm.forward_noalloc(d, out, fl)
            assert rc == 0, rc
            o = out.cpu().numpy()
            assert np.all(np.isfinite(o))
            assert np.max(np.abs(o - ref)) <= TOL32


def test_noalloc_rejects_oversize(phmm):
    import torch
    b = W.from_strings([("ACGT" * 10, "ACGT" * 300, 30, 45, 45, 10), ("ACGT", "ACGTA", 30, 45, 45, 10)])
    d = phmm.to_device(b)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    fl = torch.zeros(2, dtype=torch.uint8, device="cuda")
    assert phmm.forward_noalloc(d, out, fl) == phmm.PHMM_EINVAL  # haplotype of 1200 > 1024
    o = out.cpu().numpy()
    assert np.isnan(o[0]) and np.isfinite(o[1])
    assert (fl.cpu().numpy()[0] & phmm.PAIR_ERROR) != 0
