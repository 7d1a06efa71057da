"""kbe_op_sigma_row_noalloc: the self-energy row for callers that cannot
allocate device memory (their device memory is owned by another allocator,
or cudaMalloc/cudaFree would synchronise a latency-critical loop).

The variant keeps its scratch in a fixed device array inside libkbe. These
checks call it through the C ABI and compare its output with the existing
kbe_op_sigma_row (caller-provided scratch) on two calls in a row: the second
call is smaller than the first and so runs on top of the first call's stale
scratch, which must not leak into the result. The file is named to run last.
"""
import numpy as np
import pytest

import kbe_inputs as ki
from layout import relerr

torch = pytest.importorskip("torch")
kbe = pytest.importorskip("paper_2505_19467_gb300")

pytestmark = pytest.mark.gpu
TOL = 1e-12   # the tolerance of the Sigma-row parity tests


def _row(rng, n, nb, nk):
    Gl = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    Gg = ki.random_blocks(rng, (n + 1, nk, nb, nb))
    D = np.stack([Gl, Gg], axis=1).transpose(0, 1, 3, 4, 2)
    return torch.from_numpy(np.ascontiguousarray(D)).cuda()


def _reference(nb, L, v, n, Un, Grow, Ul=None):
    out = torch.empty_like(Grow)
    work = torch.empty(kbe.sigma_row_workspace(nb, L, n) // 16 + 1, dtype=torch.complex128, device="cuda")
    kbe.sigma_row(nb, L, v, n, Un, Grow, out, work, Ul=Ul)
    return out


def test_noalloc_matches_caller_scratch_on_two_calls_in_a_row():
    rng = np.random.default_rng(4242)
    calls = [(4, (8, 8), 40, None), (2, (6, 1), 7, rng.uniform(0.5, 1.5, 8))]
    for nb, L, n, Ul in calls:
        nk = L[0] * L[1]
        Grow = _row(rng, n, nb, nk)
        v = ki.pair_pattern(nb)
        Ul_d = None if Ul is None else torch.from_numpy(Ul).cuda()
        got = torch.full_like(Grow, float("nan"))
        kbe.sigma_row_noalloc(nb, L, v, n, 0.8, Grow, got, Ul=Ul_d)
        want = _reference(nb, L, v, n, 0.8, Grow, Ul=Ul_d)
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert np.isfinite(g).all()
        assert relerr(g, w)[1] < TOL, (nb, L, n)


def test_noalloc_rejects_rows_larger_than_its_scratch():
    nb, L = 4, (8, 8)
    # scratch of one row: 2 * (n+1) * 2 * nb^2 * nk * 16 bytes
    n = kbe.NOALLOC_SCRATCH_BYTES // (2 * 2 * nb * nb * 64 * 16)   # one row too many
    assert kbe.sigma_row_workspace(nb, L, n) > kbe.NOALLOC_SCRATCH_BYTES
    Grow = torch.zeros((1, 2, nb, nb, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(kbe.KBEError) as e:
        kbe.sigma_row_noalloc(nb, L, ki.pair_pattern(nb), n, 1.0, Grow, Grow)
    assert e.value.status == -1 and "scratch" in str(e.value)
