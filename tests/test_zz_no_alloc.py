"""The allocation-free variant of the A P + Gram entry point (for callers that cannot call
cudaMalloc): two calls in a row through the C ABI must reproduce the scratch-taking entry point's
output bit for bit (the same kernels run in the same launch shape, only the scratch differs), on the
default stream and on a stream of the caller's, and oversize requests must be rejected.
The rejection of launches wider than 1216 CTAs cannot be reached on a GB300 (152 SMs give at most
1216, 8 per SM); it is not exercised here. Collected last on purpose (file name), so a stop at the first
failure has run every other test."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_07327_gb300 as mb
    mb.lib()
    return mb


def _inputs(n, s, seed):
    A = wl.poisson2d(int(np.sqrt(n))) if seed == 0 else wl.random_spd_csr(n, seed, density=0.01)
    kp = 1 << (s - 1).bit_length()
    P = np.zeros((A.n, kp))
    P[:, :s] = wl.initial_block(A.n, s, 3)
    dev = torch.device("cuda")
    return (A, torch.as_tensor(A.row_ptr, device=dev), torch.as_tensor(A.col_idx, device=dev),
            torch.as_tensor(A.val, device=dev), torch.as_tensor(P, device=dev))


@pytest.mark.parametrize("on_stream", [False, True], ids=["default_stream", "own_stream"])
@pytest.mark.parametrize("n,s,seed", [(4096, 4, 0), (1000, 16, 5), (777, 3, 6), (100000, 8, 0)])
def test_noalloc_matches_scratch_entry_point_twice(mb, n, s, seed, on_stream):
    A, rp, ci, av, P = _inputs(n, s, seed)
    m = A.n
    dev = P.device
    AP_ref = torch.empty_like(P)
    G_ref = torch.empty((s, s), dtype=torch.float64, device=dev)
    nbytes = mb.mbpcg_k_scratch_bytes(m, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_spmm_gram(m, rp, ci, av, s, P, AP_ref, G_ref, scratch, nbytes, None) == 0
    torch.cuda.synchronize()
    stream = torch.cuda.Stream() if on_stream else None
    for _ in range(2):
        AP = torch.full_like(P, float("nan"))
        G = torch.full((s, s), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        st = mb.mbpcg_k_spmm_gram_noalloc(m, rp, ci, av, s, P, AP, G,
                                          stream.cuda_stream if stream is not None else None)
        assert st == 0, mb.last_error()
        torch.cuda.synchronize()
        assert torch.equal(AP, AP_ref)
        assert torch.equal(G, G_ref)


def test_noalloc_rejects_oversize(mb):
    A, rp, ci, av, P = _inputs(64, 32, 4)
    AP = torch.empty_like(P)
    G = torch.empty((32, 32), dtype=torch.float64, device=P.device)
    st = mb.mbpcg_k_spmm_gram_noalloc(A.n, rp, ci, av, 32, P, AP, G, None)
    assert st == 1
    assert "static scratch" in mb.last_error()
