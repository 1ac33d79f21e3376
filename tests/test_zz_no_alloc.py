"""The allocation-free variant of the A P + Gram entry point (for callers that cannot call
cudaMalloc): two calls in a row through the C ABI must reproduce the scratch-taking entry point's
output, within the tolerance the kernel tests use, and oversize requests must be rejected.
Collected last on purpose (file name), so a stop at the first failure has run every other test."""
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


@pytest.mark.parametrize("n,s,seed", [(4096, 4, 0), (1000, 16, 5), (777, 3, 6), (100000, 8, 0)])
def test_noalloc_matches_scratch_entry_point_twice(mb, n, s, seed):
    A, rp, ci, av, P = _inputs(n, s, seed)
    m = A.n
    dev = P.device
    AP_ref = torch.empty_like(P)
    G_ref = torch.empty((s, s), dtype=torch.float64, device=dev)
    nbytes = mb.mbpcg_k_scratch_bytes(m, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_spmm_gram(m, rp, ci, av, s, P, AP_ref, G_ref, scratch, nbytes, None) == 0
    torch.cuda.synchronize()
    scale_ap = AP_ref.abs().max().item() + 1e-300
    scale_g = G_ref.abs().max().item() + 1e-300
    for _ in range(2):
        AP = torch.full_like(P, float("nan"))
        G = torch.full((s, s), float("nan"), dtype=torch.float64, device=dev)
        st = mb.mbpcg_k_spmm_gram_noalloc(m, rp, ci, av, s, P, AP, G, None)
        assert st == 0, mb.last_error()
        torch.cuda.synchronize()
        assert (AP - AP_ref).abs().max().item() <= 1e-13 * scale_ap
        assert (G - G_ref).abs().max().item() <= 1e-12 * scale_g


def test_noalloc_rejects_oversize(mb):
    A, rp, ci, av, P = _inputs(64, 32, 4)
    AP = torch.empty_like(P)
    G = torch.empty((32, 32), dtype=torch.float64, device=P.device)
    st = mb.mbpcg_k_spmm_gram_noalloc(A.n, rp, ci, av, 32, P, AP, G, None)
    assert st == 1
    assert "static scratch" in mb.last_error()
