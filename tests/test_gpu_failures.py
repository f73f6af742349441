"""Failure paths that can be exercised without faulting the GPU.

A bounded device wait is made to expire by giving the GEMM's (or the network kernel's) pipeline a
limit of 1 ns: the call must report HF_ERR_TIMEOUT (the CTAs drain their own copies and tensor-core work, which complete by
themselves, before they release shared and tensor memory) and the next call must run normally.
An out-of-memory condition is injected on the host at every device allocation a fusion makes in
turn: the call that needed it must return HF_ERR_OOM, and destroying the context must give all
device memory back."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


def test_forced_wait_expiry_then_clean_call():
    import torch

    import paper_2604_05794_b300 as hf
    g = torch.Generator(device="cuda").manual_seed(7)
    M, N, K = 512, 128, 512
    a = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    ref = a.float() @ b.float().T
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        c = torch.empty((M, N), device="cuda")
        rc = hf.hair_fuse_gemm_bf16_bounded(a.data_ptr(), b.data_ptr(), c.data_ptr(), M, N, K, 1, stream)
        assert rc == hf.HF_ERR_TIMEOUT, (rc, hf.hair_fuse_last_error(None))
        assert b"bounded device wait expired" in hf.hair_fuse_last_error(None)
        c.zero_()
        rc = hf.hair_fuse_gemm_bf16_bounded(a.data_ptr(), b.data_ptr(), c.data_ptr(), M, N, K, 0, stream)
        assert rc == hf.HF_OK, hf.hair_fuse_last_error(None)
        torch.cuda.synchronize()
        assert (c - ref).abs().max().item() <= 2e-5 * ref.abs().max().item() + 1e-3


def test_network_forced_wait_expiry_then_clean_call():
    """The fused inference kernel in its test mode (a 1 ns limit on every pipeline wait, and a wait on
    a barrier nothing completes once the first tile's layer-1 steps are in flight): HF_ERR_TIMEOUT,
    with the warps draining their own copies and tensor-core steps before the CTA releases its
    memory; then, back in normal operation, the same proposals as before, bit for bit."""
    import paper_2604_05794_b300 as hf
    net = hf.ProposalNet(1024)
    net.init(3)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, size=(3000, 64)).astype(np.float32)
    x[:, 51:] = 0.0
    X = (x.view(np.uint32) >> 16).astype(np.uint16)   # bf16 codes (truncated)
    ref = net.forward(X)
    for _ in range(2):
        assert hf.hair_fuse_mlp_set_wait_limit(net.h, 1) == hf.HF_OK
        with pytest.raises(hf.HairFuseError) as e:
            net.forward(X)
        assert e.value.code == hf.HF_ERR_TIMEOUT
        assert b"bounded device wait expired" in hf.hair_fuse_mlp_last_error(net.h)
        assert hf.hair_fuse_mlp_set_wait_limit(net.h, 0) == hf.HF_OK
        assert np.array_equal(net.forward(X), ref)
    net.close()


def _fuse_once(hf, sc, H, T):
    """create, upload (host), fuse (host): the first non-OK return code, or HF_OK."""
    N = sc["N"]
    out = np.empty((N, 3), np.float32)
    cost = np.empty(N, np.float32)
    try:
        f = hf.HairFuse(H, sc["k"], T)
    except hf.HairFuseError as e:
        return e.code
    try:
        f.upload_views(sc["cams"], sc["angle"], sc["conf"])
        f.upload_points(sc["points"], sc["nbr"])
        f.fuse(out, cost)
        return hf.HF_OK
    except hf.HairFuseError as e:
        return e.code
    finally:
        f.close()


def test_injected_allocation_failure_each_allocation():
    import torch

    import paper_2604_05794_b300 as hf
    sc = scenegen.make_scene("tiny")
    H, T = 32, 4
    assert _fuse_once(hf, sc, H, T) == hf.HF_OK   # settle CUDA's own lazy allocations
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen_ok = False
    for n in range(64):
        hf.hair_fuse_fail_alloc_after(n)
        rc = _fuse_once(hf, sc, H, T)
        hf.hair_fuse_fail_alloc_after(-1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, n   # nothing leaked
        if rc == hf.HF_OK:   # n is past the fusion's last allocation
            seen_ok = True
            break
        assert rc == hf.HF_ERR_OOM, (n, rc)
    assert seen_ok and n >= 5
    assert _fuse_once(hf, sc, H, T) == hf.HF_OK
