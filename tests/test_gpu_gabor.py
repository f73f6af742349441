"""GPU parity of the Gabor orientation / confidence maps (hair_fuse_gabor, tensor cores) against the
CPU oracle on the same seeded images: the orientation index wherever the oracle's two largest
responses are further apart than the spread an FP32 evaluation can give them (the oracle's flag; at
least 95 % of the pixels of images without blank regions), the confidence within the
FP32-accumulation tolerance."""
import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(9)


def run(images, device=True):
    import torch

    import paper_2604_05794_b300 as hf
    with hf.HairFuse(8, 0, 0) as f:
        if device:
            th, cf = f.gabor(torch.from_numpy(np.ascontiguousarray(images)).cuda())
            f.sync()
            return th.cpu().numpy(), cf.cpu().numpy()
        return f.gabor(np.ascontiguousarray(images))


def compare(images, th, cf, v, idx, min_unique=0.95):
    o = oracle.gabor_pixels(images[v], idx)
    k = np.rint(th[v].ravel()[idx] * 64 / np.pi).astype(int) % 64
    ok = o["flag"] == 0
    assert ok.mean() > min_unique
    assert np.array_equal(k[ok], o["k"][ok]), np.nonzero(k[ok] != o["k"][ok])[0][:10]
    assert np.allclose(th[v].ravel()[idx][ok], o["theta"][ok], atol=1e-6)
    c = cf[v].ravel()[idx]
    assert np.all(np.abs(c - o["conf"]) <= 2e-4 + 2e-3 * (o["conf"] < 0.01)), np.max(np.abs(c - o["conf"]))
    return ok.mean()


def test_tiny_scene_views_every_pixel():
    sc = scenegen.make_scene("tiny")
    im = scenegen.strand_images(sc, seed=1)
    th, cf = run(im)
    for v in (0, 5):
        compare(im, th, cf, v, np.arange(im.shape[1] * im.shape[2]))
    # the maps find the strands: on covered pixels the angle is near the rendered one
    cov = sc["conf"] > 0
    d = np.abs((th - sc["angle"] + np.pi / 2) % np.pi - np.pi / 2)[cov]
    assert np.median(np.degrees(d)) < 15.0   # random angles would give 45


def test_ragged_sizes_and_random_images():
    for V, H, W in ((2, 37, 131), (1, 200, 256), (3, 16, 1)):
        im = RNG.random((V, H, W)).astype(np.float32)
        im[0, :, : W // 2] = 0.0
        th, cf = run(im)
        for v in range(V):   # the zeroed half of image 0 ties everywhere
            compare(im, th, cf, v, np.arange(H * W), min_unique=0.45 if v == 0 and W > 1 else 0.95)



def test_unit_boundaries_and_short_units():
    """One-row images (a CTA's tiles fewer than its accumulators), hundreds of two-row images (a CTA
    walks many units, the window-row ring and the per-tile barrier cross every unit boundary), and a
    tall single strip cut into runs of rows (several units per strip)."""
    for V, H, W, sample in ((3, 1, 7, 0), (300, 2, 130, 0), (1, 1080, 128, 6000)):
        im = RNG.random((V, H, W)).astype(np.float32)
        th, cf = run(im)
        for v in sorted({0, V // 2, V - 1}):
            idx = np.arange(H * W) if not sample else np.linspace(0, H * W - 1, sample).astype(np.int64)
            compare(im, th, cf, v, idx)


def test_full_view_sampled_and_host_path():
    sc = scenegen.make_scene("full", seed=2, knn=False)
    im = scenegen.strand_images({"conf": sc["conf"][:2]}, seed=2)
    th, cf = run(im)
    idx = np.linspace(0, im.shape[1] * im.shape[2] - 1, 4000).astype(np.int64)
    for v in range(2):
        compare(im, th, cf, v, idx)
    th2, cf2 = run(im, device=False)
    assert np.array_equal(th, th2) and np.array_equal(cf, cf2)


def test_gabor_arguments():
    import paper_2604_05794_b300 as hf
    im = np.zeros((1, 8, 8), np.float32)
    with hf.HairFuse(8, 0, 0) as f:
        for kw in (dict(n_theta=32), dict(radius=5), dict(sigma_along=0.0), dict(lambda_=float("nan"))):
            with pytest.raises(hf.HairFuseError):
                f.gabor(im, **kw)


def test_asynchronous_chunks_two_streams():
    """HF_HOST_ASYNC: chunks of views on two contexts / streams taking turns give the maps of one
    synchronous call bit for bit; pageable buffers are refused."""
    import torch

    import paper_2604_05794_b300 as hf
    im = RNG.random((7, 64, 200)).astype(np.float32)
    th, cf = run(im, device=False)
    h_im = torch.from_numpy(im).pin_memory()
    h_th = torch.empty(im.shape).pin_memory()
    h_cf = torch.empty(im.shape).pin_memory()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    fs = [hf.HairFuse(8, 0, 0, stream=s.cuda_stream) for s in streams]
    try:
        with pytest.raises(ValueError):
            fs[0].gabor(im, np.empty_like(im), np.empty_like(im), asynchronous=True)
        for q, v0 in enumerate(range(0, 7, 2)):
            fs[q & 1].gabor(h_im[v0:v0 + 2], h_th[v0:v0 + 2], h_cf[v0:v0 + 2], asynchronous=True)
        torch.cuda.synchronize()
        assert np.array_equal(h_th.numpy(), th) and np.array_equal(h_cf.numpy(), cf)
    finally:
        for f in fs:
            f.close()
