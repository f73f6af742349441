"""Pins of the CPU oracle of the Gabor orientation / confidence maps (Sec. 3.1; no GPU): bfloat16
rounding against torch, the bank's symmetries (zero-mean even kernels, odd antisymmetry, the quarter
turn), straight lines and gratings at known angles, a quarter-turned image, and flat images."""
import numpy as np
import torch

import oracle

RNG = np.random.default_rng(2)


def test_bf16_rounding_matches_torch():
    x = np.concatenate([RNG.normal(size=2000).astype(np.float32) * 10,
                        np.float32([0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 1e-30])])
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(oracle.bf16(x).view(np.uint32), want.view(np.uint32))


def test_bank_symmetries():
    b = oracle.gabor_bank()
    ev, od = b[:, 0].astype(np.float64), b[:, 1].astype(np.float64)
    # even kernels: point-symmetric and zero-mean up to their bf16 rounding; odd: antisymmetric
    assert np.array_equal(ev, ev[:, ::-1, ::-1]) and np.array_equal(od, -od[:, ::-1, ::-1])
    assert np.all(np.abs(ev.sum(axis=(1, 2))) < 225 * 2 ** -8 * np.abs(ev).max())
    # a quarter turn: orientation k + 32 is orientation k rotated by 90 degrees, to one bf16 step
    for k in range(32):
        rot = np.rot90(b[k], k=1, axes=(1, 2))      # (u, v) -> the kernel seen a quarter turn later
        d = np.abs(b[k + 32] - rot)
        assert np.all(d <= 2 ** -7 * np.abs(b[k]).max() + 1e-7) or np.all(
            np.abs(b[k + 32] - np.rot90(b[k], k=-1, axes=(1, 2))) <= 2 ** -7 * np.abs(b[k]).max() + 1e-7)


def line_image(H, W, phi, width=0.8, cx=None, cy=None):
    cx = W / 2 if cx is None else cx
    cy = H / 2 if cy is None else cy
    y, x = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    d = -(x - cx) * np.sin(phi) + (y - cy) * np.cos(phi)        # distance across the line
    return np.exp(-d * d / (2 * width * width)).astype(np.float32)


def test_lines_at_known_angles():
    for phi in np.linspace(0.0, np.pi, 13, endpoint=False) + 0.01:
        img = line_image(64, 64, phi)
        # pixels on the line, away from the border
        t = np.linspace(-15, 15, 31)
        px = (32 + t * np.cos(phi)).astype(int), (32 + t * np.sin(phi)).astype(int)
        idx = px[1] * 64 + px[0]
        r = oracle.gabor_pixels(img, idx)
        err = np.abs((r["theta"] - phi + np.pi / 2) % np.pi - np.pi / 2)
        assert np.all(err[r["flag"] == 0] <= np.pi / 64 + 0.05), np.degrees(err.max())
        assert np.all(r["conf"] > 0.3)


def test_grating_picks_its_filter():
    for k in (0, 5, 17, 40, 63):
        th = np.pi * k / 64
        y, x = np.mgrid[0:48, 0:48].astype(np.float64)
        b = -(x - 24) * np.sin(th) + (y - 24) * np.cos(th)
        img = (0.5 + 0.5 * np.cos(2 * np.pi * b / 4.0)).astype(np.float32)
        r = oracle.gabor_pixels(img, np.array([24 * 48 + 24, 20 * 48 + 27]))
        assert np.all(r["k"] == k), (k, r["k"])


def test_quarter_turn_and_flat_images():
    img = np.clip(line_image(48, 48, 0.7) + line_image(48, 48, 2.1, cx=20) * 0.5, 0, 1)
    img = oracle.bf16(img)
    inner = np.array([y * 48 + x for y in range(10, 38) for x in range(10, 38)])
    a = oracle.gabor_pixels(img, inner)
    rot = np.ascontiguousarray(np.rot90(img, k=1))              # a quarter turn of the image
    # the pixel (y, x) of img sits at (47 - x, y) of rot
    inner_rot = np.array([(47 - (q % 48)) * 48 + (q // 48) for q in inner])
    b = oracle.gabor_pixels(rot, inner_rot)
    ok = (a["flag"] == 0) & (b["flag"] == 0) & (a["conf"] > 0.05)
    dk = (b["k"] - a["k"]) % 64
    assert ok.mean() > 0.5 and np.mean(dk[ok] == 32) > 0.95, np.bincount(dk[ok])
    # a flat image: no odd response, a tiny even one (the kernels' rounded means)
    flat = np.full((40, 40), 0.6, np.float32)
    c = oracle.gabor_pixels(flat, np.array([20 * 40 + 20]))
    assert c["conf"][0] < 0.99


def test_correlations_against_scipy():
    """The window correlation written out in the oracle equals scipy's 2-D correlation (zero fill,
    window centred) of the bf16 image with each kernel of the bank; the orientation index, the
    angle and the confidence follow from those responses by their definitions."""
    from scipy.signal import correlate2d
    H, W = 40, 37
    img = oracle.bf16(RNG.random((H, W)).astype(np.float32)).astype(np.float64)
    b = oracle.gabor_bank().astype(np.float64)
    F = np.empty((64, H, W))
    S = np.empty((64, H, W))   # sums of the absolute products of both correlations
    cor = lambda a, k: correlate2d(a, k, mode="same", boundary="fill", fillvalue=0.0)
    for k in range(64):
        e, o = cor(img, b[k, 0]), cor(img, b[k, 1])
        F[k] = np.sqrt(e * e + o * o)
        S[k] = cor(np.abs(img), np.abs(b[k, 0])) + cor(np.abs(img), np.abs(b[k, 1]))
    r = oracle.gabor_pixels(img.astype(np.float32), np.arange(H * W))
    Fs = np.sort(F, axis=0)
    # the index is unique unless the two largest responses lie within the spread an FP32 evaluation
    # can give them: 15 window-row steps of relative error 2^-22 on each correlation, F^2 compared
    # at 2^-16
    margin = 2 * 15 * 2.0 ** -22 * S.max(axis=0) + 2.0 ** -16 * Fs[-1]
    unique = (Fs[-1] - Fs[-2] > margin).ravel()
    assert np.array_equal(r["flag"] == 0, unique)
    kb = np.argmax(F, axis=0).ravel()
    assert unique.mean() > 0.9 and np.array_equal(r["k"][unique], kb[unique])
    assert np.allclose(r["theta"][unique], (np.pi * kb / 64)[unique], atol=1e-6)
    conf = 1.0 - F.mean(axis=0) / F.max(axis=0)
    assert np.allclose(r["conf"], conf.ravel(), atol=2e-7, rtol=0)
