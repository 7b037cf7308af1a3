"""Display resolve (pt_tonemap) against the oracle (oracle/tonemap.py), through the C-ABI.

Every step is an FP32 operation in the same order on both sides, so without the sRGB
transfer function the 8-bit codes are identical.  With it, CUDA's powf and the host's powf
may differ by an ulp or two, which can move a code by one where the value lies that close to
a rounding boundary: codes must then be equal everywhere except at such values, where they
may differ by one.
"""
import numpy as np
import pytest

from oracle import tonemap as otm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sums(rng, h, w, spp):
    """Seeded HDR accumulator contents: log-uniform radiance over 8 decades, black pixels,
    saturated highlights, greys, values around the toe (0.08) and the knee (0.76)."""
    m = np.exp(rng.uniform(np.log(1e-4), np.log(1e4), (h, w, 3)))
    flat = m.reshape(-1, 3)
    k = len(flat)
    flat[: k // 10] = 0.0
    flat[k // 10: k // 5] = np.repeat(rng.uniform(0, 3, (k // 5 - k // 10, 1)), 3, 1)
    flat[k // 5: k // 4] = rng.uniform(0.07, 0.09, (k // 4 - k // 5, 3))
    flat[k // 4: k // 3] = rng.uniform(0.75, 0.85, (k // 3 - k // 4, 3))
    return (m * spp).astype(np.float32)


def _accum(sums, spp):
    from paper_2407_19977_gb300 import api
    h, w = sums.shape[:2]
    acc = api.Accum(w, h)
    acc.sum.copy_(torch.from_numpy(sums))
    acc.c.spp_done = spp
    return acc


@pytest.mark.parametrize("h,w", [(1, 1), (23, 37), (257, 300), (1080, 1920)])
def test_tonemap_linear_bit_exact(api, h, w):
    rng = np.random.default_rng(h * 1000 + w)
    spp = 7
    sums = _sums(rng, h, w, spp)
    acc = _accum(sums, spp)
    got = acc.tonemap(exposure=1.3, srgb=False).cpu().numpy()
    exp = otm.resolve(sums, spp, exposure=1.3, srgb=False)
    assert np.array_equal(got, exp), int((got != exp).sum())


@pytest.mark.parametrize("h,w", [(23, 37), (1080, 1920)])
def test_tonemap_srgb(api, h, w):
    rng = np.random.default_rng(7 + h)
    spp = 16
    sums = _sums(rng, h, w, spp)
    acc = _accum(sums, spp)
    got = acc.tonemap(exposure=0.8, srgb=True).cpu().numpy().astype(np.int64)
    exp = otm.resolve(sums, spp, exposure=0.8, srgb=True).astype(np.int64)
    v = otm.resolve_float(sums, spp, exposure=0.8, srgb=True).astype(np.float64) * 255.0 + 0.5
    near = np.abs(v - np.round(v)) < 1e-4          # a few ulp of the value, in code units
    diff = np.abs(got[..., :3] - exp[..., :3])
    assert np.all(diff[~near] == 0), int((diff[~near] != 0).sum())
    assert np.all(diff[near] <= 1)
    assert np.all(got[..., 3] == 255)


def test_tonemap_of_a_rendered_image(api):
    """The whole display path: a GPU render and the oracle's render of the same seeded Cornell
    frame, each tone mapped on its own side, give the same picture."""
    import oracle
    from paper_2407_19977_gb300 import api as A, scenes
    sc = scenes.cornell_box()
    g = A.Scene(sc)
    acc = g.render(sc.spp, mode=1)
    got = acc.tonemap().cpu().numpy().astype(np.int64)
    o_sum, _, _ = oracle.OracleScene(sc).render(spp=sc.spp)
    exp = otm.resolve(o_sum.astype(np.float32), sc.spp).astype(np.int64)
    diff = np.abs(got - exp)
    assert diff.max() <= 2 and (diff <= 1).mean() >= 0.999


def test_tonemap_guards_and_errors(api):
    from paper_2407_19977_gb300 import native as N
    sums = np.zeros((2, 3, 3), np.float32)
    sums[0, 0] = np.nan
    sums[0, 1] = np.inf
    sums[1, 0] = -5.0
    sums[1, 1] = 3e38
    acc = _accum(sums, 2)
    got = acc.tonemap(srgb=True).cpu().numpy()
    assert np.array_equal(got, otm.resolve(sums, 2, srgb=True))
    acc.c.spp_done = 0
    with pytest.raises(N.PtError, match="INVALID_ARG"):
        acc.tonemap()
    acc.c.spp_done = 1
    with pytest.raises(N.PtError, match="INVALID_ARG"):
        acc.tonemap(exposure=-1.0)
    with pytest.raises(N.PtError, match="INVALID_ARG"):
        acc.tonemap(exposure=float("nan"))
