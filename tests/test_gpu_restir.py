"""ReSTIR DI at the primary vertex on the GPU, through the C-ABI, against the oracle's ReSTIR
(same light candidates, same neighbours, same random numbers; the oracle's own pins are in
test_oracle_restir.py)."""
import numpy as np
import pytest

import oracle
from paper_2407_19977_gb300 import scenes
from tests.test_gpu_parity import _samples_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gpu(g, sc, restir, spp, crop=None, seed=0, s0=0, **kw):
    from paper_2407_19977_gb300 import api as A
    cam = sc.camera
    x0, y0, cw, ch = crop or (0, 0, cam.width, cam.height)
    samples = torch.zeros((ch, cw, spp, 3), dtype=torch.float32, device="cuda")
    acc = A.Accum(cw, ch)
    acc.c.spp_done = s0
    g.render(spp, seed=seed, accum=acc, crop=(x0, y0, cw, ch), sample_out=samples, restir=restir,
             **{"mode": 1, **kw})
    torch.cuda.synchronize()
    return acc, samples


def _pair(sc, restir, spp, crop=None, seed=0, **kw):
    from paper_2407_19977_gb300 import api as A
    g = A.Scene(sc)
    acc, samples = _gpu(g, sc, restir, spp, crop, seed, **kw)
    cam = sc.camera
    crop = crop or (0, 0, cam.width, cam.height)
    _, o_smp, st = oracle.OracleScene(sc).render(spp=spp, seed=seed, crop=crop, keep_samples=True, restir=restir)
    return g, acc, samples.cpu().numpy(), o_smp, st


@pytest.mark.parametrize("restir", [(1, 0, 1), (8, 0, 1), (8, 5, 4), (32, 8, 6), (8, 5, 4, 1), (8, 5, 4, 16)])
def test_restir_parity_many_lights(api, restir):
    sc = scenes.many_light_box(32, width=48, height=40, spp=4, max_depth=3, seed=1)
    g, acc, gs, os_, st = _pair(sc, restir, sc.spp, seed=3)
    _samples_check(gs, os_, f"restir {restir}", max_divergent=4e-3)
    assert g.stats()["error_flags"] == 0


def test_restir_parity_in_a_window_and_with_the_sky(api):
    """The spatial pass stays inside the rendered window, on both sides; the pushbutton crop
    adds environment candidates (sky + one quad light)."""
    sc = scenes.many_light_box(20, width=64, height=48, spp=3, max_depth=2, seed=4)
    _, _, gs, os_, _ = _pair(sc, (8, 6, 5), sc.spp, crop=(9, 7, 37, 23), seed=5)
    _samples_check(gs, os_, "restir window", max_divergent=4e-3)
    pb = scenes.pushbutton()
    _, _, gs, os_, _ = _pair(pb, (16, 5, 8, 4), 2, crop=(760, 420, 96, 64), seed=7)
    _samples_check(gs, os_, "restir pushbutton crop", max_divergent=4e-3)


def test_restir_parity_with_fuzz_materials(api):
    """The reservoirs' full target and the shading of their sample evaluate the fuzz layer
    (velvet walls and boxes in the many-light box), with later-vertex candidates too."""
    import numpy as np
    base = scenes.many_light_box(24, width=40, height=32, spp=3, max_depth=3, seed=6)
    velvet = scenes.openpbr(base_color=(0.5, 0.2, 0.1), specular_roughness=0.5, fuzz_weight=0.8,
                            fuzz_color=(0.9, 0.9, 1.0), fuzz_roughness=0.5)
    mats = np.concatenate([np.asarray(base.materials, np.float32), velvet[None]])
    mid = np.asarray(base.material_ids, np.uint32).copy()
    mid[:10] = len(mats) - 1                # the enclosure's walls
    sc = scenes.Scene(base.name, base.vertices, base.indices, mid, mats, base.lights, base.env,
                      base.camera, base.spp, base.max_depth)
    for r in ((8, 5, 4), (8, 5, 4, 4)):
        g, acc, gs, os_, st = _pair(sc, r, sc.spp, seed=13)
        _samples_check(gs, os_, f"restir fuzz {r}", max_divergent=4e-3)
        assert g.stats()["error_flags"] == 0


def test_restir_progressive_graph_and_auto_are_identical(api):
    from paper_2407_19977_gb300 import api as A
    from paper_2407_19977_gb300 import native as N
    sc = scenes.many_light_box(24, width=40, height=30, spp=5, max_depth=3, seed=2)
    g = A.Scene(sc)
    r = (8, 5, 4)
    one, s_one = _gpu(g, sc, r, 5, seed=9)
    acc = A.Accum(40, 30)
    g.render(3, seed=9, accum=acc, mode=1, restir=r)
    g.render(2, seed=9, accum=acc, mode=1, restir=r)
    torch.cuda.synchronize()
    assert torch.equal(acc.sum, one.sum) and torch.equal(acc.comp, one.comp)
    for kw in ({"use_graph": True}, {"mode": N.PT_MODE_AUTO}):
        for _ in range(2):        # the second graph call replays
            again, s_again = _gpu(g, sc, r, 5, seed=9, **kw)
            assert torch.equal(s_again, s_one), kw


def test_restir_arguments(api):
    from paper_2407_19977_gb300 import api as A
    from paper_2407_19977_gb300 import native as N
    sc = scenes.many_light_box(8, width=16, height=16, spp=1, max_depth=2)
    g = A.Scene(sc)
    acc = A.Accum(16, 16)
    for bad in ((0, 0, 1), (4, 65, 1), (4, 2, 0), (4, 2, 2, 5000)):
        with pytest.raises(N.PtError, match="INVALID_ARG"):
            g.render(1, accum=acc, mode=1, restir=bad)
    with pytest.raises(N.PtError, match="INVALID_ARG"):
        g.render(1, accum=acc, mode=1, restir=(4, 2, 2), flags=N.PT_FLAG_NO_NEE)
    with pytest.raises(N.PtError, match="UNSUPPORTED"):
        g.render(1, accum=acc, mode=N.PT_MODE_MEGAKERNEL, restir=(4, 2, 2))


def test_restir_parity_full_1080p_study_configuration(api):
    """The equal-time study's setup at full size: the many-light box at 1920x1080, depth 4,
    M 8, K 5, R 10, one sample per pixel in one wave, against the oracle's ReSTIR on all
    pixels (the spatial pass needs the whole window)."""
    sc = scenes.many_light_box(256, width=1920, height=1080, spp=1, max_depth=4, seed=0)
    g, acc, gs, os_, st = _pair(sc, (8, 5, 10), 1, seed=0, use_graph=True)
    _samples_check(gs, os_, "restir 1080p", max_divergent=4e-3)
    assert g.stats()["error_flags"] == 0
