"""Dynamic loss masking (section 6) on the GPU: the mask, running maximum,
masked loss and its gradient against the oracle (mask and history bit-exact,
the comparisons made on the same FP32 values), and the masked training step."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


@pytest.mark.parametrize("n", [1, 1000, 70001])
def test_masked_loss_matches_oracle(G, oracle, n):
    rng = np.random.default_rng(n)
    P = rng.uniform(0, 10, n).astype(np.float32)
    H = (rng.uniform(0, 10, n) * (rng.uniform(0, 1, n) < 0.5)).astype(np.float32)
    target = rng.uniform(0, 10, n).astype(np.float32)
    t_hi, t_lo = np.float32(5.0), np.float32(2.5)
    P[: n // 7] = t_lo                         # on the low threshold: kept
    H[: n // 5] = t_hi                         # on the high threshold: counts as high
    cu = lambda x: torch.as_tensor(x, device="cuda")
    hist = cu(H.copy())
    loss, dP, mask = G.geraf_masked_loss(cu(P), cu(target), hist, float(t_hi), float(t_lo))
    om, oH = oracle.dynamic_mask(P, H, 1.0, float(t_hi), float(t_lo))
    np.testing.assert_array_equal(mask.cpu().numpy(), om)
    np.testing.assert_array_equal(hist.cpu().numpy(), oH.astype(np.float32))
    oL, odP = oracle.heatmap_loss(P, target, om)
    np.testing.assert_allclose(float(loss), oL, rtol=1e-7)
    np.testing.assert_allclose(dP.cpu().numpy(), odP, rtol=1e-6, atol=1e-6)


def test_masked_training_step(G, oracle):
    from paper_2605_29097_gb300 import pipeline as PL
    wl = gi.workload("c4-small")
    geo = PL.make_geometry(wl)
    target = PL.scene_target(geo, gi.c4_scene(2), noise_seed=2)
    spec = gi.MLPSpec(center=(0.0, 0.0, 0.15), half=0.06)
    p = torch.as_tensor(gi.mlp_init(spec, seed=3, sdf_bias=0.02), device="cuda")
    field = G.MLPField(p, center=spec.center, half=spec.half)
    dm = PL.DynamicMask(target)
    # fresh history: nothing was high before, the step equals the unmasked one
    r0 = PL.forward_backward(geo, field, target, seed=1, step=0, dyn_mask=dm)
    rp = PL.forward_backward(geo, field, target, seed=1, step=0)
    assert float(r0.mask.sum()) == r0.mask.numel()
    np.testing.assert_allclose(float(r0.loss), float(rp.loss), rtol=1e-6)
    h = lambda t: t.detach().cpu().numpy()
    assert np.linalg.norm(h(r0.d_params) - h(rp.d_params)) <= 1e-5 * np.linalg.norm(h(rp.d_params))
    np.testing.assert_array_equal(h(dm.history), np.maximum(0, h(r0.P)))
    # plant a high history on every voxel and put the low threshold at the
    # median rendered power: the voxels rendered below it now drop out
    dm.t_lo = float(np.float32(np.median(h(r0.P))))
    dm.t_hi = 2 * dm.t_lo
    dm.history.fill_(2 * dm.t_hi)
    r1 = PL.forward_backward(geo, field, target, seed=1, step=0, dyn_mask=dm)
    P1 = h(r1.P)
    om, _ = oracle.dynamic_mask(P1, np.full(P1.shape, 2 * dm.t_hi, np.float32), 1.0, dm.t_hi, dm.t_lo)
    np.testing.assert_array_equal(h(r1.mask), om)
    assert 0 < om.sum() < om.size                       # some kept, some dropped
    oL, _ = oracle.heatmap_loss(P1, h(target), om)
    np.testing.assert_allclose(float(r1.loss), oL, rtol=1e-6)
