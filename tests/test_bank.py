"""Signal tracing bank (section 5.3): the patch layout on the host, and on the
GPU the bank step against the plain step, a full cycle of patches against a
full trace, and one bank step against the oracle composed on the same
inputs (trace of the patch, filter over the whole bank, filter adjoint and
tracing adjoint of the patch)."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi
from parity_helpers import away_from_clamp_kink


def _cpu_geo(nx, ny):
    from paper_2605_29097_gb300 import pipeline as PL
    from paper_2605_29097_gb300 import geraf as Gm
    ant = torch.as_tensor(gi.antenna_array(nx, ny, 0.002))
    band = Gm.Band(77e9, 1e8, 8)
    return PL.Geometry(None, 1, 1, ant, torch.zeros(3, 1), band, 1.0, 1.0, 0)


def test_patch_layout_tiles_the_array():
    from paper_2605_29097_gb300 import pipeline as PL
    nx, ny, px, py = 12, 8, 4, 2
    geo = _cpu_geo(nx, ny)
    bank = PL.SignalBank(geo, (nx, ny), (px, py))
    assert bank.n_patch == (nx // px) * (ny // py) and bank.patch_size == px * py
    assert sorted(bank.order.tolist()) == list(range(nx * ny))          # a permutation
    for k in range(bank.n_patch):
        a0, a1 = bank.rows(k)
        ids = bank.order[a0:a1]
        ix, iy = ids % nx, ids // nx
        assert ix.max() - ix.min() == px - 1 and iy.max() - iy.min() == py - 1   # one px x py tile
        np.testing.assert_array_equal(bank.patch_ant[k].numpy(), geo.ant[:, ids].numpy())
    with pytest.raises(ValueError):
        PL.SignalBank(geo, (nx, ny), (5, 2))


def _G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def _setup(G, PL, mode):
    wl = gi.workload("c4-small")
    wl.sample_mode = mode
    geo = PL.make_geometry(wl)
    target = PL.scene_target(geo, gi.c4_scene(2), noise_seed=2)
    spec = gi.MLPSpec(center=(0.0, 0.0, 0.15), half=0.06)
    p = torch.as_tensor(gi.mlp_init(spec, seed=3, sdf_bias=0.02), device="cuda")
    field = G.MLPField(p, center=spec.center, half=spec.half)
    return wl, geo, target, field


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.gpu
def test_single_patch_bank_equals_plain_step():
    G = _G()
    from paper_2605_29097_gb300 import pipeline as PL
    wl, geo, target, field = _setup(G, PL, gi.SAMPLE_STRATIFIED)
    bank = PL.SignalBank(geo, (wl.array_n, wl.array_n), (wl.array_n, wl.array_n))
    rb = PL.forward_backward_bank(bank, field, target, seed=1, step=4)
    rp = PL.forward_backward(geo, field, target, seed=1, step=4)
    assert abs(float(rb.loss) - float(rp.loss)) <= 1e-6 * abs(float(rp.loss))
    assert rel(rb.d_params.cpu(), rp.d_params.cpu()) < 1e-5


@pytest.mark.gpu
def test_cycle_of_patches_rebuilds_the_full_trace():
    G = _G()
    from paper_2605_29097_gb300 import pipeline as PL
    wl, geo, target, field = _setup(G, PL, gi.SAMPLE_UNIFORM)     # same points every step
    bank = PL.SignalBank(geo, (wl.array_n, wl.array_n), (4, 2))
    for step in range(bank.n_patch):
        PL.forward_backward_bank(bank, field, target, seed=0, step=step)
    _, s_full = PL.render_heatmap(bank.geo, field, G.SAMPLE_UNIFORM)
    assert rel(bank.s.cpu().numpy(), s_full.cpu().numpy()) < 1e-5


@pytest.mark.gpu
def test_bank_step_matches_oracle_composition(oracle):
    G = _G()
    from paper_2605_29097_gb300 import pipeline as PL
    wl, geo, target, field = _setup(G, PL, gi.SAMPLE_STRATIFIED)
    bank = PL.SignalBank(geo, (wl.array_n, wl.array_n), (4, 4))
    bank.fill(field, seed=1, step=0)
    r = PL.forward_backward_bank(bank, field, target, seed=1, step=6)     # patch 6 mod 4 = 2
    B = r.bank
    assert B["patch"] == 2
    h = lambda t: t.detach().cpu().numpy()
    a0, a1 = bank.rows(2)
    ant = h(bank.geo.ant)
    ant_p = ant[:, a0:a1]
    b = gi.Band(geo.band.f0, geo.band.df, geo.band.n_f)
    xyz, grad, w, t_eff, c_ant = (h(B[k]) for k in ("xyz", "grad", "w", "t_eff", "c_ant"))
    s_p = oracle.render(xyz, grad, w, t_eff, ant_p, c_ant, b)
    S = h(bank.s)
    assert rel(S[a0:a1], s_p) < 1e-5                       # the patch's rows hold its new trace
    vox = h(geo.vox)
    oM, oP = oracle.filter_forward(S, ant, vox, b)         # whole bank, bank order
    assert rel(h(r.P), oP) < 1e-5
    oL, odP = oracle.heatmap_loss(oP, h(target))
    np.testing.assert_allclose(float(r.loss), oL, rtol=1e-5)
    og = oracle.filter_backward(h(B["M"]), h(B["dP"]), ant_p, vox, b)   # adjoint for the patch only
    assert rel(h(B["g"]), og) < 1e-5
    ow, ot, oGd = oracle.render_backward(xyz, grad, w, t_eff, ant_p, c_ant, b, h(B["g"]))
    assert rel(h(B["d_w"]), ow) < 1e-5
    kt = away_from_clamp_kink(t_eff, c_ant)                # d_teff away from the clamp's kinks
    assert rel(h(B["d_teff"])[kt], ot[kt]) < 1e-5
    assert rel(h(B["d_G"]), oGd) < 3e-5
