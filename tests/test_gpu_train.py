"""Training workload on the GPU: the synthetic target (random ellipsoids and
boxes behind a 0.5-attenuation occluder, 10 dB noise) against the oracle, a
few optimiser steps of the MLP through the hand-written adjoints, and what the
learned proposal gains over uniform depths at the same sample count."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def test_scene_target_matches_oracle(G, oracle):
    from paper_2605_29097_gb300 import pipeline as PL
    wl = gi.workload("c4-small")
    wl.sample_mode = gi.SAMPLE_UNIFORM
    geo = PL.make_geometry(wl)
    scene = gi.c4_scene(0)
    P = PL.scene_target(geo, scene, noise_seed=0).cpu().numpy()
    # oracle chain on the same uniform points
    xyz, apr = oracle.sample(wl.grid, gi.SAMPLE_UNIFORM)
    ant = gi.antenna_array(wl.array_n, wl.array_n, wl.array_pitch)
    f, Gr, a = oracle.analytic_fields(scene, xyz)
    fa, _, _ = oracle.analytic_fields(scene, apr)
    fn, _, _ = oracle.analytic_fields(scene, ant)
    _, _, w, t_eff, c_ant = oracle.blend(f, a, wl.grid.n_ray, wl.grid.n[2], fa, fn, np.float32(wl.sharpness), 1.0)
    w = np.where(xyz[2] > gi.C4_OCCLUDER_Z, w * gi.C4_OCCLUDER_ATTEN, w)
    b = gi.band(77e9, 81e9, wl.n_f)
    s = oracle.render(xyz, Gr, w, t_eff, ant, c_ant, b)
    s = s + gi.c4_noise(0, s.shape, float((np.abs(s) ** 2).mean()))
    vox, _ = oracle.sample(wl.heat, gi.SAMPLE_UNIFORM)
    _, oP = oracle.filter_forward(s, ant, vox, b)
    assert rel(P, oP) < 1e-3


def test_training_steps_reduce_loss(G):
    from paper_2605_29097_gb300 import pipeline as PL
    wl = gi.workload("c4-small")
    geo = PL.make_geometry(wl)
    target = PL.scene_target(geo, gi.c4_scene(2), noise_seed=2)
    spec = gi.MLPSpec(center=(0.0, 0.0, 0.15), half=0.06)
    p = torch.as_tensor(gi.mlp_init(spec, seed=3, sdf_bias=0.02), device="cuda")
    field = G.MLPField(p, center=spec.center, half=spec.half)
    master = p.clone().requires_grad_(True)
    opt = torch.optim.Adam([master], lr=1e-3)
    losses = []
    for step in range(40):
        r = PL.forward_backward(geo, field, target, seed=1, step=step)
        losses.append(float(r.loss))
        opt.zero_grad()
        master.grad = r.d_params.clone()
        opt.step()
        with torch.no_grad():
            p.copy_(master)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-5:]) < 0.9 * np.mean(losses[:5])


def test_trained_proposal_beats_uniform_depths(G):
    """Same sample count (16 depths per column): proposal-drawn depths after
    online training vs uniform depths, both against a dense 256-depth render."""
    from paper_2605_29097_gb300 import pipeline as PL
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.12, (64, 64, 256))
    h = gi.cube_grid((0.0, 0.0, 0.15), 0.12, (32, 32, 32))
    wl = gi.Workload("gain", 16, 0.003, 32, g, h, gi.SAMPLE_UNIFORM, "analytic", "fp32", sharpness=2.0 / h.pitch[2])
    geo = PL.make_geometry(wl)
    scene = gi.c4_scene(1)
    field = PL.scene_field(scene)
    P_dense, _ = PL.render_heatmap(geo, field, G.SAMPLE_UNIFORM)
    geo16 = PL.geometry_with_depths(geo, 16)
    P_u16, _ = PL.render_heatmap(geo16, field, G.SAMPLE_UNIFORM)
    prop, master = PL.init_proposal(gshape=(16, 16, 64), depth=16, seed=0)
    P_before = PL.proposal_heatmap(geo16, field, prop)
    trainer = PL.ProposalTrainer(prop, master, lr=2e-2)
    losses = []
    for it in range(200):
        d_p, d_f, loss = PL.proposal_signal_dense(geo, field, prop, seed=0, step=0)
        losses.append(float(loss))
        trainer.step(d_p, d_f)
    P_prop = PL.proposal_heatmap(geo16, field, prop)
    pd = P_dense.cpu().numpy()
    e_u16 = rel(P_u16.cpu().numpy(), pd)
    e_before = rel(P_before.cpu().numpy(), pd)
    e_prop = rel(P_prop.cpu().numpy(), pd)
    print(f"heatmap rel L2 vs 256 depths: uniform16 {e_u16:.3e}, proposal untrained {e_before:.3e}, "
          f"trained {e_prop:.3e}; proposal KL {losses[0]:.3f} -> {losses[-1]:.3f}")
    assert losses[-1] < 0.5 * losses[0]
    assert e_prop < 0.5 * e_u16


def test_checkpoint_resume_repeats_the_run_bit_for_bit(G, tmp_path):
    """Training state saved at step 3 and restored into fresh tensors and
    optimisers continues exactly as the uninterrupted run: the kernels are
    deterministic (fixed-order reductions, no float atomics) and the samples
    come from counter-based generators keyed by the step."""
    from paper_2605_29097_gb300 import pipeline as PL
    wl = gi.workload("c4-small")
    geo = PL.make_geometry(wl)
    target = PL.scene_target(geo, gi.c4_scene(5), noise_seed=5)
    spec = gi.MLPSpec(center=(0.0, 0.0, 0.15), half=0.06)

    def fresh():
        p = torch.as_tensor(gi.mlp_init(spec, seed=8, sdf_bias=0.02), device="cuda")
        master = p.clone().requires_grad_(True)
        return p, master, torch.optim.Adam([master], lr=1e-3)

    def run(p, master, opt, steps):
        field = G.MLPField(p, center=spec.center, half=spec.half)
        out = []
        for step in steps:
            r = PL.forward_backward(geo, field, target, seed=4, step=step)
            out.append(float(r.loss))
            opt.zero_grad()
            master.grad = r.d_params.clone()
            opt.step()
            with torch.no_grad():
                p.copy_(master)
        return out

    p, master, opt = fresh()
    run(p, master, opt, range(3))
    ck = tmp_path / "state.pt"
    PL.save_checkpoint(ck, 3, master, opt)
    tail = run(p, master, opt, range(3, 6))
    p2, master2, opt2 = fresh()
    st = PL.load_checkpoint(ck, master2, opt2)
    with torch.no_grad():
        p2.copy_(master2)
    assert st["step"] == 3
    resumed = run(p2, master2, opt2, range(st["step"], 6))
    assert resumed == tail
    assert torch.equal(p, p2)
