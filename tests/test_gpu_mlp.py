"""MLP fields on the GPU vs the FP64 oracle: value f, reflectiveness a, the
gradient G = grad f from the forward-mode tangents, and the hand-written
parameter adjoint. FP32 path: relative L2 <= 1e-5 on every output."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


@pytest.mark.parametrize("n,n_levels,n_hidden", [(1000, 6, 4), (33, 6, 4), (257, 10, 2)])
def test_mlp_forward_backward(G, oracle, n, n_levels, n_hidden):
    spec = gi.MLPSpec(n_levels=n_levels, n_hidden=n_hidden)
    params = gi.mlp_init(spec, seed=n)
    rng = np.random.default_rng(n)
    xyz = (np.array(spec.center)[:, None] + rng.uniform(-spec.half, spec.half, (3, n))).astype(np.float32)
    field = G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=n_levels, n_hidden=n_hidden,
                       beta=spec.beta, center=spec.center, half=spec.half)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz)
    h = lambda t: t.detach().cpu().numpy()
    assert rel_l2(h(f), of) < 1e-5
    assert rel_l2(h(a), oa) < 1e-5
    assert rel_l2(h(grad), oG) < 1e-5
    d_f = rng.standard_normal(n).astype(np.float32)
    d_G = rng.standard_normal((3, n)).astype(np.float32)
    d_a = rng.standard_normal(n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a))
    ogp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    assert rel_l2(h(gp), ogp) < 1e-5
    # every layer's block individually
    off = 0
    for (o, i) in spec.shapes():
        for sz in (o * i, o):
            assert rel_l2(h(gp)[off:off + sz], ogp[off:off + sz]) < 1e-4
            off += sz


def test_mlp_origins_only_sdf(G, oracle):
    """Ray-origin evaluations ask for f alone (no gradient, no saved state)."""
    spec = gi.MLPSpec()
    params = gi.mlp_init(spec, seed=9)
    xyz = gi.antenna_array(9, 7, 0.002)
    field = G.MLPField(torch.as_tensor(params, device="cuda"))
    f, g, a, s = G.geraf_fields(field, torch.as_tensor(xyz, device="cuda"), want_grad=False, want_refl=False)
    of, _, _, _ = oracle.mlp_forward(spec, params, xyz)
    assert g is None and a is None and s is None
    assert rel_l2(f.cpu().numpy(), of) < 1e-5


@pytest.mark.parametrize("n,n_levels,n_hidden", [(1000, 6, 4), (77, 10, 3)])
def test_mlp_bf16_tensor_cores(G, oracle, n, n_levels, n_hidden):
    """BF16 network on tcgen05 vs the oracle's BF16 definition (weights and
    layer inputs rounded to bfloat16, exact sums): relative L2 <= 2e-3."""
    spec = gi.MLPSpec(n_levels=n_levels, n_hidden=n_hidden)
    params = gi.mlp_init(spec, seed=n + 1)
    rng = np.random.default_rng(n + 1)
    xyz = (np.array(spec.center)[:, None] + rng.uniform(-spec.half, spec.half, (3, n))).astype(np.float32)
    field = G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=n_levels, n_hidden=n_hidden,
                       beta=spec.beta, center=spec.center, half=spec.half, precision=G.PREC_BF16)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    h = lambda t: t.detach().cpu().numpy()
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz, precision="bf16")
    e = (rel_l2(h(f), of), rel_l2(h(a), oa), rel_l2(h(grad), oG))
    f32, G32, a32, _ = oracle.mlp_forward(spec, params, xyz)
    print(f"bf16 vs bf16 definition: f {e[0]:.2e} a {e[1]:.2e} G {e[2]:.2e}; vs fp32 network: "
          f"f {rel_l2(h(f), f32):.2e} G {rel_l2(h(grad), G32):.2e}")
    assert max(e) < 2e-3
    d_f = rng.standard_normal(n).astype(np.float32)
    d_G = rng.standard_normal((3, n)).astype(np.float32)
    d_a = rng.standard_normal(n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a))
    ogp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    assert rel_l2(h(gp), ogp) < 2e-3


def _many_tiles_case(spec, n, seed):
    params = gi.mlp_init(spec, seed=seed)
    rng = np.random.default_rng(seed)
    xyz = (np.array(spec.center)[:, None] + rng.uniform(-spec.half, spec.half, (3, n))).astype(np.float32)
    d = (rng.standard_normal(n).astype(np.float32), rng.standard_normal((3, n)).astype(np.float32),
         rng.standard_normal(n).astype(np.float32))
    return params, xyz, d


def test_mlp_fp32_persistent_tiles(G, oracle):
    """70 001 points (ragged) = 2188 tiles of 32 points over at most one CTA per
    SM: every CTA of the forward runs its persistent tile loop 14-15 times, and
    every CTA of each hidden layer's adjoint accumulates the weight gradient in
    registers over as many tiles while it prefetches the next tile's rows into
    L2. Every output and every layer's weight and bias block against the FP64
    oracle at relative L2 1e-5."""
    n = 70001
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert (n + 31) // 32 >= 8 * sms
    spec = gi.MLPSpec()
    params, xyz, (d_f, d_G, d_a) = _many_tiles_case(spec, n, 21)
    field = G.MLPField(torch.as_tensor(params, device="cuda"))
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz)
    h = lambda t: t.detach().cpu().numpy()
    assert rel_l2(h(f), of) < 1e-5
    assert rel_l2(h(a), oa) < 1e-5
    assert rel_l2(h(grad), oG) < 1e-5
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = h(G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a)))
    G.geraf_poll_device_error()
    ogp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    assert rel_l2(gp, ogp) < 1e-5
    off = 0
    for li, (o, i) in enumerate(spec.shapes()):
        for name, sz in (("W", o * i), ("b", o)):
            e = rel_l2(gp[off:off + sz], ogp[off:off + sz])
            assert e < 1e-5, f"layer {li} {name}: {e:.2e}"
            off += sz


def test_mlp_bf16_persistent_tiles(G, oracle):
    """The BF16 tensor-core kernels at 70 001 points: the forward runs pairs of
    32-point tiles (1094 pairs, ~7 per CTA), the adjoint 16-point tiles (4376,
    ~29 per CTA) with each layer's weight gradient accumulated in TMEM across
    them. Against the oracle's BF16 network definition at 2e-3."""
    n = 70001
    spec = gi.MLPSpec()
    params, xyz, (d_f, d_G, d_a) = _many_tiles_case(spec, n, 22)
    field = G.MLPField(torch.as_tensor(params, device="cuda"), precision=G.PREC_BF16)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz, precision="bf16")
    h = lambda t: t.detach().cpu().numpy()
    assert max(rel_l2(h(f), of), rel_l2(h(a), oa), rel_l2(h(grad), oG)) < 2e-3
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = h(G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a)))
    G.geraf_poll_device_error()
    ogp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    assert rel_l2(gp, ogp) < 2e-3
    off = 0
    for li, (o, i) in enumerate(spec.shapes()):
        e = rel_l2(gp[off:off + o * i], ogp[off:off + o * i])
        assert e < 2e-3, f"layer {li} W: {e:.2e}"
        off += o * i + o
