"""Field networks of the paper's size (App. C: SDF network 8 x 256 and a
separate reflectivity network 4 x 256 on a 10-octave encoding) and other
shapes that run layer by layer, on the GPU vs the FP64 oracle: f, a,
G = grad f and the adjoint of every packed parameter, FP32 path."""
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


def _field(G, nets, params):
    s = nets.sdf
    return G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=s.n_levels, width=s.width,
                      n_hidden=s.n_hidden, beta=s.beta, center=s.center, half=s.half,
                      refl_hidden=nets.refl.n_hidden, refl_width=nets.refl.width)


def _points(spec, n, seed):
    rng = np.random.default_rng(seed)
    return (np.array(spec.center)[:, None] + rng.uniform(-spec.half, spec.half, (3, n))).astype(np.float32), rng


# FP32 tolerance: every output is a chain of up to 9 FP32 dot products of
# length <= 256 (relative rounding ~ 2^-24 sqrt(256) ~ 1e-6 each, growing
# linearly with depth); the gradient tangents and the parameter adjoint carry
# one more chain. 1e-5 for values, 3e-5 for the adjoint of the 8-layer network.
@pytest.mark.parametrize("paper_size,n", [(False, 300), (True, 517)])
def test_two_networks_forward_backward(G, oracle, paper_size, n):
    if paper_size:
        nets = gi.paper_nets()
    else:
        nets = gi.FieldNets(gi.MLPSpec(4, 96, 3, 50.0, (0.0, 0.0, 0.15), 0.06, 1),
                            gi.MLPSpec(4, 64, 2, 50.0, (0.0, 0.0, 0.15), 0.06, 1))
    params = gi.nets_init(nets, seed=3, sdf_bias=0.01)
    xyz, rng = _points(nets.sdf, n, 11)
    field = _field(G, nets, params)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    of, oG, oa, cache = oracle.nets_forward(nets, params, xyz)
    h = lambda t: t.detach().cpu().numpy()
    assert rel_l2(h(f), of) < 1e-5
    assert rel_l2(h(a), oa) < 1e-5
    assert rel_l2(h(grad), oG) < 1e-5
    # value only (no tangent streams, no reflectivity network): the same f
    f1, _, _, _ = G.geraf_fields(field, xt, want_grad=False, want_refl=False)
    assert rel_l2(h(f1), of) < 1e-5
    d_f = rng.standard_normal(n).astype(np.float32)
    d_G = rng.standard_normal((3, n)).astype(np.float32)
    d_a = rng.standard_normal(n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = h(G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a)))
    ogp = oracle.nets_backward(nets, params, cache, d_f, d_G, d_a)
    tol = 3e-5 if paper_size else 1e-5
    assert rel_l2(gp, ogp) < tol
    # each network's block, and each layer's weight block of the SDF network
    ns = nets.sdf.n_params
    assert rel_l2(gp[ns:], ogp[ns:]) < tol
    off = 0
    for o, i in nets.sdf.shapes():
        assert rel_l2(gp[off:off + o * i], ogp[off:off + o * i]) < tol
        off += o * i + o


def test_paper_networks_many_splits(G, oracle):
    """The paper's two networks on 32 771 points (ragged): the adjoint's weight
    gradients run over SMs/2 = 76 splits of the rows (432 points each), their
    partials summed in FP64 in a fixed order, and the GEMMs over 257 row tiles
    of 128. Every output, each network's block and each SDF layer's weight
    block against the FP64 oracle."""
    n = 32771
    nets = gi.paper_nets()
    params = gi.nets_init(nets, seed=5, sdf_bias=0.01)
    xyz, rng = _points(nets.sdf, n, 13)
    field = _field(G, nets, params)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    of, oG, oa, cache = oracle.nets_forward(nets, params, xyz)
    h = lambda t: t.detach().cpu().numpy()
    assert rel_l2(h(f), of) < 1e-5 and rel_l2(h(a), oa) < 1e-5 and rel_l2(h(grad), oG) < 1e-5
    d_f = rng.standard_normal(n).astype(np.float32)
    d_G = rng.standard_normal((3, n)).astype(np.float32)
    d_a = rng.standard_normal(n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = h(G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a)))
    G.geraf_poll_device_error()
    ogp = oracle.nets_backward(nets, params, cache, d_f, d_G, d_a)
    assert rel_l2(gp, ogp) < 3e-5
    ns = nets.sdf.n_params
    assert rel_l2(gp[ns:], ogp[ns:]) < 3e-5
    off = 0
    for li, (o, i) in enumerate(nets.sdf.shapes()):
        e = rel_l2(gp[off:off + o * i], ogp[off:off + o * i])
        assert e < 3e-5, f"SDF layer {li}: {e:.2e}"
        off += o * i + o


def test_wide_single_trunk(G, oracle):
    """One trunk with head [f, a_logit] at width 256 runs the layer-by-layer
    kernels too; ragged point count."""
    spec = gi.MLPSpec(n_levels=6, width=256, n_hidden=3, beta=100.0, center=(0.0, 0.0, 0.15), half=0.05)
    params = gi.mlp_init(spec, seed=9)
    xyz, rng = _points(spec, 77, 5)
    field = G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=6, width=256, n_hidden=3,
                       beta=spec.beta, center=spec.center, half=spec.half)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz)
    h = lambda t: t.detach().cpu().numpy()
    assert rel_l2(h(f), of) < 1e-5 and rel_l2(h(a), oa) < 1e-5 and rel_l2(h(grad), oG) < 1e-5
    d_f, d_G, d_a = (rng.standard_normal(s).astype(np.float32) for s in ((77,), (3, 77), (77,)))
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a))
    assert rel_l2(h(gp), oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)) < 1e-5


def test_wide_network_needs_saved(G):
    nets = gi.paper_nets()
    params = torch.as_tensor(gi.nets_init(nets, seed=1), device="cuda")
    field = _field(G, nets, params.cpu().numpy())
    from paper_2605_29097_gb300 import _lib
    import ctypes
    desc = field.desc()
    xyz = torch.zeros(3, 8, device="cuda")
    f = torch.empty(8, device="cuda")
    st = _lib.lib().geraf_fields(ctypes.byref(desc), xyz.data_ptr(), 8, f.data_ptr(), None, None, None, 0, None)
    assert st == 1    # GERAF_ERR_INVALID_ARG


# BF16 networks on the tensor cores against the oracle's BF16 network reading
# (weights and every hidden layer's inputs rounded to bfloat16, FP32 sums
# stand in for exact ones): relative L2 2e-3, the BF16 path's bound.
BF16_TOL = 2e-3


def _bf16_case(G, oracle, nets, n, seed):
    params = gi.nets_init(nets, seed=seed, sdf_bias=0.01)
    xyz, rng = _points(nets.sdf, n, seed)
    s = nets.sdf
    field = G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=s.n_levels, width=s.width,
                       n_hidden=s.n_hidden, beta=s.beta, center=s.center, half=s.half,
                       refl_hidden=nets.refl.n_hidden, refl_width=nets.refl.width, precision=G.PREC_BF16)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    of, oG, oa, cache = oracle.nets_forward(nets, params, xyz, precision="bf16")
    h = lambda t: t.detach().cpu().numpy()
    errs = {"f": rel_l2(h(f), of), "a": rel_l2(h(a), oa), "G": rel_l2(h(grad), oG)}
    # value only (no tangent streams, no reflectivity network): the same f
    f1, _, _, _ = G.geraf_fields(field, xt, want_grad=False, want_refl=False)
    errs["f value-only"] = rel_l2(h(f1), of)
    d_f = rng.standard_normal(n).astype(np.float32)
    d_G = rng.standard_normal((3, n)).astype(np.float32)
    d_a = rng.standard_normal(n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = h(G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a)))
    G.geraf_poll_device_error()
    ogp = oracle.nets_backward(nets, params, cache, d_f, d_G, d_a)
    errs["d_params"] = rel_l2(gp, ogp)
    ns = nets.sdf.n_params
    errs["d_params refl"] = rel_l2(gp[ns:], ogp[ns:])
    off = 0
    for li, (o, i) in enumerate(nets.sdf.shapes()):
        errs[f"d_W sdf {li}"] = rel_l2(gp[off:off + o * i], ogp[off:off + o * i])
        errs[f"d_b sdf {li}"] = rel_l2(gp[off + o * i:off + o * i + o], ogp[off + o * i:off + o * i + o])
        off += o * i + o
    print({k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if not v < BF16_TOL}
    assert not bad, bad


def test_paper_networks_bf16_tensor_cores(G, oracle):
    """The paper's two networks (SDF 8 x 256, reflectivity 4 x 256, 10 octaves)
    in BF16 on tcgen05 at 32 771 points: every GEMM of the forward and the
    adjoint runs over 1025 row tiles (the last ragged), the weight gradients
    over 76 splits of the rows."""
    _bf16_case(G, oracle, gi.paper_nets(), 32771, 17)


def test_small_networks_bf16_tensor_cores(G, oracle):
    """Other shapes on the same kernels: a 3 x 128 SDF network and a 2 x 64
    reflectivity network on a 4-octave encoding (24 features padded to 64), 300
    points (a single partly filled row tile for the reflectivity network)."""
    nets = gi.FieldNets(gi.MLPSpec(4, 128, 3, 50.0, (0.0, 0.0, 0.15), 0.06, 1),
                        gi.MLPSpec(4, 64, 2, 50.0, (0.0, 0.0, 0.15), 0.06, 1))
    _bf16_case(G, oracle, nets, 300, 19)


def test_wide_single_trunk_bf16(G, oracle):
    """One 256-wide trunk with head [f, a_logit] in BF16 on the tensor cores."""
    spec = gi.MLPSpec(n_levels=6, width=256, n_hidden=3, beta=100.0, center=(0.0, 0.0, 0.15), half=0.05)
    params = gi.mlp_init(spec, seed=23)
    xyz, rng = _points(spec, 77, 23)
    field = G.MLPField(torch.as_tensor(params, device="cuda"), n_levels=6, width=256, n_hidden=3,
                       beta=spec.beta, center=spec.center, half=spec.half, precision=G.PREC_BF16)
    xt = torch.as_tensor(xyz, device="cuda")
    f, grad, a, saved = G.geraf_fields(field, xt, keep_saved=True)
    G.geraf_poll_device_error()
    of, oG, oa, cache = oracle.mlp_forward(spec, params, xyz, precision="bf16")
    h = lambda t: t.detach().cpu().numpy()
    assert max(rel_l2(h(f), of), rel_l2(h(a), oa), rel_l2(h(grad), oG)) < BF16_TOL
    d_f, d_G, d_a = (rng.standard_normal(s).astype(np.float32) for s in ((77,), (3, 77), (77,)))
    cu = lambda x: torch.as_tensor(x, device="cuda")
    gp = G.geraf_fields_backward(field, xt, saved, cu(d_f), cu(d_G), cu(d_a))
    G.geraf_poll_device_error()
    assert rel_l2(h(gp), oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)) < BF16_TOL
