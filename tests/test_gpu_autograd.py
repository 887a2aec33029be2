"""Hand-written adjoints behind torch.autograd.Function, end to end from the MLP
parameters to the heatmap loss:
(1) against autograd through a slow FP64 torch restatement of the same chain;
(2) against central finite differences of the FP64 oracle chain on 16 random
    MLP weights."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu
C = 299792458.0


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def _setup(n=(8, 8, 8), n_side=4, n_f=8, n_hidden=2, seed=0):
    spec = gi.MLPSpec(n_levels=4, n_hidden=n_hidden, beta=100.0)
    params = gi.mlp_init(spec, seed=seed, sdf_bias=0.0)
    grid = gi.cube_grid((0.0, 0.0, 0.15), 0.1, n)
    heat = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (6, 6, 6))
    ant = gi.antenna_array(n_side, n_side, 0.004)
    band = gi.band(77e9, 81e9, n_f)
    s_sharp = 60.0
    return spec, params, grid, heat, ant, band, s_sharp


def _torch_chain(spec, params, xyz, apr, ant, vox, band, s_sharp, a_tx, n_ray, n_z, target):
    """Slow FP64 torch restatement: PE + softplus MLP (gradient by autograd),
    NeuS blend, signal tracing and matched filter as dense tensors."""
    dev = "cuda"
    p = torch.tensor(params.astype(np.float64), device=dev, requires_grad=True)
    shapes = spec.shapes()
    c = torch.tensor(np.asarray(spec.center, np.float32).astype(np.float64), device=dev)
    half = float(np.float32(spec.half))

    def mlp(x, need_grad):
        x = x.clone().requires_grad_(need_grad)
        xt = (x - c) / half
        feats = []
        for k in range(spec.n_levels):
            feats += [torch.sin((2.0 ** k) * np.pi * xt), torch.cos((2.0 ** k) * np.pi * xt)]
        z = torch.cat(feats, 1)
        off = 0
        for li, (o, i) in enumerate(shapes):
            W = p[off:off + o * i].view(o, i); off += o * i
            b = p[off:off + o]; off += o
            z = z @ W.T + b
            if li < len(shapes) - 1:
                z = torch.nn.functional.softplus(z, beta=spec.beta, threshold=1e6)
        f, a = z[:, 0], torch.sigmoid(z[:, 1])
        Gr = torch.autograd.grad(f.sum(), x, create_graph=True)[0] if need_grad else None
        return f, Gr, a

    X = torch.tensor(xyz.T.astype(np.float64), device=dev)
    f, Gr, a = mlp(X, True)
    fa, _, _ = mlp(torch.tensor(apr.T.astype(np.float64), device=dev), False)
    fn, _, _ = mlp(torch.tensor(ant.T.astype(np.float64), device=dev), False)
    Phi = torch.sigmoid(s_sharp * f).view(n_z, n_ray)
    alpha = torch.zeros_like(Phi)
    alpha[:-1] = torch.clamp((Phi[:-1] - Phi[1:]) / Phi[:-1], min=0.0)
    T = torch.cumprod(torch.cat([torch.ones(1, n_ray, device=dev, dtype=torch.float64), 1 - alpha[:-1]], 0), 0)
    w = (a.view(n_z, n_ray) * alpha * a_tx).reshape(-1)
    t_eff = (T + torch.sigmoid(s_sharp * fa).detach()[None, :]).reshape(-1)
    c_ant = torch.sigmoid(s_sharp * fn).detach()
    A_ = torch.tensor(ant.T.astype(np.float64), device=dev)
    d = X[None, :, :] - A_[:, None, :]                       # [n_ant, n_pts, 3]
    r = torch.linalg.norm(d, dim=2)
    nrm = Gr / torch.linalg.norm(Gr, dim=1, keepdim=True)
    cosv = (d * nrm[None]).sum(2) / r
    D = torch.clamp(2 * cosv ** 2 - 1, min=0.0)
    Tp = torch.clamp(t_eff[None, :] - c_ant[:, None], 0.0, 1.0)
    Amp = w[None, :] * Tp ** 2 * D / (4 * np.pi * r) ** 2
    fr = torch.tensor(band.f0 + band.df * np.arange(band.n_f), device=dev)
    ph = 2 * np.pi * fr[None, None, :] * (2 * r / C)[:, :, None]
    s_re = (Amp[:, :, None] * torch.cos(ph)).sum(1)
    s_im = -(Amp[:, :, None] * torch.sin(ph)).sum(1)
    V = torch.tensor(vox.T.astype(np.float64), device=dev)
    rv = torch.linalg.norm(V[None, :, :] - A_[:, None, :], dim=2)
    phv = 2 * np.pi * fr[None, None, :] * (2 * rv / C)[:, :, None]
    Mr = (s_re[:, None, :] * torch.cos(phv) - s_im[:, None, :] * torch.sin(phv)).sum((0, 2))
    Mi = (s_re[:, None, :] * torch.sin(phv) + s_im[:, None, :] * torch.cos(phv)).sum((0, 2))
    P = torch.sqrt(Mr ** 2 + Mi ** 2)
    L = ((P - torch.tensor(target, device=dev, dtype=torch.float64)) ** 2).sum()
    g = torch.autograd.grad(L, p)[0]
    return P.detach().cpu().numpy(), g.cpu().numpy()


def _gpu_chain(G, spec, params, grid, heat, ant, band, s_sharp, target, seed):
    from paper_2605_29097_gb300 import autograd as AG
    gr = G.make_grid(grid.lo, grid.pitch, grid.n, grid.aperture_z)
    xyz, apr = G.geraf_sample(gr, gi.SAMPLE_UNIFORM, seed, 0)
    hg = G.make_grid(heat.lo, heat.pitch, heat.n)
    vox, _ = G.geraf_sample(hg, gi.SAMPLE_UNIFORM)
    a_t = torch.as_tensor(ant, device="cuda")
    p = torch.as_tensor(params, device="cuda").requires_grad_(True)
    kw = dict(n_levels=spec.n_levels, n_hidden=spec.n_hidden, beta=spec.beta, center=spec.center, half=spec.half)
    P = AG.heatmap(p, xyz, apr, a_t, vox, G.Band(band.f0, band.df, band.n_f), s_sharp, 1.0, grid.n_ray, grid.n[2],
                   kw)
    L = ((P - torch.as_tensor(target, device="cuda")) ** 2).sum()
    L.backward()
    return P.detach().cpu().numpy(), p.grad.cpu().numpy(), xyz.cpu().numpy(), apr.cpu().numpy(), vox.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_adjoint_chain_matches_torch_autograd(G):
    spec, params, grid, heat, ant, band, s_sharp = _setup()
    target = np.zeros(heat.n_pts, np.float32)
    P, g, xyz, apr, vox = _gpu_chain(G, spec, params, grid, heat, ant, band, s_sharp, target, 0)
    tP, tg = _torch_chain(spec, params, xyz, apr, ant, vox, band, s_sharp, 1.0, grid.n_ray, grid.n[2], target)
    assert rel(P, tP) < 1e-4
    assert rel(g, tg) < 1e-3


def test_adjoint_matches_oracle_finite_differences(G, oracle):
    """16 random MLP weights: central differences of the FP64 oracle chain."""
    spec, params, grid, heat, ant, band, s_sharp = _setup()
    rng = np.random.default_rng(3)
    target = rng.uniform(0.0, 1e-4, heat.n_pts).astype(np.float32)
    P, g, xyz, apr, vox = _gpu_chain(G, spec, params, grid, heat, ant, band, s_sharp, target, 0)

    def loss(theta):
        f, Gr, a, _ = oracle.mlp_forward(spec, theta, xyz)
        fa, _, _, _ = oracle.mlp_forward(spec, theta, apr)
        fn, _, _, _ = oracle.mlp_forward(spec, theta, ant)
        _, _, w, t_eff, c_ant = oracle.blend(f, a, grid.n_ray, grid.n[2], fa, fn, s_sharp, 1.0)
        s = oracle.render(xyz, Gr, w, t_eff, ant, c_ant, band)
        _, Pv = oracle.filter_forward(s, ant, vox, band)
        return oracle.heatmap_loss(Pv, target)[0]

    idx = rng.choice(params.size, 16, replace=False)
    th = params.astype(np.float64)
    fd = []
    for k in idx:
        h = 1e-4 * max(1.0, abs(th[k]))
        e = np.zeros_like(th); e[k] = h
        fd.append((loss(th + e) - loss(th - e)) / (2 * h))
    fd = np.array(fd)
    scale = np.abs(g).max()
    assert np.all(np.abs(g[idx] - fd) <= 2e-3 * scale + 2e-3 * np.abs(fd))
