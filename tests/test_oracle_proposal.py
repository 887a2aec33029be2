"""Pins for the oracle's learned proposal sampler: the network and its
adjoint against torch autograd, the KL loss gradient against finite
differences, and the integer inverse-CDF sampler against its distribution,
ordering and the closed form of the uniform case."""
import numpy as np
import torch
from scipy import stats

import geraf_inputs as gi


def _spec(F=8, width=16, n_hidden=2):
    shapes = [(width, F)] + [(width, width)] * (n_hidden - 1) + [(1, width)]
    rng = np.random.default_rng(0)
    parts = []
    for o, i in shapes:
        parts += [rng.uniform(-1 / np.sqrt(i), 1 / np.sqrt(i), o * i), rng.uniform(-0.1, 0.1, o)]
    return np.concatenate(parts).astype(np.float32), shapes


def test_proposal_network_and_adjoint_match_torch(oracle):
    params, shapes = _spec()
    rng = np.random.default_rng(1)
    feats = rng.standard_normal((50, 8)).astype(np.float16)
    logits, cache = oracle.proposal_logits(feats, params, 16, 2, 10.0)
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.tensor(feats.astype(np.float64), requires_grad=True)
    z, off = x, 0
    for li, (o, i) in enumerate(shapes):
        W = p[off:off + o * i].view(o, i); off += o * i
        b = p[off:off + o]; off += o
        z = z @ W.T + b
        if li < len(shapes) - 1:
            z = torch.nn.functional.softplus(z, beta=10.0, threshold=1e6)
    np.testing.assert_allclose(logits, z[:, 0].detach().numpy(), rtol=1e-12, atol=1e-13)
    g = rng.standard_normal(50)
    dp, dx = oracle.proposal_backward(feats, params, 16, 2, 10.0, cache, g)
    tp, tx = torch.autograd.grad((z[:, 0] * torch.tensor(g)).sum(), (p, x))
    np.testing.assert_allclose(dp, tp.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dx, tx.numpy(), rtol=1e-10, atol=1e-12)


def test_kl_loss_gradient_and_minimum(oracle):
    gshape = (2, 3, 8)
    rng = np.random.default_rng(2)
    logits = rng.standard_normal(48)
    hist = rng.uniform(0, 1, 48) * (rng.uniform(0, 1, 48) > 0.3)
    hist.reshape(8, 3, 2)[:, 0, 1] = 0.0          # one column without weight
    eps = 0.05
    L, d = oracle.proposal_loss(logits, gshape, eps, hist)
    assert L >= 0
    h = 1e-6
    for k in range(48):
        e = np.zeros(48); e[k] = h
        fd = (oracle.proposal_loss(logits + e, gshape, eps, hist)[0]
              - oracle.proposal_loss(logits - e, gshape, eps, hist)[0]) / (2 * h)
        np.testing.assert_allclose(d[k], fd, rtol=1e-6, atol=1e-9)
    # at eps = 0 the minimum is reached when softmax(logits) equals the histogram
    p = np.full(48, 1.0)
    L0, d0 = oracle.proposal_loss(np.zeros(48), gshape, 0.0, p)
    assert abs(L0) < 1e-14 and np.abs(d0).max() < 1e-14


def test_inverse_cdf_sampling_distribution_and_order(oracle):
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (64, 64, 64))
    gshape = (4, 4, 16)
    rng = np.random.default_rng(3)
    logits = rng.standard_normal(16 * 4 * 4) * 2
    q = oracle.proposal_q(logits, gshape, 0.01).astype(np.float32)
    D = 16
    xyz, apr, idx = oracle.proposal_sample(g, gshape, q, D, seed=5, step=1)
    z = xyz[2].reshape(D, -1)
    assert np.all(np.diff(z, axis=0) > 0)                         # sorted along every column
    np.testing.assert_array_equal(xyz[0].reshape(D, -1), np.broadcast_to(apr[0], (D, g.n_ray)))
    # cells of all samples of grid column (0, 0) vs q: 16 x 16 fine columns x 16 samples
    cell_z = idx // 16
    col = idx % 16
    sel = col == 0
    counts = np.bincount(cell_z[sel], minlength=16)
    expected = q[:, 0, 0].astype(np.float64) / q[:, 0, 0].sum() * sel.sum()
    # stratified draws: counts never differ from expectation by more than the strata allow
    assert np.abs(counts - expected).max() <= 16 + 1e-9
    assert stats.chisquare(counts + 0.0, expected).pvalue > 1e-6 or np.abs(counts - expected).max() < 3
    # samples lie inside their cells
    pz = np.float64(np.float32(g.pitch[2] * 64 / 16))
    lo = np.float64(np.float32(g.lo[2])) + cell_z * pz
    assert np.all(xyz[2] >= lo - 1e-7) and np.all(xyz[2] <= lo + pz + 1e-7)


def test_uniform_proposal_is_stratified_closed_form(oracle):
    """q uniform over 64 cells, 16 samples: sample j falls in cells 4j..4j+3 at
    z = z0 + (u + 0.5) / 2^14 * pz_cell with u = ((j << 24) + m) >> 8."""
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (8, 8, 64))
    gshape = (2, 2, 64)
    q = np.full((64, 2, 2), 1.0 / 64, np.float32)
    xyz, _, idx = oracle.proposal_sample(g, gshape, q, 16, seed=9, step=0)
    cz = (idx // 4).reshape(16, -1)
    j = np.arange(16)[:, None]
    assert np.all((cz >= 4 * j) & (cz < 4 * j + 4))
    ray = np.arange(64)
    k = (np.uint64(0) << np.uint64(42)) | (np.uint64(3) << np.uint64(40)) | (ray[None, :] * 16 + j).astype(np.uint64)
    m = (oracle.splitmix64(9, k) >> np.uint64(40)).astype(np.int64)
    u = ((j << 24) + m) >> 8
    pz = np.float64(np.float32(g.pitch[2] * 64 / 64))
    want = (np.float64(np.float32(g.lo[2])) + (u + 0.5) / 2.0 ** 14 * pz).astype(np.float32)
    np.testing.assert_array_equal(xyz[2].reshape(16, -1), want)


def _cells_case(oracle, q_fn, m, r_max, gshape=(3, 2, 12), n=(6, 4, 48), dilate=0):
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.06, n)
    G0, G1, G2 = gshape
    q = q_fn(np.random.default_rng(3), G2, G1 * G0).astype(np.float32)
    return g, q, oracle.sample_cells(g, gshape, q, m, r_max, seed=11, step=2, dilate=dilate)


def test_sample_cells_dilated_ranking(oracle):
    """With dilate = 1 a cell ranks by the largest q of itself and its two
    neighbours: the neighbours of the column's peak (cells 4 and 6 around a
    peak at 5) come before a lone cell of larger own q elsewhere (cell 10),
    and among them the larger own q first."""
    def q_fn(rng, g2, cols):
        q = np.full((g2, cols), 0.01)
        q[5, :] = 1.0
        q[6, :] = 0.05
        q[4, :] = 0.02
        q[10, :] = 0.3
        return q
    g, q, (xyz, apr, idx, keep, n_out) = _cells_case(oracle, q_fn, 3, 1, dilate=1)
    cells = set(np.unique(idx[keep == 1] // 6).tolist())
    assert cells == {4, 5, 6}
    g, q, (xyz, apr, idx, keep, n_out) = _cells_case(oracle, q_fn, 3, 1, dilate=0)
    assert set(np.unique(idx[keep == 1] // 6).tolist()) == {5, 10, 6}


def test_sample_cells_selection_and_layout(oracle):
    """Top-m cells of q per grid column (ties to the lower cell), in depth
    order; every kept sample is the dense STRATIFIED grid's own point; one
    closing sample (the next cell's first depth) after each of the first
    r_max runs; padding repeats the column's last sample; keep and idx."""
    G0, G1, G2 = 3, 2, 12
    def q_fn(rng, g2, cols):
        q = rng.uniform(0.0, 1.0, (g2, cols))
        q[5, :] = q[6, :] = 2.0                            # a tie: cells 5 and 6 both kept
        q[9, 0] = q[3, 0] = 1.5
        return q
    m, r_max = 5, 2
    g, q, (xyz, apr, idx, keep, n_out) = _cells_case(oracle, q_fn, m, r_max)
    s_fine = g.n[2] // G2
    assert n_out == m * s_fine + r_max
    dense, dapr = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=11, step=2)
    assert np.array_equal(apr.view(np.uint32), dapr.view(np.uint32))
    n_ray = g.n[0] * g.n[1]
    for ray in range(n_ray):
        ix, iy = ray % g.n[0], ray // g.n[0]
        col = (iy * G1 // g.n[1]) * G0 + (ix * G0 // g.n[0])
        want = sorted(sorted(range(G2), key=lambda c: (-q[c, col], c))[:m])
        slots = [s * n_ray + ray for s in range(n_out)]
        z = xyz[2, slots]
        kp = keep[slots]
        cells = idx[slots] // (G0 * G1)
        assert sorted(set(cells[kp == 1])) == want
        assert (kp == 1).sum() == m * s_fine
        # every sample is a dense grid point of this column, in depth order
        dz = dense[2, ray::n_ray]
        k_of = [int(np.nonzero(dz == zz)[0][0]) for zz in z]
        assert all(np.array_equal(xyz[:, p].view(np.uint32), dense[:, k * n_ray + ray].view(np.uint32))
                   for p, k in zip(slots, k_of))
        assert all(b >= a for a, b in zip(k_of, k_of[1:]))
        # closing samples: first depth of the cell after a run, keep 0
        runs = [c for i, c in enumerate(want) if i + 1 == m or want[i + 1] != c + 1]
        closing = [(c + 1) * s_fine for c in runs if c + 1 < G2][:r_max]
        emitted = [k for k, kk in zip(k_of, kp) if kk == 0]
        assert emitted[:len(closing)] == closing
        assert all(k == k_of[-1] for k in emitted[len(closing):])   # padding


def test_sample_cells_blend_equals_dense_blend_through_closed_gaps(oracle):
    """NeuS alpha telescopes: prod (1 - alpha) over consecutive samples is
    Phi(f_end)/Phi(f_start) where f decreases. On a column whose SDF falls
    monotonically in depth (a plane facing the array), the kept samples'
    T and w from the cell subset (closing samples: keep 0) equal the dense
    grid's at the same points; without the closing samples they do not."""
    G0, G1, G2 = 3, 2, 12
    def q_fn(rng, g2, cols):
        q = np.zeros((g2, cols))
        q[[0, 1, 5, 8, 9], :] = 1.0                        # runs {0, 1}, {5}, {8, 9}: every gap closed
        return q
    g, q, (xyz, apr, idx, keep, n_out) = _cells_case(oracle, q_fn, 5, 3)
    n_ray = g.n[0] * g.n[1]
    dense, dapr = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=11, step=2)
    z_plane, s_sharp = 0.15, 400.0
    f_of = lambda x: z_plane - x[2].astype(np.float64)   # decreasing in depth
    a_of = lambda x: 0.5 + 0.1 * np.sin(40.0 * x[0].astype(np.float64))
    al_d, T_d, w_d, _, _ = oracle.blend(f_of(dense), a_of(dense), n_ray, g.n[2], np.zeros(n_ray), np.zeros(1),
                                        s_sharp, 1.0)
    al_s, T_s, w_s, _, _ = oracle.blend(f_of(xyz), a_of(xyz), n_ray, n_out, np.zeros(n_ray), np.zeros(1), s_sharp,
                                        1.0, keep)
    dz = dense[2].reshape(g.n[2], n_ray)
    for p in np.nonzero(keep == 1)[0]:
        ray = p % n_ray
        k = int(np.nonzero(dz[:, ray] == xyz[2, p])[0][0])
        j = k * n_ray + ray
        np.testing.assert_allclose(T_s[p], T_d[j], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(w_s[p], w_d[j], rtol=1e-12, atol=1e-15)
    assert np.all(w_s[keep == 0] == 0.0)
    # without closing samples the alpha of each run's last sample spans the
    # gap: T after the gap still telescopes, but that sample's w takes the
    # whole gap's opacity
    _, q2, (xyz2, _, _, keep2, n2) = _cells_case(oracle, q_fn, 5, 0)
    _, T2, w2, _, _ = oracle.blend(f_of(xyz2), a_of(xyz2), n_ray, n2, np.zeros(n_ray), np.zeros(1), s_sharp, 1.0,
                                   keep2)
    dev = []
    for p in np.nonzero(keep2 == 1)[0]:
        ray = p % n_ray
        j = int(np.nonzero(dz[:, ray] == xyz2[2, p])[0][0]) * n_ray + ray
        np.testing.assert_allclose(T2[p], T_d[j], rtol=1e-12, atol=1e-15)
        dev.append(abs(w2[p] - w_d[j]) / abs(w_d).max())
    assert max(dev) > 1e-3
