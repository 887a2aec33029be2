"""Failure detection without a GPU fault: the bounded-wait path that every TMA
and tensor-core kernel relies on (a wait that runs out records the timeout in
the device error word and the kernel returns) is made to run out on purpose,
on an mbarrier nothing arrives at, with a 2 ms limit. The status reaches the
host, is cleared, and the context keeps working."""
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


def test_bounded_wait_timeout_is_reported_and_context_survives(G, oracle):
    G.geraf_poll_device_error()                       # start clean
    G.geraf_check_bounded_wait(2_000_000)
    with pytest.raises(G.GerafError) as e:
        G.geraf_poll_device_error()
    assert e.value.status == 5                        # GERAF_ERR_TIMEOUT
    G.geraf_poll_device_error()                       # the word was cleared
    # the context still computes: a small render against the oracle
    rng = np.random.default_rng(3)
    n = 200
    xyz = (np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, n))).astype(np.float32)
    grad = rng.standard_normal((3, n)).astype(np.float32)
    w = rng.uniform(0, 1, n).astype(np.float32)
    t_eff = rng.uniform(0.3, 2.0, n).astype(np.float32)
    ant = gi.antenna_array(4, 5, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, 70)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), G.Band(b.f0, b.df, b.n_f))
    G.geraf_poll_device_error()
    want = oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)
    got = s.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5


def test_bounded_wait_limits_are_checked(G):
    from paper_2605_29097_gb300 import _lib
    assert _lib.lib().geraf_check_bounded_wait(10, None) == 1            # below 1 us: INVALID_ARG
    assert _lib.lib().geraf_check_bounded_wait(5_000_000_000, None) == 1  # above 1 s
