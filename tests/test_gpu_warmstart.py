"""GPU parity of the start-vector network (rks_ws_*) against its FP64 oracle.

The network runs with FP16 copies of its weights and FP32 activations and
accumulation; the oracle (oracle/warmstart.py, pinned by finite differences)
takes the same FP16-rounded weights in FP64.  Forward outputs must agree to
FP32 rounding (1e-4 of the output's scale), gradients to 1e-3 relative (as a
whole and per layer), one Adam step to 1e-6, on grids of 32 x 32 and 40 x 48
(partial 16 x 16 tiles at the coarse levels).
"""
import numpy as np
import pytest

from oracle import warmstart as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05400_gb300 import build as B
    B.build()
    return torch


def K():
    from paper_2508_05400_gb300 import rks
    return rks


def _fp16_weights(theta):
    """The parameters as the network computes with them: weights rounded to FP16."""
    th = theta.astype(np.float64).copy()
    o = 0
    for i, sz in enumerate(W.param_sizes()):
        if i % 2 == 0:
            th[o:o + sz] = theta[o:o + sz].astype(np.float16).astype(np.float64)
        o += sz
    return th


def _sample(H, Wd, q, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((3, H, Wd)).astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((H * Wd, q)))
    return x, Q


@pytest.mark.parametrize("H,Wd", [(32, 32), (40, 48)])
def test_forward_matches_oracle(gpu, H, Wd):
    x, _ = _sample(H, Wd, 2, 1)
    with K().WarmStart(H, Wd, seed=3) as net:
        theta = net.params()
        u = net.forward(gpu.from_numpy(x).cuda()).cpu().numpy()
    uo, _ = W.forward(_fp16_weights(theta), x.astype(np.float64))
    assert np.max(np.abs(u - uo)) <= 1e-4 * np.max(np.abs(uo)), np.max(np.abs(u - uo))


@pytest.mark.parametrize("H,Wd", [(32, 32), (40, 48)])
def test_gradient_matches_oracle(gpu, H, Wd):
    x, Q = _sample(H, Wd, 4, 2)
    with K().WarmStart(H, Wd, seed=5) as net:
        theta = net.params()
        loss = net.accumulate(gpu.from_numpy(x).cuda(), gpu.from_numpy(np.ascontiguousarray(Q.T)).float().cuda())
        g = net.grad().astype(np.float64)
    th = _fp16_weights(theta)
    Lo, go, _ = W.loss_and_grad(th, x.astype(np.float64), Q.astype(np.float32).astype(np.float64))
    assert abs(loss - Lo) <= 1e-5
    assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go)
    o = 0
    for i, sz in enumerate(W.param_sizes()):
        a, b = g[o:o + sz], go[o:o + sz]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-7 * np.linalg.norm(go), i
        o += sz


def test_adam_step_matches_oracle(gpu):
    H = Wd = 32
    x, Q = _sample(H, Wd, 3, 4)
    with K().WarmStart(H, Wd, seed=6) as net:
        theta = net.params().astype(np.float64)
        net.accumulate(gpu.from_numpy(x).cuda(), gpu.from_numpy(np.ascontiguousarray(Q.T)).float().cuda())
        g = net.grad().astype(np.float64)
        net.step(1e-3)
        after = net.params().astype(np.float64)
        assert np.all(net.grad() == 0)                       # cleared by the step
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    W.adam(theta, m, v, g, 1, 1e-3)
    assert np.max(np.abs(after - theta)) <= 1e-6


def test_training_lowers_the_loss_of_a_fixed_sample(gpu):
    H = Wd = 32
    x, Q = _sample(H, Wd, 4, 7)
    xd, Qd = gpu.from_numpy(x).cuda(), gpu.from_numpy(np.ascontiguousarray(Q.T)).float().cuda()
    with K().WarmStart(H, Wd, seed=8) as net:
        first = net.accumulate(xd, Qd)
        net.step(1e-3)
        for _ in range(60):
            last = net.accumulate(xd, Qd)
            net.step(1e-3)
        # the same bits on a second network with the same seed
        with K().WarmStart(H, Wd, seed=8) as net2:
            for _ in range(61):
                net2.accumulate(xd, Qd)
                net2.step(1e-3)
            assert np.array_equal(net.params(), net2.params())
    assert last < 0.5 * first, (first, last)


def test_start_vector_is_normalised_output_plus_random_part(gpu):
    H = Wd = 32
    x, _ = _sample(H, Wd, 1, 9)
    from paper_2508_05400_gb300 import inputs as I
    with K().WarmStart(H, Wd, seed=10) as net:
        xd = gpu.from_numpy(x).cuda()
        u = net.forward(xd).cpu().numpy().ravel().astype(np.float64)
        u1 = net.start_vector(xd, eps=1e-3, seed=11).cpu().numpy()
    g = I.start_vector(H * Wd, 11)
    want = u / np.linalg.norm(u) + 1e-3 * g / np.linalg.norm(g)
    assert np.max(np.abs(u1 - want)) <= 1e-12


def test_bad_arguments_are_rejected(gpu):
    with pytest.raises(K().RKSError):
        K().WarmStart(30, 32)            # not a multiple of 8
    with K().WarmStart(16, 16) as net:
        with pytest.raises(ValueError):
            net.forward(gpu.zeros((3, 16, 8), dtype=gpu.float32, device="cuda"))
        with pytest.raises(K().RKSError):
            net.step(1e-3)               # nothing accumulated
