"""The learned start vector on held-out members of the 512 x 512 family.

The network is trained on the GPU (its own kernels) on the Schur vectors that
rKS computed for training members of the parametric convection-diffusion
family, then used for held-out members: u_1 = u / ||u|| + 1e-3 g / ||g||
(g the solver's own random start), against the random start g alone, both to
||A x - l x|| / (||A||_1 ||x||) <= 1e-8 in double-float.  The test asserts
what the network learned (a held-out subspace capture far above a random
vector's q / n) and that the warm solves converge and are not slower beyond
the run-to-run spread; it prints the restart counts and times it measured.
"""
import numpy as np
import pytest

from paper_2508_05400_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05400_gb300 import build as B
    B.build()
    return torch


def test_learned_start_on_held_out_members():
    from paper_2508_05400_gb300 import rks
    from paper_2508_05400_gb300 import warmstart as WS
    N, ntrain, ntest = 512, 16, 4
    train = WS.make_samples(range(ntrain), 10000, N)
    with rks.WarmStart(N, N, seed=0) as net:
        hist = WS.train(net, train, epochs=15, lr=1e-3, batch=8)
        rows = []
        for i in range(ntest):
            P = I.grf_convdiff2d_problem(i, seed0=20000, N=N)
            info_r, wall_r, U = WS.solve_member(P, want_basis=True)
            x = __import__("torch").from_numpy(I.grf_member_fields(i, seed0=20000, N=N)).cuda()
            cap = WS.capture(net, x, WS.target_basis(U))
            u1 = net.start_vector(x, eps=1e-3, seed=P.u1_seed).cpu().numpy()
            info_w, wall_w, _ = WS.solve_member(P, u1=u1)
            assert info_w["converged"] == 1 and info_w["max_resid"] <= P.tol
            rows.append((info_r["restarts"], info_w["restarts"], wall_r, wall_w, cap))
    r = np.array(rows)
    print(f"\ntraining loss {hist[0]:.3f} -> {hist[-1]:.3f}; held-out capture {r[:, 4].round(3)}; "
          f"restarts random {r[:, 0].astype(int)} warm {r[:, 1].astype(int)}; "
          f"time random {r[:, 2].mean():.3f} s warm {r[:, 3].mean():.3f} s")
    assert hist[-1] < hist[0]
    assert r[:, 4].mean() > 0.3            # a random vector captures q / n ~ 6e-5
    assert r[:, 1].mean() <= 1.1 * r[:, 0].mean()
