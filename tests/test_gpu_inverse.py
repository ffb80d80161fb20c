"""The synthetic inverse problem of Sec. 6.2 (paper_2504_13750_gb300/inverse.py):
the adjoint gradient of the Eq. 6.6 loss with respect to the fresh-gas
equivalence ratio against central differences of the loss, and Adam
recovering theta = 1 from both sides."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_13750_gb300 import build, inverse

    build.build()
    p = inverse.ChannelInverse(nx=100, ny=40, n_steps=40, dev_steps=150, ckpt_every=10)
    yield p
    p.close()


@pytest.mark.parametrize("theta", [0.9, 1.1])
def test_gradient_matches_central_differences(P, theta):
    L, g = P.loss_and_grad(theta)
    d = 1e-3
    Lp, _ = P.loss_and_grad(theta + d)
    Lm, _ = P.loss_and_grad(theta - d)
    fd = (Lp - Lm) / (2 * d)
    assert L > 0 and abs(g - fd) <= 2e-2 * abs(fd), (g, fd)


@pytest.mark.parametrize("theta0", [0.85, 1.15])
def test_adam_recovers_the_equivalence_ratio(P, theta0):
    hist, _ = P.optimize(theta0, iters=30, lr=0.01)
    assert abs(hist[-1][0] - 1.0) < 0.03, hist[-1]
    assert hist[-1][1] < 0.2 * hist[0][1], (hist[0], hist[-1])
