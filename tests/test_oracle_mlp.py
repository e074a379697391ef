"""Pins of the oracle's predictor network against independent routines.

The oracle's network (40 -> 64 -> 64 -> 64 -> 2, GELU, bfloat16 weights,
FP64 arithmetic) is checked against PyTorch's own CPU operators in float64:
its linear layers, its exact (erf) GELU and its automatic differentiation
for the gradient, and torch.optim.Adam for the optimiser step.  The
bfloat16 rounding is checked on hand-picked ties and against PyTorch's
float32 -> bfloat16 conversion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_stats = pytest.importorskip("scipy.stats")

IN, HID, OUT, NP = 40, 64, 2, 11074
OFF = dict(W1=0, b1=2560, W2=2624, b2=6720, W3=6784, b3=10880, W4=10944, b4=11072)


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(NP, dtype=np.float32)
    for name, shape in (("W1", (HID, IN)), ("W2", (HID, HID)), ("W3", (HID, HID)), ("W4", (OUT, HID))):
        n = shape[0] * shape[1]
        p[OFF[name]:OFF[name] + n] = (rng.uniform(-1, 1, n) * scale * np.sqrt(6.0 / shape[1]))
    for name, n in (("b1", HID), ("b2", HID), ("b3", HID), ("b4", OUT)):
        p[OFF[name]:OFF[name] + n] = rng.normal(0, 0.1, n)
    return p


def torch_net(p):
    """The network in torch float64 with bfloat16-rounded weights (leaf tensors)."""
    t = torch.from_numpy(p.copy())
    rounded = t.to(torch.bfloat16).to(torch.float64)
    full = t.to(torch.float64)
    ws = []
    for name, shape in (("W1", (HID, IN)), ("W2", (HID, HID)), ("W3", (HID, HID)), ("W4", (OUT, HID))):
        n = shape[0] * shape[1]
        ws.append(rounded[OFF[name]:OFF[name] + n].reshape(shape).clone().requires_grad_(True))
    bs = []
    for name, n in (("b1", HID), ("b2", HID), ("b3", HID), ("b4", OUT)):
        bs.append(full[OFF[name]:OFF[name] + n].clone().requires_grad_(True))

    def f(x):
        h = x
        for k in range(3):
            h = torch.nn.functional.gelu(torch.nn.functional.linear(h, ws[k], bs[k]),
                                         approximate="none")
        return torch.nn.functional.linear(h, ws[3], bs[3])
    return f, ws, bs


def test_bf16_rounding_ties_and_library(orc):
    one = np.float32(1.0)
    assert orc.bf16(one) == 1.0
    # spacing of bfloat16 at 1 is 2^-7: 1 + 2^-8 is a tie -> even (1.0);
    # 1 + 3 2^-8 is a tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert orc.bf16(np.float32(1 + 2**-8)) == 1.0
    assert orc.bf16(np.float32(1 + 3 * 2**-8)) == 1 + 2**-6
    assert orc.bf16(np.float32(1 + 2**-8 + 2**-20)) == 1 + 2**-7
    assert orc.bf16(np.float32(-1 - 3 * 2**-8)) == -(1 + 2**-6)
    rng = np.random.default_rng(5)
    w = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-30, 100),
                        rng.normal(0, 1e30, 100)]).astype(np.float32)
    want = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.bf16(w), want)


def test_gelu_is_x_phi_and_its_derivative(orc):
    for x in (-6.0, -2.5, -1.0, -0.3, 0.0, 0.4, 1.0, 2.0, 7.5):
        # the erf form cancels in the far negative tail: absolute rounding ~1e-16 |x|
        assert orc.gelu(x) == pytest.approx(x * scipy_stats.norm.cdf(x), rel=1e-14, abs=1e-15)
        # derivative: Phi(x) + x phi(x) from scipy's normal distribution
        want = scipy_stats.norm.cdf(x) + x * scipy_stats.norm.pdf(x)
        assert orc.gelu_grad(x) == pytest.approx(want, rel=1e-12, abs=1e-15)
        if abs(x) <= 3:  # and a central difference where it is well conditioned
            h = 1e-6
            fd = (orc.gelu(x + h) - orc.gelu(x - h)) / (2 * h)
            assert orc.gelu_grad(x) == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_forward_matches_torch(orc):
    p = random_params(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (50, IN))
    f, _, _ = torch_net(p)
    want = f(torch.from_numpy(X)).detach().numpy()
    got = orc.mlp_forward(p, X)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_loss_gradient_matches_autograd(orc):
    p = random_params(3)
    rng = np.random.default_rng(4)
    n = 37
    X = rng.normal(0, 1, (n, IN))
    Y = rng.normal(0, 1, (n, OUT))
    f, ws, bs = torch_net(p)
    loss_t = 0.5 * ((f(torch.from_numpy(X)) - torch.from_numpy(Y)) ** 2).sum() / n
    loss_t.backward()
    want = np.zeros(NP)
    for name, t in zip(("W1", "W2", "W3", "W4"), ws):
        want[OFF[name]:OFF[name] + t.numel()] = t.grad.numpy().ravel()
    for name, t in zip(("b1", "b2", "b3", "b4"), bs):
        want[OFF[name]:OFF[name] + t.numel()] = t.grad.numpy()
    loss, g = orc.mlp_loss_grad(p, X, Y)
    assert loss == pytest.approx(loss_t.item(), rel=1e-13)
    np.testing.assert_allclose(g, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())
    # every parameter block receives gradient
    for name in OFF:
        assert np.any(g[OFF[name]:OFF[name] + 2] != 0.0)


def test_adam_matches_torch(orc):
    rng = np.random.default_rng(6)
    p0 = rng.normal(0, 1, 300)
    grads = [rng.normal(0, 1, 300) for _ in range(5)]
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p = p0.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(grads, start=1):
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        orc.adam(p, g, m, v, t, 1e-2)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)
