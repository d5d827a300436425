"""Pins of the CPU oracle of the warm-start network (oracle/cnn.py): its convolution against
the explicit-loop definition (periodic x, zero y), its gradient against central finite
differences, and its size against the layer table.  CPU only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as C  # noqa: E402


def test_conv_matches_explicit_loops():
    rng = np.random.default_rng(0)
    B, ci, co, H, W = 2, 3, 4, 5, 6
    a = rng.normal(size=(B, ci, H, W))
    w = rng.normal(size=(co, ci, 3, 3))
    b = rng.normal(size=co)
    y = C.conv3x3(torch.tensor(a), torch.tensor(w), torch.tensor(b)).numpy()
    ref = np.zeros((B, co, H, W))
    for n in range(B):
        for o in range(co):
            for h in range(H):
                for x in range(W):
                    s = b[o]
                    for i in range(ci):
                        for dy in range(3):
                            for dx in range(3):
                                hh, xx = h + dy - 1, (x + dx - 1) % W
                                if 0 <= hh < H:
                                    s += w[o, i, dy, dx] * a[n, i, hh, xx]
                    ref[n, o, h, x] = s
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    n = C.n_params()
    p = rng.normal(scale=0.05, size=n)
    x = rng.normal(size=(2, 12, 8, 12))
    t = rng.normal(size=(2, 4, 8, 12))
    L, g, _ = C.loss_and_grad(p, x, t)
    for k in range(4):
        d = rng.normal(size=n)
        eps = 1e-6
        Lp, _, _ = C.loss_and_grad(p + eps * d, x, t)
        Lm, _, _ = C.loss_and_grad(p - eps * d, x, t)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))


def test_layer_table_and_size():
    assert C.CH == (12, 32, 32, 32, 32, 32, 4)
    assert C.n_params() == 41636
