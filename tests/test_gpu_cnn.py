"""The surrogate's hand-written CUDA kernels against the CPU FP64 oracle of the same network.

FP32-activation build: forward outputs and all parameter gradients within 1e-4 relative L2
(FP32 accumulation over 288-term sums, 6 layers).  BF16-activation build (the one trained):
stored activations carry 8 significant bits, so the bars are 3e-2 (forward) and 1e-1
(gradient), relative L2; both stated by the test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2210_07501_gb300 as p
    p.build()
    p.load()
    return p


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("bf16,fwd_bar,grad_bar", [(False, 1e-4, 1e-4), (True, 3e-2, 1e-1)])
def test_forward_and_gradients_against_oracle(pkg, bf16, fwd_bar, grad_bar):
    from oracle import cnn as C
    rng = np.random.default_rng(42)
    B, H, W = 3, 20, 40           # ragged against the 16 x 16 tiles
    net = pkg.Cnn(H, W, batch_max=4, bf16=bf16, seed=7)
    p = rng.normal(scale=0.08, size=net.n_params).astype(np.float32)
    net.set_params(p)
    x = rng.normal(size=(B, 12, H, W)).astype(np.float32)
    t = rng.normal(size=(B, 4, H, W)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    yd = torch.empty((B, 4, H, W), dtype=torch.float32, device="cuda")
    net.forward(xd, yd)
    torch.cuda.synchronize()
    L, g, y = C.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    ef = rel(yd.cpu().numpy(), y)
    gg, loss = net.gradients(xd, td)
    eg = rel(gg.astype(np.float64), g)
    print(f"bf16={bf16}: forward rel {ef:.2e}, gradient rel {eg:.2e}, loss {loss:.6e} vs {L:.6e}")
    assert ef <= fwd_bar and eg <= grad_bar
    assert abs(loss - L) <= fwd_bar * 2 * abs(L)
    g2, _ = net.gradients(xd, td)
    assert np.array_equal(g2, gg)          # deterministic
    net.close()


def test_training_reduces_loss(pkg):
    rng = np.random.default_rng(3)
    B, H, W = 8, 16, 32
    net = pkg.Cnn(H, W, batch_max=B, bf16=True, seed=1)     # on torch's current stream
    x = torch.tensor(rng.normal(size=(B, 12, H, W)).astype(np.float32), device="cuda")
    # a smooth target that depends on the inputs
    t = torch.stack([torch.tanh(x[:, 0] + 0.5 * x[:, 4]), x[:, 1] * x[:, 2], torch.sin(x[:, 3]), x[:, 5]], 1).contiguous()
    first = net.train_step(x, t, 1e-3)
    for _ in range(300):
        last = net.train_step(x, t, 1e-3)
    assert last < 0.3 * first, (first, last)
    net.close()
