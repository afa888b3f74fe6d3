"""Learned initial traces on the GPU: perceptron gradients against the FP64
oracle, trace codes, and the iterations the learned guess saves."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1710_02401_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import learn as Lrn
    from paper_1710_02401_gb300 import swr as S
    return torch, S, Lrn


def test_mlp_gradient_matches_oracle(mods):
    torch, S, Lrn = mods
    dims = [16, 64, 64, 40]
    rng = np.random.default_rng(1)
    x = rng.normal(size=(70, 16)).astype(np.float32)
    t = rng.normal(size=(70, 40)).astype(np.float32)
    p = Lrn.init_params(dims, 7)
    mlp = S.MLP(16, 64, 2, 40)
    mlp.set_params(p)
    loss, g = mlp.train_step(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), 0.0,
                             want_grad=True)
    ref_loss, ref_g = M.loss_and_grad(p.astype(np.float64), dims, x, t, bf16=True)
    assert abs(loss - ref_loss) <= 2e-3 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 1e-2 * np.linalg.norm(ref_g)
    # forward agrees too
    y = mlp.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    yr = M.forward(p.astype(np.float64), dims, x, bf16=True)[-1]
    assert np.abs(y - yr).max() <= 1e-2 * np.abs(yr).max()


def test_mlp_full_width_products_match_oracle(mods):
    # the network's real shapes: width 256, 1024 outputs, batch 300 -> several
    # 128 x 64 tensor-core tiles per product, K above one 64-wide staging block,
    # all three operand layouts (forward, weight gradient, back-propagation).
    # Measured: loss 4e-8, gradient 3e-4, output 1.2e-3 (BF16 roundings of
    # hidden activations flip where FP32 and FP64 accumulation differ)
    torch, S, Lrn = mods
    dims = [16, 256, 256, 256, 1024]
    rng = np.random.default_rng(3)
    x = rng.normal(size=(300, 16)).astype(np.float32)
    t = rng.normal(size=(300, 1024)).astype(np.float32)
    p = Lrn.init_params(dims, 5)
    mlp = S.MLP(16, 256, 3, 1024)
    mlp.set_params(p)
    loss, g = mlp.train_step(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), 0.0,
                             want_grad=True)
    ref_loss, ref_g = M.loss_and_grad(p.astype(np.float64), dims, x, t, bf16=True)
    assert abs(loss - ref_loss) <= 1e-6 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 3e-3 * np.linalg.norm(ref_g)
    y = mlp.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    yr = M.forward(p.astype(np.float64), dims, x, bf16=True)[-1]
    assert np.abs(y - yr).max() <= 1e-2 * np.abs(yr).max()


def test_mlp_training_reduces_loss(mods):
    torch, S, Lrn = mods
    rng = np.random.default_rng(2)
    x = rng.normal(size=(256, 16)).astype(np.float32)
    w = rng.normal(size=(16, 24))
    y = np.tanh(x @ w / 4.0).astype(np.float32)
    model, losses = Lrn.train(x, y, width=128, n_hidden=3, steps=400, lr=2e-3)
    assert losses[-1] < 0.05 * losses[0]


def _code_error(S_mod, Lrn, insts, S, Tm):
    s, done, _ = Lrn.solve(insts, 1e-8, 30)
    s.trace_codec(S, Tm)
    g_before = [g.copy() for g in s.robin_data()]
    code = s.trace_encode()
    s.trace_decode_set(code)
    code2 = s.trace_encode()
    err = max(np.abs(a - b).max() / np.abs(a).max() for a, b in zip(g_before, s.robin_data()))
    return code, code2, err


def test_trace_code_roundtrip(mods):
    torch, S, Lrn = mods
    insts = P.learned_trace_family(3, seed=11)
    code, code2, err_small = _code_error(S, Lrn, insts, 8, 16)
    assert float(code.abs().max()) > 0.0
    # decoding replaces the Robin data by their projection; encoding it again
    # gives back the same code (orthonormal bases: the projection is idempotent)
    assert torch.allclose(code, code2, rtol=1e-4, atol=1e-5 * float(code.abs().max()))
    # a larger code represents the data better
    _, _, err_large = _code_error(S, Lrn, insts, 16, 32)
    assert err_large < 0.5 * err_small < 0.1


def test_learned_guess_saves_schwarz_iterations(mods):
    torch, S, Lrn = mods
    train = P.learned_trace_family(160, seed=21)
    test = P.learned_trace_family(24, seed=99)
    x, y, done = Lrn.gather_training_set(train)
    assert np.all(done <= 60)
    model, losses = Lrn.train(x, y, steps=1500)
    zero, learned = Lrn.compare(model, test)
    assert np.all(zero <= 60) and np.all(learned <= 61)
    assert learned.mean() < zero.mean()
    # wall time at the same Res <= 1e-8 for every instance, inference and
    # decoding of the guess included
    t = Lrn.compare_timed(model, test)
    print(f"\nlearned guess: {t}")
    assert t["batch_iterations_learned"] <= t["batch_iterations_zero_guess"]
    assert t["seconds_inference_decode"] < 0.1 * t["seconds_learned"]
    assert t["seconds_learned"] < t["seconds_zero_guess"]
