"""Tensor-core (tcgen05/TMA/TMEM) GEMM and the surrogate MLP against CPU
references (BF16 inputs, FP32 accumulation)."""
import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu


def bf(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 200), (129, 257, 1000), (64, 128, 2048),
                                   (1024, 2048, 288), (256, 12376, 256), (8192, 2048, 2048),
                                   (2000, 3000, 96)])  # 192 ragged tiles: CTAs alternate accumulators
def test_tc_gemm_matches_cpu(M, N, K):
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(M + N + K)
    A = bf(rng.standard_normal((M, K)))
    Bm = bf(rng.standard_normal((N, K)))
    C = S.gemm(A.cuda(), Bm.cuda())
    S.sync_status()
    ref = A.double().numpy() @ Bm.double().numpy().T
    err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err


def test_tc_gemm_epilogues():
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(3)
    M, N, K = 200, 136, 320
    A = bf(rng.standard_normal((M, K)) * 0.2)
    Bm = bf(rng.standard_normal((N, K)) * 0.2)
    bias = torch.tensor(rng.standard_normal(N), dtype=torch.float32)
    acc = A.double().numpy() @ Bm.double().numpy().T
    Cb = S.gemm(A.cuda(), Bm.cuda(), S.GEMM_F32_BIAS, bias=bias.cuda())
    assert np.abs(Cb.cpu().numpy() - (acc + bias.numpy())).max() < 1e-4
    Z = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    H = S.gemm(A.cuda(), Bm.cuda(), S.GEMM_GELU, bias=bias.cuda(), aux=Z)
    zref = mlp.bf16(acc + bias.numpy())
    assert np.abs(Z.float().cpu().numpy() - zref).max() <= 1e-2 * np.abs(zref).max()
    href = mlp.bf16(mlp.gelu(Z.double().cpu().numpy()))
    assert np.abs(H.double().cpu().numpy() - href).max() <= 1e-2 * np.abs(href).max()
    D = S.gemm(A.cuda(), Bm.cuda(), S.GEMM_GELU_BWD, aux=Z)
    dref = mlp.bf16(acc * mlp.gelu_grad(Z.double().cpu().numpy()))
    assert np.abs(D.double().cpu().numpy() - dref).max() <= 1e-2 * np.abs(dref).max()
    C0 = torch.tensor(rng.standard_normal((M, N)), dtype=torch.float32, device="cuda")
    C1 = C0.clone()
    S.gemm(A.cuda(), Bm.cuda(), S.GEMM_F32_ACCUM, C=C1)
    assert np.abs(C1.cpu().numpy() - (C0.cpu().numpy() + acc)).max() < 1e-4
    S.sync_status()


def test_tc_gemm_epilogues_many_tiles():
    """More tiles than SMs (200 here), ragged on both edges, so the persistent
    CTAs walk several tiles and alternate their two TMEM accumulators while the
    fused epilogues (bias + GELU with the pre-activation, accumulate) run."""
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(4)
    M, N, K = 5000, 1100, 320
    A = bf(rng.standard_normal((M, K)) * 0.2)
    Bm = bf(rng.standard_normal((N, K)) * 0.2)
    bias = torch.tensor(rng.standard_normal(N), dtype=torch.float32)
    acc = A.double().numpy() @ Bm.double().numpy().T
    Z = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    H = S.gemm(A.cuda(), Bm.cuda(), S.GEMM_GELU, bias=bias.cuda(), aux=Z)
    zref = mlp.bf16(acc + bias.numpy())
    assert np.abs(Z.float().cpu().numpy() - zref).max() <= 1e-2 * np.abs(zref).max()
    href = mlp.bf16(mlp.gelu(Z.double().cpu().numpy()))
    assert np.abs(H.double().cpu().numpy() - href).max() <= 1e-2 * np.abs(href).max()
    C0 = torch.tensor(rng.standard_normal((M, N)), dtype=torch.float32, device="cuda")
    C1 = C0.clone()
    S.gemm(A.cuda(), Bm.cuda(), S.GEMM_F32_ACCUM, C=C1)
    assert np.abs(C1.cpu().numpy() - (C0.cpu().numpy() + acc)).max() < 1e-4
    S.sync_status()


def test_surrogate_gradients_match_cpu_mlp():
    """Weight and bias gradients of the GPU MLP (tensor-core GEMMs, BF16
    storage) against the CPU MLP with the same BF16 rounding, B = 16."""
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(21)
    P, H, L, K, Bn = 12, 64, 2, 40, 16
    model = S.Surrogate(n_phases=P, hidden=H, n_hidden_layers=L, n_outputs=K, max_batch=32, seed=5)
    params = [model.get_param(l) for l in range(L + 1)]
    phases = rng.uniform(0, 2 * np.pi, (Bn, P)).astype(np.float32)
    target = rng.dirichlet(np.ones(K), size=Bn).astype(np.float32)
    losses = torch.zeros(Bn, dtype=torch.float32, device="cuda")
    model.train_step(torch.tensor(phases, device="cuda"), torch.tensor(target, device="cuda"), 0.0, losses)
    S.sync_status()
    loss_ref, kl_ref, grads = mlp.loss_and_grads([(w.astype(np.float64), b.astype(np.float64)) for w, b in params],
                                                 phases.astype(np.float64), target.astype(np.float64), bf=True)
    assert np.abs(losses.cpu().numpy() - kl_ref).max() <= 1e-2 * np.abs(kl_ref).max()
    for l in range(L + 1):
        gw, gb = model.get_grad(l)
        rw = np.linalg.norm(gw - grads[l][0]) / np.linalg.norm(grads[l][0])
        rb = np.linalg.norm(gb - grads[l][1]) / np.linalg.norm(grads[l][1])
        assert rw <= 1e-2 and rb <= 1e-2, (l, rw, rb)
    # lr = 0 leaves the weights unchanged
    w0, _ = model.get_param(0)
    assert np.array_equal(w0, params[0][0])


def test_surrogate_input_harmonics_equal_explicit_phases():
    """With input harmonics H the model forms its phases h * x_j (index
    (h - 1) * n_x + j) itself: its outputs equal the same model fed those
    phases directly (identical weights, bitwise up to the sin/cos argument)."""
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(31)
    nx, H, K, Bn = 6, 4, 48, 16
    a = S.Surrogate(n_phases=nx * H, hidden=64, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=9)
    b = S.Surrogate(n_phases=nx * H, hidden=64, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=9)
    b.set_input_harmonics(H)
    x = rng.standard_normal((Bn, nx)).astype(np.float32)
    phases = (np.arange(1, H + 1, dtype=np.float32)[None, :, None] * x[:, None, :]).reshape(Bn, -1)
    qa = a.forward(torch.tensor(phases, device="cuda")).cpu().numpy()
    qb = b.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    S.sync_status()
    assert np.abs(qa - qb).max() <= 1e-6
    with pytest.raises(Exception):
        b.set_input_harmonics(5)  # must divide n_phases


def test_surrogate_learns_a_small_map():
    """A few hundred Adam steps on a fixed random target reduce the KL loss."""
    from paper_2602_11092_gb300 import surrogate as S
    rng = np.random.default_rng(4)
    P, K, Bn = 8, 64, 64
    model = S.Surrogate(n_phases=P, hidden=128, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=7)
    phases = torch.tensor(rng.uniform(0, 2 * np.pi, (Bn, P)), dtype=torch.float32, device="cuda")
    target = torch.tensor(rng.dirichlet(np.ones(K) * 0.5, size=Bn), dtype=torch.float32, device="cuda")
    losses = torch.zeros(Bn, dtype=torch.float32, device="cuda")
    model.train_step(phases, target, 1e-3, losses)
    first = losses.mean().item()
    for _ in range(300):
        model.train_step(phases, target, 1e-3, losses)
    S.sync_status()
    assert losses.mean().item() < 0.5 * first


def test_training_checkpoint_resume_is_bitwise(tmp_path):
    """Save weights, Adam state and the data-stream position mid-training;
    a fresh model loaded from the file continues with exactly the same losses
    and ends with exactly the same weights."""
    from paper_2602_11092_gb300.surrogate import Surrogate
    n_ph, K, Bn = 8, 64, 64

    def batch(i):
        rng = np.random.default_rng(5000 + i)
        ph = torch.tensor(rng.uniform(0, 2 * np.pi, (Bn, n_ph)), dtype=torch.float32, device="cuda")
        z = rng.standard_normal((Bn, K))
        t = np.exp(z) / np.exp(z).sum(axis=1, keepdims=True)
        return ph, torch.tensor(t, dtype=torch.float32, device="cuda")

    def run(model, start, stop):
        out = []
        for i in range(start, stop):
            ph, tg = batch(i)
            loss = torch.empty(Bn, dtype=torch.float32, device="cuda")
            model.train_step(ph, tg, 2e-3, loss_rows=loss)
            out.append(loss.clone())
        torch.cuda.synchronize()
        return out

    a = Surrogate(n_phases=n_ph, hidden=64, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=5)
    run(a, 0, 6)
    path = tmp_path / "surrogate.ckpt"
    a.save(path, stream_index=6)
    ref = run(a, 6, 10)
    b = Surrogate(n_phases=n_ph, hidden=64, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=99)
    start = b.load(path)
    assert start == 6
    got = run(b, start, 10)
    for x, y in zip(ref, got):
        assert torch.equal(x, y)
    for layer in range(3):
        wa, ba = a.get_param(layer)
        wb, bb = b.get_param(layer)
        assert np.array_equal(wa, wb) and np.array_equal(ba, bb)
    # a model of other dimensions refuses the file
    c = Surrogate(n_phases=n_ph, hidden=128, n_hidden_layers=2, n_outputs=K, max_batch=Bn, seed=1)
    with pytest.raises(Exception):
        c.load(path)
