"""GPU tests of the learned proposal: the encoder's forward and backward
kernels against the FP64 oracle, and training progress."""
import numpy as np
import pytest

from oracle import encoder_oracle as E

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccw():
    import paper_2404_00441_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("C,tj,B,M", [(2, 6, 4, 7), (3, 12, 8, 20)])
def test_encoder_gradients_match_fp64_oracle(ccw, C, tj, B, M):
    net = ccw.Net(C, tj, seed=5)
    flat = net.get(0)
    params = E.unpack(flat, C, tj)
    rng = np.random.default_rng(C + tj)
    anchors = rng.random((B, C, tj, tj)).astype(np.float32)
    cands = rng.random((M, C, tj, tj)).astype(np.float32)
    loss = net.train_step(torch.from_numpy(anchors).cuda(), torch.from_numpy(cands).cuda(),
                          tau=0.2, bf16=0, apply=0)
    torch.cuda.synchronize()
    ref_loss, ref = E.loss_and_grads(params, anchors, cands, tau=0.2)
    assert abs(float(loss.item()) - ref_loss) <= 1e-4 * max(1.0, abs(ref_loss))
    got = E.unpack(net.get(1), C, tj)
    for name, _ in E.shapes(C, tj):
        a, b = got[name], ref[name]
        scale = max(np.abs(b).max(), 1e-6)
        assert np.abs(a - b).max() <= 2e-3 * scale, name
    # embeddings
    x = torch.from_numpy(anchors).cuda()
    emb = net.embed(x, bf16=0).cpu().numpy()
    ref_e, _ = E.forward(params, anchors.astype(np.float64))
    assert np.abs(emb - ref_e).max() < 1e-4


def test_training_reduces_the_loss(ccw):
    """Two views of the same random pattern (one masked) become neighbours."""
    net = ccw.Net(2, 12, seed=1)
    rng = np.random.default_rng(0)
    base = rng.random((512, 2, 12, 12)).astype(np.float32)
    masked = base.copy()
    masked[:, :, 3:, 3:] = 0.0
    a = torch.from_numpy(masked).cuda()
    c = torch.from_numpy(base).cuda()
    losses = []
    for it in range(60):
        i0 = (it * 64) % 512
        l = net.train_step(a[i0:i0 + 64], c[i0:i0 + 64], tau=0.1, lr=2e-3, bf16=1)
        losses.append(float(l.item()))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5])


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).bfloat16().float().numpy()


@pytest.mark.parametrize("C,tj,N", [(2, 12, 7 * 9 + 3), (3, 16, 3 * 5 + 2), (2, 9, 8 * 3 + 1),
                                    (1, 7, 1), (2, 20, 6)])
def test_inference_pass_matches_the_encoder(ccw, C, tj, N):
    """The proposal's inference pass (the tcgen05 implicit-GEMM kernel where
    the shape fits, several sample groups and a ragged last group) embeds like
    the FP64 encoder oracle with BF16 weights and non-zero biases, and like
    the fused FP32-lane kernel up to the BF16 rounding of the activations."""
    net = ccw.Net(C, tj, seed=11)
    rng = np.random.default_rng(C * 100 + tj)
    d = E.unpack(net.get(0), C, tj)
    for name in ("b1", "b2", "b3", "bf"):
        d[name] = rng.normal(0.0, 0.05, d[name].shape)
    flat = E.pack(d, C, tj).astype(np.float32)
    net.set(flat)
    ref_p = {k: (_bf16(v).astype(np.float64) if k[0] == "w" else v.astype(np.float32)
                 .astype(np.float64)) for k, v in E.unpack(flat, C, tj).items()}
    # inputs as the proposal makes them: block counts / 2^(d J), exact in BF16
    x = (rng.integers(0, 17, (N, C, tj, tj)) / 16.0).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    tc = net.embed(xt, bf16=2).cpu().numpy().astype(np.float64)
    simt = net.embed(xt, bf16=3).cpu().numpy().astype(np.float64)
    ref, _ = E.forward(ref_p, x.astype(np.float64))
    for got in (tc, simt):
        assert np.all(np.abs(np.linalg.norm(got, axis=1) - 1.0) < 1e-5)
        assert np.all((got * ref).sum(1) >= 0.998)
        assert np.abs(got - ref).max() <= 0.03
    assert np.abs(tc - simt).max() <= 0.02
