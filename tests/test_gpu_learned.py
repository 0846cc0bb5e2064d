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
