"""Pin of the FP64 encoder oracle: its analytic gradients equal central
finite differences of its own loss (a check of the backpropagation against
the definition of the derivative, independent of the code that computes it)."""
import numpy as np

from oracle import encoder_oracle as E


def test_encoder_gradients_equal_finite_differences():
    rng = np.random.default_rng(0)
    C, tj, B, M = 2, 6, 3, 5
    params = {name: rng.normal(0, 0.4, shp) for name, shp in E.shapes(C, tj)}
    anchors = rng.random((B, C, tj, tj))
    cands = rng.random((M, C, tj, tj))
    loss, grads = E.loss_and_grads(params, anchors, cands, tau=0.5)
    assert np.isfinite(loss)
    h = 1e-6
    for name, _ in E.shapes(C, tj):
        flat = params[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = E.loss_and_grads(params, anchors, cands, tau=0.5)
            flat[i] = old - h
            lm, _ = E.loss_and_grads(params, anchors, cands, tau=0.5)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (name, i, fd, an)


def test_embeddings_are_unit_vectors():
    rng = np.random.default_rng(1)
    params = {name: rng.normal(0, 0.3, shp) for name, shp in E.shapes(3, 12)}
    e, _ = E.forward(params, rng.random((4, 3, 12, 12)))
    assert e.shape == (4, 64)
    assert np.allclose(np.linalg.norm(e, axis=1), 1.0)
