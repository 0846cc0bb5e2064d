"""FP64 NumPy oracle of the learned proposal's encoder and its InfoNCE loss
(test infrastructure only; the learned proposal is not part of the paper).

Network on inputs [N, C, tj, tj]: conv 3x3 C->32 pad 1 + ReLU, conv 3x3
32->32 stride 2 pad 1 + ReLU, conv 3x3 32->32 stride 2 pad 1 + ReLU, linear
(32 h3 h3) -> 64, L2 normalisation. Loss over B anchors and M candidates
(candidate i is the positive of anchor i): mean_i of
-log softmax_j(a_i . c_j / tau)[i]. Gradients by explicit backpropagation.
The flat parameter layout matches the CUDA library's: w1, b1, w2, b2, w3, b3,
wf, bf.
"""
from __future__ import annotations

import numpy as np


def shapes(C: int, tj: int):
    h2 = (tj - 1) // 2 + 1
    h3 = (h2 - 1) // 2 + 1
    flat = 32 * h3 * h3
    return [("w1", (32, C, 3, 3)), ("b1", (32,)), ("w2", (32, 32, 3, 3)), ("b2", (32,)),
            ("w3", (32, 32, 3, 3)), ("b3", (32,)), ("wf", (64, flat)), ("bf", (64,))]


def unpack(flat: np.ndarray, C: int, tj: int) -> dict:
    out, o = {}, 0
    for name, shp in shapes(C, tj):
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp).astype(np.float64)
        o += n
    assert o == flat.size
    return out


def pack(d: dict, C: int, tj: int) -> np.ndarray:
    return np.concatenate([d[name].reshape(-1) for name, _ in shapes(C, tj)])


def _conv(x, w, b, stride):
    N, Ci, H, W = x.shape
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((N, w.shape[0], Ho, Wo)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            y += np.einsum("nchw,oc->nohw", patch, w[:, :, ky, kx])
    return y


def _conv_back(dy, x, w, stride):
    """Gradients of y = conv(x) wrt x, w and b."""
    N, Ci, H, W = x.shape
    Ho, Wo = dy.shape[2], dy.shape[3]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky, ky + stride * (Ho - 1) + 1, stride),
                  slice(kx, kx + stride * (Wo - 1) + 1, stride))
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, xp[sl])
            dxp[sl] += np.einsum("nohw,oc->nchw", dy, w[:, :, ky, kx])
    return dxp[:, :, 1:-1, 1:-1], dw, dy.sum(axis=(0, 2, 3))


def forward(p: dict, x: np.ndarray):
    a1 = np.maximum(_conv(x, p["w1"], p["b1"], 1), 0)
    a2 = np.maximum(_conv(a1, p["w2"], p["b2"], 2), 0)
    a3 = np.maximum(_conv(a2, p["w3"], p["b3"], 2), 0)
    z = a3.reshape(len(x), -1) @ p["wf"].T + p["bf"]
    nrm = np.sqrt((z * z).sum(axis=1, keepdims=True))
    return z / nrm, (x, a1, a2, a3, z, nrm)


def loss_and_grads(p: dict, anchors: np.ndarray, cands: np.ndarray, tau: float):
    B = len(anchors)
    x = np.concatenate([anchors, cands]).astype(np.float64)
    e, (x, a1, a2, a3, z, nrm) = forward(p, x)
    A, Cm = e[:B], e[B:]
    logits = A @ Cm.T / tau
    mx = logits.max(axis=1, keepdims=True)
    pr = np.exp(logits - mx)
    pr /= pr.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(pr[np.arange(B), np.arange(B)])))
    g = pr.copy()
    g[np.arange(B), np.arange(B)] -= 1.0
    g /= B
    de = np.concatenate([g @ Cm / tau, g.T @ A / tau])
    dz = (de - e * (e * de).sum(axis=1, keepdims=True)) / nrm
    grads = {"wf": dz.T @ a3.reshape(len(x), -1), "bf": dz.sum(axis=0)}
    d3 = (dz @ p["wf"]).reshape(a3.shape) * (a3 > 0)
    d2, grads["w3"], grads["b3"] = _conv_back(d3, a2, p["w3"], 2)
    d2 = d2 * (a2 > 0)
    d1, grads["w2"], grads["b2"] = _conv_back(d2, a1, p["w2"], 2)
    d1 = d1 * (a1 > 0)
    _, grads["w1"], grads["b1"] = _conv_back(d1, x, p["w1"], 1)
    return loss, grads
