"""FP64 CPU oracle of the learned warm start's network (TEST INFRASTRUCTURE
ONLY: used by the tests and nowhere in the product path).

The network maps per-pixel input channels to 9 logits, one per cell of the
pixel's 3x3 cell window (slot t = (dy+1)*3 + (dx+1), scan order as in the
assignment of Eq. 1). Four 3x3 convolutions with zero padding and ReLU
between them: C0 -> 32 -> 32 -> 32 -> 9.

Input channels (C0 = 14, zero-padded to 16 on the device): L/100, a/128,
b/128, (x mod S)/S, (y mod S)/S, and D_t/100 for t = 0..8, the Eq. (1)
distance to the grid-initialised centre of slot t (2.0 for an off-grid
slot) -- the information of the first assignment.

Precision model of the device path, mirrored here when ``bf16=True``:
weights and the activations stored between layers are rounded to bfloat16
(round to nearest even); every sum is exact (FP64 here, FP32 accumulation
on the device). The loss is the mean softmax cross-entropy over pixels, with
off-grid slots excluded from the softmax. Gradients (``backward``) are the
plain FP64 chain rule of that loss, pinned by central finite differences in
the tests. With ``bf16_grad=True`` the loss gradient of every layer's
pre-activation (dL/dz: the softmax gradient, and each propagated gradient
after the ReLU mask) is rounded to bfloat16 where the device stores it
between its backward kernels; the weight and bias gradients are exact sums
of those stored values.
"""
from __future__ import annotations

import numpy as np

C0, C_HID, N_SLOTS = 14, 32, 9
LAYERS = [(C0, C_HID), (C_HID, C_HID), (C_HID, C_HID), (C_HID, N_SLOTS)]


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0):
    """He-normal weights [3,3,Cin,Cout] and zero biases, FP32 master values."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in LAYERS:
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), (3, 3, cin, cout)).astype(np.float32)
        params.append((w, np.zeros(cout, np.float32)))
    return params


def grid_distances(lab: np.ndarray, S: int, m: float) -> np.ndarray:
    """D[H,W,9]: Eq. (1) distance of each pixel to the grid-initialised centre
    (Sec. 3 initialisation) of each slot of its 3x3 cell window; inf off-grid."""
    H, W, _ = lab.shape
    ns_c, ns_r = -(-W // S), -(-H // S)
    ys, xs = np.mgrid[0:H, 0:W]
    D = np.full((H, W, 9), np.inf)
    for t in range(9):
        cx = xs // S + t % 3 - 1
        cy = ys // S + t // 3 - 1
        ok = (cx >= 0) & (cx < ns_c) & (cy >= 0) & (cy < ns_r)
        cxc, cyc = np.clip(cx, 0, ns_c - 1), np.clip(cy, 0, ns_r - 1)
        xk = (cxc * S + np.minimum((cxc + 1) * S, W) - 1) / 2.0
        yk = (cyc * S + np.minimum((cyc + 1) * S, H) - 1) / 2.0
        ck = lab[np.floor(yk).astype(int), np.floor(xk).astype(int)]
        d = np.sqrt(((lab - ck) ** 2).sum(-1)) + (m / S) * np.sqrt((xs - xk) ** 2 + (ys - yk) ** 2)
        D[..., t] = np.where(ok, d, np.inf)
    return D


def input_channels(lab: np.ndarray, S: int, m: float = 10.0) -> np.ndarray:
    """lab [H,W,3] -> network input [H,W,14]."""
    H, W, _ = lab.shape
    ys, xs = np.mgrid[0:H, 0:W]
    D = grid_distances(lab, S, m)
    Dn = np.where(np.isfinite(D), D / 100.0, 2.0)
    base = np.stack([lab[..., 0] / 100.0, lab[..., 1] / 128.0, lab[..., 2] / 128.0,
                     (xs % S) / S, (ys % S) / S], axis=-1)
    return np.concatenate([base, Dn], axis=-1).astype(np.float64)


def slot_mask(H: int, W: int, S: int) -> np.ndarray:
    """valid[H,W,9]: slot t's cell lies in the grid."""
    ns_c, ns_r = -(-W // S), -(-H // S)
    ys, xs = np.mgrid[0:H, 0:W]
    cx, cy = xs // S, ys // S
    valid = np.zeros((H, W, 9), bool)
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        valid[..., t] = (cx + dx >= 0) & (cx + dx < ns_c) & (cy + dy >= 0) & (cy + dy < ns_r)
    return valid


def slots_from_labels(labels: np.ndarray, S: int) -> np.ndarray:
    """Slot index of each pixel's label relative to its own cell (labels must
    lie in the 3x3 cell window, as assignment labels do)."""
    H, W = labels.shape
    ns_c = -(-W // S)
    ys, xs = np.mgrid[0:H, 0:W]
    dx = labels % ns_c - xs // S
    dy = labels // ns_c - ys // S
    assert np.all(np.abs(dx) <= 1) and np.all(np.abs(dy) <= 1)
    return ((dy + 1) * 3 + (dx + 1)).astype(np.int64)


def labels_from_slots(slots: np.ndarray, S: int) -> np.ndarray:
    H, W = slots.shape
    ns_c = -(-W // S)
    ys, xs = np.mgrid[0:H, 0:W]
    return ((ys // S + slots // 3 - 1) * ns_c + xs // S + slots % 3 - 1).astype(np.int32)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[y,x,o] = b[o] + sum_{dy,dx,i} x[y+dy-1, x+dx-1, i] w[dy,dx,i,o], zero padding."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b.astype(np.float64), (H, W, w.shape[3])).copy()
    for dy in range(3):
        for dx in range(3):
            out += xp[dy:dy + H, dx:dx + W, :] @ w[dy, dx].astype(np.float64)
    return out


def forward(x0: np.ndarray, params, bf16: bool = True):
    """Logits [H,W,9] and the per-layer cache (inputs, pre-activations)."""
    cache = []
    a = bf16_round(x0) if bf16 else np.asarray(x0, np.float64)
    for li, (w, b) in enumerate(params):
        wq = bf16_round(w) if bf16 else np.asarray(w, np.float64)
        z = conv3x3(a, wq, np.asarray(b, np.float64))
        cache.append((a, wq, z))
        if li < len(params) - 1:
            a = np.maximum(z, 0.0)
            if bf16:
                a = bf16_round(a)
        else:
            a = z
    return a, cache


def masked_log_softmax(logits: np.ndarray, valid: np.ndarray) -> np.ndarray:
    z = np.where(valid, logits, -np.inf)
    m = np.max(z, axis=-1, keepdims=True)
    e = np.where(valid, np.exp(z - m), 0.0)
    return z - m - np.log(np.sum(e, axis=-1, keepdims=True))


def loss(logits: np.ndarray, target: np.ndarray, valid: np.ndarray) -> float:
    """Mean softmax cross-entropy over pixels (off-grid slots excluded)."""
    lp = masked_log_softmax(logits, valid)
    return float(-np.mean(np.take_along_axis(lp, target[..., None], axis=-1)))


def backward(x0: np.ndarray, params, target: np.ndarray, valid: np.ndarray, bf16: bool = True,
             bf16_grad: bool = False, return_dz: bool = False):
    """Loss and its gradients [(dW, db), ...] by the chain rule in FP64
    (dL/dz rounded to bfloat16 at each layer when ``bf16_grad``); with
    ``return_dz`` also each layer's dL/dz [H,W,Cout] and its input [H,W,Cin]."""
    stored = bf16_round if bf16_grad else (lambda v: v)
    logits, cache = forward(x0, params, bf16)
    H, W, _ = logits.shape
    lp = masked_log_softmax(logits, valid)
    p = np.where(valid, np.exp(lp), 0.0)
    onehot = np.zeros_like(p)
    np.put_along_axis(onehot, target[..., None], 1.0, axis=-1)
    dz = stored((p - onehot) / (H * W))
    grads = [None] * len(params)
    dzs = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        a_in, wq, z = cache[li]
        dzs[li] = (dz, a_in)
        # dW[dy,dx,i,o] = sum_{y,x} a_in[y+dy-1, x+dx-1, i] dz[y,x,o]
        ap = np.pad(a_in, ((1, 1), (1, 1), (0, 0)))
        dw = np.zeros(wq.shape)
        for dy in range(3):
            for dx in range(3):
                dw[dy, dx] = np.einsum("yxi,yxo->io", ap[dy:dy + H, dx:dx + W, :], dz)
        grads[li] = (dw, dz.sum(axis=(0, 1)))
        if li > 0:
            # da_in[y,x,i] = sum_{dy,dx,o} dz[y-dy+1, x-dx+1, o] w[dy,dx,i,o]
            dzp = np.pad(dz, ((1, 1), (1, 1), (0, 0)))
            da = np.zeros(a_in.shape)
            for dy in range(3):
                for dx in range(3):
                    da += dzp[2 - dy:2 - dy + H, 2 - dx:2 - dx + W, :] @ wq[dy, dx].T
            z_prev = cache[li - 1][2]
            dz = stored(da * (z_prev > 0))
    if return_dz:
        return loss(logits, target, valid), grads, dzs
    return loss(logits, target, valid), grads
