"""Learned warm start: a small convolutional network predicts each pixel's
cell among the 9 of its 3x3 cell window; its labels give initial centres
(member means), after which one or two SLIC iterations replace the usual
five to ten. The network, its training (forward, backward, Adam) and its
inference are the library's own CUDA kernels (``slic_net_*`` in
include/slic.h); this module only drives them.

Training targets are the slots of full-iteration SLIC labels (S=16, m=10,
10 iterations, before connectivity) computed by this library's batched GPU
path on seeded synthetic 256x256 images.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
from . import synth


def slots_from_labels(labels: np.ndarray, S: int) -> np.ndarray:
    """Slot (dy+1)*3 + (dx+1) of each pixel's label relative to its own cell
    (labels [..., H, W] must lie in the 3x3 cell window, as assignment labels do)."""
    H, W = labels.shape[-2:]
    ns_c = -(-W // S)
    ys, xs = np.mgrid[0:H, 0:W]
    dx = labels % ns_c - xs // S
    dy = labels // ns_c - ys // S
    if np.any(np.abs(dx) > 1) or np.any(np.abs(dy) > 1):
        raise ValueError("labels outside the 3x3 cell window")
    return ((dy + 1) * 3 + (dx + 1)).astype(np.uint8)


class WarmStartNet:
    """The network on one geometry (width x height, grid interval S)."""

    def __init__(self, width: int, height: int, S: int = 16, max_batch: int = 64, seed: int = 0, m: float = 10.0):
        self.W, self.H, self.S, self.m, self.max_batch = width, height, S, m, max_batch
        self.handle = B.slic_net_create(max_batch, width, height, S, m, seed)

    def close(self):
        if getattr(self, "handle", None):
            B.slic_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters / checkpoints
    def params(self) -> np.ndarray:
        return B.slic_net_get_params(self.handle, 0)

    def grads(self) -> np.ndarray:
        return B.slic_net_get_params(self.handle, 1)

    def set_params(self, p: np.ndarray):
        B.slic_net_set_params(self.handle, p)

    def save(self, path: str):
        np.savez(path, params=self.params(), W=self.W, H=self.H, S=self.S)

    def load(self, path: str):
        z = np.load(path)
        self.set_params(z["params"])

    # compute
    def forward(self, images, logits=None, labels=None, stream: int = 0):
        """images: uint8 CUDA tensor [n, H, W, 3]; logits float32 [n, H, W, 16]
        and/or labels int32 [n, H, W] CUDA tensors to fill."""
        n = images.shape[0]
        B.slic_net_forward(self.handle, n, images.data_ptr(), logits.data_ptr() if logits is not None else None,
                           labels.data_ptr() if labels is not None else None, stream)

    def gradients(self, images, targets, stats=None, stream: int = 0):
        B.slic_net_gradients(self.handle, images.shape[0], images.data_ptr(), targets.data_ptr(),
                             stats.data_ptr() if stats is not None else None, stream)

    def status(self):
        """Raises SlicError(SLIC_ERR_TIMEOUT) if a bounded wait of the tensor-core kernels gave up."""
        B.slic_net_status(self.handle)

    def train_step(self, images, targets, lr: float, stats=None, stream: int = 0):
        B.slic_net_train_step(self.handle, images.shape[0], images.data_ptr(), targets.data_ptr(), lr,
                              stats.data_ptr() if stats is not None else None, stream)


def reference_labels(images_u8, S: int = 16, m: float = 10.0, iterations: int = 10):
    """Full-iteration SLIC labels before connectivity, by the batched GPU path.
    images_u8: uint8 CUDA tensor [n, H, W, 3] -> int32 CUDA tensor [n, H, W]."""
    import torch
    from . import BatchSegmenter
    n, H, W, _ = images_u8.shape
    bs = BatchSegmenter([dict(width=W, height=H, S=S, m=m)] * n, iterations=iterations,
                        enforce_connectivity=False, device=images_u8.device)
    bs.bind([images_u8[i] for i in range(n)])
    labels, _ = bs.segment()
    out = torch.stack(labels)
    bs.status()
    bs.close()
    return out


def training_batch(first: int, count: int, device, S: int = 16, m: float = 10.0, iterations: int = 10):
    """Seeded 256x256 training images first..first+count-1 and their target slots."""
    import torch
    host = np.stack([synth.train_image(i) for i in range(first, first + count)])
    imgs = torch.from_numpy(host).to(device)
    labels = reference_labels(imgs, S, m, iterations).cpu().numpy()
    slots = slots_from_labels(labels, S)
    return imgs, torch.from_numpy(slots).to(device)


def train(net: WarmStartNet, n_images: int, batch: int = 32, epochs: int = 1, lr: float = 2e-3,
          first_image: int = 0, log_every: int = 0, chunk: int = 1024):
    """Train on images first_image..first_image+n_images-1 (targets computed
    chunk by chunk on the GPU). Returns the per-step (loss, accuracy) history."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stats = torch.zeros(2, dtype=torch.float32, device=dev)
    hist = []
    px = net.W * net.H
    step = 0
    for _ in range(epochs):
        for c0 in range(first_image, first_image + n_images, chunk):
            cn = min(chunk, first_image + n_images - c0)
            imgs, slots = training_batch(c0, cn, dev, net.S)
            order = torch.randperm(cn, device=dev)
            for b0 in range(0, cn - batch + 1, batch):
                idx = order[b0:b0 + batch]
                x = imgs[idx].contiguous()
                t = slots[idx].contiguous()
                # cosine decay over the whole run
                total = max(1, epochs * (n_images // batch))
                lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * min(step, total) / total))
                net.train_step(x, t, lr_t, stats)
                if log_every and step % log_every == 0:
                    s = stats.cpu().numpy()
                    hist.append((step, float(s[0]) / (batch * px), float(s[1]) / (batch * px)))
                step += 1
    torch.cuda.synchronize()
    return hist


def warm_start_segment(net: WarmStartNet, images_u8, iterations: int, m: float = 10.0,
                       enforce_connectivity: bool = True):
    """Segment frames [n, H, W, 3] starting from the network's labels: centres
    are the member means of the predicted labels (slic_update), then
    `iterations` assignments (iterations - 1 updates between them) and
    connectivity. Returns (labels list, centres list)."""
    import torch
    from . import BatchSegmenter, Segmenter
    n, H, W, _ = images_u8.shape
    dev = images_u8.device
    net_labels = torch.empty((n, H, W), dtype=torch.int32, device=dev)
    net.forward(images_u8, labels=net_labels)
    seg = Segmenter(W, H, S=net.S, m=m, iterations=0)
    init = []
    for i in range(n):
        feat = seg.convert(images_u8[i])
        c0 = seg.init_centres(feat)
        init.append(seg.update(feat, net_labels[i], c0))
    bs = BatchSegmenter([dict(width=W, height=H, S=net.S, m=m)] * n, iterations=iterations - 1,
                        enforce_connectivity=enforce_connectivity, device=dev)
    bs.bind([images_u8[i] for i in range(n)], init_centres=init)
    labels, centres = bs.segment()
    return [l.clone() for l in labels], [c.clone() for c in centres]


def agreement(a, b) -> float:
    """Fraction of equal labels between two lists of int32 CUDA tensors."""
    import torch
    eq = sum(int((x == y).sum().item()) for x, y in zip(a, b))
    return eq / sum(x.numel() for x in a)


def plain_segment(images_u8, iterations: int, S: int = 16, m: float = 10.0, enforce_connectivity: bool = True):
    """Plain batched SLIC (grid initialisation) on frames [n, H, W, 3]."""
    from . import BatchSegmenter
    n, H, W, _ = images_u8.shape
    bs = BatchSegmenter([dict(width=W, height=H, S=S, m=m)] * n, iterations=iterations,
                        enforce_connectivity=enforce_connectivity, device=images_u8.device)
    bs.bind([images_u8[i] for i in range(n)])
    labels, centres = bs.segment()
    return [l.clone() for l in labels], [c.clone() for c in centres]


class WarmStartPipeline:
    """The learned path for a fixed set of frames, with every buffer
    allocated up front so that `run` only enqueues kernels (and can be
    captured into a CUDA graph): network labels -> member-mean centres per
    frame -> `iterations` assignments of the batched path -> connectivity."""

    def __init__(self, net: WarmStartNet, images, iterations: int, m: float = 10.0,
                 enforce_connectivity: bool = True):
        import torch
        from . import BatchSegmenter, Segmenter
        self.net = net
        self.images = list(images)
        n = len(self.images)
        H, W, _ = self.images[0].shape
        dev = self.images[0].device
        self.stacked = torch.stack(self.images)
        self.net_labels = torch.empty((n, H, W), dtype=torch.int32, device=dev)
        self.seg = Segmenter(W, H, S=net.S, m=m, iterations=0)
        self.feat = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        self.c0 = torch.empty((self.seg.K_eff, 6), dtype=torch.float32, device=dev)
        self.init = [torch.empty((self.seg.K_eff, 6), dtype=torch.float32, device=dev) for _ in range(n)]
        self.bs = BatchSegmenter([dict(width=W, height=H, S=net.S, m=m)] * n, iterations=iterations - 1,
                                 enforce_connectivity=enforce_connectivity, device=dev)
        self.bs.bind(self.images, init_centres=self.init)

    def run(self, stream=None):
        import torch
        s = int((stream if stream is not None else torch.cuda.current_stream()).cuda_stream)
        B.slic_net_forward(self.net.handle, len(self.images), self.stacked.data_ptr(), None,
                           self.net_labels.data_ptr(), s)
        h = self.seg.handle
        for i, img in enumerate(self.images):
            B.slic_convert(h, img.data_ptr(), self.feat.data_ptr(), s)
            B.slic_init_centres(h, self.feat.data_ptr(), self.c0.data_ptr(), s)
            B.slic_update(h, self.feat.data_ptr(), self.net_labels[i].data_ptr(), self.c0.data_ptr(),
                          self.init[i].data_ptr(), s)
        B.slic_batch_segment(self.bs.handle, s)
        return self.bs.labels, self.bs.centres
