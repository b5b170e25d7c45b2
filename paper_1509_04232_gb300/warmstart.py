"""Learned warm start: a small convolutional network predicts each pixel's
cell among the 9 of its 3x3 cell window; its labels give initial centres
(member means), after which a few SLIC iterations replace the usual five
to ten. The network, its training (forward, backward, Adam), its inference
and the warm-started segmentation (``slic_batch_set_warmstart``) are the
library's own CUDA kernels behind include/slic.h; this module only drives
them (data, the learning-rate schedule, the order of the calls).

Training targets are the slots of full-iteration SLIC labels (S=16, m=10,
10 iterations, before connectivity) computed by this library's batched GPU
path on seeded synthetic 256x256 images (``slic_net_slots``).
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
from . import synth


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


def target_slots(net: "WarmStartNet", labels_i32):
    """Slots (dy+1)*3 + (dx+1) of labels int32 CUDA [n, H, W] relative to
    each pixel's own cell (the library's slic_net_slots), as uint8 CUDA
    [n, H, W]; raises if a label lies outside its pixel's 3x3 cell window."""
    import torch
    n = labels_i32.shape[0]
    slots = torch.empty(labels_i32.shape, dtype=torch.uint8, device=labels_i32.device)
    bad = torch.zeros(1, dtype=torch.int32, device=labels_i32.device)
    s = int(torch.cuda.current_stream().cuda_stream)
    B.slic_net_slots(net.handle, n, labels_i32.data_ptr(), slots.data_ptr(), bad.data_ptr(), s)
    if int(bad.item()) != 0:
        raise ValueError(f"{int(bad.item())} labels outside the 3x3 cell window")
    return slots


def training_batch(net: "WarmStartNet", first: int, count: int, device, m: float = 10.0, iterations: int = 10):
    """Seeded 256x256 training images first..first+count-1 and their target
    slots (the network's geometry: width, height and S)."""
    import torch
    host = np.stack([synth.train_image(i) for i in range(first, first + count)])
    imgs = torch.from_numpy(host).to(device)
    labels = reference_labels(imgs, net.S, m, iterations)
    return imgs, target_slots(net, labels.contiguous())


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
            imgs, slots = training_batch(net, c0, cn, dev, net.m)
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
    """Segment frames [n, H, W, 3] from the network's labels (the library's
    warm start: member means of the predicted labels replace the grid
    centres), then an assignment, `iterations` x {update, assignment} and
    connectivity. Returns (labels list, centres list)."""
    from . import BatchSegmenter
    n, H, W, _ = images_u8.shape
    bs = BatchSegmenter([dict(width=W, height=H, S=net.S, m=m)] * n, iterations=iterations,
                        enforce_connectivity=enforce_connectivity, device=images_u8.device)
    bs.bind([images_u8[i] for i in range(n)])
    bs.set_warmstart(net)
    labels, centres = bs.segment()
    out = [l.clone() for l in labels], [c.clone() for c in centres]
    bs.status()
    bs.close()
    return out


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
    """The learned path for a fixed set of frames: one warm-started batch
    (network labels -> member-mean centres -> assignment, `iterations` x
    {update, assignment} -> connectivity, all enqueued by one library call),
    so `run` can be captured into a CUDA graph."""

    def __init__(self, net: WarmStartNet, images, iterations: int, m: float = 10.0,
                 enforce_connectivity: bool = True):
        from . import BatchSegmenter
        self.net = net
        self.images = list(images)
        H, W, _ = self.images[0].shape
        self.bs = BatchSegmenter([dict(width=W, height=H, S=net.S, m=m)] * len(self.images), iterations=iterations,
                                 enforce_connectivity=enforce_connectivity, device=self.images[0].device)
        self.bs.bind(self.images)
        self.bs.set_warmstart(net)

    def run(self, stream=None):
        return self.bs.segment(stream)

    def close(self):
        self.bs.close()
