"""The permutation-invariant quality measures of the video report, on small
hand-built label maps (CPU tensors)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1509_04232_gb300.video import boundary_recall, centre_drift, segmentation_accuracy  # noqa: E402


def _blocks(H, W, bw):
    y, x = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    return ((y // bw) * (W // bw) + x // bw).to(torch.int32)


def test_segmentation_accuracy_ignores_numbering():
    ref = _blocks(12, 12, 4)
    assert segmentation_accuracy(ref, ref) == 1.0
    assert segmentation_accuracy(8 - ref, ref) == 1.0   # renumbered
    # one segment covering two reference blocks gets only the larger one right
    merged = ref.clone()
    merged[merged == 1] = 0
    assert segmentation_accuracy(merged, ref) == pytest.approx(1.0 - 16 / 144)
    # finer segments than the reference lose nothing
    assert segmentation_accuracy(_blocks(12, 12, 2), ref) == 1.0


def test_boundary_recall_tolerance():
    ref = torch.zeros((8, 20), dtype=torch.int32)
    ref[:, 10:] = 1                       # boundary between columns 9 and 10
    assert boundary_recall(ref, ref) == 1.0
    shifted = torch.zeros_like(ref)
    shifted[:, 12:] = 1                   # two pixels to the right
    assert boundary_recall(shifted, ref, tol=2) == 1.0
    assert boundary_recall(shifted, ref, tol=1) == pytest.approx(0.5)   # column 10 is within 1, column 9 is not
    assert boundary_recall(torch.zeros_like(ref), ref) == 0.0


def test_centre_drift_in_cells():
    W, H, S = 32, 16, 8                    # 4 x 2 cells, midpoints at 3.5, 11.5, ...
    K = 8
    c = torch.zeros((K, 6))
    c[:, 5] = 1.0
    for k in range(K):
        c[k, 3] = (k % 4) * 8 + 3.5
        c[k, 4] = (k // 4) * 8 + 3.5
    assert centre_drift(c, W, H, S) == 0.0
    c[5, 3] += 12.0                        # 1.5 cells to the right
    assert centre_drift(c, W, H, S) == pytest.approx(1.5)
    c[5, 5] = 0.0                          # an empty cluster does not count
    assert centre_drift(c, W, H, S) == 0.0
