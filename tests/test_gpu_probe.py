"""The measurement probes the rooflines come from: every width (8, 32, 64
bytes) and every reads-in-flight count runs at the launch shapes the
bench's sweep uses, a block the kernel cannot run with is refused with
CK_EINVAL (not a failed launch), and bad arguments are refused; the
random atomics run for each kind."""
import pytest
import torch

from paper_1605_05236_gb300 import ck

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [8, 32, 64])
def test_gather_probe_shapes(width):
    buf = torch.ones((1 << 22) // 8, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda")
    ran = 0
    for per_thread in (1, 2, 4, 8):
        for block in (128, 256, 512):
            try:
                ck.gather_probe_ex(buf, width, 1 << 16, 7, per_thread, block, 152 * 8, sink)
                ran += 1
            except RuntimeError as e:
                # only the 64-byte kernel with 8 reads in flight is too large for 512 threads
                assert (width, per_thread, block) == (64, 8, 512) and "(-1)" in str(e), e
    torch.cuda.synchronize()
    assert ran == (11 if width == 64 else 12)
    ck.gather_probe(buf, width, 1 << 16, 3, sink)
    torch.cuda.synchronize()


def test_gather_probe_refuses_bad_arguments():
    buf = torch.ones(1 << 10, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda")
    for width, per_thread, block in ((16, 1, 128), (32, 3, 128), (32, 1, 100), (32, 1, 2048)):
        with pytest.raises(RuntimeError):
            ck.gather_probe_ex(buf, width, 1 << 10, 1, per_thread, block, 0, sink)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_atomic_probe_runs(kind):
    buf = torch.zeros((1 << 22) // 8, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1024, dtype=torch.int64, device="cuda")
    ck.atomic_probe(buf, kind, 1 << 16, 5, sink)
    torch.cuda.synchronize()
