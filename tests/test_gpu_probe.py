"""The read-bandwidth probe (ssgi_read_bandwidth_probe) runs and leaves its buffer untouched."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_read_bandwidth_probe_runs_and_only_reads():
    import paper_2504_01358_gb300 as S
    buf = torch.arange(1 << 18, device="cuda", dtype=torch.float32)  # 1 MiB
    ref = buf.clone()
    sink = torch.zeros(1, device="cuda", dtype=torch.int32)
    S.ssgi_read_bandwidth_probe(buf, 3, sink)
    S.ssgi_read_bandwidth_probe(buf[:4], 1, sink)  # 16 bytes: one thread's tail loop
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)
    assert int(sink.item()) in (0, 1, 2)
    with pytest.raises(Exception):
        S.ssgi_read_bandwidth_probe(buf[1:4], 1, sink)  # 12 bytes, not 16-byte aligned
