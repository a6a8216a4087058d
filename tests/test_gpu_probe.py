"""The random-read probe behind bench.py's sector-roofline context: it runs
through the C ABI, leaves the buffer unchanged, and reports a positive time
that grows with the number of reads."""
import pytest

pytestmark = pytest.mark.gpu


def test_random_read_probe_runs():
    import torch
    from paper_2404_16370_gb300 import mp
    words = torch.arange(1 << 20, dtype=torch.int32, device="cuda")
    ref = words.clone()
    ms_small = mp.mp_probe_random_reads(words, 64, 16, repeats=3)
    ms_large = mp.mp_probe_random_reads(words, 64, 1024, repeats=3)
    torch.cuda.synchronize()
    assert ms_small > 0 and ms_large > ms_small
    assert torch.equal(words, ref)


def test_random_read_probe_rejects_bad_sizes():
    import torch
    from paper_2404_16370_gb300 import mp
    words = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MPError):
        mp.mp_probe_random_reads(words, 0, 16)
