"""The benchmark's measurement helpers (libmp_probe.so, include/mp_probe.h):
the random-read probe leaves its buffer unchanged and takes longer for more
reads; the FMA probes report positive rates in a plausible order (FP64 far
below FP32 on this GPU); host buffers and bad sizes are refused."""
import pytest

pytestmark = pytest.mark.gpu


def test_random_read_probe_runs():
    import torch
    from paper_2404_16370_gb300 import mp
    words = torch.arange(1 << 20, dtype=torch.int32, device="cuda")
    ref = words.clone()
    ms_small, n_small = mp.mp_probe_random_reads(words, 64, 16, repeats=3)
    ms_large, n_large = mp.mp_probe_random_reads(words, 64, 1024, repeats=3)
    torch.cuda.synchronize()
    assert n_small == 64 * 256 * 16 and n_large == 64 * 256 * 1024
    assert ms_small > 0 and ms_large > ms_small
    assert torch.equal(words, ref)


def test_random_read_probe_rejects_bad_arguments():
    import ctypes as C
    import torch
    from paper_2404_16370_gb300 import mp
    words = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MPError):
        mp.mp_probe_random_reads(words, 0, 16)
    host = torch.zeros(16, dtype=torch.int32).pin_memory()
    ms, n = C.c_float(), C.c_int64()
    assert mp.probe_lib().mp_probe_random_reads(C.c_void_p(host.data_ptr()), 16, 1, 16, 1, None, C.byref(ms),
                                                C.byref(n)) == mp.MP_EINVAL


def test_fma_probes():
    from paper_2404_16370_gb300 import mp
    rates = {}
    for kind, iters in ((mp.MP_FMA_FP32, 2000), (mp.MP_FMA_FP32X2, 2000), (mp.MP_FMA_FP64, 200)):
        ms, flops = mp.mp_probe_fma_rate(kind, 152 * 4, iters, repeats=2)
        assert ms > 0 and flops == 2 * 16 * iters * 152 * 4 * 256
        rates[kind] = flops / (ms * 1e-3)
    assert rates[mp.MP_FMA_FP32] > 5 * rates[mp.MP_FMA_FP64]
    with pytest.raises(mp.MPError):
        mp.mp_probe_fma_rate(3, 1, 1)
