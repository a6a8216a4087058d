"""The Python binding's argument checks (no GPU): the C ABIs take raw
pointers and read or write exactly the elements the caller describes, so
the binding refuses, before any call, a torch tensor or an output of the
wrong element type, an array of the wrong shape or size, a non-contiguous
output, and batched scans that differ from the sizes the batch was made for.
Inputs given as numpy arrays of another type are converted."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2404_16370_gb300 import mp


def test_numpy_inputs_are_converted_and_kept_alive():
    x = np.arange(12, dtype=np.float64).reshape(4, 3)
    p, keep = mp._ptr(x, np.float32, shape=(-1, 3))
    assert keep.dtype == np.float32 and keep.flags.c_contiguous and np.array_equal(keep, x)
    assert p.value == keep.ctypes.data


def test_torch_inputs_must_have_the_library_type():
    scan16 = torch.zeros((8, 3), dtype=torch.float16)
    with pytest.raises(TypeError):
        mp.mp_step(None, scan16)
    with pytest.raises(TypeError):
        mp.mp_set_buffer(None, mp.MP_BUF_NBR_IDS, torch.zeros((4, 16), dtype=torch.int64))
    with pytest.raises(ValueError):
        mp.mp_step(None, torch.zeros((8, 3), dtype=torch.float32).t())      # not contiguous
    p, keep = mp._ptr(torch.zeros((8, 3), dtype=torch.float32), np.float32, shape=(-1, 3))
    assert p.value == keep.data_ptr()


def test_shapes_and_sizes_are_checked():
    with pytest.raises(ValueError):
        mp.mp_step(None, np.zeros((8, 2), np.float32))                        # n x 2, not n x 3
    with pytest.raises(ValueError):
        mp.mp_step(None, np.zeros((8, 3), np.float32), odom_T=np.eye(3))      # 9 values, not 16
    with pytest.raises(ValueError):
        mp.mp_step(None, np.zeros((8, 3), np.float32), odom_cov=np.eye(5))
    with pytest.raises(ValueError):
        mp.mp_init_particles(None, 10, poses=np.zeros((9, 7), np.float32))
    with pytest.raises(ValueError):
        mp.mp_init_particles(None, 10, lo=np.zeros(5), hi=np.zeros(6))
    with pytest.raises(ValueError):
        mp.mp_init_map(np.zeros((100, 4), np.float32), None)
    with pytest.raises(ValueError):
        mp.mp_set_scan(None, np.zeros(24, np.float32))


def test_outputs_must_have_the_buffer_type_and_be_writeable_in_place():
    with pytest.raises(TypeError):
        mp.mp_get_buffer(None, mp.MP_BUF_GN, out=torch.zeros((4, 29), dtype=torch.float16))
    with pytest.raises(TypeError):
        mp.mp_get_buffer(None, mp.MP_BUF_GN, out=np.zeros((4, 29), np.float64))
    with pytest.raises(TypeError):
        mp.mp_get_buffer(None, mp.MP_BUF_GN, out=np.zeros((29, 4), np.float32).T)   # not C-contiguous


def test_batched_scans_match_the_batch():
    fake = 123457
    mp._batch_nscan[fake] = [4, 5]
    try:
        with pytest.raises(ValueError):
            mp.mp_batch_step(fake, [np.zeros((4, 3), np.float32)])                       # one scan for two
        with pytest.raises(ValueError):
            mp.mp_batch_step(fake, [np.zeros((4, 3), np.float32), np.zeros((6, 3), np.float32)])
        with pytest.raises(TypeError):
            mp.mp_batch_step(fake, [np.zeros((4, 3), np.float32), torch.zeros((5, 3))])
    finally:
        del mp._batch_nscan[fake]
    with pytest.raises(ValueError):
        mp.mp_batch_step(fake, [np.zeros((4, 3), np.float32)])                           # not a live batch


def test_proposal_tensors_are_checked():
    with pytest.raises(TypeError):
        mp._dev(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):
        mp._dev(torch.zeros((4, 6)), (4, 7))
    with pytest.raises(ValueError):
        mp._dev(torch.zeros((4, 7)), (4, 7))                                   # a host tensor
    with pytest.raises(TypeError):
        mp.mp_pn_forward(None, torch.zeros((2, 5, 3), dtype=torch.float16), torch.zeros((2, mp.MP_PN_OUT)))
    with pytest.raises(ValueError):
        mp.mp_pn_forward(None, torch.zeros((2, 5, 3)), torch.zeros((3, mp.MP_PN_OUT)))
    with pytest.raises(ValueError):
        mp.mp_pn_sample(None, torch.zeros(mp.MP_PN_OUT - 1), 3, 0, torch.zeros((3, 7)))
    with pytest.raises(ValueError):
        mp.mp_pn_sample(None, torch.zeros(mp.MP_PN_OUT), 3, 0, torch.zeros((4, 7)))
    with pytest.raises(ValueError):
        mp.mp_pn_sim_box_room(torch.zeros((3, 7)), 5.0, 3.0, torch.zeros((2, 7)), torch.zeros((8, 3)), 0.0, 0,
                              torch.zeros((2, 9, 3)))


def test_noalloc_refuses_host_arrays_before_any_call():
    """The allocation-free posterior dereferences its pointers as device
    memory: numpy arrays and CPU tensors are refused by the binding (the C
    entry point also refuses them, by cudaPointerGetAttributes)."""
    n = 16
    ll_np = np.zeros(n, np.float32)
    post_np = np.zeros(n, np.float64)
    best_np = np.zeros(1, np.int64)
    with pytest.raises(TypeError):
        mp.mp_posterior_init_noalloc(None, ll_np, post_np, best_np)
    ll_t = torch.zeros(n, dtype=torch.float32)
    post_t = torch.zeros(n, dtype=torch.float64)
    best_t = torch.zeros(1, dtype=torch.int64)
    with pytest.raises(TypeError):
        mp.mp_posterior_init_noalloc(None, ll_t, post_t, best_t)
    with pytest.raises(TypeError):
        mp.mp_posterior_init_noalloc(torch.zeros(n, dtype=torch.float64), ll_t, post_t, best_t)
