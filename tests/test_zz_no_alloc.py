"""Eq. 1 through the entry point that allocates nothing (bn_evaluate_energy_noalloc).

It is meant for callers that cannot allocate device memory, e.g. code living inside another
framework's memory pool, or a real-time loop that must never stall on the allocator: they hand
in the count fields and an output buffer, and the library uses only a fixed scratch array of its
own.  The GPU test checks it against bn_evaluate_energy on two calls in a row (the second call
must not see anything left over from the first).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2105_12620_gb300 import _lib as L

E_REL = 1e-5  # the energy tolerance of the other GPU tests


def _call(counts_ptr, n_fields, W, H, N, T, out_ptr, stream=None, sigma=2.1, radius=6):
    lib = L.load()
    return lib.bn_evaluate_energy_noalloc(counts_ptr, n_fields, W, H, N, T, sigma, radius,
                                          out_ptr, stream)


def test_noalloc_rejects_bad_arguments_on_the_host():
    from paper_2105_12620_gb300 import build
    build.build()
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    rc = _call(dummy, 65, 32, 32, 16, 8, dummy)
    assert rc == L.BN_ERR_INVALID_ARG
    assert "scratch" in L.load().bn_last_error().decode()
    assert _call(None, 1, 32, 32, 16, 8, dummy) == L.BN_ERR_INVALID_ARG
    assert _call(dummy, 1, 32, 32, 12, 8, dummy) == L.BN_ERR_INVALID_ARG
    assert _call(dummy, 1, 32, 32, 16, 8, dummy, radius=9) == L.BN_ERR_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_energy_matches_the_sampler_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_12620_gb300 import build
    build.build()
    import paper_2105_12620_gb300 as pkg
    W, H, N, T = 40, 36, 16, 100
    s = pkg.Sampler(W, H, N, T, seed=31, n_pairs=2)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call:
            s.optimize(15, stats=False)   # the fields change between the calls
        fields = np.stack([s.counts(0), s.counts(1)]).astype(np.int32)
        dev = torch.from_numpy(fields).cuda()
        rc = _call(ctypes.c_void_p(dev.data_ptr()), 2, W, H, N, T,
                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == L.BN_OK, L.load().bn_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = s.energy()
        assert np.all(np.abs(got - want) <= E_REL * np.abs(want)), (call, got, want)
    s.close()
