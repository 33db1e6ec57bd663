"""Eq. 1 through the entry point that allocates nothing (bn_evaluate_energy_noalloc).

It is meant for callers that cannot allocate device memory, e.g. code living inside another
framework's memory pool, or a real-time loop that must never stall on the allocator: they hand
in the count fields and an output buffer, and the library uses only a fixed scratch array of its
own.  The GPU tests check it against the FP64 oracle's Eq. 1 (at several radii, on a 4 x 4 torus,
on a tile narrower than the stencil, and at the 64-field limit of the scratch array) and against
bn_evaluate_energy on two calls in a row (the second call must not see anything left over from
the first).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_12620_gb300 import build
    build.build()
    return torch


# (n_fields, W, H, N, T, radius, sigma): the 64-field limit, a 4 x 4 torus (every other pixel
# is a neighbour), a tile narrower than 2 r + 1 (min-image aliases removed), radius 1, 3 and 8
# (29 distance classes of the 32 the scratch holds per field), ragged non-square tiles
NOALLOC_CASES = [
    (64, 9, 7, 16, 24, 6, 2.1),
    (1, 4, 4, 16, 40, 6, 2.1),
    (3, 8, 5, 64, 70, 6, 2.1),
    (2, 21, 13, 8, 33, 1, 2.1),
    (2, 19, 23, 32, 65, 3, 1.5),
    (1, 37, 29, 64, 130, 8, 3.0),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", NOALLOC_CASES, ids=lambda c: "f%d_%dx%d_N%d_T%d_r%d" % c[:6])
def test_noalloc_energy_matches_the_oracle(case):
    torch = _torch_cuda()
    n_fields, W, H, N, T, r, sigma = case
    rng = np.random.default_rng(7 + n_fields * 1000 + W * 31 + r)
    fields = rng.integers(0, N + 1, size=(n_fields, W * H, T), dtype=np.int32)
    want = np.array([oracle.energy(W, H, N, fields[f], sigma, r)[0] for f in range(n_fields)])
    dev = torch.from_numpy(fields).cuda()
    out = torch.full((n_fields,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # the second call must not see the first one's sums
        rc = _call(ctypes.c_void_p(dev.data_ptr()), n_fields, W, H, N, T,
                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream), sigma=sigma,
                   radius=r)
        assert rc == L.BN_OK, L.load().bn_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - want) <= E_REL * np.abs(want)), (call, got, want)


@pytest.mark.gpu
def test_noalloc_energy_matches_the_sampler_on_two_calls():
    torch = _torch_cuda()
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
        ref = np.array([oracle.energy(W, H, N, fields[i], 2.1, 6)[0] for i in range(2)])
        assert np.all(np.abs(got - ref) <= E_REL * np.abs(ref)), (call, got, ref)
    s.close()
