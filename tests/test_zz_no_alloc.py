"""qs_norm_noalloc, the norm for callers that cannot allocate device memory
(their GPU memory is reserved up front by another allocator, their budget
is fixed at start-up, or they must stay off the driver's allocation path).
It keeps its scratch in a fixed array inside the library; this test checks
it against qs_norm on two calls in a row, so stale contents of the shared
array from the first call cannot leak into the second.  The file is named to
be collected last."""

import numpy as np
import pytest
import torch

from paper_2008_00216_gb300 import binding as B
from workloads.rng import random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_norm_noalloc_matches_norm_twice(qs, dtype):
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    for n, seed, scale in ((14, 1, 1.0), (9, 2, 0.37)):   # second call: other size and values
        t = torch.from_numpy(random_state(n, seed) * scale).to(tdt).cuda()
        ref = B.State(n, dtype, tensor=t, init=None).norm()
        got = B.norm_noalloc(t, n, dtype)
        assert abs(got - ref) <= 1e-13 * ref, (n, got, ref)
        assert abs(got - scale * scale) < (1e-6 if dtype == "c64" else 1e-13)


def test_norm_noalloc_rejects_bad_arguments(qs):
    """The C entry point's own checks (the binding's are bypassed here)."""
    import ctypes as ct
    lib = B.load()
    t = torch.zeros(16, dtype=torch.complex64, device="cuda")
    v = ct.c_double()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.qs_norm_noalloc(ct.c_void_p(t.data_ptr()), 0, B.QS_C64, stream, ct.byref(v)) == 1   # n = 0
    # 8-byte offset: not 16-byte aligned
    assert lib.qs_norm_noalloc(ct.c_void_p(t[1:].data_ptr()), 3, B.QS_C64, stream, ct.byref(v)) == 1
    with pytest.raises(ValueError):                     # and through the binding: too few amplitudes
        B.norm_noalloc(t[:8], 4, "c64")
