"""The allocation-free inner product, spl_dot_f64_noalloc.

It serves callers that cannot let the library allocate device memory (a
host framework that owns all device memory through its own pool, a
device-memory budget fixed at start-up, loops that cannot afford
cudaMalloc's implicit synchronisation).  Its partial sums live in a fixed
device array inside the library, so the test checks that two calls in a row
(with different inputs, the second reusing the array the first left behind)
agree with the workspace-based spl_dot_f64 through the C ABI.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_dot_matches_workspace_dot_twice():
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import spl

    B.build()
    L = spl.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(4242)
    work = spl.dot_workspace(dev)
    for n in (1000003, 4099):
        a = torch.tensor(rng.normal(size=n).astype(np.float32), device=dev)
        b = torch.tensor(rng.normal(size=n).astype(np.float32), device=dev)
        ref = torch.zeros(1, dtype=torch.float64, device=dev)
        got = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        spl.check(L.spl_dot_f64(n, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                C.c_void_p(ref.data_ptr()), C.c_void_p(work.data_ptr()), work.numel(), stream))
        spl.check(L.spl_dot_f64_noalloc(n, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                        C.c_void_p(got.data_ptr()), stream))
        torch.cuda.synchronize()
        r, g = float(ref.item()), float(got.item())
        exact = float(np.dot(a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
        scale = float(np.sum(np.abs(a.cpu().numpy().astype(np.float64) * b.cpu().numpy())))
        assert abs(g - r) <= 1e-12 * scale, (g, r)
        assert abs(g - exact) <= 1e-12 * scale, (g, exact)
    # sizes beyond the stated maximum are rejected before any launch
    assert L.spl_dot_f64_noalloc((1 << 40) + 1, C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), None) == 1
