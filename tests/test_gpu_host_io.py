"""Host state transfers through the C ABI: a page-locked (pinned) host buffer is read and
written by the conversion kernel directly through its device mapping, a pageable one is
staged through device memory; both must give bitwise the same states, in every combination
of the context's type and the buffer's type, before and after steps."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("ctx_dtype", ["f64", "f32"])
@pytest.mark.parametrize("io", [np.float64, np.float32])
def test_pinned_and_pageable_host_buffers_agree(torch, ctx_dtype, io):
    from paper_1901_02955_gb300 import Context
    w = W.add_random_motion(W.moist_bubble(nx=45, nz=35))
    Y = np.ascontiguousarray(w.Y.astype(io))
    tio = torch.float64 if io == np.float64 else torch.float32
    a = Context(w, dtype=ctx_dtype)
    b = Context(w, dtype=ctx_dtype)
    a.set_state(Y)                                   # pageable
    pin_in = torch.from_numpy(Y.copy()).pin_memory()
    assert pin_in.is_pinned()
    b.set_state(pin_in)                              # pinned, read in place by the kernel
    for steps in (0, 2):
        if steps:
            a.step(steps, dt_fixed=0.02)
            b.step(steps, dt_fixed=0.02)
        ref = a.get_state(dtype=io)                  # pageable
        out = torch.empty(Y.shape, dtype=tio).pin_memory()
        b.get_state(out=out)                         # pinned, written in place by the kernel
        assert np.array_equal(out.numpy(), ref), steps
    a.close()
    b.close()
