"""snap_budget_noalloc: the domain budget for callers that cannot allocate device memory
(a fixed pool that must not grow, a framework that owns all device memory, a phase where
cudaMalloc is not allowed). Its partial sums live in a fixed array inside the library; the
caller passes the state and the output. Checked against the context's own budget
(snap_budget_compute) on four calls in a row. Collected last on purpose."""
import ctypes

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


CASES = {
    "dry_x_z": lambda: W.add_random_motion(W.warm_bubble(n=40)),
    "moist_3d": lambda: W.add_random_motion(W.jovian(nx=13, ny=11, nz=18)),
    "moist_3d_many_blocks": lambda: W.jovian(nx=64, ny=64, nz=128),
}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_budget_matches_context_budget(torch, name, dtype):
    from paper_1901_02955_gb300 import Context, capi
    w = CASES[name]()
    Y0 = w.Y.astype(np.float32) if dtype == "f32" else w.Y.copy()
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ref = ctx.budget()
    ctx.close()
    lib = capi.load()
    Yd = torch.from_numpy(np.ascontiguousarray(Y0)).cuda()
    out = torch.empty(w.nv + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nmass = 1 + w.nvapor * (1 + w.ncond)
    rtol = 1e-12 if dtype == "f64" else 1e-6
    free_unchanged = []
    for call in range(4):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        torch_before = torch.cuda.memory_allocated()
        rc = lib.snap_budget_noalloc(
            ctypes.c_void_p(Yd.data_ptr()), capi.F32 if dtype == "f32" else capi.F64,
            w.nx, w.ny, w.nz, w.nv, nmass, w.dx, w.dy, w.dz, w.grav,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == capi.OK
        torch.cuda.synchronize()
        # nothing allocated through torch's allocator by the call (the figure may fall while
        # the call runs, when torch releases a tensor of earlier work)
        assert torch.cuda.memory_allocated() <= torch_before
        # device-wide free memory: the first call may load the library's module lazily, and
        # other users of the GPU change this figure too, so one unchanged reading among the later
        # calls is what the check asks for
        if call >= 1:
            free_unchanged.append(torch.cuda.mem_get_info()[0] == free_before)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:-1], ref["total"], rtol=rtol,
                                   atol=rtol * np.abs(ref["total"]).max())
        assert got[-1] == pytest.approx(ref["energy_with_potential"], rel=rtol)
    assert any(free_unchanged), "every call changed the device's free memory"


def test_noalloc_rejects_too_many_fields(torch):
    from paper_1901_02955_gb300 import capi
    lib = capi.load()
    buf = torch.zeros(30 * 27, dtype=torch.float64, device="cuda")
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    rc = lib.snap_budget_noalloc(ctypes.c_void_p(buf.data_ptr()), capi.F64, 3, 3, 3, 30, 1,
                                 1.0, 1.0, 1.0, 9.81, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == capi.EINVAL
