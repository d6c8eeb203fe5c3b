"""Ensemble launch modes (many domains in the same launches): every tile shape and the persistent one-launch
step give the same result as the default three-launch step (the per-cell and per-face
arithmetic does not depend on the tiling), and the autotuner leaves the state untouched.
Dry layouts agree bitwise. With the saturation adjustment two compiled instances of the same
per-cell code may round a cell's transfer one unit in the last place apart (the assembler
fuses multiply-adds by context), which the iteration's stop test then keeps: moist layouts
agree to a few units in the last place of each field. The oracle comparison of an ensemble
is in test_gpu_parity.py."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()


def members():
    return [W.add_random_motion(W.moist_bubble(n=n, A=A, R=R), seed=W.BASE_SEED + n)
            for n, A, R in [(20, 0.5, 200.0), (64, 1.5, 300.0), (37, 1.0, 150.0), (96, 2.0, 390.0)]]


def run(ws, dtype, variant=None, persistent=False, steps=3, graph=True):
    from paper_1901_02955_gb300 import Context
    ctx = Context(ws, dtype=dtype)
    if variant is not None:
        ctx.set_tile_variant(variant)
    ctx.use_persistent(persistent)
    ctx.use_graph(graph)
    for d, w in enumerate(ws):
        ctx.set_state(w.Y, domain=d)
    ctx.step(steps)
    out = [ctx.get_state(domain=d) for d in range(len(ws))]
    info = ctx.info()
    ctx.close()
    return out, info


def agree(a, b, exact):
    """Bitwise, or (moist) within 1e-6 of each field's largest magnitude."""
    if exact:
        return np.array_equal(a, b)
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    d = np.abs(a - b).reshape(b.shape[0], -1).max(axis=1)
    return bool(np.all(d <= 1e-6 * np.maximum(scale, 1e-30)))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tile_variants_and_persistent_step_agree(dtype):
    ws = members()
    ref, info = run(ws, dtype)
    assert info["kernel_launches_per_step"] == 3
    for v in range(info["n_tile_variants"]):
        for persistent in (False, True):
            for graph in (True, False):
                out, inf = run(ws, dtype, v, persistent, graph=graph)
                assert inf["tile_variant"] == v
                assert inf["kernel_launches_per_step"] == (1 if persistent else 3)
                for a, b in zip(out, ref):
                    assert agree(a, b, exact=False), (v, persistent, graph)


def test_persistent_step_on_3d_and_dry_layouts():
    for ws, exact in (([W.add_random_motion(W.jovian(nx=13, ny=11, nz=18))], False),
                      ([W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f32"))], True),
                      ([W.add_random_motion(W.dry_bubble_3d(nx=19, ny=10, nz=9))], True)):
        ref, info = run(ws, "f32")
        for v in range(info["n_tile_variants"]):
            for persistent in (False, True):
                out, _ = run(ws, "f32", v, persistent)
                assert all(agree(a, b, exact) for a, b in zip(out, ref)), (v, persistent)


def test_dry_fp64_tile_variants_agree_bitwise():
    """The FP64 dry x-z family has two tile shapes (32 x 28 and 32 x 14): both, in both launch
    modes, on a grid that leaves ragged tiles in x and z."""
    ws = [W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f64"))]
    ref, info = run(ws, "f64")
    assert info["n_tile_variants"] == 2
    for v in range(2):
        for persistent in (False, True):
            out, _ = run(ws, "f64", v, persistent)
            assert np.array_equal(out[0], ref[0]), (v, persistent)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [(1024, 256), (256, 256), (40, 40)])
def test_default_tile_fills_the_sms(dtype, n):
    """A new context starts on the first tile shape whose tiles cover every SM at least once,
    else on the shape with the most tiles."""
    import torch
    from paper_1901_02955_gb300 import Context
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    w = W.density_current(nx=n[0], nz=n[1], dtype=dtype)
    ctx = Context(w, dtype=dtype)
    chosen = ctx.info()["tile_variant"]
    tiles = []
    for v in range(ctx.info()["n_tile_variants"]):
        ctx.set_tile_variant(v)
        tiles.append(ctx.info()["tiles_total"])
    ctx.close()
    full = [v for v, t in enumerate(tiles) if t >= nsm]
    expect = full[0] if full else int(np.argmax(tiles))
    assert chosen == expect, (tiles, chosen)


def test_autotune_keeps_state_and_picks_a_mode():
    from paper_1901_02955_gb300 import Context
    ws = members()
    ctx = Context(ws, dtype="f32")
    for d, w in enumerate(ws):
        ctx.set_state(w.Y, domain=d)
    before = [ctx.get_state(domain=d) for d in range(len(ws))]
    res = ctx.autotune(steps=3)
    assert res["ms_per_step"] > 0
    info = ctx.info()
    if res["variant"] is None:  # every size class on its own shape
        assert info["per_class_tiles"] == 1 and info["persistent"] == 0
    else:
        assert info["tile_variant"] == res["variant"] and info["persistent"] == res["persistent"]
    after = [ctx.get_state(domain=d) for d in range(len(ws))]
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    ctx.step(3)
    ref, _ = run(ws, "f32")
    assert all(agree(ctx.get_state(domain=d), ref[d], exact=False) for d in range(len(ws)))


def test_persistent_barrier_timeout_reports_and_recovers():
    """A persistent step whose grid-barrier waits run out -- CTA 0 told to skip its arrivals,
    every wait limited to about 1 ms -- returns SNAP_ETIMEOUT instead of hanging, and the
    next normal step starts from a cleared barrier: bitwise the three-launch step."""
    from paper_1901_02955_gb300 import Context, SnapError, capi
    ws = [W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f32"))]
    ref, _ = run(ws, "f32", steps=2)
    ctx = Context(ws, dtype="f32")
    ctx.use_persistent(True)
    assert ctx.info()["persistent_grid"] >= 2
    ctx.set_state(ws[0].Y)
    ctx.set_barrier_test(spin_cycles=2_000_000, absent_cta=0)
    with pytest.raises(SnapError) as err:
        ctx.step(1)
    assert err.value.code == capi.ETIMEOUT
    ctx.set_barrier_test(0, -1)
    ctx.reset_flags()
    ctx.set_state(ws[0].Y)
    ctx.step(2)
    assert np.array_equal(ctx.get_state(), ref[0])
    ctx.close()


def test_resident_step_matches_three_launches():
    """The resident step (one tile per CTA for all three stages, neighbour flags between
    stages) against three launches: bitwise for dry layouts (ragged tiles, walls, periodic,
    3-D, several domains), to the moist tolerance with the saturation adjustment."""
    cases = [
        ([W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f32"))], "f32", True),
        ([W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f64"))], "f64", True),
        ([W.add_random_motion(W.dry_bubble_3d(nx=19, ny=10, nz=9))], "f32", True),
        ([W.add_random_motion(W.warm_bubble(n=5))], "f64", True),
        (members(), "f32", False),
    ]
    for ws, dtype, exact in cases:
        ref, _ = run(ws, dtype, steps=4)
        out, info = run(ws, dtype, persistent=2, steps=4)
        assert info["persistent"] == 2 and info["kernel_launches_per_step"] == 1
        for a, b in zip(out, ref):
            assert agree(a, b, exact), (ws[0].name, dtype)


def test_resident_step_on_the_density_current_grid():
    """The 1024 x 256 density current: 304 tiles of 64 x 14 cells, two per SM -- the grid the
    resident step is for; bitwise the three-launch step, with the CFL time step carried from
    step to step through the launch's last CTA."""
    ws = [W.density_current(dtype="f32")]
    ref, _ = run(ws, "f32", steps=3)
    out, info = run(ws, "f32", persistent=2, steps=3)
    assert info["tiles_total"] == 304
    assert np.array_equal(out[0], ref[0])


def test_resident_step_refuses_grids_beyond_one_wave():
    from paper_1901_02955_gb300 import Context, SnapError, capi
    ctx = Context(W.density_current(nx=4096, nz=256, dtype="f32"), dtype="f32")
    with pytest.raises(SnapError) as e:
        ctx.use_persistent(2)
    assert e.value.code == capi.ENOTSUP
    ctx.close()


def test_per_class_tile_shapes_agree():
    """Each size class on its own tile shape (one launch per class and stage, the classes in
    parallel): bitwise the one-shape step for dry domains, to the moist tolerance with the
    saturation adjustment; with and without graph capture."""
    from paper_1901_02955_gb300 import Context
    dry = [W.add_random_motion(W.density_current(nx=n, nz=m, dtype="f32"), seed=W.BASE_SEED + n)
           for n, m in [(70, 37), (40, 20), (70, 37), (33, 45)]]
    for ws, exact in ((dry, True), (members() + [members()[0]], False)):
        ref, _ = run(ws, "f32")
        for graph in (True, False):
            ctx = Context(ws, dtype="f32")
            info = ctx.info()
            nc, nv = info["n_size_classes"], info["n_tile_variants"]
            assert nc == len({(w.nx, w.ny, w.nz) for w in ws})
            for c in range(nc):
                ctx.set_class_tile_variant(c, (c + 1) % nv)
            info = ctx.info()
            assert info["per_class_tiles"] == 1 and info["kernel_launches_per_step"] == 3 * nc
            assert [k["variant"] for k in info["classes"]] == [(c + 1) % nv for c in range(nc)]
            assert sum(k["domains"] for k in info["classes"]) == len(ws)
            ctx.use_graph(graph)
            for d, w in enumerate(ws):
                ctx.set_state(w.Y, domain=d)
            ctx.step(3)
            out = [ctx.get_state(domain=d) for d in range(len(ws))]
            ctx.close()
            assert all(agree(a, b, exact) for a, b in zip(out, ref)), graph


def test_autotune_over_size_classes_keeps_state():
    from paper_1901_02955_gb300 import Context
    ws = members() + [members()[1]]
    ctx = Context(ws, dtype="f32")
    for d, w in enumerate(ws):
        ctx.set_state(w.Y, domain=d)
    before = [ctx.get_state(domain=d) for d in range(len(ws))]
    res = ctx.autotune(steps=2)
    info = ctx.info()
    if res["variant"] is None:
        assert info["per_class_tiles"] == 1
        assert res["per_class"] == [k["variant"] for k in info["classes"]]
    else:
        assert info["per_class_tiles"] == 0 and info["tile_variant"] == res["variant"]
    after = [ctx.get_state(domain=d) for d in range(len(ws))]
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    ctx.step(3)
    ref, _ = run(ws, "f32")
    assert all(agree(ctx.get_state(domain=d), ref[d], exact=False) for d in range(len(ws)))
    ctx.close()
