"""GPU parity: the CUDA stream-collide path against the CPU oracle.

Bar: FP32 arithmetic (every storage format) is bit-for-bit the oracle's FP32
arithmetic in the paper's operation order (Sec. 2.2), because both sides
round the same operations in the same order and the codecs are bit-exact.
FP64 arithmetic with FP64 storage is within a relative L2 of 1e-12 of the
FP64 textbook definition.  Lattices span several thread blocks with ragged
edges; geometries mix every cell kind.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def P():
    import paper_2112_08926_gb300 as pkg
    return pkg


SHAPES = {"D2Q9": (1, 27, 45), "D3Q19": (7, 19, 37), "D3Q27": (5, 11, 35)}
FORCE = {"D2Q9": (1e-5, -2e-5, 0.0), "D3Q19": (1e-5, -2e-5, 3e-5), "D3Q27": (-1e-5, 2e-5, 1e-5)}
ALL_STORAGE = ["FP64", "FP32", "FP16", "FP16S", "FP16C", "P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"]


def geometry(vs, scheme, seed):
    shape = SHAPES[vs]
    if scheme == "AA":
        return W.random_geometry(shape, seed, outflow=0.0, freeslip_frac=0.0)
    return W.random_geometry(shape, seed)


def run_gpu(vs, coll, storage, arith, scheme, steps, force, geo, fields, tau=0.66, block=(32, 8)):
    nz, ny, nx = SHAPES[vs]
    g = P().Lattice(nx, ny, nz, vs, coll, storage, arith, scheme, tau=tau, trt_lambda=0.2, force=force)
    g.set_block(*block)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    g.step(steps)
    out = g.f(), g.rho_u(), g.reduce()
    g.close()
    return out


def run_oracle(vs, coll, arith, storage, steps, force, geo, fields, tau=0.66):
    nz, ny, nx = SHAPES[vs]
    o = oracle.Lattice(nx, ny, nz, vs, coll, arith, storage, tau=tau, trt_lambda=0.2, force=force)
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    o.step(steps)
    return o.f(), o.rho_u(), o.reduce()


@pytest.mark.parametrize("vs", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("storage", ALL_STORAGE)
def test_fp32_arithmetic_bitwise(vs, coll, scheme, storage):
    geo = geometry(vs, scheme, 11)
    fields = W.random_fields(SHAPES[vs], 12)
    force = FORCE[vs] if storage in ("FP32", "FP16C", "P16_1S") else (0.0, 0.0, 0.0)
    steps = 21 if scheme == "AA" else 20      # AA: odd count ends on the natural layout
    gf, grho, gred = run_gpu(vs, coll, storage, "FP32", scheme, steps, force, geo, fields)
    of, orho, ored = run_oracle(vs, coll, "ORD32", storage, steps, force, geo, fields)
    assert np.array_equal(gf, of), f"max |diff| {np.abs(gf - of).max():.3e}"
    for a, b in zip(grho, orho):
        assert np.array_equal(a, b)
    assert gred[0] == pytest.approx(ored[0], rel=1e-13)
    assert gred[1] == pytest.approx(ored[1], rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("vs", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
def test_fp64_tier_matches_definition(vs, coll, scheme):
    geo = geometry(vs, scheme, 21)
    fields = W.random_fields(SHAPES[vs], 22)
    gf, grho, gred = run_gpu(vs, coll, "FP64", "FP64", scheme, 30, FORCE[vs], geo, fields)
    of, orho, ored = run_oracle(vs, coll, "DEF64", "FP64", 30, FORCE[vs], geo, fields)
    assert np.linalg.norm(gf - of) / np.linalg.norm(of) < 1e-12
    for a, b in zip(grho[1:], orho[1:]):
        assert np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300) < 1e-12
    assert gred[0] == pytest.approx(ored[0], rel=1e-13)


@pytest.mark.parametrize("storage", ["FP64", "FP32"])
def test_fp64_arithmetic_bitwise_against_ordered_fp64(storage):
    vs, coll = "D3Q19", "SRT"
    geo = geometry(vs, "AB", 31)
    fields = W.random_fields(SHAPES[vs], 32)
    gf, _, _ = run_gpu(vs, coll, storage, "FP64", "AB", 15, FORCE[vs], geo, fields)
    of, _, _ = run_oracle(vs, coll, "ORD64", storage, 15, FORCE[vs], geo, fields)
    assert np.array_equal(gf, of)


@pytest.mark.parametrize("storage", ["FP32", "FP16S", "P16_2C"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
def test_flag_free_periodic_kernel(storage, scheme):
    vs = "D3Q19"
    nz, ny, nx = 9, 17, 70
    fields = W.random_fields((nz, ny, nx), 5)
    g = P().Lattice(nx, ny, nz, vs, "SRT", storage, "FP32", scheme, tau=0.53)
    g.set_rho_u(*fields)
    g.step(13)
    o = oracle.Lattice(nx, ny, nz, vs, "SRT", "ORD32", storage, tau=0.53)
    o.set_rho_u(*fields)
    o.step(13)
    assert np.array_equal(g.f(), o.f())
    assert g.info().has_flags == 0


@pytest.mark.parametrize("shape,block", [
    ((1, 1, 1), (32, 1)), ((1, 1, 33), (32, 1)), ((3, 2, 1), (32, 1)), ((2, 3, 129), (128, 2)),
    ((4, 5, 6), (256, 1)), ((3, 40, 3), (32, 8)),
])
def test_degenerate_and_ragged_sizes(shape, block):
    nz, ny, nx = shape
    geo = W.random_geometry(shape, 7, outflow=0.0)
    fields = W.random_fields(shape, 8)
    g = P().Lattice(nx, ny, nz, "D3Q19", "TRT", "FP16C", "FP32", "AB", tau=0.9, force=(1e-5, 0, 0))
    g.set_block(*block)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    g.step(9)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "TRT", "ORD32", "FP16C", tau=0.9, force=(1e-5, 0, 0))
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    o.step(9)
    assert np.array_equal(g.f(), o.f())


def test_set_f_round_trip_and_nan_detection():
    nz, ny, nx = 4, 5, 6
    rng = np.random.default_rng(1)
    f = rng.uniform(-0.01, 0.01, (19, nz, ny, nx))
    for storage in ("FP64", "FP16S"):
        arith = "FP64" if storage == "FP64" else "FP32"
        g = P().Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, "AA", tau=0.8)
        g.set_f(f)
        o = oracle.Lattice(nx, ny, nz, "D3Q19", "SRT", "DEF64" if storage == "FP64" else "ORD32", storage, tau=0.8)
        o.set_f(f)
        # a periodic lattice pulls each population from its upstream neighbour
        assert np.array_equal(g.f(), o.f())
        g.step(3)
        o.step(3)
        if storage == "FP16S":
            assert np.array_equal(g.f(), o.f())
    bad = f.copy()
    bad[3, 1, 2, 3] = np.nan
    g = P().Lattice(nx, ny, nz, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.8)
    g.set_f(bad)
    g.step(2)
    with pytest.raises(P().LBMError) as ei:
        g.reduce()
    assert ei.value.status == 5


def test_unsupported_geometry_for_in_place_streaming():
    shape = (3, 4, 5)
    flags = np.zeros(shape, np.uint8)
    flags[0, 0, 0] = W.OUTFLOW
    g = P().Lattice(5, 4, 3, "D3Q19", "SRT", "FP32", "FP32", "AA", tau=0.8)
    with pytest.raises(P().LBMError) as ei:
        g.set_geometry(flags)
    assert ei.value.status == 4
    flags[0, 0, 0] = W.MOVING            # MOVING without WALL
    with pytest.raises(P().LBMError) as ei:
        g.set_geometry(flags)
    assert ei.value.status == 1


@pytest.mark.parametrize("nx,scheme,flags", [(40, "AA", True), (64, "AA", True), (64, "AB", False), (128, "AB", False)])
def test_autotune_keeps_results(nx, scheme, flags):
    """The autotuner times the kernel variants that apply (and with them the
    layout: structure of arrays or chunked) and then block shapes; whatever
    it keeps, the lattice's values equal those of an untuned twin."""
    shape = (6, 13, nx)
    geo = W.random_geometry(shape, 3, outflow=0.0, freeslip_frac=0.0)
    fields = W.random_fields(shape, 4)
    res = []
    for tune in (False, True):
        g = P().Lattice(nx, 13, 6, "D3Q19", "SRT", "FP16S", "FP32", scheme, tau=0.7)
        if flags:
            g.set_geometry(*geo)
        g.set_rho_u(*fields)
        if tune:
            bx, by = g.autotune(trial_steps=2)
            assert bx * by % 32 == 0
            assert g.variant() in ("generic", "paired", "staged")
            done = g.info().step
        else:
            done = 0
        res.append((g, done))
    g0, _ = res[0]
    g1, done = res[1]
    g0.step(done)
    assert np.array_equal(g0.f(), g1.f())


@pytest.mark.parametrize("shape", [(3, 9, 128), (2, 6, 256), (2, 3, 512), (1, 1, 128), (1, 2, 256)])
@pytest.mark.parametrize("storage", ["FP32", "FP16S", "FP16C", "P16_1S", "P16_2C"])
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
def test_staged_kernel_bitwise(shape, storage, coll):
    nz, ny, nx = shape
    fields = W.random_fields(shape, 17)
    g = P().Lattice(nx, ny, nz, "D3Q19", coll, storage, "FP32", "AB", tau=0.57, trt_lambda=0.2)
    g.set_variant("staged")
    assert g.variant() == "staged"
    g.set_rho_u(*fields)
    g.step(7)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", coll, "ORD32", storage, tau=0.57, trt_lambda=0.2)
    o.set_rho_u(*fields)
    o.step(7)
    assert np.array_equal(g.f(), o.f())


@pytest.mark.parametrize("vs,shape,block", [
    ("D3Q19", (3, 9, 128), (32, 4)), ("D3Q19", (2, 5, 70), (32, 8)), ("D3Q19", (2, 3, 2), (32, 1)),
    ("D3Q19", (1, 3, 198), (64, 2)), ("D2Q9", (1, 17, 132), (32, 8)), ("D2Q9", (1, 4, 66), (32, 4)),
])
@pytest.mark.parametrize("storage", ["FP16", "FP16S", "FP16C", "P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"])
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
def test_paired_kernel_bitwise(vs, shape, block, storage, coll):
    nz, ny, nx = shape
    fields = W.random_fields(shape, 19)
    force = (1e-5, -1e-5, 0.0) if coll == "TRT" else (0.0, 0.0, 0.0)
    g = P().Lattice(nx, ny, nz, vs, coll, storage, "FP32", "AB", tau=0.61, trt_lambda=0.2, force=force)
    g.set_block(*block)
    g.set_variant("paired")
    assert g.variant() == "paired"
    g.set_rho_u(*fields)
    g.step(5)
    o = oracle.Lattice(nx, ny, nz, vs, coll, "ORD32", storage, tau=0.61, trt_lambda=0.2, force=force)
    o.set_rho_u(*fields)
    o.step(5)
    assert np.array_equal(g.f(), o.f())


@pytest.mark.parametrize("vs,shape", [("D3Q19", (3, 5, 128)), ("D3Q19", (2, 3, 64)), ("D3Q19", (1, 9, 192)),
                                      ("D2Q9", (1, 11, 128)), ("D2Q9", (1, 3, 64))])
@pytest.mark.parametrize("storage", ["FP16", "FP16S", "FP16C", "P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"])
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
def test_chunked_layout_bitwise(vs, shape, storage, coll):
    nz, ny, nx = shape
    fields = W.random_fields(shape, 23)
    force = (2e-5, 1e-5, 0.0) if coll == "SRT" else (0.0, 0.0, 0.0)
    g = P().Lattice(nx, ny, nz, vs, coll, storage, "FP32", "AB", tau=0.59, trt_lambda=0.2, force=force)
    g.set_rho_u(*fields)
    assert g.info().layout == 1 and g.variant() == "paired"
    g.step(6)
    o = oracle.Lattice(nx, ny, nz, vs, coll, "ORD32", storage, tau=0.59, trt_lambda=0.2, force=force)
    o.set_rho_u(*fields)
    o.step(6)
    assert np.array_equal(g.f(), o.f())
    r1, r2 = g.rho_u(), o.rho_u()
    for a, b in zip(r1, r2):
        assert np.array_equal(a, b)
    # switching kernels converts the layout without changing a value
    g.set_variant("generic")
    assert g.info().layout == 0
    g.step(3)
    o.step(3)
    assert np.array_equal(g.f(), o.f())
    g.set_variant("auto")
    assert g.info().layout == 1
    g.step(2)
    o.step(2)
    assert np.array_equal(g.f(), o.f())


def test_chunked_lattice_takes_flags_later():
    shape = (3, 4, 64)
    fields = W.random_fields(shape, 29)
    geo = W.random_geometry(shape, 30)
    g = P().Lattice(64, 4, 3, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.7)
    g.set_rho_u(*fields)
    assert g.info().layout == 1
    g.step(4)
    o = oracle.Lattice(64, 4, 3, "D3Q19", "SRT", "ORD32", "FP16S", tau=0.7)
    o.set_rho_u(*fields)
    o.step(4)
    g.set_geometry(*geo)
    o.set_geometry(*geo)
    assert g.info().layout == 1          # flags keep the chunked layout (boundary cells from a list)
    g.step(5)
    o.step(5)
    assert np.array_equal(g.f(), o.f())
    g.set_f(o.f())
    o.set_f(o.f())
    g.set_geometry(None)
    o.set_geometry(None)
    g.set_f(o.f())
    o.set_f(o.f())
    assert g.info().layout == 1
    g.step(3)
    o.step(3)
    assert np.array_equal(g.f(), o.f())
    # flags again: the flag bytes and wall masks are allocated anew
    g.set_geometry(*geo)
    o.set_geometry(*geo)
    g.step(4)
    o.step(4)
    assert np.array_equal(g.f(), o.f())


# ---------------------------------------------------------------- no DDF shifting
def _pair(vs, coll, storage, arith, oarith, scheme, shifting, steps, force, geo, fields):
    nz, ny, nx = SHAPES[vs]
    g = P().Lattice(nx, ny, nz, vs, coll, storage, arith, scheme, tau=0.66, trt_lambda=0.2, force=force,
                    shifting=shifting)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    g.step(steps)
    gout = g.f(), g.rho_u()
    g.close()
    o = oracle.Lattice(nx, ny, nz, vs, coll, oarith, "FP64" if oarith == "DEF64" else storage, tau=0.66,
                       trt_lambda=0.2, force=force, shifting=shifting)
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    o.step(steps)
    return gout, (o.f(), o.rho_u())


@pytest.mark.parametrize("vs", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("storage", ["FP32", "FP16", "FP16S", "FP16C", "P16_1S", "P16_2C"])
def test_unshifted_fp32_arithmetic_bitwise(vs, scheme, storage):
    """The no-shifting ablation (appendix, without DDF-shifting): stored f,
    rho = sum f, plain equilibrium; bit for bit the ordered FP32 oracle."""
    geo = geometry(vs, scheme, 41)
    fields = W.random_fields(SHAPES[vs], 42)
    (gf, gu), (of, ou) = _pair(vs, "TRT" if storage in ("FP16S", "P16_2C") else "SRT", storage, "FP32", "ORD32",
                               scheme, False, 21 if scheme == "AA" else 20, FORCE[vs], geo, fields)
    assert np.array_equal(gf, of)
    for a, b in zip(gu, ou):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("vs", ["D3Q19", "D3Q27"])
def test_unshifted_fp64_tier_matches_definition(vs):
    geo = geometry(vs, "AB", 43)
    fields = W.random_fields(SHAPES[vs], 44)
    (gf, _), (of, _) = _pair(vs, "SRT", "FP64", "FP64", "DEF64", "AB", False, 30, FORCE[vs], geo, fields)
    assert np.linalg.norm(gf - of) / np.linalg.norm(of) < 1e-12


def test_unshifted_lattice_starts_at_rest_and_chunked_layout_applies():
    g = P().Lattice(128, 6, 5, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.7, shifting=False)
    r, ux, uy, uz = g.rho_u()
    assert np.abs(r - 1).max() < 1e-3 and np.abs(ux).max() == 0
    assert g.info().layout == 1          # flag-free 16-bit A-B: chunked paired kernel
    fields = W.random_fields((5, 6, 128), 45)
    g.set_rho_u(*fields)
    g.step(9)
    o = oracle.Lattice(128, 6, 5, "D3Q19", "SRT", "ORD32", "FP16S", tau=0.7, shifting=False)
    o.set_rho_u(*fields)
    o.step(9)
    assert np.array_equal(g.f(), o.f())
    g.close()


# ---------------------------------------------------------------- chunked layout, every scheme
CH_SHAPES = {"D2Q9": (1, 9, 128), "D3Q19": (3, 7, 128)}


@pytest.mark.parametrize("vs", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("geo_kind", ["free", "flags"])
@pytest.mark.parametrize("storage", ["FP16", "FP16S", "FP16C", "P16_1S", "P16_2C", "P16_0"])
def test_chunked_layout_every_scheme_bitwise(vs, scheme, geo_kind, storage):
    """16-bit lattices with nx a multiple of 64 run on the chunked layout with
    the paired kernels, for A-B and both A-A halves, flag-free or with a
    random geometry (plain cells paired, boundary cells from the list).
    D3Q27 has its own test (test_d3q27_chunked_bitwise)."""
    nz, ny, nx = CH_SHAPES[vs]
    shape = (nz, ny, nx)
    fields = W.random_fields(shape, 51)
    if geo_kind == "flags":
        extra = {"outflow": 0.0, "freeslip_frac": 0.0} if scheme == "AA" else {}
        geo = W.random_geometry(shape, 52, **extra)
    coll = "TRT" if storage in ("FP16S", "P16_2C") else "SRT"
    force = FORCE[vs] if storage == "FP16C" else (0.0, 0.0, 0.0)
    g = P().Lattice(nx, ny, nz, vs, coll, storage, "FP32", scheme, tau=0.66, trt_lambda=0.2, force=force)
    if geo_kind == "flags":
        g.set_geometry(*geo)
    g.set_rho_u(*fields)
    assert g.info().layout == 1 and g.variant() == "paired"
    steps = 21 if scheme == "AA" else 20
    g.step(steps)
    o = oracle.Lattice(nx, ny, nz, vs, coll, "ORD32", storage, tau=0.66, trt_lambda=0.2, force=force)
    if geo_kind == "flags":
        o.set_geometry(*geo)
    o.set_rho_u(*fields)
    o.step(steps)
    assert np.array_equal(g.f(), o.f())
    for a, b in zip(g.rho_u(), o.rho_u()):
        assert np.array_equal(a, b)
    # one more step on the other A-A half, then switch to the SoA layout mid-run
    g.step(1)
    o.step(1)
    g.set_variant("generic")
    assert g.info().layout == 0
    g.step(2)
    o.step(2)
    assert np.array_equal(g.f(), o.f())
    g.close()


@pytest.mark.parametrize("vs,shape", [("D3Q19", (5, 6, 128)), ("D3Q19", (4, 7, 37)), ("D2Q9", (1, 9, 64)),
                                      ("D3Q27", (4, 5, 22))])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("storage", ["FP32", "FP16S", "FP16C"])
def test_plain_bounce_back_cells_in_fast_kernels(vs, shape, scheme, storage):
    """Static walls only (the x = 0 and x = nx - 1 planes and a solid block):
    every boundary cell needs plain bounce-back, which the fast kernels do
    themselves (generic and paired; the odd A-A half of the paired kernel
    leaves them to the list).  Bit-equal to the oracle after an odd step
    count, i.e. after both A-A halves."""
    nz, ny, nx = shape
    flags = np.zeros(shape, np.uint8)
    flags[:, :, 0] = flags[:, :, -1] = 1
    flags[nz // 2:nz // 2 + 2, 2:4, nx // 2:nx // 2 + 3] = 1
    fields = W.random_fields(shape, 61)
    force = FORCE[vs]
    g = P().Lattice(nx, ny, nz, vs, "SRT", storage, "FP32", scheme, tau=0.7, force=force)
    g.set_geometry(flags)
    g.set_rho_u(*fields)
    g.step(13)
    o = oracle.Lattice(nx, ny, nz, vs, "SRT", "ORD32", storage, tau=0.7, force=force)
    o.set_geometry(flags)
    o.set_rho_u(*fields)
    o.step(13)
    assert np.array_equal(g.f(), o.f())
    for a, b in zip(g.rho_u(), o.rho_u()):
        assert np.array_equal(a, b)
    g.close()


@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("storage", ["FP32", "FP16S"])
def test_graph_replayed_steps_bitwise(scheme, storage):
    """Calls of 64 steps or more on lattices up to 2^23 cells replay runs of
    32 steps from a CUDA graph: bit-equal to one launch per step and to the
    oracle, from either step parity (the graphs are keyed by it) and after
    calls that change what a step launches (kernel variant, geometry)."""
    nz, ny, nx = 5, 9, 64
    shape = (nz, ny, nx)
    fields = W.random_fields(shape, 71)
    extra = {"outflow": 0.0, "freeslip_frac": 0.0} if scheme == "AA" else {}
    geo = W.random_geometry(shape, 72, **extra)

    def make():
        g = P().Lattice(nx, ny, nz, "D3Q19", "SRT", storage, "FP32", scheme, tau=0.7)
        g.set_geometry(*geo)
        g.set_rho_u(*fields)
        return g

    a, b = make(), make()
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "SRT", "ORD32", storage, tau=0.7)
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    a.step(101)                      # three replays and five launches
    for _ in range(101):
        b.step(1)
    o.step(101)
    assert np.array_equal(a.f(), b.f())
    assert np.array_equal(a.f(), o.f())
    a.step(64)                       # odd start: the graph of the other parity
    o.step(64)
    assert np.array_equal(a.f(), o.f())
    a.set_variant("generic")         # another kernel: the graphs are captured again
    a.step(65)
    o.step(65)
    assert np.array_equal(a.f(), o.f())
    a.set_geometry(*geo)             # a new cell list
    a.step(66)
    o.step(66)
    assert np.array_equal(a.f(), o.f())
    a.close()
    b.close()


def test_d3q27_software_codecs_stay_generic():
    """D3Q27 takes the chunked paired kernel only with the hardware
    conversions (FP16, FP16S); the software codecs keep the generic kernel."""
    g = P().Lattice(64, 3, 2, "D3Q27", "SRT", "FP16C", "FP32", "AB", tau=0.7)
    g.set_variant("paired")
    assert g.variant() == "generic" and g.info().layout == 0
    g.close()


@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("geo_kind", ["free", "flags"])
@pytest.mark.parametrize("storage,coll", [("FP16S", "TRT"), ("FP16", "SRT")])
def test_d3q27_chunked_bitwise(scheme, geo_kind, storage, coll):
    """D3Q27 on the chunked layout: the paired kernel takes a lane's two
    cells one after the other (27 code pairs); bit-equal to the oracle for
    A-B and both A-A halves, flag-free or with a random geometry."""
    nz, ny, nx = 3, 5, 128
    shape = (nz, ny, nx)
    fields = W.random_fields(shape, 81)
    force = FORCE["D3Q27"]
    g = P().Lattice(nx, ny, nz, "D3Q27", coll, storage, "FP32", scheme, tau=0.66, trt_lambda=0.2, force=force)
    o = oracle.Lattice(nx, ny, nz, "D3Q27", coll, "ORD32", storage, tau=0.66, trt_lambda=0.2, force=force)
    if geo_kind == "flags":
        extra = {"outflow": 0.0, "freeslip_frac": 0.0} if scheme == "AA" else {}
        geo = W.random_geometry(shape, 82, **extra)
        g.set_geometry(*geo)
        o.set_geometry(*geo)
    g.set_rho_u(*fields)
    o.set_rho_u(*fields)
    assert g.info().layout == 1 and g.variant() == "paired"
    g.step(21)
    o.step(21)
    assert np.array_equal(g.f(), o.f())
    for a, b in zip(g.rho_u(), o.rho_u()):
        assert np.array_equal(a, b)
    g.close()


@pytest.mark.parametrize("storage,shape", [("FP16S", (3, 7, 128)), ("FP32", (5, 9, 37)), ("P16_1S", (4, 6, 64))])
def test_scheme_switch_keeps_values(storage, shape):
    """lbm_set_scheme: A-B <-> in-place A-A on a live lattice (even step counts)."""
    nz, ny, nx = shape
    geo = W.random_geometry(shape, 61, outflow=0.0, freeslip_frac=0.0)
    fields = W.random_fields(shape, 62)
    g = P().Lattice(nx, ny, nz, "D3Q19", "TRT", storage, "FP32", "AB", tau=0.7)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "TRT", "ORD32", storage, tau=0.7)
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    g.step(10)
    mem_ab = g.info().device_bytes
    g.set_scheme("AA")
    assert g.info().device_bytes < mem_ab
    g.step(11)
    with pytest.raises(P().LBMError) as e:      # odd step count
        g.set_scheme("AB")
    assert e.value.status == 7
    g.step(1)
    g.set_scheme("AB")
    g.step(3)
    o.step(25)
    assert np.array_equal(g.f(), o.f())
    g.close()


def test_ensemble_autotune_picks_scheme_bitwise():
    specs = W.ensemble_cavities(count=6, n_min=6, n_max=19, seed=5)
    def members():
        out = []
        for s in specs:
            g = P().Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=s.tau)
            g.set_geometry(W.cavity_flags(s.n))
            g.set_nodes(*W.cavity_lid(s.n, s.u_lid))
            g.set_rho_u()
            out.append(g)
        return out
    a, b = members(), members()
    e = P().Ensemble(a)
    e.autotune(trial_steps=3)
    assert e.scheme() in ("AB", "AA")
    done = a[0].info().step              # the trial steps are real steps
    e.step(20)
    for g in b:
        g.step(done + 20)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())
    e.close()


# ---------------------------------------------------------------- MRT (D3Q19)
@pytest.mark.parametrize("storage", ["FP32", "FP16S", "FP16C"])
@pytest.mark.parametrize("scheme", ["AB", "AA"])
@pytest.mark.parametrize("shape", [(7, 19, 37), (3, 7, 128)])
def test_mrt_fp32_arithmetic_bitwise(storage, scheme, shape):
    """D3Q19 MRT (moment basis and rates of d'Humieres et al. 2002) in the
    fixed transform order: bit for bit the ordered FP32 oracle, with
    boundaries and forcing."""
    nz, ny, nx = shape
    extra = {"outflow": 0.0, "freeslip_frac": 0.0} if scheme == "AA" else {}
    geo = W.random_geometry(shape, 81, **extra)
    fields = W.random_fields(shape, 82)
    force = (1e-5, -2e-5, 3e-5)
    steps = 21 if scheme == "AA" else 20
    g = P().Lattice(nx, ny, nz, "D3Q19", "MRT", storage, "FP32", scheme, tau=0.66, force=force)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    g.step(steps)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "MRT", "ORD32", storage, tau=0.66, force=force)
    o.set_geometry(*geo)
    o.set_rho_u(*fields)
    o.step(steps)
    assert np.array_equal(g.f(), o.f())
    g.close()


def test_mrt_fp64_tier():
    shape = (7, 19, 37)
    nz, ny, nx = shape
    geo = W.random_geometry(shape, 83)
    fields = W.random_fields(shape, 84)
    force = (1e-5, -2e-5, 3e-5)
    g = P().Lattice(nx, ny, nz, "D3Q19", "MRT", "FP64", "FP64", "AB", tau=0.7, force=force)
    g.set_geometry(*geo)
    g.set_rho_u(*fields)
    g.step(20)
    gf = g.f()
    g.close()
    for arith, check in (("DEF64", "l2"), ("ORD64", "bitwise")):
        o = oracle.Lattice(nx, ny, nz, "D3Q19", "MRT", arith, "FP64", tau=0.7, force=force)
        o.set_geometry(*geo)
        o.set_rho_u(*fields)
        o.step(20)
        of = o.f()
        if check == "l2":
            assert np.linalg.norm(gf - of) / np.linalg.norm(of) < 1e-12
        else:
            assert np.array_equal(gf, of)


def test_mrt_unsupported_combinations():
    for vs, storage, arith, nz in (("D2Q9", "FP32", "FP32", 1), ("D3Q19", "P16_1S", "FP32", 4)):
        with pytest.raises(P().LBMError) as e:
            P().Lattice(8, 4, nz, vs, "MRT", storage, arith, "AB")
        assert e.value.status == 4



def test_stream_auto_picks_a_scheme_and_keeps_results():
    """LBM_STREAM_AUTO: created as A-B where both copies fit; lbm_autotune
    times A-B against in-place A-A and keeps the faster.  Every choice gives
    the populations of a fixed-scheme run bit for bit (same step count)."""
    import paper_2112_08926_gb300 as P
    shape = (12, 10, 64)
    nz, ny, nx = shape
    fields = W.random_fields(shape, seed=31)
    flags = W.cavity(nx, 0.05, ny=ny, nz=nz)
    g = P.Lattice(nx, ny, nz, "D3Q19", "TRT", "FP16S", "FP32", "AUTO", tau=0.6)
    assert g.scheme == "AB"
    g.set_geometry(*flags)
    g.set_rho_u(*fields)
    g.autotune(trial_steps=7)
    assert g.scheme in ("AB", "AA")
    steps = g.info().step
    g.step(10 + (steps & 1))
    ref = P.Lattice(nx, ny, nz, "D3Q19", "TRT", "FP16S", "FP32", "AB", tau=0.6)
    ref.set_geometry(*flags)
    ref.set_rho_u(*fields)
    ref.step(g.info().step)
    assert np.array_equal(g.f(), ref.f())
    g.close()
    ref.close()


def _quotient_edge_populations(nz, ny, nx, big):
    """Shifted D3Q19 populations whose cells reach every branch of the
    velocity quotient: ordinary values, exact zeros (numerators 0 of either
    sign), a density below 2^-20 (f_0 = -1 plus one 2^-22), a negative
    density, and large values (FP16: 6e4)."""
    rng = np.random.default_rng(17)
    f = rng.uniform(-0.01, 0.01, (19, nz, ny, nx))
    flat = f.reshape(19, -1)
    n = flat.shape[1]
    flat[:, 0:n:7] = 0.0                          # at rest: zero momenta
    flat[1:, 1:n:7] = -0.0
    flat[:, 2:n:7] = 0.0                          # rho = 2^-22
    flat[0, 2:n:7] = -1.0
    flat[1, 2:n:7] = 2.0 ** -22
    flat[0, 3:n:7] = -1.5                         # rho < 0
    flat[0, 4:n:7] = big                          # large density and momentum
    flat[1, 4:n:7] = big / 2
    return f


@pytest.mark.parametrize("storage", ["FP16", "FP16S", "P16_2C", "FP32"])
@pytest.mark.parametrize("force", [(0.0, 0.0, 0.0), (1e-30, 0.0, 2e-5), (2.0 ** -76, -(2.0 ** -70), 0.0),
                                   (-(2.0 ** 90), 0.0, 1e-3)])
@pytest.mark.parametrize("nx", [64, 6])
def test_velocity_quotient_ranges_bitwise(storage, force, nx):
    """u_a = (j_a + F_a/2) / rho is the IEEE quotient on every route: the
    corrected reciprocal, the 16-bit storage shortcut that checks only the
    largest numerator (force components 0 or within [2^-76, 2^90]), and the
    division taken for numerators below 2^-100 (a 1e-30 force), densities
    outside [2^-20, 2^20] and non-finite values.  Bit for bit against the
    oracle after one and two steps, on the paired (nx = 64) and the generic
    (nx = 6) kernels."""
    nz, ny = 3, 5
    big = 6.0e4 if storage in ("FP16", "FP32") else 1.5
    f = _quotient_edge_populations(nz, ny, nx, big)
    g = P().Lattice(nx, ny, nz, "D3Q19", "SRT", storage, "FP32", "AB", tau=0.8, force=force)
    g.set_f(f)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "SRT", "ORD32", storage, tau=0.8, force=force)
    o.set_f(f)
    assert np.array_equal(g.f(), o.f(), equal_nan=True)
    for _ in range(2):
        g.step(1)
        o.step(1)
        assert np.array_equal(g.f(), o.f(), equal_nan=True)
    g.close()
