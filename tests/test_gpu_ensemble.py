"""Ensembles: one launch per step over many uneven lattices must give exactly
the result of one launch per member (same per-cell routine), and members
must match the CPU oracle bit for bit (FP32 arithmetic, FP16S storage)."""
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


def make_members(specs, storage, scheme, P):
    out = []
    for s in specs:
        g = P.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", storage, "FP32", scheme, tau=s.tau)
        flags, node_u = W.cavity(s.n, s.u_lid)
        g.set_geometry(flags, node_u)
        g.set_rho_u()
        out.append(g)
    return out


@pytest.mark.parametrize("scheme", ["AB", "AA"])
def test_ensemble_equals_per_member_launches(scheme):
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=7, n_min=6, n_max=21)
    a = make_members(specs, "FP16S", scheme, P)
    b = make_members(specs, "FP16S", scheme, P)
    ea, eb = P.Ensemble(a), P.Ensemble(b)
    ea.step(150)          # two graph replays of 64 steps and 22 single launches
    eb.step_each(150)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())
    ea.set_block(64, 1)
    ea.step(3)
    eb.step_each(3)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())


@pytest.mark.parametrize("storage,coll", [("FP16S", "SRT"), ("FP16", "TRT")])
def test_paired_ensemble_equals_per_member_launches(storage, coll):
    """The paired ensemble kernel (two cells per thread, 32-bit code pairs,
    runs of 64 linear cells) on cavities of odd and even edges (every parity
    of source and destination pairs), with 1, 2 and 4 runs per tile, against
    one launch per member."""
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=9, n_min=5, n_max=23, seed=7)

    def members():
        out = []
        for s in specs:
            g = P.Lattice(s.n, s.n, s.n, "D3Q19", coll, storage, "FP32", "AB", tau=s.tau)
            flags, node_u = W.cavity(s.n, s.u_lid)
            g.set_geometry(flags, node_u)
            g.set_rho_u(*W.random_fields((s.n, s.n, s.n), seed=s.n))
            out.append(g)
        return out

    a, b = members(), members()
    ea, eb = P.Ensemble(a), P.Ensemble(b)
    for layout, warps in (("soa", 4), ("soa", 1), ("chunked", 2), ("chunked", 4)):
        ea.set_layout(layout)
        ea.set_variant("paired", warps)
        assert ea.variant() == "paired" and ea.layout() == layout
        ea.step(70)          # a graph replay of 64 steps and 6 single launches
        eb.step_each(70)
        for ga, gb in zip(a, b):
            assert np.array_equal(ga.f(), gb.f()), (layout, warps)


@pytest.mark.parametrize("scheme", ["AB", "AA"])
def test_chunked_member_layout_every_kernel(scheme):
    """Members on the chunked layout (64-cell chunks of the linear cell
    index, any nx): the per-cell ensemble kernel, one launch per member on
    the same layout (lbm_ensemble_step_each), and the members' readbacks,
    against members on the structure of arrays."""
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=6, n_min=5, n_max=19, seed=3)
    a = make_members(specs, "FP16C", scheme, P)
    b = make_members(specs, "FP16C", scheme, P)
    c = make_members(specs, "FP16C", scheme, P)
    ea, eb, ec = P.Ensemble(a), P.Ensemble(b), P.Ensemble(c)
    ea.set_layout("chunked")
    eb.set_layout("chunked")
    assert a[0].info().layout == 1
    ea.step(70)
    eb.step_each(70)
    ec.step(70)
    for ga, gb, gc in zip(a, b, c):
        fa = ga.f()
        assert np.array_equal(fa, gb.f()) and np.array_equal(fa, gc.f())
        assert np.array_equal(ga.rho_u()[1], gc.rho_u()[1])
    ea.close()
    assert a[0].info().layout == 0       # back to the members' own layout
    for ga, gc in zip(a, c):
        assert np.array_equal(ga.f(), gc.f())


def test_paired_ensemble_open_faces_and_every_cell_kind():
    """Members whose faces hold fluid cells (periodic in every direction) and
    every kind of boundary cell: the face cells take the per-cell path inside
    the paired launch, the listed cells the list launch; the result equals
    one launch per member bit for bit."""
    import paper_2112_08926_gb300 as P
    # (9, 3, 5): odd q N, and the last run's lanes past the member read
    # source elements beyond the copy (clamped to its last aligned word)
    shapes = [(7, 9, 11), (6, 10, 64), (5, 5, 33), (12, 3, 17), (9, 3, 5)]

    def members():
        out = []
        for k, shp in enumerate(shapes):
            nz, ny, nx = shp
            g = P.Lattice(nx, ny, nz, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.7, force=(1e-5, 0.0, -2e-5))
            g.set_geometry(*W.random_geometry(shp, 40 + k))
            g.set_rho_u(*W.random_fields(shp, seed=50 + k))
            out.append(g)
        return out

    a, b = members(), members()
    ea, eb = P.Ensemble(a), P.Ensemble(b)
    for layout in ("soa", "chunked"):
        ea.set_layout(layout)
        ea.set_variant("paired", 2)
        ea.step(70)
        eb.step_each(70)
        for ga, gb in zip(a, b):
            assert np.array_equal(ga.f(), gb.f()), layout


def test_members_on_their_own_streams():
    """Members created on different streams: the ensemble's launches wait
    for the members' initialisation and layout changes, and the members'
    readbacks on their own streams wait for the ensemble's steps."""
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=6, n_min=6, n_max=20, seed=11)
    streams = [torch.cuda.Stream() for _ in range(3)]

    def members(on_streams):
        out = []
        for k, s in enumerate(specs):
            st = streams[k % 3].cuda_stream if on_streams else None
            g = P.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=s.tau, stream=st)
            flags, node_u = W.cavity(s.n, s.u_lid)
            g.set_geometry(flags, node_u)
            g.set_rho_u(*W.random_fields((s.n, s.n, s.n), seed=s.n))
            out.append(g)
        return out

    a, b = members(True), members(False)
    ea, eb = P.Ensemble(a), P.Ensemble(b)
    ea.step(70)
    eb.step(70)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())
    ea.set_layout("chunked")
    ea.set_variant("paired", 2)
    ea.step(66)
    eb.step_each(66)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())
    ea.close()
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.f(), gb.f())


def test_paired_ensemble_members_match_oracle():
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=3, n_min=5, n_max=12, seed=98)
    mem = make_members(specs, "FP16S", "AB", P)
    e = P.Ensemble(mem)
    e.set_layout("chunked")
    e.set_variant("paired", 4)
    e.step(70)
    for s, g in zip(specs, mem):
        o = oracle.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "ORD32", "FP16S", tau=s.tau)
        flags, node_u = W.cavity(s.n, s.u_lid)
        o.set_geometry(flags, node_u)
        o.set_rho_u()
        o.step(70)
        assert np.array_equal(g.f(), o.f())


def test_ensemble_members_match_oracle():
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=3, n_min=5, n_max=12, seed=99)
    mem = make_members(specs, "FP16S", "AB", P)
    e = P.Ensemble(mem)
    e.step(70)
    for s, g in zip(specs, mem):
        o = oracle.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "ORD32", "FP16S", tau=s.tau)
        flags, node_u = W.cavity(s.n, s.u_lid)
        o.set_geometry(flags, node_u)
        o.set_rho_u()
        o.step(70)
        assert np.array_equal(g.f(), o.f())


def test_member_stepped_outside_is_detected():
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=2, n_min=5, n_max=8)
    mem = make_members(specs, "FP32", "AB", P)
    e = P.Ensemble(mem)
    mem[0].step(1)
    with pytest.raises(P.LBMError) as ei:
        e.step(1)
    assert ei.value.status == 7
    # a member whose copies changed outside (A-A keeps one copy): the
    # ensemble's tables no longer hold its buffers and it refuses to step
    mem2 = make_members(specs, "FP32", "AB", P)
    e2 = P.Ensemble(mem2)
    e2.step(2)
    mem2[1].set_scheme("AA")
    with pytest.raises(P.LBMError) as ei:
        e2.step(1)
    assert ei.value.status == 7
    e2.close()


def _full_ensemble(P, specs, storage, arith):
    mem = []
    for s in specs:
        g = P.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", storage, arith, "AB", tau=s.tau)
        g.set_geometry(W.cavity_flags(s.n))
        g.set_nodes(*W.cavity_lid(s.n, s.u_lid))
        g.set_rho_u()
        mem.append(g)
    return mem, P.Ensemble(mem)


def test_full_ensemble_error_against_fp64():
    """The 512-cavity workload (edges 16..128, splitmix64 seed 20211216):
    FP16S members advanced by the batched launch against the same members in
    FP64, 500 steps; every member's velocity error at 2048 sampled cells is
    stated, and 16 seeded members equal the CPU oracle bit for bit."""
    import paper_2112_08926_gb300 as P
    specs = W.ensemble_cavities(count=512, seed=20211216)
    steps = 500
    lo, elo = _full_ensemble(P, specs, "FP16S", "FP32")
    hi, ehi = _full_ensemble(P, specs, "FP64", "FP64")
    elo.autotune(trial_steps=2)            # trial steps are real steps: match them on the FP64 side
    done = lo[0].info().step
    ehi.step(done)
    elo.step(steps - done)
    ehi.step(steps - done)
    rng = np.random.default_rng(5)
    errs = []
    for s, a, b in zip(specs, lo, hi):
        cells = rng.integers(0, s.n ** 3, 2048)
        ua = np.stack(a.rho_u_cells(cells)[1:])
        ub = np.stack(b.rho_u_cells(cells)[1:])
        errs.append(np.linalg.norm(ua - ub) / max(np.linalg.norm(ub), 1e-300))
    errs = np.array(errs)
    print(f"\n512 cavities, FP32/FP16S vs FP64/FP64 after {steps} steps: relative L2 of u at sampled cells: "
          f"median {np.median(errs):.3e}, 90th percentile {np.percentile(errs, 90):.3e}, max {errs.max():.3e}")
    assert np.median(errs) < 2e-2 and errs.max() < 1e-1
    # 16 seeded members (the smallest edges) against the oracle, bit for bit
    order = np.argsort([s.n for s in specs], kind="stable")[:16]
    for k in order:
        s = specs[k]
        o = oracle.Lattice(s.n, s.n, s.n, "D3Q19", "SRT", "ORD32", "FP16S", tau=s.tau)
        flags, node_u = W.cavity(s.n, s.u_lid)
        o.set_geometry(flags, node_u)
        o.set_rho_u()
        o.step(steps)
        assert np.array_equal(lo[k].f(), o.f()), (k, s)
    elo.close()
    ehi.close()
    for g in lo + hi:
        g.close()
