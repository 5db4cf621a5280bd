"""GPU tests of the ensemble path (independent boxes of uneven sizes evolved together).

Every box of an ensemble follows eq. ALCtimestep exactly as a single-box plan with the same
configuration: the ensemble kernels run the same per-row / per-column / per-particle device
code as the single-box kernels, only grouped differently into blocks and launches, and the
deposit sums are integers (order-independent).  So each box's result must equal the
single-box result bit for bit -- and the single-box path is the one checked against the
float64 oracle in test_gpu_parity.py.  The same holds for every launch shape the autotuner
may pick with the single-box FFT factorisation (radix variant 0), for the per-box launch mode
(each box's single-box launches in the step graph) and for graph replay versus direct
launches; the second factorisation (variant 1) agrees to float32 rounding.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# mesh sizes 64, 96, 128, 192 and 256 (every size the ensemble kernels support), two boxes
# of the same size with different seeds, box sizes with the 0.78 Mpc/h cells of the
# 48-box mock ensemble and a different one
BOXES = [(32, 64, 50.0), (48, 96, 75.0), (64, 128, 100.0), (96, 192, 150.0), (128, 256, 200.0), (32, 64, 120.0)]
SEEDS = [11, 12, 13, 14, 15, 16]


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


@pytest.fixture(scope="module")
def ens(cola):
    return cola.Ensemble(BOXES)


@pytest.fixture(scope="module")
def single_runs(cola):
    out = []
    for (n_p, ng, box), seed in zip(BOXES, SEEDS):
        plan = cola.Plan(np_side=n_p, ng=ng, box=box)
        s, v, s1, s2 = plan.run(plan.noise(seed))
        _, delta = plan.density(s, rho=False)
        k, pk, nm = plan.power(delta, 32)
        plan.status()
        out.append(dict(s=s, v=v, s1=s1, s2=s2, delta=delta, pk=pk, nm=nm))
    torch.cuda.synchronize()
    return out


def test_offsets_follow_the_box_sizes(ens):
    assert ens.poff[0] == 0 and ens.moff[0] == 0
    assert list(np.diff(ens.poff)) == [b[0] ** 3 for b in BOXES]
    assert list(np.diff(ens.moff)) == [b[1] ** 3 for b in BOXES]


def test_ensemble_run_equals_single_box_runs(cola, ens, single_runs):
    noise = ens.noise(SEEDS)
    s, v, s1, s2 = ens.run(noise)
    ens.status()
    delta = ens.density(s)
    k, pk, nm = ens.power(delta, 32)
    ens.status()
    torch.cuda.synchronize()
    for b, ref in enumerate(single_runs):
        for name, x in (("s1", s1), ("s2", s2), ("s", s), ("v", v)):
            assert torch.equal(ens.split(x)[b], ref[name]), (b, name)
        assert torch.equal(ens.split_mesh(delta)[b], ref["delta"]), b
        assert torch.equal(pk[b], ref["pk"]) and torch.equal(nm[b], ref["nm"]), b


def run_steps(ens, seeds, nsteps):
    s, v, s1, s2 = ens.ic_2lpt(ens.noise(seeds))
    for i in range(nsteps):
        ens.step(i, s, v, s1, s2)
    ens.step(ens.nsteps, s, v, s1, s2)  # the final kick + L+ as well
    torch.cuda.synchronize()
    return s, v


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("tile_shape", [0, 1])
@pytest.mark.parametrize("blocks_per_sm", [0, 2])
@pytest.mark.parametrize("radix", [0, 1])
def test_every_launch_shape_gives_the_same_result(ens, threads, tile_shape, blocks_per_sm, radix):
    # radix variant 0 is the single-box factorisation: bit-identical; variant 1 factorises the
    # transforms differently, so it agrees to float32 rounding -- amplified where a particle's
    # position lands on the other side of a 2^-16-cell quantisation step (measured after two
    # steps and the final kick: 1.2e-4 cell at most); bound 5e-4 cell and 5e-4 of the rms v
    ens.tuning = (256, 0, 0, 0)
    ref_s, ref_v = run_steps(ens, SEEDS, 2)
    ens.tuning = (threads, tile_shape, blocks_per_sm, radix)
    assert ens.tuning == (threads, tile_shape, blocks_per_sm, radix, 0, 0)
    s, v = run_steps(ens, SEEDS, 2)
    ens.status()
    if radix == 0:
        assert torch.equal(s, ref_s) and torch.equal(v, ref_v)
    else:
        for b, (n_p, ng, box) in enumerate(BOXES):
            sb, rb = ens.split(s)[b], ens.split(ref_s)[b]
            vb, rvb = ens.split(v)[b], ens.split(ref_v)[b]
            assert float((sb - rb).abs().max()) <= 5e-4 * box / ng, b
            assert float((vb - rvb).abs().max()) <= 5e-4 * float(rvb.pow(2).mean().sqrt()), b


@pytest.mark.parametrize("streams", [1, 2, 4])
def test_per_box_launch_mode_gives_the_same_result(ens, streams):
    ens.tuning = (256, 0, 0, 0)
    ref_s, ref_v = run_steps(ens, SEEDS, 2)
    ens.tuning = (128, 0, 0, 0, streams)
    assert ens.tuning == (128, 0, 0, 0, streams, 0)
    for graphs in (True, False):
        ens.use_graphs(graphs)
        s, v = run_steps(ens, SEEDS, 2)
        ens.status()
        assert torch.equal(s, ref_s) and torch.equal(v, ref_v)
    ens.use_graphs(True)
    ens.tuning = (256, 0, 0, 0)


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("mesh_streams", [1, 2, 4])
def test_hybrid_mode_gives_the_same_result(ens, threads, mesh_streams):
    # multi-box binning, gather and kick around every box's own single-box mesh passes (on 1, 2
    # or 4 forked streams): the boxes bin as their plans do, so the result is bit-identical
    ens.tuning = (256, 0, 0, 0)
    ref_s, ref_v = run_steps(ens, SEEDS, 2)
    ens.tuning = (threads, 0, 0, 0, 0, mesh_streams)
    assert ens.tuning == (threads, 0, 0, 0, 0, mesh_streams)
    for graphs in (True, False):
        ens.use_graphs(graphs)
        s, v = run_steps(ens, SEEDS, 2)
        ens.status()
        assert torch.equal(s, ref_s) and torch.equal(v, ref_v)
    ens.use_graphs(True)
    ens.tuning = (256, 0, 0, 0)


def test_graph_replay_equals_direct_launches(cola, ens):
    ens.tuning = (256, 0, 0, 0)
    ens.use_graphs(True)
    s_g, v_g = run_steps(ens, SEEDS, 3)
    s_g2, v_g2 = run_steps(ens, SEEDS, 3)  # second pass replays the recorded graphs
    ens.use_graphs(False)
    s_e, v_e = run_steps(ens, SEEDS, 3)
    ens.use_graphs(True)
    assert torch.equal(s_g, s_e) and torch.equal(v_g, v_e)
    assert torch.equal(s_g2, s_e) and torch.equal(v_g2, v_e)


@pytest.mark.parametrize("launch,mesh_streams,per_step",
                         [(0, 0, 12), (0, 2, 7 + 5 * len(BOXES)), (1, 0, 12 * len(BOXES)), (2, 0, 12 * len(BOXES))])
def test_graph_replay_launch_count_per_step(cola, ens, launch, mesh_streams, per_step):
    # keys, three scan passes, scatter, deposit + x r2c, forward y, z + Green, inverse y,
    # inverse x, gather in bin order, kick/drift: once for all boxes (launch 0), per box (launch
    # 1, 2), or the five mesh passes per box and the rest once (hybrid)
    ens.tuning = (256, 0, 0, 0, launch, mesh_streams)
    s, v, s1, s2 = ens.ic_2lpt(ens.noise(SEEDS))
    ens.step(0, s, v, s1, s2)  # records the graph for these pointers
    torch.cuda.synchronize()
    lib = cola.load_library()
    import ctypes
    c0, c1 = ctypes.c_uint64(), ctypes.c_uint64()
    lib.cola_launch_count(ctypes.byref(c0))
    ens.step(0, s, v, s1, s2)
    lib.cola_launch_count(ctypes.byref(c1))
    assert c1.value - c0.value == per_step
    ens.tuning = (256, 0, 0, 0)


def test_autotuner_picks_the_fastest_candidate(cola, ens):
    s, v, s1, s2 = ens.ic_2lpt(ens.noise(SEEDS))
    best, ms = ens.tune(s, reps=2)
    assert (best.threads, best.tile_shape, best.blocks_per_sm, best.radix, best.launch, best.mesh_streams) == ens.tuning
    assert np.all(ms > 0) and len(ms) == 25
    order = [(t, sh, b, r, 0, 0) for t in (128, 256) for sh in (0, 1) for b in (0, 2) for r in (0, 1)]
    order += [(128, 0, 0, 0, 1, 0), (128, 0, 0, 0, 2, 0), (128, 0, 0, 0, 4, 0)]
    order += [(t, 0, 0, 0, 0, m) for m in (1, 2, 4) for t in (128, 256)]
    assert order[int(np.argmin(ms))] == ens.tuning
    ens.status()


def test_nonfinite_displacement_is_reported_with_its_box(cola, ens):
    s, v, s1, s2 = ens.ic_2lpt(ens.noise(SEEDS))
    ens.split(s)[3][1, 5] = float("nan")
    ens.step(0, s, v, s1, s2)
    with pytest.raises(cola.ColaError) as e:
        ens.status()
    assert "box 3" in str(e.value)
    ens.status()  # cleared
