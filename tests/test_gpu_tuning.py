"""The launch-shape autotuner on the GPU.

Every tunable kernel (reconstruction, gas-kinetic face flux, KFVS face flux,
colour sweep) computes each cell or face with the same arithmetic whatever
its launch shape, so results must agree BIT FOR BIT across shapes, between
tuned and untuned solvers, and between the tuning cycles (plain launches)
and the graph replays that follow them.  The tuner must try every shape of
every kernel the cycle launches, time it, and keep the fastest.
"""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact
from tests.test_gpu_parity import case

pytestmark = pytest.mark.gpu
GAM = 1.4
UNITS = 3 * 5        # tuning units per kernel: 3 rounds of 5 shapes


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_09965_gb300 import cgks
    cgks.lib()
    return cgks


def case3():
    mesh = MG.box3(3, 2, 3, jitter=0.2, seed=2, cells="prism", tags=(2, 2, 2, 2, 0, 1))
    vel = (0.2, 0.0, 0.0)
    spec = dict(gamma=GAM, mu=0.01,
                bcs=[dict(kind="slip"), dict(kind="noslip", uw=(0.1, 0.05, 0.0)),
                     dict(kind="farfield", rho=1.0, u=vel, p=1 / GAM)])
    rho, p = 1.0, 1 / GAM
    W = np.tile([rho, rho * vel[0], rho * vel[1], rho * vel[2], p / (GAM - 1) + 0.5 * rho * vel[0] ** 2],
                (mesh.n_cells, 1))
    rng = np.random.default_rng(11)
    W[:, 0] *= 1 + 0.02 * rng.standard_normal(mesh.n_cells)
    return mesh, spec, (W, None)


def run(cg, mesh, spec, state, cycles, **over):
    s = cg.Solver(cg.Mesh(mesh), dict(spec, **over))
    s.set_state(*state)
    h = s.pmg_cycle(cycles)
    return s, s.get_state(), h


def test_shapes_are_distinct_and_valid(cg):
    shapes = [cg.tune_shape(k) for k in range(cg.TUNE_SHAPES)]
    assert len(set(shapes)) == cg.TUNE_SHAPES
    for bs, ipt, minb in shapes:
        assert bs % 32 == 0 and 64 <= bs <= 256 and ipt >= 1 and minb >= 1
    with pytest.raises(cg.CgksError):
        cg.tune_shape(cg.TUNE_SHAPES)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dim", [2, 3])
def test_every_shape_gives_bitwise_equal_results(cg, dim, precision):
    if dim == 2:
        mesh, spec, state = case("mixed_slip_farfield")
    else:
        mesh, spec, state = case3()
    spec = dict(spec, precision=precision, autotune=0)
    ref = None
    for shp in range(cg.TUNE_SHAPES):
        s = cg.Solver(cg.Mesh(mesh), spec)
        s.set_tuning([shp] * cg.TUNE_KERNELS)
        t = s.tuning()
        assert all(t[k]["shape"] == shp and t[k]["done"] for k in cg.TUNE_NAMES)
        s.set_state(*state)
        h = s.pmg_cycle(3)
        s.explicit_steps(1)
        W, Wx = s.get_state()
        if ref is None:
            ref = (W, Wx, h)
            continue
        assert np.array_equal(W, ref[0]) and np.array_equal(Wx, ref[1]), shp
        assert np.array_equal(h, ref[2]), shp


@pytest.mark.parametrize("dim", [2, 3])
def test_tuner_times_every_shape_and_keeps_the_fastest(cg, dim):
    if dim == 2:
        mesh, spec, state = case("cylinder_viscous")
    else:
        mesh, spec, state = case3()
    n = UNITS + 5
    tuned, (Wt, Xt), ht = run(cg, mesh, spec, state, n, autotune=1)
    fixed, (Wf, Xf), hf = run(cg, mesh, spec, state, n, autotune=0)
    assert np.array_equal(Wt, Wf) and np.array_equal(Xt, Xf) and np.array_equal(ht, hf)
    t = tuned.tuning()
    for k in cg.TUNE_NAMES:
        ms = t[k]["ms"]
        assert t[k]["done"], (k, t[k])
        assert all(x > 0.0 for x in ms), (k, ms)
        assert ms[t[k]["shape"]] == min(ms), (k, t[k])
    # without the tuner the default shapes stay and nothing is timed
    f = fixed.tuning()
    assert all(f[k]["done"] and not any(f[k]["ms"]) for k in cg.TUNE_NAMES)
    # the tuned solver replays its graph after tuning: same launches per cycle
    assert tuned.launches_per_call(True) == fixed.launches_per_call(True)


def test_tuning_spans_calls_and_explicit_steps(cg):
    """Tuning units are counted per kernel across calls; explicit steps tune
    only the kernels they launch."""
    mesh, spec, state = case("cavity8")
    s = cg.Solver(cg.Mesh(mesh), dict(spec, time_scheme="S2O4"))
    s.set_state(*state)
    s.explicit_steps(UNITS - 1)
    t = s.tuning()
    assert not t["k_face"]["done"] and not t["k_lo_face"]["done"]
    s.explicit_steps(1)
    t = s.tuning()
    assert t["k_face"]["done"] and t["k_recon"]["done"]
    assert not t["k_lo_face"]["done"] and not t["k_sweep"]["done"]
    assert not any(t["k_sweep"]["ms"])
    for _ in range(UNITS):
        s.pmg_cycle(1)
    t = s.tuning()
    assert all(t[k]["done"] for k in cg.TUNE_NAMES), t
    # the same state as an untuned solver after the same calls
    r = cg.Solver(cg.Mesh(mesh), dict(spec, time_scheme="S2O4", autotune=0))
    r.set_state(*state)
    r.explicit_steps(UNITS)
    r.pmg_cycle(UNITS)
    assert np.array_equal(s.get_state()[0], r.get_state()[0])


def test_set_tuning_rejects_bad_shapes(cg):
    mesh, spec, state = case("cavity8")
    s = cg.Solver(cg.Mesh(mesh), spec)
    with pytest.raises(cg.CgksError):
        s.set_tuning([0, 0, 0, cg.TUNE_SHAPES])
    with pytest.raises(cg.CgksError):
        s.set_tuning([-1, 0, 0, 0])
    with pytest.raises(ValueError):
        s.set_tuning([0, 0, 0])


def test_server_batch_is_tuned(cg):
    """The server tunes its batch in its first cycles; the solves still
    match standalone runs bit for bit."""
    reqs = []
    for name in ("cavity8", "cylinder_viscous"):
        mesh, spec, (W, _) = case(name)
        reqs.append((mesh, dict(spec, cfl_hi=0.4), W))
    K = UNITS + 2
    srv = cg.Server(4 << 30, max_active=4, max_cycles=K)
    assert not srv.tuning()["k_face"]["done"]
    meshes = [cg.Mesh(m) for m, _, _ in reqs]
    ids = [srv.submit(gm, spec, W, 1e-300) for gm, (_, spec, W) in zip(meshes, reqs)]
    for _ in range(K):
        srv.step()
    t = srv.tuning()
    assert all(t[k]["done"] for k in cg.TUNE_NAMES), t
    for rid, gm, (mesh, spec, W) in zip(ids, meshes, reqs):
        st, Wb = srv.poll(rid)
        s = cg.Solver(gm, dict(spec, autotune=0))
        s.set_state(W)
        s.pmg_cycle(K)
        assert np.array_equal(Wb, s.get_state()[0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dim", [2, 3])
def test_programmatic_launch_is_bitwise_equal(cg, dim, precision):
    """Programmatic dependent launch only moves when a kernel is scheduled;
    each kernel still waits on the device for its predecessor, so cycles,
    explicit steps and the server give identical results with it on or off,
    replayed from a graph or launched one by one."""
    if dim == 2:
        mesh, spec, state = case("cylinder_viscous")
    else:
        mesh, spec, state = case3()
    out = []
    for pdl, graph in ((1, 1), (0, 1), (1, 0)):
        s = cg.Solver(cg.Mesh(mesh), dict(spec, precision=precision, programmatic_launch=pdl, use_graph=graph))
        s.set_state(*state)
        h = s.pmg_cycle(UNITS + 4)
        s.explicit_steps(3)
        out.append((s.get_state(), h))
    for (W, X), h in out[1:]:
        assert np.array_equal(W, out[0][0][0]) and np.array_equal(X, out[0][0][1])
        assert np.array_equal(h, out[0][1])
