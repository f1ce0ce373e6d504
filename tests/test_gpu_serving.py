"""Batched solves and the serving loop (continuous batching) on the GPU.

A batch concatenates several solves into one index space; every solve's
arithmetic is the same as running it alone, so the states and residuals
must agree BIT FOR BIT with a standalone solver after the same number of
V-cycles, whatever the batch composition, admission order or rebuilds in
between.  Admission must keep the device bytes of the active batch within
the budget.
"""
import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact
from tests.test_gpu_parity import case

pytestmark = pytest.mark.gpu
GAM = 1.4
NEVER = 1e-300   # residual drop no solve reaches: every solve runs max_cycles


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2109_09965_gb300 import cgks
    cgks.lib()
    return cgks


def requests():
    """Four different solves: walls, far field, mixed cells, viscous and
    inviscid, different sizes (several padding remainders)."""
    out = []
    for name in ("cavity8", "mixed_slip_farfield", "cylinder_viscous", "linear_fallback"):
        mesh, spec, (W, _) = case(name)
        spec = dict(spec, cfl_hi=0.4)
        out.append((name, mesh, spec, W))
    return out


def standalone(cg, mesh, spec, W, cycles, precision):
    gm = cg.Mesh(mesh)
    s = cg.Solver(gm, dict(spec, precision=precision))
    s.set_state(W)
    hist = s.pmg_cycle(cycles)
    Wf, _ = s.get_state()
    return Wf, hist


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_standalone_bitwise(cg, precision):
    K = 6
    reqs = requests()
    srv = cg.Server(8 << 30, precision=precision, max_active=8, max_cycles=K)
    meshes = [cg.Mesh(m) for _, m, _, _ in reqs]
    ids = [srv.submit(gm, spec, W, NEVER) for gm, (_, _, spec, W) in zip(meshes, reqs)]
    for _ in range(K):
        assert srv.step() == len(reqs)
    for rid, (name, mesh, spec, W) in zip(ids, reqs):
        st, Wb = srv.poll(rid)
        assert st["state"] == "stopped" and st["cycles"] == K, (name, st)
        Ws, hist = standalone(cg, mesh, spec, W, K, precision)
        assert np.array_equal(Wb, Ws), (name, np.abs(Wb - Ws).max())
        assert st["res_last"] == hist[-1] and st["res_first"] == hist[0], name
    assert srv.step() == 0
    info = srv.info()
    assert info["n_active"] == 0 and info["n_queued"] == 0
    assert 0 < info["device_bytes"] <= 8 << 30


def test_staggered_admission_and_budget(cg):
    """A budget for about three of four equal solves and a late submission
    mid-run: solves are admitted as space frees up, retired ones leave
    holes that later ones reuse, continuing solves keep running in place,
    the device bytes stay within the budget, and every result is bitwise
    the standalone one."""
    K = 5
    reqs = []
    for k in range(5):
        mesh = MG.cavity(24, jitter=0.1, seed=10 + k)
        lid = 0.1 + 0.02 * k
        spec = dict(gamma=GAM, mu=lid / 400.0, bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(lid, 0.0))])
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
        reqs.append((f"cavity24_{k}", mesh, spec, W))
    meshes = [cg.Mesh(m) for _, m, _, _ in reqs]
    probe = cg.Server(1 << 30, max_cycles=K)
    fp = probe.footprint(meshes[0])
    probe.close()
    budget = int(3.2 * fp)
    srv = cg.Server(budget, max_active=8, max_cycles=K)
    ids = [srv.submit(gm, spec, W, NEVER) for gm, (_, _, spec, W) in zip(meshes[:4], reqs[:4])]
    late = None
    steps, counts = 0, []
    while True:
        n = srv.step()
        info = srv.info()
        assert info["device_bytes"] <= budget
        counts.append(n)
        steps += 1
        if steps == 3:
            _, _, spec, W = reqs[4]
            late = srv.submit(meshes[4], spec, W, NEVER)
        if n == 0 and info["n_queued"] == 0 and late is not None:
            break
        assert steps < 100
    assert 1 <= max(counts) <= 3
    for rid, (name, mesh, spec, W) in zip(ids + [late], reqs):
        st, Wb = srv.poll(rid)
        assert st["state"] == "stopped" and st["cycles"] == K, (name, st)
        assert st["t_submit"] <= st["t_admit"] <= st["t_done"]
        Ws, hist = standalone(cg, mesh, spec, W, K, "fp64")
        assert np.array_equal(Wb, Ws), (name, np.abs(Wb - Ws).max())
        assert st["res_last"] == hist[-1]


def test_convergence_retires_and_poll_steps(cg):
    """A viscous cylinder converges by 3 decades and retires on its own;
    poll with a timeout drives the server; an oversize request is rejected."""
    mesh = MG.cylinder(24, 4, 6, growth=1.2, R_far=5.0)
    spec = dict(gamma=GAM, mu=0.01,
                bcs=[dict(kind="noslip"), dict(kind="farfield", rho=1.0, u=(0.38, 0.0), p=1 / GAM)])
    W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.38, 0.0, 1 / GAM), (mesh.n_cells, 1))
    gm = cg.Mesh(mesh)
    srv = cg.Server(1 << 30, max_cycles=5000)
    rid = srv.submit(gm, spec, W, 1e-3)
    st, Wf = srv.poll(rid, timeout_ms=120000)
    assert st["state"] == "converged", st
    assert st["res_last"] <= 1e-3 * st["res_first"]
    Ws, hist = standalone(cg, mesh, spec, W, st["cycles"], "fp64")
    assert np.array_equal(Wf, Ws)
    assert np.all(hist[1:-1] > 1e-3 * hist[0])   # not converged earlier
    tiny = cg.Server(1 << 20)
    with pytest.raises(cg.CgksError) as e:
        tiny.submit(gm, spec, W, 1e-3)
    assert e.value.status == -7
    st, Wr = tiny.poll(max(tiny.n_cells))
    assert st["state"] == "rejected" and Wr is None


def test_diverged_solve_does_not_disturb_others(cg):
    """A solve started from a state with negative pressure is reported
    diverged after its first cycle; the solves batched with it carry on
    bitwise unchanged."""
    K = 4
    reqs = requests()[:2]
    meshes = [cg.Mesh(m) for _, m, _, _ in reqs]
    srv = cg.Server(8 << 30, max_cycles=K)
    ids = [srv.submit(gm, spec, W, NEVER) for gm, (_, _, spec, W) in zip(meshes, reqs)]
    bad_mesh = MG.cavity(6)
    bad_W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (bad_mesh.n_cells, 1))
    bad_W[:, 3] = 0.01 * bad_W[:, 3]
    bad_W[:, 1] = 0.5        # kinetic energy above total energy: p < 0
    bad = srv.submit(cg.Mesh(bad_mesh), dict(gamma=GAM, mu=0.001,
                                             bcs=[dict(kind="noslip"), dict(kind="noslip")]), bad_W, NEVER)
    for _ in range(K + 1):
        srv.step()
    st, _ = srv.poll(bad)
    assert st["state"] == "diverged" and st["cycles"] == 1
    for rid, (name, mesh, spec, W) in zip(ids, reqs):
        st, Wb = srv.poll(rid)
        Ws, _ = standalone(cg, mesh, spec, W, K, "fp64")
        assert np.array_equal(Wb, Ws), name


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_admitted_into_a_diverged_solves_space(cg, precision):
    """A solve that diverges leaves NaN in its part of the arena; the solves
    admitted into that space afterwards (one of the same size, one smaller,
    so that its padding cells cover stale NaN) must still be bitwise the
    standalone ones."""
    K = 6
    def cavity(n, seed, lid):
        mesh = MG.cavity(n, jitter=0.1, seed=seed)
        spec = dict(gamma=GAM, mu=lid / 400.0, bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(lid, 0.0))])
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
        return mesh, spec, W
    good = cavity(24, 20, 0.1)
    bad_mesh, bad_spec, bad_W = cavity(24, 21, 0.1)
    bad_W[:, 3] = 0.01 * bad_W[:, 3]
    bad_W[:, 1] = 0.5        # kinetic energy above total energy: p < 0
    late = [cavity(24, 22, 0.12), cavity(21, 23, 0.14)]
    probe = cg.Server(1 << 30, precision=precision, max_cycles=K)
    fp = probe.footprint(cg.Mesh(good[0]))
    probe.close()
    srv = cg.Server(int(4 * fp), precision=precision, max_active=2, max_cycles=K)
    g = srv.submit(cg.Mesh(good[0]), good[1], good[2], NEVER)
    b = srv.submit(cg.Mesh(bad_mesh), bad_spec, bad_W, NEVER)
    for _ in range(3):
        srv.step()
        st, _ = srv.poll(b)
        if st["state"] != "queued":
            break
    assert st["state"] == "diverged" and st["cycles"] == 1, st
    ids = [srv.submit(cg.Mesh(m), sp, W, NEVER) for m, sp, W in late]
    for _ in range(4 * K):
        if srv.step() == 0 and srv.info()["n_queued"] == 0:
            break
    for rid, (m, sp, W) in zip([g] + ids, [good] + late):
        st, Wb = srv.poll(rid)
        assert st["state"] == "stopped" and st["cycles"] == K, st
        Ws, hist = standalone(cg, m, sp, W, K, precision)
        assert np.array_equal(Wb, Ws), np.nanmax(np.abs(Wb - Ws))
        assert st["res_last"] == hist[-1]


def test_many_solves_use_cell_lists(cg):
    """More solves than the sweep's per-launch range table holds (64): the
    sweeps switch to cell lists; results stay bitwise the standalone ones."""
    K = 3
    srv = cg.Server(8 << 30, max_active=80, max_cycles=K)
    cases = []
    for k in range(70):
        mesh = MG.cavity(3, jitter=0.1, seed=100 + k)
        lid = 0.1 + 0.001 * k
        spec = dict(gamma=GAM, mu=lid / 100.0,
                    bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(lid, 0.0))])
        W = np.tile(exact.cons_from_prim(GAM, 1.0, 0.0, 0.0, 1 / GAM), (mesh.n_cells, 1))
        cases.append((mesh, spec, W, srv.submit(cg.Mesh(mesh), spec, W, NEVER)))
    for _ in range(K):
        assert srv.step() == 70
    for mesh, spec, W, rid in (cases[0], cases[33], cases[69]):
        st, Wb = srv.poll(rid)
        assert st["state"] == "stopped"
        Ws, _ = standalone(cg, mesh, spec, W, K, "fp64")
        assert np.array_equal(Wb, Ws)


def test_per_request_cycle_cap(cg):
    """A request's own cycle cap stops it early; the others keep running."""
    reqs = requests()[:2]
    meshes = [cg.Mesh(m) for _, m, _, _ in reqs]
    srv = cg.Server(8 << 30, max_cycles=6)
    a = srv.submit(meshes[0], reqs[0][2], reqs[0][3], NEVER, max_cycles=2)
    b = srv.submit(meshes[1], reqs[1][2], reqs[1][3], NEVER)
    counts = [srv.step() for _ in range(7)]
    assert counts == [2, 2, 1, 1, 1, 1, 0]
    assert srv.poll(a)[0]["cycles"] == 2 and srv.poll(b)[0]["cycles"] == 6
    Ws, _ = standalone(cg, reqs[0][1], reqs[0][2], reqs[0][3], 2, "fp64")
    assert np.array_equal(srv.poll(a)[1], Ws)


LIMITED = dict(flux_hi="full", weno_eps=1e-2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_flux_classes_in_one_batch(cg, precision):
    """Smooth and limited requests (the full flux of Eq. (2nd-flux) with
    compact WENO, Section 4's setting for transonic flow) share one batch:
    each class's launches skip the other class's solves, and every result
    is bitwise the standalone solver's with the same settings."""
    K = 5
    reqs = requests()
    reqs = [(n, m, dict(s, **LIMITED) if k % 2 else s, W) for k, (n, m, s, W) in enumerate(reqs)]
    srv = cg.Server(8 << 30, precision=precision, max_active=8, max_cycles=K)
    meshes = [cg.Mesh(m) for _, m, _, _ in reqs]
    ids = [srv.submit(gm, spec, W, NEVER) for gm, (_, _, spec, W) in zip(meshes, reqs)]
    for _ in range(K):
        assert srv.step() == len(reqs)
    for rid, (name, mesh, spec, W) in zip(ids, reqs):
        st, Wb = srv.poll(rid)
        assert st["state"] == "stopped" and st["cycles"] == K, (name, st)
        Ws, hist = standalone(cg, mesh, spec, W, K, precision)
        assert np.array_equal(Wb, Ws), (name, spec.get("flux_hi"), np.abs(Wb - Ws).max())
        assert st["res_last"] == hist[-1]
    # a limited request with other constants, or characteristic WENO, is refused
    name, mesh, spec, W = reqs[0]
    for bad in (dict(LIMITED, weno_eps=1e-3), dict(LIMITED, weno_vars="characteristic"), dict(flux_hi="full")):
        with pytest.raises(cg.CgksError):
            srv.submit(meshes[0], dict(spec, **bad), W, NEVER)


@pytest.mark.parametrize("limited", [False, True])
def test_server_result_matches_oracle(cg, oracle_lib, limited):
    """A served FP64 request against the CPU oracle: a viscous cylinder run
    for 6 batched V-cycles (the per-request cap), its final state within the
    FP64 bar of the oracle's 6 V-cycles; smooth and limited classes, each
    batched with a request of the other class."""
    O = oracle_lib
    K = 6
    _, mesh, spec, W = requests()[2]                     # cylinder_viscous
    other = requests()[0]
    if limited:
        spec = dict(spec, **LIMITED)
    else:
        other = (other[0], other[1], dict(other[2], **LIMITED), other[3])
    srv = cg.Server(8 << 30, precision="fp64", max_active=4, max_cycles=K)
    rid = srv.submit(cg.Mesh(mesh), spec, W, NEVER)
    srv.submit(cg.Mesh(other[1]), other[2], other[3], NEVER)
    for _ in range(K):
        srv.step()
    st, Wb = srv.poll(rid)
    assert st["state"] == "stopped" and st["cycles"] == K
    o = O.OracleSolver(O.OracleMesh(mesh), spec)
    o.set_state(W)
    h = o.pmg_cycles(K)
    Wo, _ = o.get_state()
    e = np.linalg.norm(Wb - Wo) / np.linalg.norm(Wo)
    assert e < 1e-12, e
    assert abs(st["res_last"] - h[-1]) <= 1e-9 * h[-1]
