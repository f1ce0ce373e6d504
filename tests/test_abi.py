"""CPU checks of the C ABI: the library loads, exports every entry point
declared in include/cgks.h, builds meshes on the host, reproduces the
oracle's sweep order bit for bit, rejects bad meshes, and refuses to run
without a GPU instead of falling back to the CPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cg():
    from paper_2109_09965_gb300 import cgks
    cgks.lib()
    return cgks


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cgks_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(cg):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(cg.lib_path())
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(cg.SIGNATURES), set(names) ^ set(cg.SIGNATURES)


def test_tune_shapes_and_defaults(cg):
    """The autotuner's launch shapes are distinct, legal block sizes, and
    the defaults turn the tuner on (host-only calls, no GPU needed)."""
    shapes = [cg.tune_shape(k) for k in range(cg.TUNE_SHAPES)]
    assert len(set(shapes)) == cg.TUNE_SHAPES
    for bs, ipt, minb in shapes:
        assert bs % 32 == 0 and 64 <= bs <= 256 and 1 <= ipt <= 2 and 1 <= minb
        assert bs * minb <= 2048          # resident threads per SM
    for bad in (-1, cg.TUNE_SHAPES):
        with pytest.raises(cg.CgksError):
            cg.tune_shape(bad)
    P = cg.CgksParams()
    cg.lib().cgks_default_params(C.byref(P))
    assert P.autotune == 1 and P.low_order_fused == 0 and P.use_graph == 1 and P.programmatic_launch == 1
    O = cg.CgksServerOpts()
    cg.lib().cgks_server_default_opts(C.byref(O))
    assert O.autotune == 1 and O.programmatic_launch == 1 and O.max_active == 64


@pytest.mark.parametrize("mesh", [MG.cavity(8), MG.cylinder(24, 3, 5),
                                  MG.box(7, 5, jitter=0.2, seed=2, cells="mixed",
                                         quad_mask=lambda i, j: (i + j) % 3 == 0)],
                         ids=["cavity", "cylinder", "mixed"])
def test_host_mesh_and_ordering_match_oracle(cg, oracle_lib, mesh):
    gm = cg.Mesh(mesh)
    om = oracle_lib.OracleMesh(mesh)
    assert gm.n_faces == om.n_faces
    assert gm.n_colours == om.n_colours
    rcm, col = gm.ordering()
    orcm, ocol = om.ordering()
    np.testing.assert_array_equal(rcm, orcm)
    np.testing.assert_array_equal(col, ocol)
    assert gm.device_bytes > 0


def test_bad_meshes_are_rejected(cg):
    m = MG.box(3, 3)
    # clockwise cell
    bad = MG.box(3, 3)
    nodes = bad.cell_nodes.copy()
    a, b = bad.cell_ptr[0], bad.cell_ptr[1]
    nodes[a:b] = nodes[a:b][::-1]
    bad.cell_nodes = nodes
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(bad)
    assert e.value.status == -3
    # boundary edge without a tag
    bad2 = MG.box(3, 3)
    bad2.bface_ptr = bad2.bface_ptr[:-1]
    bad2.bface_tag = bad2.bface_tag[:-1]
    bad2.bface_nodes = bad2.bface_nodes[:-2]
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(bad2)
    assert e.value.status == -3
    # 2-D cell types handed in as a 3-D mesh are rejected; dim 4 is invalid
    m3 = MG.box(2, 2)
    m3.dim = 3
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(m3)
    assert e.value.status == -3
    m3.dim = 4
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(m3)
    assert e.value.status == -1
    # 3-D: a negatively ordered tet, and a boundary face without a tag
    b3 = MG.box3(2, 2, 2, cells="tet")
    nodes = b3.cell_nodes.copy()
    a = b3.cell_ptr[0]
    nodes[a], nodes[a + 1] = nodes[a + 1], nodes[a]
    b3.cell_nodes = nodes
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(b3)
    assert e.value.status == -3
    c3 = MG.box3(2, 2, 2, cells="hex")
    c3.bface_ptr = c3.bface_ptr[:-1]
    c3.bface_tag = c3.bface_tag[:-1]
    c3.bface_nodes = c3.bface_nodes[:-4]
    with pytest.raises(cg.CgksError) as e:
        cg.Mesh(c3)
    assert e.value.status == -3


@pytest.mark.parametrize("mesh", [MG.box3(3, 2, 2, jitter=0.2, seed=1, cells="tet"),
                                  MG.box3(2, 3, 2, jitter=0.2, seed=2, cells="prism"),
                                  MG.box3(2, 2, 2, jitter=0.1, seed=3, cells="pyramid"),
                                  MG.sphere(1, 3, 2, R_far=4.0)],
                         ids=["tet", "prism", "pyramid", "sphere"])
def test_host_mesh3_and_ordering_match_oracle(cg, mesh):
    from oracle import oracle3 as O3
    gm = cg.Mesh(mesh)
    om = O3.OracleMesh3(mesh)
    assert gm.dim == 3 and gm.nv == 5
    assert gm.n_faces == om.n_faces
    assert gm.n_colours == om.n_colours
    rcm, col = gm.ordering()
    orcm, ocol = om.ordering()
    np.testing.assert_array_equal(rcm, orcm)
    np.testing.assert_array_equal(col, ocol)
    assert gm.device_bytes > 0


def test_no_cpu_fallback_without_gpu(cg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    gm = cg.Mesh(MG.cavity(4))
    with pytest.raises(cg.CgksError) as e:
        cg.Solver(gm, dict(bcs=[dict(kind="noslip"), dict(kind="noslip")]), use_torch=False)
    assert e.value.status == -4


def test_default_params(cg):
    """The C library fills the defaults; reading them back through the
    ctypes mirror checks the mirror's field offsets."""
    P = cg.make_params({})
    assert P.gamma == 1.4 and P.cfl_lo == 1000.0 and P.n_implicit == 6 and P.n_sweeps == 2
    assert P.alpha == 0.5 and P.use_graph == 1
    assert P.autotune == 1 and P.programmatic_launch == 1 and P.flux_lo == 0 and P.flux_hi == 0
    assert P.weno_vars == 0 and P.tau_c1 == 0.01 and P.tau_c2 == 1.0 and P.weno_eps == 0.0 and P.weno_g0 == 0.95
    assert P.stream is None and not P.alloc_ctx


def test_params_mapping(cg):
    P = cg.make_params(dict(flux_hi="full", weno_eps=1e-2, weno_vars="characteristic", tau_c1=0.2, tau_c2=3.0,
                            flux_lo="lf", bcs=[dict(kind="dirichlet", rho=1.7, u=(2.6, -0.5), p=1.5),
                                               dict(kind="outflow")]))
    assert (P.flux_hi, P.weno_vars, P.flux_lo) == (cg.FLUX_FULL, cg.WENO_CHARACTERISTIC, cg.FLUX_LF)
    assert (P.weno_eps, P.tau_c1, P.tau_c2, P.weno_g0) == (1e-2, 0.2, 3.0, 0.95)
    assert P.n_bc == 2 and P.bc[0].kind == cg.BC_DIRICHLET and P.bc[1].kind == cg.BC_OUTFLOW
    assert (P.bc[0].rho, P.bc[0].u[0], P.bc[0].u[1], P.bc[0].u[2], P.bc[0].p) == (1.7, 2.6, -0.5, 0.0, 1.5)


def test_empty_mesh_is_rejected(cg):
    """A mesh without cells or nodes is an invalid argument, in 2-D and
    3-D, before anything touches a device."""
    import types
    for dim in (2, 3):
        e = types.SimpleNamespace(dim=dim, nodes=np.zeros((0, dim)), cell_type=np.zeros(0, np.uint8),
                                  cell_ptr=np.zeros(1, np.int64), cell_nodes=np.zeros(0, np.int64),
                                  bface_ptr=np.zeros(1, np.int64), bface_nodes=np.zeros(0, np.int64),
                                  bface_tag=np.zeros(0, np.int32), n_cells=0, n_nodes=0, n_bfaces=0)
        with pytest.raises(cg.CgksError) as err:
            cg.Mesh(e)
        assert err.value.status == -1



def test_full_flux_weno_and_new_boundaries_validated_before_the_device(cg):
    """Parameter checks run before any device call: bad values and options
    the 3-D path does not have (characteristic WENO, Dirichlet / outflow)
    are invalid arguments (-1); valid ones reach the device step (-4 here,
    without a GPU)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    mesh, spec, _ = MG.shock_reflection_case(6, 2, weno_eps=1e-2)
    gm = cg.Mesh(mesh)

    def status(m, sp):
        with pytest.raises(cg.CgksError) as e:
            cg.Solver(m, sp, use_torch=False)
        return e.value.status
    assert status(gm, spec) == -4
    for bad in (dict(weno_eps=-1.0), dict(tau_c1=-0.1), dict(tau_c2=float("nan")), dict(weno_g0=1.0)):
        assert status(gm, dict(spec, **bad)) == -1, bad
    g3 = cg.Mesh(MG.box3(2, 2, 2, cells="hex"))
    ok3 = dict(gamma=1.4, bcs=[dict(kind="slip")] * 6)
    assert status(g3, ok3) == -4
    for extra in (dict(weno_eps=1e-2, weno_vars="characteristic"), dict(bcs=[dict(kind="outflow")] * 6),
                  dict(bcs=[dict(kind="dirichlet", rho=1.0, p=1.0)] * 6)):
        assert status(g3, dict(ok3, **extra)) == -1, extra
    assert status(g3, dict(ok3, flux_hi="full", weno_eps=1e-2)) == -4
