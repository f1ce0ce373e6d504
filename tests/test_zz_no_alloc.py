"""GPU test of cgks_density_residual_noalloc, the entry point for callers
that cannot allocate device memory when they call the library (serving
processes with device memory fixed at start-up, host frameworks that own
all device memory).  Its result must equal the residual that the solver
itself reports through cgks_residual, on two calls in a row sharing the
library's fixed scratch array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_residual_matches_solver_residual():
    import torch
    from paper_2109_09965_gb300 import cgks
    L = cgks.lib()
    mesh = MG.cavity(16)
    spec = dict(gamma=1.4, mu=0.15 / 100, cfl_hi=0.5,
                bcs=[dict(kind="noslip"), dict(kind="noslip", uw=(0.15, 0.0))])
    s = cgks.Solver(cgks.Mesh(mesh), spec)
    W0 = np.zeros((mesh.n_cells, 4))
    W0[:, 0] = 1.0
    W0[:, 3] = 1.0 / 1.4 / 0.4
    s.set_state(W0)
    s.explicit_steps(3)                    # a non-trivial density field first
    stream = torch.cuda.current_stream()
    res_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):                  # two calls in a row share the scratch
        W_old = torch.from_numpy(s.get_state()[0]).cuda()
        s.explicit_steps(1)
        ref, _ = s.residual()              # the existing entry point
        W_new = torch.from_numpy(s.get_state()[0]).cuda()
        torch.cuda.synchronize()
        rc = L.cgks_density_residual_noalloc(C.c_void_p(W_new.data_ptr()), C.c_void_p(W_old.data_ptr()),
                                            mesh.n_cells, C.c_void_p(res_dev.data_ptr()),
                                            C.c_void_p(stream.cuda_stream))
        assert rc == 0
        got = float(res_dev.item())
        assert ref > 0 and abs(got - ref) <= TOL * ref, (call, got, ref)
    # sizes beyond the fixed scratch are refused, not run
    rc = L.cgks_density_residual_noalloc(C.c_void_p(W_new.data_ptr()), C.c_void_p(W_old.data_ptr()),
                                        1_048_577, C.c_void_p(res_dev.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == -1
