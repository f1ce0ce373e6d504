"""Pin of the oracle's S1O2 step (Section 2.4, Eqs. s1o2 and flux-operator;
Section 2.3 for the gradient update from the interface state at t^{n+1}).

With the smooth flux and tau = 0, one S1O2 step from fixed data is a
polynomial in dt: the cell average is W^n + dt a + dt^2 b with a = L(W^n)
and b = (1/2) dL/dt (W^n), and the Gauss-Green gradient is linear in dt,
GG(W^c) + dt GG(W_t^c).  For the translating isentropic vortex the exact
cell averages give the targets in closed form: dW/dt and d^2W/dt^2 of the
cell averages of W0(x - t, y), and d/dt of their averaged gradients.  The
coefficients are read off three steps of different dt, and their errors
against the exact derivatives must fall under mesh refinement.

A wrong time coefficient on F1 (dt instead of dt/2, or F1 dropped) leaves
2b a fixed fraction away from d^2W/dt^2 on every mesh; gradients taken from
the interface state at t = 0 or t = dt/2 instead of t^{n+1} leave the
gradient's slope a fixed fraction off.  The second test plants each of
these mistakes in a copy of the oracle and checks that the pin fails."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2109_09965_gb300 import meshgen as MG
from tests import exact

GAM = 1.4
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DELTA = 0.05      # the step's dt values are DELTA, 2 DELTA, 3 DELTA
EPS_T = 1e-3      # central differences in t of the exact cell averages


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def s1o2_coefficient_errors(O, n):
    """Relative errors of one S1O2 step's dt coefficients against the exact
    time derivatives of the vortex's cell averages on an n x n jittered
    triangle mesh of [-5, 5]^2."""
    L = 5.0
    mesh = MG.box(n, n, -L, L, -L, L, jitter=0.1, seed=3, cells="tri", tags=(0, 0, 0, 0))
    om = O.OracleMesh(mesh)
    spec = dict(gamma=GAM, mu=0.0, time_scheme="S1O2",
                bcs=[dict(kind="farfield", rho=1.0, u=(1.0, 0.0), p=1.0)])
    W0, X0 = exact.cell_averages(mesh, exact.isentropic_vortex(GAM))
    steps = []
    for k in (1, 2, 3):
        s = O.OracleSolver(om, spec)
        s.set_state(W0, X0)
        s.highorder_step(k * DELTA)
        steps.append(s.get_state())
    (W1, X1), (W2, X2), (W3, X3) = steps
    a = (4 * W1 - W2 - 3 * W0) / (2 * DELTA)
    b = (W2 - 2 * W1 + W0) / (2 * DELTA ** 2)
    g = (X2 - X1) / DELTA
    Wp, Xp = exact.cell_averages(mesh, exact.isentropic_vortex(GAM, t=EPS_T))
    Wm, Xm = exact.cell_averages(mesh, exact.isentropic_vortex(GAM, t=-EPS_T))
    return {
        # the step really is quadratic (W) and linear (W_x) in dt
        "w_quadratic": rel(W0 + 3 * DELTA * a + 9 * DELTA ** 2 * b, W3),
        "wx_linear": rel(X3, X2 + DELTA * g),
        "a": rel(a, (Wp - Wm) / (2 * EPS_T)),
        "b": rel(2 * b, (Wp - 2 * W0 + Wm) / EPS_T ** 2),
        "grad_slope": rel(g, (Xp - Xm) / (2 * EPS_T)),
    }


def pin_failures(O):
    """Names of the pin's checks that fail for oracle module O."""
    e16, e32 = s1o2_coefficient_errors(O, 16), s1o2_coefficient_errors(O, 32)
    bad = []
    if not (e16["w_quadratic"] < 1e-12 and e32["w_quadratic"] < 1e-12):
        bad.append("w_quadratic")
    if not (e16["wx_linear"] < 1e-10 and e32["wx_linear"] < 1e-10):
        bad.append("wx_linear")
    # dL/dt: about first order in h here (0.48 -> 0.25); the targets are exact
    for key, bar in (("a", 0.06), ("b", 0.35), ("grad_slope", 0.2)):
        if not (e32[key] < bar and e32[key] < 0.6 * e16[key]):
            bad.append(key)
    return bad, e16, e32


def test_s1o2_step_matches_the_exact_time_derivatives(oracle_lib):
    bad, e16, e32 = pin_failures(oracle_lib)
    assert not bad, (bad, e16, e32)


def _oracle_variant(tmp_path, old, new, tag):
    src = open(os.path.join(ROOT, "oracle", "cgks_oracle.c")).read()
    assert src.count(old) == 1, old
    d = tmp_path / tag
    d.mkdir()
    (d / "cgks_oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_{tag}", os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC, mod._LIB_PATH = str(d / "cgks_oracle.c"), str(d / "liboracle.so")
    mod.build(force=True)
    return mod


S1O2_UPDATE = "net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, Rlag);"
S1O2_GRADIENT = "    gauss_green(s, s->Wc, s->Wt, dt, Wxn);\n  } else {"


@pytest.mark.parametrize("tag,old,new,caught_by", [
    ("f1_full_dt", S1O2_UPDATE, S1O2_UPDATE.replace("0.5 * dt", "1.0 * dt"), "b"),
    ("f1_dropped", S1O2_UPDATE, S1O2_UPDATE.replace("0.5 * dt", "0.0 * dt"), "b"),
    ("gradient_at_t0", S1O2_GRADIENT, S1O2_GRADIENT.replace("Wt, dt,", "Wt, 0.0,"), "grad_slope"),
    ("gradient_at_half_dt", S1O2_GRADIENT, S1O2_GRADIENT.replace("Wt, dt,", "Wt, 0.5 * dt,"), "grad_slope"),
])
def test_s1o2_pin_catches_planted_mistakes(oracle_lib, tmp_path, tag, old, new, caught_by):
    bad, e16, e32 = pin_failures(_oracle_variant(tmp_path, old, new, tag))
    assert caught_by in bad, (bad, e16, e32)
