"""Writes the oracle regression fixtures of tests/golden/ (run from the
repository root: python tests/golden/make_golden.py).

The paper prints no worked example of the scheme's values, so these
fixtures are the FP64 oracle's own output on small seeded cases.  They are
not an independent pin (the pins are in tests/test_oracle_*pins.py); they
make any later change of the oracle's arithmetic visible, so that the
change has to be made, with its justification, together with a rewrite of
the fixture by this script.  Only oracle/ is called.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402

CASES = {
    # name: (dims, bc, form, solver)
    "cavity_6x5x4_advective_jacobi": ((6, 5, 4), "cavity", "advective", "jacobi"),
    "periodic_8x4x4_flux_multigrid": ((8, 4, 4), "periodic", "flux", "mg"),
    # the discrete adjoint of two Jacobi-solve steps: gradients of
    # L = 1/2 sum u_T^2 with respect to u_0, p_0 and nu
    "cavity_6x5x4_flux_adjoint": ((6, 5, 4), "cavity", "flux", "adjoint"),
}

HEADERS = {
    "jacobi": "2 RK2 steps;\n# u, v, w, p interiors",
    "mg": "2 RK2 steps;\n# u, v, w, p interiors",
    "adjoint": "gradient of L = 1/2 |u_T|^2 after 2 RK2 steps;\n"
               "# dL/du_0, dL/dv_0, dL/dw_0, dL/dp_0 interiors, then dL/dnu",
}


def run_case(name):
    dims, bc, form, solver = CASES[name]
    h = tuple(1.0 / d for d in dims)
    rng = np.random.default_rng(20)
    fields = {c: 0.1 * rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}
    o = Oracle(dims, ghost=1, h=h, bc=bc, nu=0.05, form=form)
    u, p = o.state(fields)
    dt = 0.05 * min(h)
    if solver == "adjoint":
        _, du, dp, dnu = o.gradient(u, p, dt, 5, 2, lambda ut: (
            0.5 * sum(float((a * a).sum()) for a in ut), [a.copy() for a in ut]))
        return np.concatenate([a.ravel() for a in du + [dp]] + [[dnu]])
    if solver == "jacobi":
        o.run(u, p, dt, 5, 2)
    else:
        o.rk2_step_mg(u, p, dt, 2, steps=2)
    return np.concatenate([o.interior(a).ravel() for a in u + [p]])


def path(name):
    return os.path.join(HERE, "oracle_%s.txt" % name)


if __name__ == "__main__":
    for name, (dims, bc, form, solver) in CASES.items():
        vals = run_case(name)
        with open(path(name), "w") as f:
            f.write("# FP64 oracle, %s grid %s, %s form, %s pressure solve, %s "
                    "(z, y, x order), written by make_golden.py\n"
                    % (bc, "x".join(map(str, dims)), form,
                       "jacobi" if solver == "adjoint" else solver, HEADERS[solver]))
            for v in vals:
                f.write("%.17e\n" % v)
        print("wrote", path(name), len(vals))
