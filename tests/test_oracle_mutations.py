"""The pins are sensitive: plant plausible mistakes in a copy of the oracle and check that the pin
suite fails for every one of them (CPU only; the mutated copy is built in a temporary folder)."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "eq11_sign": ("dLdp += gm * (image[pa * C + c] - image[pb * C + c]);",
                  "dLdp += gm * (image[pb * C + c] - image[pa * C + c]);"),
    "eq11_half": ("double gm = 0.5 * (", "double gm = 1.0 * ("),
    "overhang_foreground": ("fg = a_in_b ? 0 : 1;", "fg = a_in_b ? 1 : 0;"),
    "eq12_sign": ("double dpdr_a = -nB[1] / den_a;", "double dpdr_a = nB[1] / den_a;"),
    "eq12_slice_axis": ("double nA[2] = {NA[axis], NA[2]}", "double nA[2] = {NA[1 - axis], NA[2]}"),
    "gather_pixel": ("else gather(scr, tris, tb, xb, yb, g, grad_scr, m, grad_abs);",
                     "else gather(scr, tris, tb, xa, ya, g, grad_scr, m, grad_abs);"),
    "perspective_bary": ("b[i] = ddiv(dmul(lam[i], z[i]), s);", "b[i] = lam[i];"),
    "depth_derivative": ("I[sh->depth_ch] = ddiv(dconst(1.0), s);", "I[sh->depth_ch] = dconst(1.0 / s.v);"),
    "dual_quotient_rule": ("(a.d[k] * b.v - a.v * b.d[k])", "(a.d[k] * b.v + a.v * b.d[k])"),
    "texture_fraction": ("dual fx = dsub(x, dconst(x0));", "dual fx = dconst(x.v - x0);"),
    "top_left_rule": ("if (!(ga > 0 || (ga == 0 && gb > 0))) return 0;", "if (!(ga >= 0)) return 0;"),
    "depth_tie_break": ("(z == z1[p] && t < index[p])", "(z == z1[p] && t > index[p])"),
    "projection_operand": ("xs = (cam->fx * Xc) * zeta + cam->cx;", "xs = (cam->fx * Yc) * zeta + cam->cx;"),
    "backface_sign": ("return (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0) > 0;",
                      "return (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0) < 0;"),
    "forward_grad_half": ("const double h = 0.5 * (image[pa * C + c] - image[pb * C + c]);",
                          "const double h = 1.0 * (image[pa * C + c] - image[pb * C + c]);"),
    "forward_grad_axis": ("dpdt = dr[axis];", "dpdt = dr[1 - axis];"),
    "project_jvp_depth": ("o[2] = -dZ * iz * iz;", "o[2] = dZ * iz * iz;"),
    "crossing_weight_order": ("wout[0] = 1.0 - u; wout[1] = u;", "wout[0] = u; wout[1] = 1.0 - u;"),
    "crossing_first_edge": ("(__int128)eF * bden < (__int128)bnum * (eF - eO)",
                            "(__int128)eF * bden > (__int128)bnum * (eF - eO)"),
    "pixel_depth_reciprocal": ("Z = 1.0 / s;", "Z = s;"),
    "pixel_bary_screen_linear": ("for (int i = 0; i < 3; ++i) b[i] = lam[i] * scr[3 * tri[i] + 2] / s;",
                                 "for (int i = 0; i < 3; ++i) b[i] = lam[i];"),
    "texel_eps_too_small": ("double eps = n * 32.0 * ulp * ext", "double eps = n * 2.0 * ulp * ext"),
    "texel_clamp_edge": ("amb = fabs(xc) <= eps || fabs(xc - (n - 1)) <= eps ||",
                         "amb = fabs(xc - (n - 1)) <= eps ||"),
    "project_backward_transpose": ("grad_verts[3 * v + 0] += R[0] * gX + R[3] * gY + R[6] * gZ;",
                                   "grad_verts[3 * v + 0] += R[0] * gX + R[1] * gY + R[2] * gZ;"),
}


def _run_mutation(name: str, folder: str):
    """Builds the oracle with mutation `name` in `folder` and runs the pin suites against it; returns
    (pytest's exit code, the tail of its output)."""
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name  # the first occurrence: the backward (a copy may sit in the forward gradients)
    mutated = os.path.join(folder, "oracle_mut.c")
    with open(mutated, "w") as f:
        f.write(src.replace(old, new, 1))
    lib = os.path.join(folder, "liboracle_mut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", lib, mutated, "-lm"],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_forward.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutation_results(tmp_path_factory):
    """Every mutation's pin run, several at once (each in its own process and folder)."""
    from concurrent.futures import ThreadPoolExecutor

    folders = {n: str(tmp_path_factory.mktemp("mut_" + n)) for n in MUTATIONS}
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        futures = {n: ex.submit(_run_mutation, n, folders[n]) for n in sorted(MUTATIONS)}
        return {n: f.result() for n, f in futures.items()}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, mutation_results):
    rc, out = mutation_results[name]
    assert rc != 0, f"mutation {name} survived the pins:\n{out}"
