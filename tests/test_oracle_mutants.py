"""The oracle's pins catch plausible mistakes (no GPU).

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, index or factor), builds it, and runs the fast pin tests
against that build in a child process: at least one pin must fail.  The
mistakes are planted only in a temporary copy on the CPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

# the free-surface branch of the density ghost on a horizontal (y) and on a
# vertical (x) wall
_FS1_Y = "if (bc == BC_FREE && p->fs_order == 1)\n      return 2.0 * rho[(size_t)yb"
_FS1_X = "if (bc == BC_FREE && p->fs_order == 1)\n      return 2.0 * rho[(size_t)y * p->nx + xb]"

MUTANTS = {
    # elastic force with the wrong sign (Eq. 9)
    "lambda_sign": ("Gx = Lambda * bb * gx_rho;", "Gx = -Lambda * bb * gx_rho;"),
    # half-force shift dropped from the physical flux (Eqs. 12, 22)
    "no_half_shift": ("jx = (mx + 0.5 * (Gx + Fx)) / (1.0 + 0.5 * A);", "jx = mx / (1.0 + 0.5 * A);"),
    # equilibrium second-order term with 1/b^4 instead of 1/(2 b^4) (Eq. 14)
    "feq_factor": ("feq[i] = wt[i] * (rho + cj / bb + pn_h / (2.0 * bb * bb));",
                   "feq[i] = wt[i] * (rho + cj / bb + pn_h / (bb * bb));"),
    # P^n without the rho b^2 I shift (Eq. 15)
    "pn_shift": ("double pnxx = pxx - rho * bb, pnyy = pyy - rho * bb, pnxy = pxy;",
                 "double pnxx = pxx, pnyy = pyy, pnxy = pxy;"),
    # forcing prefactor (1 - 1/tau) instead of (1 - 1/(2 tau)) (Eq. 18)
    "force_prefactor": ("(1.0 - 1.0 / (2.0 * tau)) * si[i]", "(1.0 - 1.0 / tau) * si[i]"),
    # density gradient taken along the wrong axis (Eq. 10)
    "grad_axis": ("double gx = 0.5 * (rho_ghost(rho, p, x + 1, y) - rho_ghost(rho, p, x - 1, y));\n        double gy",
                  "double gx = 0.5 * (rho_ghost(rho, p, x, y + 1) - rho_ghost(rho, p, x, y - 1));\n        double gy"),
    # bounce-back returning the incoming instead of the outgoing population (Eq. 36)
    "bb_index": ("double fk = cplane(fs, p, k)[c];\n  if (bc == BC_RIGID) return fk;",
                 "double fk = cplane(fs, p, k)[c];\n  if (bc == BC_RIGID) return cplane(fs, p, i)[c];"),
    # free-surface extrapolation weights swapped (Eq. 39)
    "abb_extrapolation": ("rho_air = 1.5 * rb - 0.5 * ri;", "rho_air = 0.5 * rb + 0.5 * ri;"),
    # constant free-surface extrapolation taking the inner cell (reading of Eq. 39)
    "abb_constant": ("rho_air = rb;\n", "rho_air = ri;\n"),
    # anti-bounce-back without the sign flip (Eq. 38)
    "abb_sign": ("return -fk + 2.0 * wt[k] *", "return fk + 2.0 * wt[k] *"),
    # a diagonal weight off (Sec. 2, D2Q9)
    "weight": ("1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 35.0};"),
    # Ricker with the wrong sign of the quadratic term (Sec. 5)
    "ricker": ("return (1.0 - 2.0 * a) * exp(-a);", "return (1.0 + 2.0 * a) * exp(-a);"),
    # periodic minimum image dropped from the source distance (Sec. 5)
    "min_image": ("if (p->bc_left == BC_PERIODIC) dx -= p->nx * floor(dx / p->nx + 0.5);", ""),
    # sponge depth off by one (absorbing-layer reading)
    "sponge_depth": ("d[0] = p->sp_top - y;", "d[0] = p->sp_top - y + 1;"),
    # density ghosts of Eq. 10 at walls (reading): rigid wall extrapolated
    # linearly instead of mirrored, on a horizontal and on a vertical wall
    "ghost_rigid_linear_y": (_FS1_Y, _FS1_Y.replace("bc == BC_FREE && p->fs_order == 1",
                                                    "bc != BC_FREE || p->fs_order == 1")),
    "ghost_rigid_linear_x": (_FS1_X, _FS1_X.replace("bc == BC_FREE && p->fs_order == 1",
                                                    "bc != BC_FREE || p->fs_order == 1")),
    # ghost set to zero (rigid wall and constant-order free surface)
    "ghost_zero_y": ("    return rho[(size_t)yb * p->nx + x];", "    return 0.0;"),
    "ghost_zero_x": ("    return rho[(size_t)y * p->nx + xb];", "    return 0.0;"),
    # ghost set to zero (linear-order free surface)
    "ghost_zero_fs1_y": ("return 2.0 * rho[(size_t)yb * p->nx + x] - rho[(size_t)yin * p->nx + x];",
                         "return 0.0;"),
    "ghost_zero_fs1_x": ("return 2.0 * rho[(size_t)y * p->nx + xb] - rho[(size_t)y * p->nx + xin];",
                         "return 0.0;"),
    # free-surface ghosts of the two extrapolation orders swapped
    "ghost_fs_swap_y": (_FS1_Y, _FS1_Y.replace("p->fs_order == 1", "p->fs_order == 0")),
    "ghost_fs_swap_x": (_FS1_X, _FS1_X.replace("p->fs_order == 1", "p->fs_order == 0")),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "lbm_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liblbm_oracle_mutant.so"
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    str(mutated), "-o", str(lib), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, LBM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_lattice.py"),
                        os.path.join(ROOT, "tests", "test_oracle_step.py"),
                        os.path.join(ROOT, "tests", "test_oracle_walls.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin failed for mutant {name}:\n{r.stdout[-2000:]}"
