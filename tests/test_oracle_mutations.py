"""The oracle's pins catch plausible mistakes.

Each case plants one slip in a copy of the oracle source (on the CPU),
compiles it to a temporary library and runs the pin tests (including the
whole-solve cross-check against tests/numpy_solve.py) against it: at least
one pin must fail.  This checks the pins, not the CUDA path.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mppi_oracle.c")

MUTATIONS = [
    ("philox round: high words swapped",
     "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;"),
    ("uniform offset 1/2 instead of 1",
     "((double)(x >> 8) + 1.0)", "((double)(x >> 8) + 0.5)"),
    ("box-muller cos/sin swapped",
     "z[0] = r * cos(two_pi * ub);", "z[0] = r * sin(two_pi * ub);"),
    ("rotation matrix transposed (one entry)",
     "R[2] = 2 * (x * z + w * y);", "R[2] = 2 * (x * z - w * y);"),
    ("quaternion product sign",
     "dx[7] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);",
     "dx[7] = 0.5 * (q[0] * w[0] - q[2] * w[2] + q[3] * w[1]);"),
    ("gyroscopic term sign",
     "dx[10 + i] = (tau[i] - cx[i]) / Jd[i];", "dx[10 + i] = (tau[i] + cx[i]) / Jd[i];"),
    ("drag applied in the world frame",
     "for (int i = 0; i < 3; ++i) DRtv[i] = md->drag[i] * Rtv[i];",
     "for (int i = 0; i < 3; ++i) DRtv[i] = md->drag[i] * v[i];"),
    ("RK4 weights 1-1-1-1",
     "(k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i])", "(1.5 * k1[i] + 1.5 * k2[i] + 1.5 * k3[i] + 1.5 * k4[i])"),
    ("near-gate term on p_{k+1}",
     "double d0 = sqrt(dist2(x, g0));", "double d0 = sqrt(dist2(xn, g0));"),
    ("temporal rule off by one step",
     "prev_at(cx, k) <= passed", "prev_at(cx, k + 1) <= passed"),
    ("crossing accepted on s = 0 at the start",
     "if (!(sa < 0.0 && sb >= 0.0)) return 0;", "if (!(sa <= 0.0 && sb >= 0.0)) return 0;"),
    ("lag and contouring weights swapped",
     "double lag = pr->q_lag *", "double lag = pr->q_cont *"),
    ("terminal tracking weight Q instead of Q_N",
     "stage += track_err(xn, cx->xref + 13 * N, pr->QN);", "stage += track_err(xn, cx->xref + 13 * N, pr->Q);"),
    ("temperature multiplies instead of divides",
     "w[m] = isfinite(J[m]) ? exp(-(J[m] - Jmin) / pr->lambda) : 0.0;",
     "w[m] = isfinite(J[m]) ? exp(-(J[m] - Jmin) * pr->lambda) : 0.0;"),
    ("warm start without the shift",
     "(k + 1 < N ? k + 1 : N - 1);", "k;"),
    ("kept warm start shifted anyway",
     "pr->warm_start == 1 ? k :", "pr->warm_start == 1 ? (k + 1 < N ? k + 1 : N - 1) :"),
    ("nominal candidate perturbed like the others",
     "if (pr->nominal_sample && m == 0) {", "if (pr->nominal_sample && m < 0) {"),
    ("rotor roll torque pattern mirrored",
     "a * (T[0] + T[1] - T[2] - T[3])", "a * (T[0] - T[1] - T[2] + T[3])"),
    ("rotor yaw torque pattern of the roll axis",
     "md->c_tau * (T[0] - T[1] + T[2] - T[3])", "md->c_tau * (T[0] + T[1] - T[2] - T[3])"),
    ("rotor thrust does not saturate",
     "T[s] = v < md->thrust_min ? md->thrust_min : (v > md->thrust_max ? md->thrust_max : v);", "T[s] = v;"),
    ("rotor stage 2 uses the start-of-step thrusts",
     "or_deriv_rotor(md, xs, Th, k2);", "or_deriv_rotor(md, xs, T0, k2);"),
    ("rotor tracking effort about hover",
     "double hover = rotor ? 0.0 : md->mass * md->gravity;", "double hover = md->mass * md->gravity;"),
    ("rotor state not advanced by u0",
     "or_rotor_at(md, T0, Unew, pr->dt, st->rotor);", "or_rotor_at(md, T0, Unew, 0.0, st->rotor);"),
    ("near-plane flag misses the end of the segment",
     "if (fabs(info[0]) < eps || fabs(info[1]) < eps) flag |= 1;", "if (fabs(info[0]) < eps) flag |= 1;"),
    ("near-edge flag on one side of the opening only",
     "if (fabs(fabs(info[2]) - g[4]) < eps", "if (fabs(info[2] - g[4]) < eps"),
    ("near-sphere flag never set",
     "if (fabs(d0 - pr->r_near) < eps) flag |= 4;", "if (fabs(d0 - pr->r_near) < 0.0) flag |= 4;"),
    ("gate cost scale drops the start distance",
     "Jabs += fabs(dist2(xn, g)) + fabs(dist2(x, g)) + fabs(near);", "Jabs += fabs(dist2(xn, g)) + fabs(near);"),
    ("contouring cost scale subtracts the progress reward",
     "Jabs += lag + con + om + dv + dT + fabs(prog);", "Jabs += lag + con + om + dv + dT - prog;"),
    ("path tangent not renormalised",
     "for (int i = 0; i < 3; ++i) Tn[i] /= n;", "(void)n;"),
    ("contouring state terms on the start state",
     "double e[3] = {xn[0] - P[0], xn[1] - P[1], xn[2] - P[2]};", "double e[3] = {x[0] - P[0], x[1] - P[1], x[2] - P[2]};"),
    ("5th normal drawn per step instead of four steps per draw",
     "(uint32_t)(k & ~3), st->iter, 1u, z4);", "(uint32_t)k, st->iter, 1u, z4);"),
    ("samples not clamped",
     "u[j] = clampd(Unom[OR_NU * k + j] + pr->sigma[j] * z[j], md->u_min[j], md->u_max[j]);",
     "u[j] = Unom[OR_NU * k + j] + pr->sigma[j] * z[j];"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must appear exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so),
                           str(mut), "-lm"])
    env = dict(os.environ, MPPI_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
