"""Mutation check of the oracle's pins (test infrastructure, CPU only).

Each entry below is one plausible mistake in the oracle: a dropped factor, a wrong sign, a
swapped operand, a wrong tie rule. For each, a mutated copy of rwmi_oracle.c is compiled into a
temporary directory with the oracle's own flags. The CPU pins (tests/test_oracle_*.py) then run
against it through RWMI_ORACLE_LIB. A mutation must make at least one pin fail. The real
source and library are never touched, so an interrupted run leaves nothing behind.

    python tests/mutation_check.py               # all mutations (about 15 minutes on 8 cores)
    python tests/mutation_check.py Guo DEM       # those whose name contains a given word
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_SRC = os.path.join(ROOT, "oracle", "rwmi_oracle.c")
sys.path.insert(0, ROOT)
from oracle.oracle import CFLAGS  # noqa: E402

PINS = ["tests/test_oracle_rng.py", "tests/test_oracle_metaball.py", "tests/test_oracle_lbm.py",
        "tests/test_oracle_walkers.py", "tests/test_oracle_ibb.py", "tests/test_oracle_dem.py"]

# (name, passage it breaks, exact source text, replacement)
MUTATIONS = [
    ("Guo prefactor 1-1/tau", "Guo forcing",
     "double guo = 1.0 - 0.5 / tau;", "double guo = 1.0 - 1.0 / tau;"),
    ("velocity with F, not F/2", "Guo forcing",
     "u[a] = (jm[a] + 0.5 * F[a]) / rho;", "u[a] = (jm[a] + F[a]) / rho;"),
    ("equilibrium 4.5 -> 4.0", "Eq. 13",
     "(1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu)", "(1.0 + 3.0 * eu + 4.0 * eu * eu - 1.5 * uu)"),
    ("PSM weight B denominator", "PSM (Noble-Torczynski)",
     "((1.0 - eps) + (tau - 0.5))", "((1.0 - eps) + tau)"),
    ("PSM solid term u and u_s swapped", "PSM (Noble-Torczynski)",
     "om = fi[mo] - feq(q, mo, rho, u) - fi[m] + feq(q, m, rho, us);",
     "om = fi[mo] - feq(q, mo, rho, us) - fi[m] + feq(q, m, rho, u);"),
    ("Guo source not weighted by 1-B", "PSM with forcing",
     "+ B * om + (1.0 - B) * S;", "+ B * om + S;"),
    ("bounce-back takes f_i, not f_opp", "no-slip walls",
     "if (blocked) fi[m] = o->f[(size_t)opposite(m) * o->ncell + c];",
     "if (blocked) fi[m] = o->f[(size_t)m * o->ncell + c];"),
    ("Algorithm 1 tolerance 1e-1", "Algorithm 1",
     "if (fabs(fm - 1.0) < 1e-3) {", "if (fabs(fm - 1.0) < 1e-1) {"),
    ("Algorithm 2 projection, not mirror", "Algorithm 2 / Eq. 22",
     "(ti[d] - 2.0 * tn * n[d])", "(ti[d] - 1.0 * tn * n[d])"),
    ("noise amplitude sqrt(D)", "Eq. 2",
     "double amp = sqrt(2.0 * o->D * 1.0);", "double amp = sqrt(o->D * 1.0);"),
    ("Box-Muller angle pi U", "Eq. 2 (normal noise)",
     "double ang = 2.0 * M_PI * ub;", "double ang = M_PI * ub;"),
    ("Philox with 9 rounds", "walker noise generator",
     "for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)"),
    ("refill radius without cube root", "type II refill (Section 2.4.2)",
     "double rad = sqrt(2.0 * o->D) * cbrt(u24(r[2]));", "double rad = sqrt(2.0 * o->D) * u24(r[2]);"),
    ("advection dropped", "Eq. 2",
     "xf[d] = x[d] + u[d] * 1.0 + amp * z[d];", "xf[d] = x[d] + amp * z[d];"),
    ("trilinear node offset", "Section 2.4.1 interpolation",
     "if (!o->wall[a]) {\n        double s = xa - 0.5;", "if (!o->wall[a]) {\n        double s = xa;"),
    ("minimum image off", "periodic metaballs",
     "if (d > 0.5 * n) d -= n;", "if (d > 2.0 * n) d -= n;"),
    ("raster sub-sample offset", "solid fraction",
     "(float)i + (0.125f + 0.25f * (float)cx)", "(float)i + (0.25f * (float)cx)"),
    ("raster owner tie to the higher index", "solid fraction owner",
     "if (npart[cand[m]] > best) { best = npart[cand[m]]; owner = cand[m]; }",
     "if (npart[cand[m]] >= best) { best = npart[cand[m]]; owner = cand[m]; }"),
    ("walls clamp instead of reflecting", "walker walls",
     "if (x[a] < 0.0) x[a] = -x[a];\n            else if (x[a] > n) x[a] = 2.0 * n - x[a];",
     "if (x[a] < 0.0) x[a] = 0.0;\n            else if (x[a] > n) x[a] = n;"),
    ("binning rounds, not floors", "Eq. 16",
     "long long i = (long long)floor(x[a]);", "long long i = (long long)floor(x[a] + 0.5);"),
    ("variance over N-1", "Eqs. 38-40 moments",
     "out[4 + a] = vd[a] / (double)o->nw;", "out[4 + a] = vd[a] / (double)(o->nw - 1);"),
    ("DEM normal damping sign", "DEM contact law",
     "double Fn = o->dem_kn * delta - o->dem_etan * vn;", "double Fn = o->dem_kn * delta + o->dem_etan * vn;"),
    ("DEM normal force may attract", "DEM contact law",
     "if (Fn < 0.0) Fn = 0.0;", "if (Fn < -1e300) Fn = 0.0;"),
    ("DEM Coulomb limit without mu_s", "Eq. 5",
     "double lim = o->dem_mus * Fn;", "double lim = Fn;"),
    ("DEM spring not projected", "Eq. 5",
     "for (int a = 0; a < 3; ++a) xi[a] = (xi[a] - xn * n[a]) + vt[a] * dt;",
     "for (int a = 0; a < 3; ++a) xi[a] = xi[a] + vt[a] * dt;"),
    ("DEM explicit, not symplectic, Euler", "Eq. 4 integration",
     "st[7 + a] = st[7 + a] + dt * (F[a] / m);\n            st[a] = st[a] + dt * st[7 + a];",
     "st[a] = st[a] + dt * st[7 + a];\n            st[7 + a] = st[7 + a] + dt * (F[a] / m);"),
    ("DEM gyroscopic term sign", "Eq. 4 rotation",
     "double rhs[3] = {T[0] - gyro[0], T[1] - gyro[1], T[2] - gyro[2]}",
     "double rhs[3] = {T[0] + gyro[0], T[1] + gyro[1], T[2] + gyro[2]}"),
    ("DEM spin applied in the body frame", "Eq. 4 rotation",
     "qv[0] + h * (qw * w[0] + wxq[0]),", "qv[0] + h * (qw * w[0] - wxq[0]),"),
    ("IBB q <= 1/2 interpolation swapped", "Eq. 24",
     "if (qf <= 0.5) us[a] = 2.0 * qf * uf[a] + (1.0 - 2.0 * qf) * uff[a];",
     "if (qf <= 0.5) us[a] = 2.0 * qf * uff[a] + (1.0 - 2.0 * qf) * uf[a];"),
    ("PSM force on the particle with the wrong sign", "PSM force (momentum exchange)",
     "double Fc[3] = {-dp[0], -dp[1], -dp[2]}, r[3];", "double Fc[3] = {dp[0], dp[1], dp[2]}, r[3];"),
    ("PSM solid velocity without the spin", "PSM solid velocity",
     "us[0] = v[0] + w[1] * r[2] - w[2] * r[1];", "us[0] = v[0];"),
    ("Guo source without its second-order term", "Guo forcing",
     "S += (3.0 * (e[a] - u[a]) + 9.0 * eu * e[a]) * F[a];", "S += (3.0 * (e[a] - u[a])) * F[a];"),
    ("body force cos, not sin", "oscillating drive (Eq. 37)",
     "if (o->Fperiod > 0.0) s = sin(2.0 * M_PI * (double)t / o->Fperiod);",
     "if (o->Fperiod > 0.0) s = cos(2.0 * M_PI * (double)t / o->Fperiod);"),
    ("seeding covers half the box", "walker seeding",
     "volatile double off = u24(r[d]) * span;", "volatile double off = u24(r[d]) * span * 0.5;"),
    ("IBB force on the particle with the wrong sign", "momentum exchange",
     "for (int a = 0; a < 3; ++a) o->Fp[3 * p + a] += Fl[a];", "for (int a = 0; a < 3; ++a) o->Fp[3 * p + a] -= Fl[a];"),
    ("IBB refill at rest, not at the rigid velocity", "Eq. 27",
     "rigid_velocity(o, &fr, nprev[c] - 1, xc, un);", "un[0] = un[1] = un[2] = 0.0;"),
    ("DEM wall normal outward", "Eqs. 10-11",
     "double sg = side ? -1.0 : 1.0;", "double sg = side ? 1.0 : -1.0;"),
    ("PSM torque, x component sign", "PSM torque",
     "o->Tp[3 * p + 0] += r[1] * Fc[2] - r[2] * Fc[1];", "o->Tp[3 * p + 0] -= r[1] * Fc[2] - r[2] * Fc[1];"),
    ("IBB torque, x component sign", "momentum-exchange torque",
     "o->Tp[3 * p + 0] += r[1] * Fl[2] - r[2] * Fl[1];", "o->Tp[3 * p + 0] -= r[1] * Fl[2] - r[2] * Fl[1];"),
    ("type IV keeps a reflected point inside a particle", "multiple reflections (Section 2.4.2)",
     "if (beyond_wall(o, tr) || inside_any64(o, fr1, tr) >= 0) {", "if (beyond_wall(o, tr)) {"),
    ("type IV keeps a reflected point beyond a wall", "multiple reflections (Section 2.4.2)",
     "if (beyond_wall(o, tr) || inside_any64(o, fr1, tr) >= 0) {", "if (inside_any64(o, fr1, tr) >= 0) {"),
    ("type III refilled instead of moving out", "walker types (Section 2.4.2)",
     "        o->cnt_type[2]++;\n        for (int d = 0; d < 3; ++d) xnew[d] = xf[d];",
     "        o->cnt_type[2]++;\n        if (!refill(o, fr1, pin, x, id, t, xnew)) o->refill_fail++;"),
    ("Eq. 9 contact point past the overlap", "Eq. 9",
     "for (int a = 0; a < 3; ++a) xcp[a] = xc0[a] + (Rs0 - 0.5 * delta) * nrm[a];",
     "for (int a = 0; a < 3; ++a) xcp[a] = xc0[a] + (Rs0 + 0.5 * delta) * nrm[a];"),
    ("DEM mass sampled at h = 1/2", "Eq. 4 mass properties",
     "#define DEM_MASS_H 0.25", "#define DEM_MASS_H 0.5"),
    ("IBB q bisection with 12 steps", "Eq. 25",
     "for (int it = 0; it < 24; ++it) {", "for (int it = 0; it < 12; ++it) {"),
    ("seeding keeps points inside particles", "initial removal (Section 2.4.2)",
     "ok = (o->P == 0) || inside_any32(o, &fr, xs) < 0;", "ok = 1;"),
    ("Eq. 7 Newton on the gradient of f0 only", "Eq. 7",
     "double G[3] = {g0[0] + g1[0], g0[1] + g1[1], g0[2] + g1[2]};",
     "double G[3] = {g0[0], g0[1], g0[2]};"),
    ("Eq. 8 single first-order step", "Eq. 8",
     "    if (inside) {\n        q = hi;", "    if (0) {\n        q = hi;"),
    ("walled binning wraps instead of clamping", "Eq. 16 on walled axes",
     "if (o->wall[a]) { if (i < 0) i = 0; if (i > o->n[a] - 1) i = o->n[a] - 1; }",
     "if (0) { if (i < 0) i = 0; if (i > o->n[a] - 1) i = o->n[a] - 1; }"),
    ("moments: mean of x, not of x - x0", "Eqs. 38-40 moments",
     "md[a] += o->x[3 * w + a] - o->x0[3 * w + a];", "md[a] += o->x[3 * w + a];"),
    ("IBB node owner: the highest index", "node classes (Fig. 3)",
     "                        node[c] = p + 1;\n                        break;",
     "                        node[c] = p + 1;"),
    ("IBB node at the cell corner", "node classes (Fig. 3)",
     "float xs[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};\n                node[c] = 0;",
     "float xs[3] = {(float)i, (float)j, (float)k};\n                node[c] = 0;"),
    ("DEM pair without the periodic image", "DEM on periodic axes",
     "if (!o->wall[a]) d -= (double)o->n[a] * floor(d / (double)o->n[a] + 0.5);", "(void)0;"),
    ("walker noise not keyed by the step", "Eq. 2 (noise per step)",
     "trilinear(o, ufield, x, u);\n    uint32_t ctr[4] = {id, t, 0u, 0u}, r[4];",
     "trilinear(o, ufield, x, u);\n    uint32_t ctr[4] = {id, 0u, 0u, 0u}, r[4];"),
    ("interpolation wall layer held at the node value", "Section 2.4.1 at walls",
     "wt[1] = xa / 0.5; wt[0] = 1.0 - wt[1];", "wt[1] = 1.0; wt[0] = 0.0;"),
    ("PSM solid velocity without the minimum image", "PSM solid velocity on periodic axes",
     "for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, xn[a] - fr->o[3 * owner + a]);",
     "for (int a = 0; a < 3; ++a) r[a] = xn[a] - fr->o[3 * owner + a];"),
    ("DEM pair torque arm from the other body", "Eq. 4 (contact torque)",
     "double ri[3] = {xcp[0] - si[0], xcp[1] - si[1], xcp[2] - si[2]};",
     "double ri[3] = {xcp[0] - oj[0], xcp[1] - oj[1], xcp[2] - oj[2]};"),
    ("DEM wall torque with the wrong sign", "Eq. 4 (contact torque)",
     "    cross3(r, Fw, Tw);\n}", "    cross3(Fw, r, Tw);\n}"),
    ("DEM wall contact point outside the overlap", "Eq. 11",
     "for (int d = 0; d < 3; ++d) xcp[d] = xcw[d] + 0.5 * delta * nrm[d];",
     "for (int d = 0; d < 3; ++d) xcp[d] = xcw[d] - 0.5 * delta * nrm[d];"),
    ("momentum exchange without the wall velocity", "Galilean-invariant momentum exchange",
     "for (int a = 0; a < 3; ++a) Fl[a] = (eip[a] - uw[a]) * Gp - (e[a] - uw[a]) * fi[m];",
     "for (int a = 0; a < 3; ++a) Fl[a] = eip[a] * Gp - e[a] * fi[m];"),
    ("IBB moving-wall term sign", "Eq. 23",
     "return feq(q, ip, rho_f, ud) + gneq + 6.0 * lattice_weight(q, ip) * rho_f * eu;",
     "return feq(q, ip, rho_f, ud) + gneq - 6.0 * lattice_weight(q, ip) * rho_f * eu;"),
]


def run(names=()) -> list:
    """Returns [(mutation, passage, caught, failing pins, seconds)]."""
    src = open(ORACLE_SRC).read()
    out = []
    with tempfile.TemporaryDirectory() as tmp:
        for name, passage, old, new in MUTATIONS:
            if names and not any(w in name for w in names):
                continue
            if src.count(old) != 1:
                raise SystemExit(f"mutation '{name}': its source text occurs {src.count(old)} times")
            t0 = time.time()
            csrc = os.path.join(tmp, "mutant.c")
            lib = os.path.join(tmp, f"mutant_{len(out)}.so")
            with open(csrc, "w") as f:
                f.write(src.replace(old, new))
            subprocess.check_call(["gcc", *CFLAGS, "-o", lib, csrc, "-lm"])
            env = dict(os.environ, RWMI_ORACLE_LIB=lib)
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                               cwd=ROOT, env=env, capture_output=True, text=True)
            failed = [ln.split("::", 1)[1].split(" ")[0] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
            out.append((name, passage, r.returncode != 0, failed, time.time() - t0))
            print(f"{'caught' if r.returncode else 'MISSED':6s}  {name:38s}  {', '.join(failed)}", flush=True)
    return out


if __name__ == "__main__":
    res = run(tuple(sys.argv[1:]))
    missed = [r[0] for r in res if not r[2]]
    print(f"{len(res) - len(missed)} of {len(res)} mutations caught" + (f"; missed: {missed}" if missed else ""))
    sys.exit(1 if missed else 0)
