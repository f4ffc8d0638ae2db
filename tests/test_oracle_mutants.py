"""Planted mistakes in the oracle must fail its pins.

Each case copies oracle/vct_oracle.c, plants one plausible slip (a dropped
term or factor, a wrong sign, index or transposed operand), compiles the copy
into a temporary library and runs the named pin tests against it in a
separate process (VCT_ORACLE_LIB points the oracle's front end at the copy).
The case passes only if those pins FAIL on the mutant, which shows the pins
can see that mistake.  The unmodified oracle passes the same pins in the
normal run of the suite.  Nothing here touches the committed oracle source.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vct_oracle.c")
PINS = "tests/test_oracle_pins.py"
PRED = "tests/test_oracle_predictor_pins.py"
REG = "tests/test_oracle_regularise.py"
ISPH = "tests/test_oracle_isph_pins.py"
SLIP = "tests/test_oracle_free_slip.py"

# (name, original snippet, planted snippet, pin files or test ids that must fail)
MUTANTS = [
    # SPH(2) and the map (Sec. 2.2, Eq. sec_SPH2)
    ("p_ij sign", "pv[a] = pr->q[a] - s;", "pv[a] = pr->q[a] + s;", [PINS]),
    ("c0 cross factor", "+ 2.0 * (ab[1] * ab[6] + ab[2] * ab[7])", "+ (ab[1] * ab[6] + ab[2] * ab[7])",
     [PINS, PRED]),
    ("c3 drops s^2", "met[4] = al * al + sx * sx + sy * sy;", "met[4] = al * al;", [PINS]),
    ("2-D keeps y curvature", "ab[2] = ab[4] = ab[7] = ab[9] = 0.0;", "ab[2] = ab[7] = 0.0;", [PRED]),
    ("kernel constant 2-D", "10.0 / (7.0 * M_PI * l * l)", "10.0 / (7.0 * l * l)", [PINS]),
    ("grad w sign (pass 1)", "for (int K = 0; K < d; ++K) gw[K] = -dw / rr * r[K];",
     "for (int K = 0; K < d; ++K) gw[K] = dw / rr * r[K];", [PINS]),
    ("cross output not halved", "ct[2] = 0.5 * met[5];", "ct[2] = met[5];", [PRED]),
    ("density self term dropped", "rho += W->V0 * kern_w(0.0, W->l, d);", "rho += 0.0;", [PRED]),
    # predictor (Eq. VCT_predictor, Sec. 3.4)
    ("c0 on the x^ gradient", "double lap = W->met[7 * i + 3] * gv[c * d + (d - 1)];",
     "double lap = W->met[7 * i + 3] * gv[c * d + 0];", [PRED]),
    ("strain product transposed", "term += (G[c * d + J2] + G[J2 * d + c]) * gn[J2];",
     "term += (G[c * d + J2] + G[c * d + J2]) * gn[J2];", [PRED]),
    ("grad nu without J", "for (int K = 0; K < d; ++K) s += Jm[I * d + K] * gnh[K];",
     "for (int K = 0; K < d; ++K) s += (I == K ? 1.0 : 0.0) * gnh[K];", [PRED]),
    ("S:S without 1/2", "double sij = 0.5 * (G[I * d + c] + G[c * d + I]);",
     "double sij = (G[I * d + c] + G[c * d + I]);", [PRED]),
    ("wall damping d0/ds inverted", "exp(-10.0 * P->d0 / P->ds * dwall / W->re)",
     "exp(-10.0 * P->ds / P->d0 * dwall / W->re)", [PRED]),
    ("wall damping factor 10 dropped", "exp(-10.0 * P->d0 / P->ds * dwall / W->re)",
     "exp(-P->d0 / P->ds * dwall / W->re)", [PRED]),
    ("nu_K dropped", "W->nu[i] = P->nu_k + nue;", "W->nu[i] = nue;", [PRED]),
    # pressure right side and walls (Eqs. VCT_ppe, VCT_ppe_w, PNC)
    ("divergence J transposed", "div += Jm[I * d + K] * X[I * d + K];",
     "div += Jm[K * d + I] * X[I * d + K];", [PRED]),
    ("rho/dt dropped", "rhs[i] = P->rho / P->dt * div", "rhs[i] = P->rho * div", [PRED]),
    ("stabilisation sign", "gamma * (P->rho * fac - W.rho_hat[i])", "gamma * (W.rho_hat[i] - P->rho * fac)",
     [PRED]),
    ("Jbar/J inverted", "S->jbar[i] / W.met[7 * i];", "W.met[7 * i] / S->jbar[i];", [PRED]),
    ("PNC sign", "pij = P->rho * s;", "pij = -P->rho * s;", [PINS]),
    # ISPH operator set (Eqs. sec_0th, gra_sum)
    ("E-R constant", "c = d == 2 ? 4.0 : 5.0", "c = d == 2 ? 5.0 : 5.0", [ISPH]),
    ("E-R drops delta", "k[0] = f * (c * r[0] * r[0] / rr2 - 1.0);",
     "k[0] = f * (c * r[0] * r[0] / rr2);", [ISPH]),
    ("E-R cross undoubled", "k[2] = 2.0 * f * c * r[0] * r[1] / rr2;", "k[2] = f * c * r[0] * r[1] / rr2;",
     [ISPH]),
    ("summation as a difference", "g[K] += pp[k].V * (f[pp[k].j] + f[i]) * pp[k].gw[K];",
     "g[K] += pp[k].V * (f[pp[k].j] - f[i]) * pp[k].gw[K];", [ISPH]),
    # free-slip walls (Sec. 3.5)
    ("slip normal not transformed", "for (int K = 0; K < d; ++K) nn[I] += Jm[I * d + K] * nh[K];",
     "for (int K = 0; K < d; ++K) nn[I] += (I == K ? 1.0 : 0.0) * nh[K];", [SLIP]),
    ("slip projects instead of reflecting", "W->vw[3 * (size_t)j + c] = v[c] - 2.0 * vn * nn[c];",
     "W->vw[3 * (size_t)j + c] = v[c] - vn * nn[c];", [SLIP]),
    # regularisation (Sec. 4.1, restated methods)
    ("DS fluid share", "double mu = S->type[j] == ORC_FLUID ? 0.5 : 1.0;",
     "double mu = S->type[j] == ORC_FLUID ? 1.0 : 1.0;", [REG]),
    ("XSPH sign", "xs[c] += V0 * (ud[3 * j + c] - ud[3 * i + c]) * wv;",
     "xs[c] += V0 * (ud[3 * i + c] - ud[3 * j + c]) * wv;", [REG]),
]


def _run_mutant(case, tmp):
    name, old, new, targets = case
    src = open(SRC).read()
    assert src.count(old) >= 1, f"snippet of '{name}' not found in the oracle"
    tag = "".join(c if c.isalnum() else "_" for c in name)
    csrc = os.path.join(tmp, f"m_{tag}.c")
    lib = os.path.join(tmp, f"m_{tag}.so")
    with open(csrc, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-w", csrc,
                           "-o", lib, "-lm"])
    env = dict(os.environ, VCT_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"] + targets,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return name, r.returncode, r.stdout[-600:]


@pytest.mark.slow
def test_planted_mistakes_fail_the_pins():
    tmp = tempfile.mkdtemp(prefix="vct_mutants_")
    try:
        workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
        with ThreadPoolExecutor(workers) as ex:
            results = list(ex.map(lambda c: _run_mutant(c, tmp), MUTANTS))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    # pytest exit code 1 = some test failed: the pins saw the mistake
    survived = [(n, rc, out) for n, rc, out in results if rc != 1]
    assert not survived, "mutants not caught:\n" + "\n".join(
        f"--- {n} (exit {rc})\n{out}" for n, rc, out in survived)
