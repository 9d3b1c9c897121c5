"""Mutation check of the oracle's pins: plausible mistakes planted in copies of the
oracle source (compiled on the CPU, loaded in child processes) must each fail at least
one pin, while the unmodified oracle passes all of them."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spinsys_oracle.c")

# (name, original text, mistaken text)
MUTANTS = [
    ("anisotropy field without factor 2", "double a = 2.0 * s->k_u[i] / mu * sdote;",
     "double a = s->k_u[i] / mu * sdote;"),
    ("exchange bonds counted twice in the field", "    H[0] = sx / mu;\n    H[1] = sy / mu;\n    H[2] = sz / mu;",
     "    H[0] = 2.0 * sx / mu;\n    H[1] = 2.0 * sy / mu;\n    H[2] = 2.0 * sz / mu;"),
    ("applied field with the wrong sign", "    H[0] += s->H_app[0];\n    H[1] += s->H_app[1];\n    H[2] += s->H_app[2];",
     "    H[0] -= s->H_app[0];\n    H[1] -= s->H_app[1];\n    H[2] -= s->H_app[2];"),
    ("Neel field without factor 2", "        H[0] += 2.0 / mu * kx;", "        H[0] += 1.0 / mu * kx;"),
    ("damping term with the wrong sign", "    dS[0] = pre * (c0 + lambda * d0);\n    dS[1] = pre * (c1 + lambda * d1);\n"
     "    dS[2] = pre * (c2 + lambda * d2);", "    dS[0] = pre * (c0 - lambda * d0);\n    dS[1] = pre * (c1 - lambda * d1);\n"
     "    dS[2] = pre * (c2 - lambda * d2);"),
    ("LLG prefactor without 1/(1+lambda^2)", "double pre = -gamma / (1.0 + lambda * lambda);", "double pre = -gamma;"),
    ("transposed cross product", "    double c0 = S[1] * H[2] - S[2] * H[1];", "    double c0 = S[2] * H[1] - S[1] * H[2];"),
    ("noise variance with a (1+lambda^2) factor",
     "double sigma = sqrt(2.0 * lambda * ORC_KB * Tn / (gamma * s->mu_s[i] * s->dt));",
     "double sigma = sqrt(2.0 * lambda * ORC_KB * Tn * (1.0 + lambda * lambda) / (gamma * s->mu_s[i] * s->dt));"),
    ("corrector started from the predicted spin", "            v[0] = S[3 * i + 0] + 0.5 * (dS[3 * i + 0] + dSp[0]) * s->dt;",
     "            v[0] = Sp[3 * i + 0] + 0.5 * (dS[3 * i + 0] + dSp[0]) * s->dt;"),
    ("corrector without renormalisation", "            orc_normalise(v);\n            /* S_i is only read",
     "            /* S_i is only read"),
    ("exchange energy without the factor 1/2", "eex += -0.5 * (Si[0] * hex[0]", "eex += -1.0 * (Si[0] * hex[0]"),
    ("third Gaussian reusing the first angle", "    g[2] = r2 * cos(phi2);", "    g[2] = r2 * cos(phi1);"),
    ("Philox key not advanced", "            k0 += 0x9E3779B9u;", ""),
    ("Philox multipliers swapped", "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;",
     "uint64_t p0 = (uint64_t)0xCD9E8D57u * (uint64_t)x0;"),
    # Monte Carlo
    ("Metropolis test with the wrong sign", "(dE <= -ORC_KB * T * log(u))", "(dE <= ORC_KB * T * log(u))"),
    ("Metropolis test without kB", "(dE <= -ORC_KB * T * log(u))", "(dE <= -T * log(u))"),
    ("exchange counted twice in the energy change", "    double e = -(X[0] * hx + X[1] * hy + X[2] * hz);",
     "    double e = -2.0 * (X[0] * hx + X[1] * hy + X[2] * hz);"),
    ("anisotropy energy with the wrong sign", "    e += -s->k_u[i] * xe * xe;", "    e += s->k_u[i] * xe * xe;"),
    ("applied-field energy without the moment",
     "    e += -s->mu_s[i] * (X[0] * s->H_app[0] + X[1] * s->H_app[1] + X[2] * s->H_app[2]);",
     "    e += -(X[0] * s->H_app[0] + X[1] * s->H_app[1] + X[2] * s->H_app[2]);"),
    ("Gaussian move not renormalised", "        Sn[2] = Si[2] + sigma_g * g[2];\n        orc_normalise(Sn);",
     "        Sn[2] = Si[2] + sigma_g * g[2];"),
    ("every move a Gaussian move", "    int move = (int)(((uint64_t)wb[0] * 3u) >> 32);", "    int move = 1;"),
    ("cone width with exponent 1/4", "pow(ORC_KB * T / ORC_MUB, 0.2)", "pow(ORC_KB * T / ORC_MUB, 0.25)"),
    ("colouring ignores the neighbours", "        while (c < cap && seen[c] == i) ++c;", "        c = 0;"),
    ("record taken after the step", "        if (rec) orc_moment_energy(s, S, rec + 8 * k);\n        int64_t acc = 0;",
     "        int64_t acc = 0;"),
    # demagnetising field
    ("self term without the factor 1/3", "- ORC_MU0 / 3.0 * m[3 * a + 0] / V;", "- ORC_MU0 * m[3 * a + 0] / V;"),
    ("dipole term with 2 (m.r)r", "            hz += (3.0 * mdotu * uz - m[3 * b + 2]) / r3;",
     "            hz += (2.0 * mdotu * uz - m[3 * b + 2]) / r3;"),
    ("cell centre not weighted by the moment",
     "            p[3 * c + a] += mu * s->pos[3 * i + a];\n        }\n        w[c] += mu;",
     "            p[3 * c + a] += s->pos[3 * i + a];\n        }\n        w[c] += 1.0;"),
    ("cell volume from the cube edge", "        double V = na[a] * s->demag_vatom;",
     "        double V = s->demag_cell * s->demag_cell * s->demag_cell;"),
    ("demagnetising field updated every step",
     "(k == 0 || (step0 + k) % (s->demag_every > 0 ? s->demag_every : 1) == 0)", "(1)"),
    # tensorial exchange and cubic anisotropy
    ("exchange tensors applied transposed",
     "            sx += t[0] * S[3 * j + 0] + t[1] * S[3 * j + 1] + t[2] * S[3 * j + 2];\n"
     "            sy += t[3] * S[3 * j + 0] + t[4] * S[3 * j + 1] + t[5] * S[3 * j + 2];\n"
     "            sz += t[6] * S[3 * j + 0] + t[7] * S[3 * j + 1] + t[8] * S[3 * j + 2];",
     "            sx += t[0] * S[3 * j + 0] + t[3] * S[3 * j + 1] + t[6] * S[3 * j + 2];\n"
     "            sy += t[1] * S[3 * j + 0] + t[4] * S[3 * j + 1] + t[7] * S[3 * j + 2];\n"
     "            sz += t[2] * S[3 * j + 0] + t[5] * S[3 * j + 1] + t[8] * S[3 * j + 2];"),
    ("one tensor row transposed", "            sx += t[0] * S[3 * j + 0] + t[1] * S[3 * j + 1] + t[2] * S[3 * j + 2];",
     "            sx += t[0] * S[3 * j + 0] + t[3] * S[3 * j + 1] + t[6] * S[3 * j + 2];"),
    ("cubic field without factor 2", "        double c = -2.0 * s->k_c[i] / mu;", "        double c = -1.0 * s->k_c[i] / mu;"),
    ("cubic energy with the wrong sign", "            ea += 0.5 * s->k_c[i] * (x2 * x2 + y2 * y2 + z2 * z2);",
     "            ea -= 0.5 * s->k_c[i] * (x2 * x2 + y2 * y2 + z2 * z2);"),
    ("cubic term missing from the Monte Carlo energy", "        e += 0.5 * s->k_c[i] * (x2 * x2 + y2 * y2 + z2 * z2);",
     "        e += 0.0;"),
    # midpoint integrator
    ("midpoint iteration on S^(k) instead of the midpoint", "M[i] = 0.5 * (S[i] + X[i]);", "M[i] = X[i];"),
    ("midpoint iterations skipped", "        for (int it = 0; it < iters; ++it) {", "        for (int it = 0; it < 0; ++it) {"),
    # semi-implicit predictor-corrector
    ("semi-implicit corrector with the field at S_n", "            orc_site_field(s, M, i, hex, H);\n            for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];\n            orc_sib_a(gamma, lambda, M + 3 * i, H, A);",
     "            orc_site_field(s, S, i, hex, H);\n            for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];\n            orc_sib_a(gamma, lambda, M + 3 * i, H, A);"),
    ("semi-implicit damping term at S_n in the corrector", "            orc_sib_a(gamma, lambda, M + 3 * i, H, A);",
     "            orc_sib_a(gamma, lambda, S + 3 * i, H, A);"),
    ("midpoint without the demagnetising field", "            for (int64_t q = 0; q < 3 * n; ++q) Hth[q] += Hd[q];  /* both are held over the step */\n        /* Euler predictor",
     "            (void)0;\n        /* Euler predictor"),
    ("semi-implicit solve with b x c added", "X[k] = (c[k] - bxc[k] + bc * b[k]) / (1.0 + bb);",
     "X[k] = (c[k] + bxc[k] + bc * b[k]) / (1.0 + bb);"),
]


def _build(name, text, tmp):
    path = os.path.join(tmp, f"lib_{abs(hash(name))}.so")
    csrc = path.replace(".so", ".c")
    open(csrc, "w").write(text)
    import oracle

    subprocess.run(["gcc", *oracle.FLAGS, "-o", path, csrc, "-lm"], check=True)
    return path


def _run(lib):
    env = dict(os.environ, SPINSYS_ORACLE_LIB=lib, PYTHONPATH=ROOT, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_mutant_pins.py")], capture_output=True,
                         text=True, env=env, timeout=600).stdout
    return [line.split()[1] for line in out.splitlines() if line.startswith("FAIL")], out


@pytest.mark.filterwarnings("ignore")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = open(SRC).read()
    jobs = {"(unmodified)": base}
    for name, a, b in MUTANTS:
        assert base.count(a) == 1, f"mutant text not found once: {name}"
        jobs[name] = base.replace(a, b)
    libs = {name: _build(name, text, str(tmp_path)) for name, text in jobs.items()}
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(libs, ex.map(_run, libs.values())))
    failed, out = results.pop("(unmodified)")
    assert failed == [], out
    survivors = [name for name, (f, _) in results.items() if not f]
    assert survivors == [], f"mistakes no pin detects: {survivors}"
