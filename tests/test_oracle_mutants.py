"""Mutation check of the oracle's pins: each plausible slip planted in a copy of oracle.c (a wrong
weight, a transposed operand, a dropped term or factor, a wrong sign or index) must make at least
one pin of test_oracle_pins.py fail.  The mutants are built and run on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "trilinear x weight flipped": ("double wx = (c & 1) ? x[0] : 1.0 - x[0];",
                                   "double wx = (c & 1) ? 1.0 - x[0] : x[0];"),
    "corner bits y/z swapped": ("double wy = (c & 2) ? x[1] : 1.0 - x[1];\n            double wz = (c & 4) ? x[2] : 1.0 - x[2];",
                                "double wy = (c & 4) ? x[1] : 1.0 - x[1];\n            double wz = (c & 2) ? x[2] : 1.0 - x[2];"),
    "explin factor dropped": ("return x > 1.1 ? x : 1.1 * exp(x / 1.1 - 1.0);", "return x > 1.1 ? x : exp(x / 1.1 - 1.0);"),
    "colour offset dropped": ("double c = 0.5;", "double c = 0.0;"),
    "depth at entry, not midpoint": ("e->mid = 0.5 * (sg->t0 + sg->t1);", "e->mid = sg->t0;"),
    "weight without transmittance": ("double w = T * e.alpha;", "double w = e.alpha;"),
    "overlap owned twice": ("double a = hits[k].a > cur ? hits[k].a : cur;", "double a = hits[k].a;"),
    "view direction reversed": ("g[a] = lo[a] + 0.5 * s - ol[a];", "g[a] = ol[a] - (lo[a] + 0.5 * s);"),
    "left Riemann samples": ("double t = sg->t0 + ((double)k + 0.5) * l / (double)K;",
                             "double t = sg->t0 + ((double)k) * l / (double)K;"),
    "backward depth suffix dropped": ("gtau += gD * (Tn * e->mid - RD);", "gtau += gD * (Tn * e->mid);"),
    "backward alpha term dropped": ("double gtau = gA * Tend;", "double gtau = 0.0;"),
    "backward colour suffix sign": ("gtau += gC[ch] * (Tn * e->rgb[ch] - RC[ch]);", "gtau += gC[ch] * (Tn * e->rgb[ch] + RC[ch]);"),
    "SH gradient ignores the clamp": ("if (!(g->pre[ch] > 0.0)) continue;", "if (0) continue;"),
    "SH gradient without the weight": ("r.g_rgb[ch] = gC[ch] * w;", "r.g_rgb[ch] = gC[ch];"),
    "normal points up the density gradient": ("n_loc[a] = gn > 0.0 ? -g[a] / gn : 0.0;", "n_loc[a] = gn > 0.0 ? g[a] / gn : 0.0;"),
    "normal left in the local frame": ("n_world[r] = P->R[r * 3 + 0] * n_loc[0] + P->R[r * 3 + 1] * n_loc[1] + P->R[r * 3 + 2] * n_loc[2];",
                                       "n_world[r] = n_loc[r];"),
    "normal gradient without the tangent projection": ("dg[a] = -(dn[a] - n_loc[a] * nd) / gn;", "dg[a] = -dn[a] / gn;"),
    "normal suffix dropped": ("gtau += gN[a] * (Tn * e->nrm[a] - RN[a]);", "gtau += gN[a] * (Tn * e->nrm[a]);"),
    "SH sign flipped": ("Y[1] = -k1 * y;", "Y[1] = k1 * y;"),
    "pose rotation transposed": ("for (int r = 0; r < 3; ++r) q[r] = P->R[0 * 3 + r] * w[0] + P->R[1 * 3 + r] * w[1] + P->R[2 * 3 + r] * w[2];",
                                 "for (int r = 0; r < 3; ++r) q[r] = P->R[r * 3 + 0] * w[0] + P->R[r * 3 + 1] * w[1] + P->R[r * 3 + 2] * w[2];"),
    "early stop before the crossing segment": ("            T *= (1.0 - e.alpha);\n            ++used;\n            if (T < J->opt->eps_stop) break;",
                                               "            if (T * (1.0 - e.alpha) < J->opt->eps_stop) break;\n            T *= (1.0 - e.alpha);\n            ++used;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mut = src.replace(old, new)
    c = tmp_path / "oracle_mut.c"
    c.write_text(mut)
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(lib), str(c),
                           "-lm", "-lpthread"])
    env = dict(os.environ, DV_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], env=env, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutant '{name}'"
