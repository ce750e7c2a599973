"""Planted mistakes in a copy of the oracle: each plausible slip (a dropped
factor, a wrong sign, a transposed index, a left-out term, a wrong update
order) is written into a copy of nep_oracle.c, the copy is compiled with the
oracle's own flags, and the pins (tests/test_oracle_descriptor.py,
_forces.py, _functions.py, _md_training.py) run against it in a separate
process: at least one pin must fail for every mistake, while the unaltered
copy passes them all.  This checks the pins, not the oracle; it runs on the
CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_descriptor.py", "tests/test_oracle_forces.py", "tests/test_oracle_functions.py",
        "tests/test_oracle_md_training.py"]

# (what the mistake is, text in nep_oracle.c, the text that replaces it)
MISTAKES = [
    ("factor 2 of the angular descriptor derivative (Eq. 25) dropped",
     "double t1 = 2.0 * E->dgA", "double t1 = 1.0 * E->dgA"),
    ("the pair's partial force added to F_j instead of subtracted (Eqs. 4-5)",
     "F[3 * (size_t)j + c] -= pij[c];", "F[3 * (size_t)j + c] += pij[c];"),
    ("per-atom virial transposed (Eq. 6)",
     "W[9 * (size_t)j + 3 * a + b] += -rij[a] * pij[b];", "W[9 * (size_t)j + 3 * a + b] += -rij[b] * pij[a];"),
    ("the k = j term of the angular double sum (Eq. 13) left out",
     "if (!(E->rn[b] < h->rc_A)) continue;\n            double c = cos_angle(E, a, b);",
     "if (!(E->rn[b] < h->rc_A) || b == a) continue;\n            double c = cos_angle(E, a, b);"),
    ("hidden-layer bias with a plus sign (Eq. 21)",
     "x[mu] = tanh(a - b1[mu]);", "x[mu] = tanh(a + b1[mu]);"),
    ("SNES: sigma updated before the mean (Eqs. 38-39)",
     "        m[p] += eta_m * s[p] * gm;\n        s[p] *= exp(0.5 * eta_s * gs);",
     "        s[p] *= exp(0.5 * eta_s * gs);\n        m[p] += eta_m * s[p] * gm;"),
    ("Chebyshev recurrence with the wrong sign (App. A)",
     "T[k] = 2.0 * x * T[k - 1] - T[k - 2];", "T[k] = 2.0 * x * T[k - 1] + T[k - 2];"),
    ("cutoff function with the wrong sign (Eq. 15)",
     "return 0.5 * (1.0 + cos(ORC_PI * r / rc));", "return 0.5 * (1.0 - cos(ORC_PI * r / rc));"),
]


def _build_copy(tmp_path, name, old=None, new=None):
    src = open(os.path.join(ROOT, "oracle", "nep_oracle.c")).read()
    if old is not None:
        assert src.count(old) == 1, (name, src.count(old))
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "nep_oracle.h"), d / "nep_oracle.h")
    (d / "nep_oracle.c").write_text(src)
    from oracle import oracle as orc
    lib = d / "liboracle.so"
    subprocess.run(["gcc"] + orc.GCC_FLAGS + [str(d / "nep_oracle.c"), "-o", str(lib), "-lm"], check=True)
    return str(lib)


def _run_pins(lib, first_failure=True):
    env = dict(os.environ, NEP_ORACLE_LIB=lib, OMP_NUM_THREADS="4")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + \
        (["-x"] if first_failure else []) + PINS
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_an_unaltered_copy(tmp_path):
    r = _run_pins(_build_copy(tmp_path, "unaltered"), first_failure=False)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,old,new", MISTAKES, ids=[m[0][:40] for m in MISTAKES])
def test_every_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    r = _run_pins(_build_copy(tmp_path, "mutant", old, new))
    assert r.returncode != 0, f"no pin caught: {what}\n{r.stdout[-1500:]}"
