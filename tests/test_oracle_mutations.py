"""The oracle's pins are not self-referential: each plausible mistake planted
in a copy of oracle.c (on the CPU) makes at least one pin fail.

Each mutant is compiled into a temporary library and the pins run in a child
pytest process with HLB_ORACLE_LIB pointing at it.  The unmodified oracle
passes the same pins (test_clean_oracle_passes_selected_pins)."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle" / "oracle.c"

FAST = ["tests/test_oracle_equilibrium.py", "tests/test_oracle_kinematics.py", "tests/test_oracle_adjoint.py"]
LADD = ["tests/test_oracle_ladd.py"]
LADD_FLOW = ["tests/test_oracle_flow.py::test_ladd_inlet_flux_matches_profile_integral",
             "tests/test_oracle_flow.py::test_ladd_near_inlet_profile"]

# (name, original text, mutated text, pins that must catch it)
MUTANTS = [
    ("feq drops the 1/2 on (c.u)^2", "cu * cu * b", "cu * cu * 2.0 * b", FAST),
    ("feq flips the sign of u.u", "- uu * c);", "+ uu * c);", FAST),
    ("velocity without division by rho", "u[a] = j[a] / r;", "u[a] = j[a];", FAST),
    ("collision relaxes with 1 - 1/tau", "(f[i] - feq[i]) * omega;", "(f[i] - feq[i]) * (1.0 - omega);", FAST),
    ("bounce-back into the same direction", "o->fn[x * Q + ib] = val;", "o->fn[x * Q + i] = val;", FAST),
    ("Ladd correction with the wrong sign", "val = fp[i] - 2.0 * weight(i) * r * cu_w / CS2;",
     "val = fp[i] + 2.0 * weight(i) * r * cu_w / CS2;", FAST),
    ("adjoint drops the Ladd density term", "if (!o->ladd_rho_one) arho += m", "if (0) arho += m", FAST),
    ("adjoint tau derivative with 1/tau", "dtau += lam[i] * (f[i] - feq[i]) / (tau * tau);",
     "dtau += lam[i] * (f[i] - feq[i]) / tau;", FAST),
    ("WSS with (1 - 1/tau)", "-(1.0 - 1.0 / (2.0 * o->tau))", "-(1.0 - 1.0 / o->tau)",
     ["tests/test_oracle_flow.py::test_wss_poiseuille"]),
    ("Ladd correction without the factor 2", "val = fp[i] - 2.0 * weight(i) * r * cu_w / CS2;",
     "val = fp[i] - weight(i) * r * cu_w / CS2;", LADD),
    ("Ladd correction over cs^4", "val = fp[i] - 2.0 * weight(i) * r * cu_w / CS2;",
     "val = fp[i] - 2.0 * weight(i) * r * cu_w / (CS2 * CS2);", LADD),
    ("Ladd density fixed at 1", "double r = o->ladd_rho_one ? 1.0 : rho;\n        val = fp[i]",
     "double r = 1.0;\n        val = fp[i]", LADD),
    ("Ladd weight at the site, not the link midpoint", "m[a] = p[a] + 0.5 * CV[i][a];", "m[a] = p[a];", LADD),
    ("Ladd weight with the diameter as radius", "r2 / (io->R * io->R)", "r2 / (4.0 * io->R * io->R)", LADD),
    ("Ladd correction without the factor 2 (flow pins)", "val = fp[i] - 2.0 * weight(i) * r * cu_w / CS2;",
     "val = fp[i] - weight(i) * r * cu_w / CS2;", LADD_FLOW),
    ("Ladd weight at the site (flow pins)", "m[a] = p[a] + 0.5 * CV[i][a];", "m[a] = p[a];", LADD_FLOW),
    ("WSS fallback normal not normalised", "nv[a] = l > 0 ? nsum[a] / l : 0;", "nv[a] = nsum[a];", LADD),
    ("ghost velocity not projected on the normal", "for (int a = 0; a < 3; ++a) ug[a] = un * io->nrm[a];",
     "for (int a = 0; a < 3; ++a) ug[a] = un * io->nrm[a] + u[a];",
     ["tests/test_oracle_flow.py::test_pressure_driven_linear"]),
]


def _build(text, path):
    path.write_text(text)
    lib = path.with_suffix(".so")
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", str(lib), str(path), "-lm"],
                   check=True, capture_output=True)
    return lib


def _run_pins(lib, pins):
    env = dict(os.environ, HLB_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


def test_clean_oracle_passes_selected_pins(tmp_path):
    lib = _build(SRC.read_text(), tmp_path / "clean.c")
    rc, out = _run_pins(lib, FAST + LADD + LADD_FLOW)
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, pins):
    text = SRC.read_text()
    assert text.count(old) == 1, f"mutation site not unique: {old!r}"
    lib = _build(text.replace(old, new), tmp_path / "mutant.c")
    rc, out = _run_pins(lib, pins)
    assert rc != 0, f"mutant survived: {name}\n{out}"
