"""Every plausible mistake planted in a copy of the oracle must fail at least
one pin (CPU only).  The mistakes are planted here, in temporary copies of
``oracle/mech_oracle.c``; the oracle itself is never modified."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle
from tests import oracle_pins

# (name, text in the oracle source, replacement, which occurrence (0 = first)).
# Dropping the explicit self-pair skip is not listed: the self pair has d = 0
# and the d > 0 test removes it anyway, so that change is not a mistake.
MUTANTS = [
    ("repulsion_sign", "c = sqrt(ccri * ccrj) * (t * t);", "c = -sqrt(ccri * ccrj) * (t * t);", 0),
    ("adhesion_sign", "c = c - sqrt(ccai * ccaj) * (ta * ta);", "c = c + sqrt(ccai * ccaj) * (ta * ta);", 0),
    ("coefficient_no_sqrt", "c = sqrt(ccri * ccrj) * (t * t);", "c = (ccri * ccrj) * (t * t);", 0),
    ("coefficient_one_cell", "c = c - sqrt(ccai * ccaj) * (ta * ta);", "c = c - ccai * (ta * ta);", 0),
    ("repulsion_not_squared", "c = sqrt(ccri * ccrj) * (t * t);", "c = sqrt(ccri * ccrj) * t;", 0),
    ("adhesion_uses_S", "double ta = 1.0 - d / AS;", "double ta = 1.0 - d / S;", 0),
    ("cutoff_S_only", "if (!(d < AS)) return 0;", "if (!(d < S)) return 0;", 0),
    ("S_is_twice_Ri", "double S = Ri + Rj;", "double S = Ri + Ri;", 0),
    ("transposed_dx", "double dx = xi[0] - xj[0];", "double dx = xj[0] - xi[0];", 0),
    ("wrong_component", "acc[1] += s * dy;", "acc[1] += s * dz;", 0),
    ("no_unit_vector", "double s = c / d;", "double s = c;", 0),
    ("no_d_positive_check", "if (!(d > 0.0)) return 0;", "", 0),
    ("half_stencil", "for (int dz = -1; dz <= 1; ++dz) {", "for (int dz = 0; dz <= 1; ++dz) {", 0),
    ("key_axis_swap", "key[i] = (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy", "key[i] = (uint32_t)iy + (uint32_t)g.n[0] * ((uint32_t)ix", 0),
    ("round_not_floor", "double f = floor(t);", "double f = round(t);", 0),
    ("clamp_high_off_by_one", "if (f >= (double)(n - 1)) return n - 1;", "if (f >= (double)(n - 1)) return n - 2;", 0),
    ("sort_unstable", "for (int64_t i = 0; i < n; ++i) order[fill[key[i]]++] = i;",
     "for (int64_t i = n - 1; i >= 0; --i) order[fill[key[i]]++] = i;", 0),
    ("scan_inclusive", "start[v] = (uint32_t)run; run += count[v];", "run += count[v]; start[v] = (uint32_t)run;", 0),
    ("ab2_euler", "xyz[k] = xyz[k] + dt * (1.5 * v[k] - 0.5 * vprev[k]);", "xyz[k] = xyz[k] + dt * v[k];", 0),
    ("ab2_wrong_weights", "xyz[k] = xyz[k] + dt * (1.5 * v[k] - 0.5 * vprev[k]);",
     "xyz[k] = xyz[k] + dt * (1.5 * v[k] + 0.5 * vprev[k]);", 0),
    ("vprev_not_updated", "vprev[k] = v[k];", "(void)0;", 0),
    # caught by the new pins: FP32 face decision, subset indexing, the
    # hand-evaluated two-cell values, the scalar AB2 recursion
    ("f32_face_to_lower_voxel", "float f = floorf(t);", "float f = ceilf(t) - 1.0f;", 0),
    ("subset_rows_by_cell", "velocity_one(idx[k], &b, xyz, R, ccr, cca, A, &v[3 * k]);",
     "velocity_one(idx[k], &b, xyz, R, ccr, cca, A, &v[3 * (k > 0 ? k - 1 : k)]);", 0),
    ("subset_ignores_list", "velocity_one(idx[k], &b, xyz, R, ccr, cca, A, &v[3 * k]);",
     "velocity_one(k, &b, xyz, R, ccr, cca, A, &v[3 * k]);", 0),
    ("adhesion_cubed", "c = c - sqrt(ccai * ccaj) * (ta * ta);", "c = c - sqrt(ccai * ccaj) * (ta * ta * ta);", 0),
    ("ab2_first_step_euler_weight", "xyz[k] = xyz[k] + dt * (1.5 * v[k] - 0.5 * vprev[k]);",
     "xyz[k] = xyz[k] + dt * (1.5 * v[k] - 0.45 * vprev[k]);", 0),
]


def _replace_nth(text, old, new, nth):
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation anchor not found: {old!r}"
    return text[:pos] + new + text[pos + len(old):]


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory(prefix="oracle_mutants_") as d:
        yield d


@pytest.mark.parametrize("name,old,new,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, name, old, new, nth):
    src = oracle.source_text()
    mutated = _replace_nth(src, old, new, nth)
    assert mutated != src
    path = os.path.join(workdir, f"lib_{name}.so")
    oracle.compile_variant(mutated, path).lib = None
    # run the pins in a child process: a planted mistake may also crash the oracle
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys\n"
        "import oracle\n"
        "from tests import oracle_pins\n"
        f"lib = oracle.OracleLib({path!r})\n"
        "failed = []\n"
        "for pin in oracle_pins.ALL_PINS:\n"
        "    try:\n"
        "        pin(lib)\n"
        "    except Exception as e:\n"
        "        failed.append(pin.__name__)\n"
        "print('FAILED:' + ','.join(failed))\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return  # the planted mistake crashed the oracle: caught
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")][-1]
    failures = [f for f in line[len("FAILED:"):].split(",") if f]
    assert failures, f"planted mistake {name!r} passed every pin"
