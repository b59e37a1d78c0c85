"""Every plausible mistake planted in a copy of the velocity-variant oracle
must fail at least one variant pin (CPU only).  The mistakes are planted
here, in temporary copies of ``oracle/mech_oracle.c``; the oracle itself is
never modified."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

# (name, text in the oracle source, replacement)
MUTANTS = [
    ("affinity_row_only", "return w->aff[(int64_t)w->type[i] * w->ntypes + w->type[j]];",
     "return w->aff[(int64_t)w->type[i] * w->ntypes + w->type[i]];"),
    ("affinity_ignored", "c = c - (aij * sqrt(ccai * ccaj)) * (ta * ta);", "c = c - sqrt(ccai * ccaj) * (ta * ta);"),
    ("affinity_on_repulsion", "c = sqrt(ccri * ccrj) * (t * t);\n    }\n    double ta = 1.0 - d / AS;\n    c = c - (aij",
     "c = aij * sqrt(ccri * ccrj) * (t * t);\n    }\n    double ta = 1.0 - d / AS;\n    c = c - (aij"),
    ("wall_sign", "acc[axis] += high ? -push : push;", "acc[axis] += high ? push : -push;"),
    ("wall_cutoff_doubled", "if (!(dw < Ri)) continue;", "if (!(dw < 2.0 * Ri)) continue;"),
    ("wall_grows_outside", "double t = dw > 0.0 ? 1.0 - dw / Ri : 1.0;", "double t = 1.0 - dw / Ri;"),
    ("wall_not_squared", "double push = w->cw * (t * t);", "double push = w->cw * t;"),
    ("wall_axis", "int axis = f / 2;", "int axis = f % 3;"),
    ("wall_low_face_from_high", "x[axis] - w->wlo[axis];", "x[axis] - w->whi[axis];"),
    ("wall_mask_ignored", "if (!(w->mask & (1 << f))) continue;", "if (!w->mask) continue;"),
    ("walls_skipped", "    wall_terms(&xyz[3 * i], R[i], w, acc);\n", "\n"),
]


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory(prefix="variant_mutants_") as d:
        yield d


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_variant_mutant_is_caught(workdir, name, old, new):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mutated = src.replace(old, new)
    path = os.path.join(workdir, f"lib_{name}.so")
    oracle.compile_variant(mutated, path)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import oracle\n"
        "from tests import variant_pins\n"
        f"lib = oracle.OracleLib({path!r})\n"
        "failed = []\n"
        "for pin in variant_pins.ALL_VARIANT_PINS:\n"
        "    try:\n"
        "        pin(lib)\n"
        "    except Exception:\n"
        "        failed.append(pin.__name__)\n"
        "print('FAILED:' + ','.join(failed))\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return  # the planted mistake crashed the oracle: caught
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")][-1]
    failures = [f for f in line[len("FAILED:"):].split(",") if f]
    assert failures, f"planted mistake {name!r} passed every variant pin"
