"""Every plausible mistake planted in a copy of the diffusion oracle must fail
at least one diffusion pin (CPU only).  The mistakes are planted here, in
temporary copies of ``oracle/diffusion_oracle.c`` built with the unchanged
mechanics oracle; the oracle itself is never modified."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_ORACLE = os.path.join(_ROOT, "oracle")

# (name, text in the diffusion oracle source, replacement)
MUTANTS = [
    ("face_rows_interior", "else if (i == 0 || i == n - 1) diag = 1.0 + k + e;", "else if (0) diag = 1.0 + k + e;"),
    ("face_rows_without_k", "else if (i == 0 || i == n - 1) diag = 1.0 + k + e;",
     "else if (i == 0 || i == n - 1) diag = 1.0 + e;"),
    ("pivot_not_eliminated", "m[i] = i == 0 ? diag : diag + k * c[i - 1];", "m[i] = diag;"),
    ("pivot_wrong_sign", "m[i] = i == 0 ? diag : diag + k * c[i - 1];",
     "m[i] = i == 0 ? diag : diag - k * c[i - 1];"),
    ("c_sign", "if (i < n - 1) c[i] = -k / m[i];", "if (i < n - 1) c[i] = k / m[i];"),
    ("forward_sign", "p[i * stride] = (p[i * stride] + k * p[(i - 1) * stride]) / m[i];",
     "p[i * stride] = (p[i * stride] - k * p[(i - 1) * stride]) / m[i];"),
    ("first_pivot_skipped", "p[0] = p[0] / m[0];", "p[0] = p[0];"),
    ("backward_skips_first", "for (int64_t i = n - 2; i >= 0; --i)", "for (int64_t i = n - 2; i >= 1; --i)"),
    ("k_uses_dx", "const double k = D[s] * dt / (dx * dx);", "const double k = D[s] * dt / dx;"),
    ("decay_not_split", "const double e = lambda[s] * dt / 3.0;", "const double e = lambda[s] * dt;"),
    ("y_lines_wrong_stride", "solve_line(r + x + nx * ny * z, nx, ny, k, m, c);",
     "solve_line(r + x + nx * ny * z, 1, ny, k, m, c);"),
    ("z_axis_skipped", "solve_line(r + x + nx * y, nx * ny, nz, k, m, c);", "(void)0;"),
    ("central_difference_halved", "else g = (r[v + stride[a]] - r[v - stride[a]]) / (2.0 * dx);",
     "else g = (r[v + stride[a]] - r[v - stride[a]]) / dx;"),
    ("face_difference_reversed", "else if (i == 0) g = (r[v + stride[a]] - r[v]) / dx;",
     "else if (i == 0) g = (r[v] - r[v + stride[a]]) / dx;"),
    ("gradient_axis_swap", "const int64_t i = a == 0 ? x : (a == 1 ? y : z);",
     "const int64_t i = a == 0 ? y : (a == 1 ? x : z);"),
]


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory(prefix="diffusion_mutants_") as d:
        yield d


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(workdir, name, old, new):
    with open(os.path.join(_ORACLE, "diffusion_oracle.c")) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mutated = src.replace(old, new)
    csrc = os.path.join(workdir, f"diffusion_{name}.c")
    lib = os.path.join(workdir, f"lib_{name}.so")
    with open(csrc, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", *oracle.CFLAGS, os.path.join(_ORACLE, "mech_oracle.c"), csrc, "-o", lib, "-lm"],
                   check=True)
    # run the pins in a child process: a planted mistake may also crash the oracle
    code = (
        "import oracle\n"
        "from tests import diffusion_pins\n"
        f"lib = oracle.OracleLib({lib!r})\n"
        "failed = []\n"
        "for pin in diffusion_pins.ALL_DIFFUSION_PINS:\n"
        "    try:\n"
        "        pin(lib)\n"
        "    except Exception:\n"
        "        failed.append(pin.__name__)\n"
        "print('FAILED:' + ','.join(failed))\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=_ROOT, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return  # the planted mistake crashed the oracle: caught
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")][-1]
    failures = [f for f in line[len("FAILED:"):].split(",") if f]
    assert failures, f"planted mistake {name!r} passed every pin"
