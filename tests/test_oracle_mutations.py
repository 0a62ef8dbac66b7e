"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a scratch copy of the C oracle (a torque
of the wrong sign, the spring turned the wrong way or not rescaled, the
tangential dashpot twice as strong, the spin left out of the contact
velocity, half the tangential stiffness), builds it, and runs the pins of
the tangential law against it: at least one of them must fail.  Nothing
here touches the CUDA library.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "wall torque of the wrong sign": ("            Ti[k] += R * nFt[k];", "            Ti[k] -= R * nFt[k];"),
    "spring turned the wrong way": (
        "    xi[0] -= xn * n[0];\n    xi[1] -= xn * n[1];\n    xi[2] -= xn * n[2];",
        "    xi[0] += xn * n[0];\n    xi[1] += xn * n[1];\n    xi[2] += xn * n[2];"),
    "spring not rescaled": ("        double sc = old / nw;", "        double sc = 1.0; (void)old; (void)nw;"),
    "tangential dashpot doubled": ("    double gt = 2.0 * sqrt(5.0 / 6.0) * beta * sqrt(kt * ms);",
                                   "    double gt = 4.0 * sqrt(5.0 / 6.0) * beta * sqrt(kt * ms);"),
    "spin left out of the wall contact velocity": (
        "        double rw[3] = {R * w[0], R * w[1], R * w[2]};",
        "        double rw[3] = {0.0 * w[0], 0.0 * w[1], 0.0 * w[2]};"),
    "half the tangential stiffness": ("    double kt = 8.0 * Gs * a;", "    double kt = 4.0 * Gs * a;"),
}

PINS = ("five_sevenths or frame_indifferent or tangent_plane or dashpot or mindlin or coulomb")


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "cgdem_oracle.c")).read()
    a, b = MUTATIONS[name]
    assert a in src
    d = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (d / "oracle" / "cgdem_oracle.c").write_text(src.replace(a, b))
    for sub in ("tests", "paper_2211_06142_gb300"):
        os.symlink(os.path.join(ROOT, sub), d / sub)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-p",
                        "no:cacheprovider", "-m", "not gpu", "-k", PINS],
                       cwd=d, capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(d)))
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]
