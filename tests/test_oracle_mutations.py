"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a scratch copy of the C oracle (a torque
of the wrong sign, the spring turned the wrong way or not rescaled, the
tangential dashpot twice as strong, the spin left out of the contact
velocity, half the tangential stiffness; the porosity cube spread with the
sphere's diameter as its side, or its overlap measured from the wrong cell
face), builds it, and runs the pins of the tangential law and the porosity
spread against it: at least one of them must fail.  The same
for the preparation stages (the original JKR separating at C or solved on
the modified branch, the plate's servo of the wrong sign, the tool's
normal without its axial part, the tool turning back late, its driving
force ignored) against the preparation pins.  Nothing here touches the
CUDA library.
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
    "cube spread with the sphere's diameter as its side": ("    double side = 2.0 * R * ORA_CUBE_SIDE;",
                                                          "    double side = 2.0 * R;"),
    "cube spread overlap measured from the wrong face": ("double o = fmin(hi[k], b1) - fmax(lo[k], b0);",
                                                         "double o = fmin(hi[k], b1) - fmin(lo[k], b0);"),
}

# planted in the preparation stages, caught by tests/test_oracle_prep.py
PREP_MUTATIONS = {
    "original JKR separating at C": (
        "if (orig ? ora_contact_separates(delta, Rs, Es, gamma) : ora_bond_breaks(delta, Rs, Es, gamma)) {",
        "if (ora_bond_breaks(delta, Rs, Es, gamma)) {"),
    "original JKR on the modified branch": (
        "        a = orig ? ora_jkr_contact_radius_s(delta, Rs, Es, gamma)",
        "        a = orig ? ora_jkr_contact_radius(delta, Rs, Es, gamma)"),
    "plate servo of the wrong sign": (
        "            double v = s->stage.plate_gain * (stress - s->stage.plate_stress);",
        "            double v = s->stage.plate_gain * (s->stage.plate_stress - stress);"),
    "tool normal without its axial part": ("    n[2] = dz / d;", "    n[2] = 0.0;"),
    "tool turning back late": ("if (s->pen_dir < 0 && s->pen_z <= s->stage.pen_z_stop) s->pen_dir = 1;",
                               "if (s->pen_dir < 0 && s->pen_z < s->stage.pen_z_stop - 1e-6) s->pen_dir = 1;"),
    "tool's driving force ignored": ("                f = 1.0 - (double)tq * ORA_TWO_M40 / s->stage.pen_force;",
                                     "                f = 1.0;"),
}

PINS = ("five_sevenths or frame_indifferent or tangent_plane or dashpot or mindlin or coulomb or cube")


@pytest.mark.parametrize("name", list(MUTATIONS) + list(PREP_MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "cgdem_oracle.c")).read()
    prep = name in PREP_MUTATIONS
    a, b = PREP_MUTATIONS[name] if prep else MUTATIONS[name]
    assert a in src
    d = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (d / "oracle" / "cgdem_oracle.c").write_text(src.replace(a, b))
    for sub in ("tests", "paper_2211_06142_gb300"):
        os.symlink(os.path.join(ROOT, sub), d / sub)
    pins = ["tests/test_oracle_prep.py"] if prep else ["tests/test_oracle_pins.py", "-k", PINS]
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"],
                       cwd=d, capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(d)))
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]
