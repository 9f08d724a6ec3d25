"""Sensitivity of the oracle's pins.  Each mutant plants one plausible
mistake in a copy of oracle/mamute_oracle.cpp (on the CPU: a text
substitution, built under oracle/_build/mutants beside the oracle's own
build), and the pins that must catch it run in a subprocess with that
library loaded in place of the oracle; they must fail.  (A sponge kept on
the top face under a free surface is an equivalent mutant and is not
listed: the planes above the surface hold zero whatever their damping.)"""
import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mamute_oracle.cpp")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = "tests/test_oracle_pins.py::"
BOUNDARY = "tests/test_oracle_boundary.py::"

# name: ([(text, replacement), ...] applied to every occurrence, [pins that must fail])
MUTANTS = {
    "source without sqrt(rho)": (
        [("* M.srho[sh.src.node[e]]);", ");"), ("* M.srho[src.node[e]]);", ");")],
        [PINS + "test_uniform_density_equals_constant_density"]),
    "receivers without sqrt(rho)": (
        [("P.w[e] *= M.srho[P.node[e]];", "P.w[e] *= 1.0;"),
         ("rp.w[e] *= M.srho[rp.node[e]];", "rp.w[e] *= 1.0;")],
        [PINS + "test_uniform_density_equals_constant_density"]),
    "rho for sqrt(rho)": (
        [("M.srho[d.at(i, j, k)] = std::sqrt(rho[src]);", "M.srho[d.at(i, j, k)] = rho[src];")],
        [PINS + "test_density_mass_term_closed_form"]),
    "imaging term: sign of the m^2 u term": (
        [("c.g[p] * (l - c.m2[p] * u1[p]);", "c.g[p] * (l + c.m2[p] * u1[p]);")],
        [PINS + "test_gn_jacobian_column_matches_finite_differences"]),
    "imaging term: laplacian doubled": (
        [("c.g[p] * (l - c.m2[p] * u1[p]);", "c.g[p] * (2.0 * l - c.m2[p] * u1[p]);")],
        [PINS + "test_gn_jacobian_column_matches_finite_differences"]),
    "free surface: even image": (
        [("      sign = T(-1);\n", "      sign = T(1);\n")],
        [BOUNDARY + "test_free_surface_equals_odd_image_source"]),
    "free surface: image one plane off": (
        [("      c = 2 * d.zs - c;\n", "      c = 2 * d.zs - c + 1;\n")],
        [BOUNDARY + "test_free_surface_equals_odd_image_source"]),
    "trilinear weights swapped": (
        [("w *= up ? t[a] : 1.0 - t[a];", "w *= up ? 1.0 - t[a] : t[a];")],
        [BOUNDARY + "test_trilinear_receiver_and_source_are_weighted_node_sums"]),
}

CONTROL = "unmodified"  # the same build and runner with no substitution: every pin passes

RUNNER = """
import ctypes, sys
sys.path.insert(0, {root!r})
from oracle import oracle as O
O._lib = ctypes.CDLL({lib!r})
O.build = lambda force=False: {lib!r}
import pytest
sys.exit(pytest.main(["-q", "-p", "no:cacheprovider"] + {tests!r}))
"""


def _run(name):
    reps, tests = MUTANTS[name] if name != CONTROL else ([], sorted({t for _, ts in MUTANTS.values()
                                                                     for t in ts}))
    with open(SRC) as f:
        s = f.read()
    for a, b in reps:
        assert a in s, (name, a)
        s = s.replace(a, b)
    stem = re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")
    cpp, lib = os.path.join(OUT, stem + ".cpp"), os.path.join(OUT, stem + ".so")
    with open(cpp, "w") as f:
        f.write(s)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                           cpp])
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib, tests=tests)],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def results():
    os.makedirs(OUT, exist_ok=True)
    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
        names = list(MUTANTS) + [CONTROL]
        return dict(zip(names, ex.map(_run, names)))


def test_unmodified_build_passes_the_pins(results):
    rc, out = results[CONTROL]
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_fails_its_pins(results, name):
    rc, out = results[name]
    assert rc == 1, (name, rc, out)  # 1: pytest ran the pins and some failed
