"""The mixed-precision refinement's inner-tolerance policy (csrc/refine.h),
compiled on its own with the host compiler (no GPU): the values it returns
for hand-worked cases of the rule

  inner = min(0.1, max(inner_tol, tol / rel));
  from the second sweep on, a sweep that did not halve the residual is
  followed by one that asks for min(inner, 1e-3) (not below inner_tol), and
  one that asked for max(1e-3, inner_tol) and still did not halve it ends
  the refinement (returned as a negative value).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_2108_10481_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "refine.h"
int main(int argc, char** argv) {
    for (int i = 1; i + 5 < argc; i += 6) {
        const double v = pb::refine_inner_tol(atoi(argv[i]), atof(argv[i + 1]), atof(argv[i + 2]),
                                              atof(argv[i + 3]), atof(argv[i + 4]), atof(argv[i + 5]));
        printf("%.17g\n", v);
    }
    return 0;
}
"""

# (sweeps, rel, prev, inner_last, tol, inner_min) -> expected
CASES = [
    ((0, 1.0, 1.0, 1.0, 1e-6, 1e-4), 1e-4),        # first sweep: the inner_tol floor
    ((1, 1e-4, 1.0, 1e-4, 1e-6, 1e-4), 1e-2),      # tol / rel
    ((2, 3.5e-6, 1e-4, 1e-2, 1e-6, 1e-4), 0.1),    # capped at 0.1
    ((2, 2e-5, 1e-4, 1e-2, 1e-6, 1e-4), 0.05),     # halved: tol / rel
    ((3, 1.6e-6, 2.5e-6, 0.1, 1e-6, 1e-4), 1e-3),  # stalled on a loose inner solve: retry at 1e-3
    ((4, 1.3e-6, 1.6e-6, 1e-3, 1e-6, 1e-4), -1.0), # stalled although it asked for 1e-3: stop
    ((6, 2e-8, 2.1e-8, 5e-3, 1e-10, 1e-4), 1e-3), # reference solve (tol 1e-10): one retry...
    ((7, 2e-8, 2e-8, 1e-3, 1e-10, 1e-4), -1.0),   # ...then the floor
    ((3, 1.6e-6, 2.5e-6, 0.1, 1e-6, 2e-2), 2e-2), # a large inner_tol bounds the retry from below
    ((4, 1.5e-6, 1.6e-6, 2e-2, 1e-6, 2e-2), -1.0), # and the stop takes it as the tightest ask
    ((1, 0.9, 1.0, 1e-4, 1e-6, 1e-4), 1e-4),       # no stall test before the second sweep
]


@pytest.fixture(scope="module")
def policy(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("refine")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + SRC, str(src), "-o", str(exe)], check=True)

    def run(cases):
        args = [str(x) for c in cases for x in c]
        out = subprocess.run([str(exe), *args], check=True, capture_output=True, text=True).stdout.split()
        return [float(v) for v in out]

    return run


def test_refine_policy_cases(policy):
    got = policy([c for c, _ in CASES])
    for (case, want), v in zip(CASES, got):
        if want < 0:
            assert v < 0, (case, v)
        else:
            assert v == pytest.approx(want, rel=1e-12), (case, v)


def test_refine_policy_never_loosens_after_a_stall(policy):
    """A stalled sweep is never followed by a looser inner solve than the one it had."""
    cases = [(s, r, r * 1.2, last, 1e-6, 1e-4) for s in (2, 5) for r in (1e-6, 3e-6, 1e-5)
             for last in (1e-1, 3e-2, 1e-2, 5e-3)]
    for c, v in zip(cases, policy(cases)):
        assert 0 < v <= min(c[3], 1e-3) + 1e-18, (c, v)
