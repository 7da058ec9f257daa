"""The library's host line search (the state machine in csrc/linesearch.h that
etdm_minimize and the batched minimizer drive, Eq. 25-29 with the bracketing
and zoom conventions of the oracle) against the oracle's line search, on the
CPU: the header is compiled with the host compiler into a small driver, and
both searches see the same values of analytic functions phi(alpha) =
E(a + alpha p) with their slopes phi'(alpha) = g(a + alpha p) . p.

Pinned per function: every step length the driver asks for equals the
oracle's trial sequence, and so do the accepted step, its energy and the trial
count.  Where no trial is acceptable within 20 trials, the driver evaluates
the best point once more (the device keeps only the last evaluation's
gradient) or, when the best point is the start point, gives up; the oracle
returns that best point directly or nothing."""
import math
import os
import shutil
import subprocess

import pytest

from oracle.etdm_oracle import line_search

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_12597_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("ls") / "linesearch_driver")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC,
                    os.path.join(ROOT, "tests", "linesearch_driver.cpp"), "-o", exe],
                   check=True)
    p = subprocess.Popen([exe], stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True,
                         bufsize=1)
    yield p
    p.stdin.write("quit\n")
    p.stdin.close()
    p.wait(timeout=10)


def run_driver(p, phi, E0, d0):
    """The library's search on phi: the step lengths it evaluated and its result."""
    p.stdin.write(f"start {E0!r} {d0!r}\n")
    asked = []
    while True:
        f = p.stdout.readline().split()
        if f[0] == "eval":
            a = float(f[1])
            asked.append(a)
            E, d = phi(a)
            p.stdin.write(f"{E!r} {d!r}\n")
        else:
            assert f[0] == "done"
            return asked, bool(int(f[1])), int(f[2]), float(f[3]), float(f[4])


def run_oracle(phi, E0, d0):
    seen = []

    def rec(a):
        seen.append(a)
        E, d = phi(a)
        return E, d, a

    alpha, E, d, pay, trials = line_search(rec, E0, d0)
    return seen, pay is not None, trials, alpha, E


def quad(amin, kappa=2.0, c=0.0):
    return lambda t: (0.5 * kappa * (t - amin) ** 2 + c, kappa * (t - amin))


CASES = {
    # quadratics: overshoot (bracket [0, 1], one cubic step), undershoot
    # (doubling: the exact cubic's minimum lies beyond 4 alpha), alpha = 1
    # accepted at once
    "quad_overshoot": quad(0.2),
    "quad_far": quad(30.0),
    "quad_tiny": quad(0.01, kappa=50.0, c=-3.0),
    "quad_short": quad(2.5),
    "quad_accept": quad(1.5),
    "quad_huge": quad(1e3, kappa=1e-3),
    # non-polynomial: the cubic is not exact, so the zoom iterates; a quartic
    # whose minimum lies far out takes a doubling, then a cubic extrapolation
    # inside [1.1, 4] times the step, then a zoom
    "quartic_extrapolate": lambda t: (-t + t ** 4 / 864.0, -1.0 + t ** 3 / 216.0),
    "sixth_power": lambda t: ((t - 0.35) ** 6 - 0.001 * t, 6 * (t - 0.35) ** 5 - 0.001),
    "exp_well": lambda t: (-t * math.exp(-t / 30.0), -(1.0 - t / 30.0) * math.exp(-t / 30.0)),
    "double_well": lambda t: (0.25 * (t * t - 1.0) ** 2 - 0.2 * t, (t * t - 1.0) * t - 0.2),
    "steep_wall": lambda t: (-t + math.exp(20.0 * (t - 0.3)),
                             -1.0 + 20.0 * math.exp(20.0 * (t - 0.3))),
    # alpha = 1 lowers E but the slope there is positive and large: the
    # bracket is [1, 0] (low end at alpha = 1)
    "positive_slope": lambda t: (-t + t ** 3 / 1.08, -1.0 + t * t / 0.36),
    # Eq. 27-28: a step whose energy change is below the noise of E
    "noisy_flat": lambda t: (-1000.0 - 1e-12 * t + 0.5e-12 * t * t + 1e-10,
                             -1e-12 + 1e-12 * t),
    # slopes that never satisfy Eq. 26 or Eq. 27: 20 trials, then the best point
    "never_ok": lambda t: (t * t - 0.5 * t, -1.0),
    # no point below the start: 20 trials, nothing taken
    "no_descent": lambda t: (t, -1.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_line_search_equals_oracle(driver, name):
    phi = CASES[name]
    E0, d0 = phi(0.0)
    assert d0 < 0.0
    asked, ok, trials, alpha, E = run_driver(driver, phi, E0, d0)
    seen, ok_o, trials_o, alpha_o, E_o = run_oracle(phi, E0, d0)
    assert ok == ok_o and trials == trials_o
    # the trials themselves, then (no acceptable trial) the best point again
    extra = asked[len(seen):]
    assert len(extra) == (1 if (ok and trials == 20) else 0)
    for a, b in zip(asked, seen):
        assert a == pytest.approx(b, rel=1e-13, abs=1e-300)
    if ok:
        assert alpha == pytest.approx(alpha_o, rel=1e-13)
        assert E == pytest.approx(E_o, rel=1e-13, abs=1e-300)
        if extra:
            assert extra[0] == pytest.approx(alpha_o, rel=1e-13)


def test_cases_cover_every_exit(driver):
    """The functions above reach each way out of the search: acceptance on the
    first trial, after bracketing, after zooming, on Eq. 27-28 alone, the best
    point after 20 trials, and no step."""
    out = {n: run_driver(driver, CASES[n], *CASES[n](0.0)) for n in CASES}
    assert out["quad_accept"][2] == 1 and out["quad_accept"][3] == 1.0
    assert out["noisy_flat"][1] and out["noisy_flat"][2] == 1
    assert out["quad_far"][2] == 3 and out["quad_far"][3] == 4.0
    q = out["quartic_extrapolate"][0]  # 1, 2 (doubling), cubic extrapolation, zoom
    assert q[:2] == [1.0, 2.0] and 2.2 <= q[2] <= 8.0 and q[2] != 4.0 and len(q) == 4
    assert out["positive_slope"][1] and out["positive_slope"][3] < 1.0
    assert max(o[2] for o in out.values() if o[1] and len(o[0]) == o[2]) >= 3
    assert out["never_ok"][1] and out["never_ok"][2] == 20 and len(out["never_ok"][0]) == 21
    assert not out["no_descent"][1] and out["no_descent"][2] == 20
