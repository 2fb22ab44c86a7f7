"""Stored fixtures under tests/golden/ (written by committed scripts that call only the oracle):
the workload CFL factors stay below the oracle scheme's 1-D stability limits, and Eq. (7) with a
literal CFL_N = 0.9 exceeds them for N >= 2 (Sec. 3.4)."""
import os

from paper_1905_07987_gb300 import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def limits():
    out = {}
    for line in open(os.path.join(HERE, "cfl_limits.txt")):
        if line.startswith("#") or not line.strip():
            continue
        N, nu = line.split()
        out[int(N)] = float(nu)
    return out


def test_workload_cfl_factors_are_below_the_stability_limits():
    lim = limits()
    assert sorted(lim) == [1, 2, 3, 4, 5, 6]
    for N, nu in lim.items():
        courant = synth.cfl_number(N) / (2 * N + 1)   # Eq. (7) with d = 1
        assert courant <= 0.9 * nu * 1.0001, (N, courant, nu)
        assert synth.KAPPA[N] <= (2 * N + 1) * nu + 1e-5  # file holds 6 decimals


def test_literal_eq7_exceeds_the_limits_for_N_at_least_2():
    lim = limits()
    assert abs(lim[1] - 1.0 / 3.0) < 1e-5      # order 1: the classical 1/(2N+1) bound is sharp
    for N in range(2, 7):
        assert 0.9 / (2 * N + 1) > lim[N]
