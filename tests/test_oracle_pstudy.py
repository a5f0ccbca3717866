"""The p-study of the paper's last experiment (eq. 10.3, Table 4) on the oracle: on a fixed
mesh, the relative errors of eq. 10.1 decay geometrically in k for a smooth solution, so
log(e_k / e_{k+1}) / log(e_{k+1} / e_{k+2}) is close to 1 (Table 4: 0.78 to 1.13).  Degrees
0..4."""
import numpy as np
import pytest

from oracle import hdg
from workloads import get_problem


def p_ratios(errs, key):
    e = [x[key] for x in errs]
    return [np.log(e[i] / e[i + 1]) / np.log(e[i + 1] / e[i + 2]) for i in range(len(e) - 2)]


@pytest.mark.parametrize("s", [2, 3])
def test_p_convergence_ratios(s):
    errs = []
    for k in (0, 1, 2, 3, 4):
        prob = get_problem("cube4_k1").at(s=s, k=k)
        r = hdg.solve_problem(prob)
        errs.append(hdg.errors(r["mesh"], k, r["q"], r["u"], r["uhat"], r["ustar"], prob))
    for key in ("e_q", "e_u", "e_uhat"):
        e = [x[key] for x in errs]
        # geometric decay: the k = 0 -> 1 step (k = 0 converges only like h) with 0.45, the
        # steps between k >= 1 with 0.35
        assert e[1] < 0.45 * e[0], (key, e)
        assert all(e[i + 1] < 0.35 * e[i] for i in range(1, 4)), (key, e)
        for ratio in p_ratios(errs, key):
            assert 0.7 < ratio < 1.3, (key, ratio)


def test_k0_converges_like_h():
    """k = 0: the errors of eq. 10.1 decay like h (the paper's remark on k = 0)."""
    errs = []
    for s in (4, 8):
        prob = get_problem("cube4_k1").at(s=s, k=0)
        r = hdg.solve_problem(prob)
        errs.append(hdg.errors(r["mesh"], 0, r["q"], r["u"], r["uhat"], r["ustar"], prob))
    for key in ("e_q", "e_u", "e_uhat"):
        rate = np.log2(errs[0][key] / errs[1][key])
        assert abs(rate - 1.0) < 0.25, (key, rate)
