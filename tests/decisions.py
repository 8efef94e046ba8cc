"""Decision-by-decision comparison of a column-generation run (Sec. 2.2,
Fig. 1) with the FP64 oracle.

Which aperture the pricing picks is an argmin over prices, and a price is
the derivative of Eq. 3 at the solution of the previous master problem.  A
decision is only defined as far as that solution is: the oracle's own prices
move by up to 2e-5 relative between a master tolerance of 1e-8 and 1e-12
(tiny phantom), so decisions whose margin is below that are not fixed by a
1e-8 solve.  The comparison therefore takes
  - the oracle converged to KKT 1e-12 (ORACLE_EPS), its row scans in FP32
    as the kernel takes them (the decision in the kernel's precision);
  - the library converged to KKT 1e-9 (GPU_KKT), the tightest its
    compensated FP32 master reaches on every phantom tested (at 1e-10 it
    stalls on its rounding floor);
  - a near-tie: best price within NEAR_TIE = 1e-6 relative of the runner-up
    beam, or of the runner-up interval of one of its rows (FP64 enumeration).
Every decision that is not a near-tie must agree bit for bit; at a near-tie
either choice is valid, and the library's must price within PRICE_RTOL of
the oracle's best."""
import numpy as np

import oracle

NEAR_TIE = 1e-6
ORACLE_EPS = 1e-12
GPU_KKT = 1e-9
PRICE_RTOL = 1e-5
COST_RTOL = 1e-5


def oracle_plan(prob, **kw):
    """The oracle's column generation at the comparison's tolerance."""
    kw.setdefault("eps", ORACLE_EPS)
    return oracle.colgen(prob, f32_pricing=True, **kw)


def margin(ref, t):
    return min(ref["margin"][t], ref["row_margin"][t])


def forced(ref, R):
    """The oracle's decisions as a replay: (beams, left leaves, right leaves)."""
    fl = np.array([ref["lleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    fr = np.array([ref["rleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    return ref["k"], fl, fr


def _same(k, l, r, ref, t, R):
    kr = ref["k"][t]
    return (k == kr and np.array_equal(l, ref["lleaf"][kr * R:(kr + 1) * R])
            and np.array_equal(r, ref["rleaf"][kr * R:(kr + 1) * R]))


def check_unforced(gpu, ref, R):
    """The library's own plan against the oracle's: identical beams and
    leaves up to the first near-tie, costs within COST_RTOL while they
    agree.  Returns the number of leading iterations that agree."""
    n = len(ref["k"])
    for t in range(n):
        k = gpu["k"][t]
        if not _same(k, gpu["lleaf"][k * R:(k + 1) * R], gpu["rleaf"][k * R:(k + 1) * R], ref, t, R):
            assert margin(ref, t) <= NEAR_TIE, (
                f"iteration {t}: beam {k} vs oracle {ref['k'][t]} without a near-tie "
                f"(margin {ref['margin'][t]:.3e}, row margin {ref['row_margin'][t]:.3e})")
            np.testing.assert_allclose(gpu["cost"][:t], ref["cost"][:t], rtol=COST_RTOL)
            return t
    np.testing.assert_allclose(gpu["cost"], ref["cost"], rtol=COST_RTOL)
    return n


def check_replay(rep, ref, R):
    """The oracle's plan replayed on the library (forced apertures): at every
    iteration the library's own pricing result on the replayed state equals
    the oracle's decision unless that decision is a near-tie; its price is
    within PRICE_RTOL of the oracle's; every master cost within COST_RTOL.
    Returns (decisions compared bit for bit, near-ties)."""
    n = len(ref["k"])
    np.testing.assert_array_equal(rep["k"], ref["k"])  # the forced beams were added
    np.testing.assert_allclose(rep["cost"], ref["cost"], rtol=COST_RTOL)
    compared = ties = 0
    floor = 1e-12 * abs(ref["p"][0])  # an exact zero price (closed rows only) on both sides
    for t in range(n):
        p, pg = ref["p"][t], rep["p"][t]
        assert abs(pg - p) <= PRICE_RTOL * abs(p) + floor, f"iteration {t}: price {pg!r} vs oracle {p!r}"
        if margin(ref, t) <= NEAR_TIE:
            ties += 1
            continue
        assert _same(rep["priced_k"][t], rep["priced_l"][t], rep["priced_r"][t], ref, t, R), (
            f"iteration {t}: library priced beam {rep['priced_k'][t]} leaves "
            f"{rep['priced_l'][t].tolist()}/{rep['priced_r'][t].tolist()}, oracle beam {ref['k'][t]} "
            f"(margin {ref['margin'][t]:.3e}, row margin {ref['row_margin'][t]:.3e})")
        compared += 1
    return compared, ties
