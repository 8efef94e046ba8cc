"""Decision-by-decision comparison of a column-generation run (Sec. 2.2,
Fig. 1) with the FP64 oracle.

Which aperture the pricing picks is an argmin over prices, and a price is
the derivative of Eq. 3 at the solution of the previous master problem.  A
decision is only defined as far as that solution is: the oracle's own prices
move by up to 2e-5 relative between a master tolerance of 1e-8 and 1e-12
(tiny phantom), so decisions whose margin is below that are not fixed by a
1e-8 solve.  The comparison therefore takes
  - the oracle converged to KKT 1e-13 (ORACLE_EPS), its row scans in FP32
    as the kernel takes them (the decision in the kernel's precision);
  - the library in its extended-precision master mode
    (vmat_set_master_precision: float-pair dose excess, F', columns and
    partial sums, FP64 price sums) converged to KKT 1e-12 (GPU_KKT).  The
    default FP32 master stops improving near 1e-9 to 4e-8, where prices
    still differ by up to ~1e-5 relative.  The KKT tolerance is relative to
    the plan's first residual, the size of its first (largest) price, while
    a margin is relative to the current best price, which late in a plan can
    be 1,000x smaller: a 1e-6 margin there needs the solve to ~1e-12;
  - a near-tie: best price within NEAR_TIE = 1e-6 relative of the runner-up
    beam, or of the runner-up interval of one of its rows (FP64 enumeration),
    or within the single-precision resolution of the row scans that decide it
    (one unit in the last place of a row's largest prefix sum; the oracle
    records it): both sides take the decision in FP32, and below that
    resolution a one-ulp difference in a single beamlet price decides it.
Every decision that is not a near-tie must agree bit for bit; at a near-tie
either choice is valid, and the library's must price within PRICE_RTOL of
the oracle's best."""
import numpy as np

import oracle

NEAR_TIE = 1e-6
ORACLE_EPS = 1e-13
GPU_KKT = 1e-12
PRICE_RTOL = 1e-5
COST_RTOL = 1e-5


def precise(plan):
    """Put a plan in the comparison's master mode (before it has columns)."""
    plan.set_master_precision(True)
    return plan


def oracle_plan(prob, **kw):
    """The oracle's column generation at the comparison's tolerance."""
    kw.setdefault("eps", ORACLE_EPS)
    return oracle.colgen(prob, f32_pricing=True, **kw)


def margin(ref, t):
    return min(ref["margin"][t], ref["row_margin"][t])


def near_tie(ref, t):
    """The decision of iteration t is not fixed to the comparison's precision."""
    return (margin(ref, t) <= NEAR_TIE or ref["margin"][t] <= ref["f32_res"][t]
            or ref["row_res"][t] <= 1.0)


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
            assert near_tie(ref, t), (
                f"iteration {t}: beam {k} vs oracle {ref['k'][t]} without a near-tie "
                f"(margin {ref['margin'][t]:.3e}, row margin {ref['row_margin'][t]:.3e}, "
                f"single-precision resolution {ref['f32_res'][t]:.3e})")
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
        if near_tie(ref, t):
            ties += 1
            continue
        assert _same(rep["priced_k"][t], rep["priced_l"][t], rep["priced_r"][t], ref, t, R), (
            f"iteration {t}: library priced beam {rep['priced_k'][t]} leaves "
            f"{rep['priced_l'][t].tolist()}/{rep['priced_r'][t].tolist()}, oracle beam {ref['k'][t]} "
            f"(margin {ref['margin'][t]:.3e}, row margin {ref['row_margin'][t]:.3e})")
        compared += 1
    return compared, ties
