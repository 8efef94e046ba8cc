"""Host logic of the multi-plan batch: the list schedule of plans on SM
tokens.  Whatever the actual run times, two plans that hold a common SM must
be ordered by the dependencies, so cooperative master kernels that may run
at the same time always fit the GPU together."""
import numpy as np
import pytest

from paper_1005_4396_b300 import vmat


def _ancestors(deps):
    n = len(deps)
    anc = [set() for _ in range(n)]

    def visit(p, seen):
        for q in deps[p]:
            if q not in seen:
                seen.add(q)
                visit(q, seen)
        return seen
    for p in range(n):
        anc[p] = visit(p, set())
    return anc


@pytest.mark.parametrize("seed", range(12))
def test_list_schedule_invariants(seed):
    rng = np.random.default_rng(seed)
    sms = int(rng.choice([148, 132, 37]))
    n = int(rng.integers(1, 24))
    budget = rng.integers(1, sms + 1, n)
    if seed % 3 == 0:
        budget[:] = sms // int(rng.integers(1, 5))  # equal shares
    est = rng.uniform(0.0, 10.0, n)
    if seed % 4 == 1:
        est[: n // 2] = est[0]  # ties in estimated work
    order, deps, tokens = vmat.vmat_list_schedule(budget, est, sms, want_tokens=True)
    # capture order: a permutation by decreasing estimated work, stable
    assert sorted(order.tolist()) == list(range(n))
    ref = sorted(range(n), key=lambda p: -est[p])
    assert order.tolist() == ref
    pos = {p: i for i, p in enumerate(order.tolist())}
    # each plan holds exactly its budget, waits only for plans captured before it
    assert np.array_equal(tokens.sum(1), budget)
    for p in range(n):
        assert all(pos[q] < pos[p] for q in deps[p])
        assert len(set(deps[p])) == len(deps[p])
    # plans sharing an SM are ordered: one is an ancestor of the other
    anc = _ancestors(deps)
    for p in range(n):
        for q in range(p + 1, n):
            if np.any(tokens[p] & tokens[q]):
                assert q in anc[p] or p in anc[q], (p, q)


def test_list_schedule_packs_small_plans_side_by_side():
    # four plans of a quarter of the SMs each: all start at once, no waits
    order, deps, tokens = vmat.vmat_list_schedule([37] * 4, [1.0] * 4, 148, want_tokens=True)
    assert all(len(d) == 0 for d in deps)
    assert tokens.sum(0).max() == 1
    # whole-GPU plans run one after another
    order, deps, _ = vmat.vmat_list_schedule([148] * 3, [3.0, 2.0, 1.0], 148)
    assert order.tolist() == [0, 1, 2] and deps == [[], [0], [1]]


def test_list_schedule_rejects_bad_sizes():
    with pytest.raises(vmat.VmatError):
        vmat.vmat_list_schedule([0], [1.0], 148)
    with pytest.raises(vmat.VmatError):
        vmat.vmat_list_schedule([149], [1.0], 148)
    with pytest.raises(vmat.VmatError):
        vmat.vmat_list_schedule([10], [-1.0], 148)
