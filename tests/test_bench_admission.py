"""The batched form's admission plan (bench.py): the systems handed to
kbe_batch_create smallest-of-each-N_b-class first, then ascending by size, and
what the call's in-order rule admits under a byte budget. Host logic only."""
import numpy as np

import bench
import kbe_inputs as ki


def test_admission_order_and_rule_small_case():
    nbs = [16, 2, 4, 2, 16, 4]
    need = [50, 5, 10, 3, 40, 20]
    order, admitted, used = bench.batch_admission(nbs, need, 60)
    assert order == [3, 2, 4, 1, 5, 0]           # classes 2, 4, 16 by their smallest; then by size
    assert admitted == [3, 2, 4, 1] and used == 58
    order, admitted, used = bench.batch_admission(nbs, need, 2)
    assert admitted == [] and used == 0


def test_admission_on_the_uneven_draw():
    """on the 64-system draw with a size model ~ N_b^2 n_k N_t^2: every class leads,
    the admitted set fits, and every system left out did not fit at its turn"""
    systems = ki.batched(64)
    nbs = [x.nb for x in systems]
    need = [x.nb ** 2 * x.nk * (x.nt + 1) * (x.nt + 2) // 2 * 32 for x in systems]
    budget = int(0.1 * sum(need))
    order, admitted, used = bench.batch_admission(nbs, need, budget)
    assert sorted(order) == list(range(64))
    classes = sorted(set(nbs))
    assert [nbs[i] for i in order[:len(classes)]] == classes
    for c, i in zip(classes, order[:len(classes)]):
        assert need[i] == min(need[j] for j in range(64) if nbs[j] == c)
    rest = order[len(classes):]
    assert all(need[a] <= need[b] for a, b in zip(rest, rest[1:]))
    assert used == sum(need[i] for i in admitted) <= budget
    run = 0
    for i in order:   # the in-order rule, replayed
        if i in admitted:
            run += need[i]
        else:
            assert run + need[i] > budget
    assert len(admitted) > len(classes)
    assert np.isclose(used, run)
