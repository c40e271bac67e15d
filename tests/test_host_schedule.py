"""Host logic of the tensor-core product's work schedule (no GPU needed): the
split of Step I (Alg. 2) and of the K_BB a products (Alg. 5) over the CTAs of
one GPU, walked on the host through the kernel's own run decoding."""

import pytest

from paper_2505_13723_b300 import binding as lib

ROWS = [1, 127, 128, 129, 1000, 2500, 4096, 4999, 9999, 10000, 20000, 100000]
COLS = [1, 128, 129, 1000, 10001, 20011, 50001, 65536, 262144, 1048576]


@pytest.mark.parametrize("ctas", [0, 144, 147, 37, 8, 1])
def test_every_tile_and_slot_covered_once(ctas):
    flat = 0
    for m in ROWS:
        for n in COLS:
            st, ns, fl = lib.schedule_check(m, n, ctas)
            assert st == 0, (m, n, ctas, ns, fl)
            assert ns >= 1
            flat += fl
    if ctas in (0, 144, 147):
        assert flat > 0           # the equal-run schedule is exercised


def test_which_products_take_equal_runs():
    # the ten 10,000 x 10,000 K_BB a products of the regress workload: three slots a row
    assert lib.schedule_check(10000, 10000, 148) == (0, 3, True)
    # Step I of the regress workload keeps the (row tile x split) items: equal runs of
    # 4,494 tiles per CTA would give up the L2 sharing of column tiles
    st, ns, fl = lib.schedule_check(10000, 1 << 20, 144)
    assert st == 0 and not fl
    # too few tiles for every CTA to get two
    st, ns, fl = lib.schedule_check(129, 1000, 148)
    assert st == 0 and not fl


def test_invalid_arguments():
    assert lib.schedule_check(0, 10, 0)[0] == 1      # ADASAP_EINVAL
    assert lib.schedule_check(10, 0, 0)[0] == 1
