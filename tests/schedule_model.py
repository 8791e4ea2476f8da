"""A model of THIS library's Strassen-Winograd accumulate schedule (not a
formula of the paper, whose Section 6.2 prices 22 additions per level): per
level 4 explicit additions of the n/2 x k/2 halves of A, 4 of the k/2 x m/2
halves of B and 8 of n/2 x m/2 products into quadrants of C; the other four
accumulations are fused into the products' stores.  The op-counting build's
counters are checked against it (tests/test_gpu_op_counts.py), and it is
pinned by tests/test_cost_model.py; the oracle does not use it."""


def strassen_additions(n: int, k: int, m: int, b: int, levels: int) -> int:
    """Words written by the explicit additions of `levels` levels."""
    if levels == 0:
        return 0
    n2, k2, m2 = n // 2, k // 2, m // 2
    here = 4 * n2 * (k2 // b) + 4 * k2 * (m2 // b) + 8 * n2 * (m2 // b)
    return here + 7 * strassen_additions(n2, k2, m2, b, levels - 1)
