"""The popping measure of bench.py: order flips between two blend orders are the pairs
of common Gaussians in opposite order (the Kendall distance restricted to the common
elements), counted here against brute force on random orders, with padding and
truncation."""
import sys
from pathlib import Path

import numpy as np
import torch

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402


def brute(a, b):
    pos = {g: k for k, g in enumerate(b)}
    c = [g for g in a if g in pos]
    flips = sum(1 for i in range(len(c)) for j in range(i + 1, len(c)) if pos[c[i]] > pos[c[j]])
    return flips, len(c) * (len(c) - 1) // 2


def test_order_flips_match_brute_force():
    rng = np.random.default_rng(3)
    P, L = 64, 12
    A = np.full((P, L), -1, np.int32)
    B = np.full((P, L), -1, np.int32)
    la, lb = np.zeros(P, np.int32), np.zeros(P, np.int32)
    want = [0, 0, 0]
    for p in range(P):
        na, nb = rng.integers(0, L + 1), rng.integers(0, L + 1)
        a, b = rng.choice(24, na, replace=False), rng.choice(24, nb, replace=False)
        A[p, :na], B[p, :nb], la[p], lb[p] = a, b, na, nb
        f, c = brute(list(a), list(b))
        want[0] += f
        want[1] += f > 0
        want[2] += c
    got = bench.order_flips(torch.tensor(A), torch.tensor(la), torch.tensor(B), torch.tensor(lb), torch, batch=7)
    assert list(got) == want


def test_order_flips_identical_and_reversed_orders():
    a = torch.tensor([[5, 9, 2, 7]], dtype=torch.int32)
    n = torch.tensor([4], dtype=torch.int32)
    assert bench.order_flips(a, n, a, n, torch) == (0, 0, 6)
    r = torch.tensor([[7, 2, 9, 5]], dtype=torch.int32)
    assert bench.order_flips(a, n, r, n, torch) == (6, 1, 6)


def test_order_flips_truncated_lengths_count_the_stored_entries():
    a = torch.tensor([[1, 2, 3]], dtype=torch.int32)
    b = torch.tensor([[3, 2, 1]], dtype=torch.int32)
    # a length past the stored entries (a truncated probe) counts the stored entries only
    assert bench.order_flips(a, torch.tensor([9]), b, torch.tensor([9]), torch) == (3, 1, 3)
