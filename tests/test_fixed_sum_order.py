"""The quadrature's fixed summation order (CPU only).

The oracle sums level by level (32-term chunks left to right, then
neighbouring pairs, an unpaired last entry moving up); the CUDA library
streams the same order with a binary-counter stack of chunk sums.  Both
forms are written out here in plain Python (IEEE doubles, one rounding per
addition) and must agree bit for bit for every length, including the ragged
ones around powers of two."""
import random

import pytest

CHUNK = 32


def level_sum(t):
    if not t:
        return 0.0
    c = []
    for k in range(0, len(t), CHUNK):
        a = 0.0
        for v in t[k:k + CHUNK]:
            a = a + v
        c.append(a)
    while len(c) > 1:
        nxt = [c[2 * k] + c[2 * k + 1] for k in range(len(c) // 2)]
        if len(c) % 2:
            nxt.append(c[-1])
        c = nxt
    return c[0]


def streamed_sum(t):
    stack, chunks, cur, inn = [], 0, 0.0, 0

    def push(s):
        nonlocal chunks
        chunks += 1
        n = chunks
        while n % 2 == 0:
            s = stack.pop() + s
            n //= 2
        stack.append(s)

    for v in t:
        cur = cur + v
        inn += 1
        if inn == CHUNK:
            push(cur)
            cur, inn = 0.0, 0
    if inn:
        push(cur)
    if not stack:
        return 0.0
    r = stack[-1]
    for s in reversed(stack[:-1]):
        r = s + r
    return r


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 63, 64, 65, 95, 96, 97, 2401,
                               32 * 77, 32 * 128 - 1, 32 * 128, 32 * 128 + 1,
                               14001, 100001])
def test_streamed_form_equals_level_order(n):
    rng = random.Random(n)
    # magnitudes spread over many binades so that the grouping changes the
    # rounding (a different order would almost surely give another double)
    t = [rng.random() * 10.0 ** rng.randint(-8, 3) for _ in range(n)]
    a, b = level_sum(t), streamed_sum(t)
    assert a == b or (a != a and b != b)


def test_order_is_not_the_serial_one():
    rng = random.Random(5)
    t = [rng.random() * 10.0 ** rng.randint(-8, 3) for _ in range(2401)]
    serial = 0.0
    for v in t:
        serial = serial + v
    assert serial != level_sum(t)          # the order matters at this size
    assert abs(serial - level_sum(t)) <= 2401 * 2.0 ** -53 * sum(t)
