"""The closed form that the exact box check evaluates (the Bernstein
coefficients of a quadratic on [s/n, (s+1)/n], n = 2^d, scaled by n^2)
against d successive de Casteljau halvings of the same row, in exact
rationals, for random rows, depths and positions; and the 3D tensor version
against halving a random 27-coefficient box along a random path of
children."""
import random
from fractions import Fraction as F


def halve(row, right):
    p0, p1, p2 = row
    m = (p0 + 2 * p1 + p2) / 4
    return (m, (p1 + p2) / 2, p2) if right else (p0, (p0 + p1) / 2, m)


def closed_form(row, d, s):
    n = 2 ** d
    a, b, am = n - s, s + 1, n - s - 1
    w = ((a * a, 2 * s * a, s * s), (a * am, a * b + s * am, s * b), (am * am, 2 * b * am, b * b))
    return tuple(sum(F(wi[m]) * row[m] for m in range(3)) / (n * n) for wi in w)


def test_rows():
    rng = random.Random(11)
    for _ in range(300):
        row = tuple(F(rng.randint(-10**6, 10**6), rng.randint(1, 1000)) for _ in range(3))
        d = rng.randint(0, 15)
        s = rng.randrange(2 ** d)
        r = row
        for bit in range(d - 1, -1, -1):  # most significant bit first: the first split
            r = halve(r, (s >> bit) & 1)
        assert r == closed_form(row, d, s)


def test_weights_are_nonnegative_and_sum_to_n2():
    for d in range(16):
        n = 2 ** d
        for s in {0, n // 3, n // 2, n - 1}:
            a, b, am = n - s, s + 1, n - s - 1
            for w in ((a * a, 2 * s * a, s * s), (a * am, a * b + s * am, s * b),
                      (am * am, 2 * b * am, b * b)):
                assert min(w) >= 0 and sum(w) == n * n and max(w) < 2 ** 31


def test_tensor_box():
    rng = random.Random(12)
    for _ in range(20):
        box = {(i, j, k): F(rng.randint(-999, 999), rng.randint(1, 50))
               for i in range(3) for j in range(3) for k in range(3)}
        root = dict(box)
        d = rng.randint(1, 6)
        pos = [0, 0, 0]
        for _ in range(d):
            o = [rng.randint(0, 1) for _ in range(3)]
            for axis in range(3):
                new = {}
                for key in box:
                    if key[axis] != 0:
                        continue
                    line = [box[tuple(key[:axis]) + (m,) + tuple(key[axis + 1:])] for m in range(3)]
                    h = halve(line, o[axis])
                    for m in range(3):
                        new[tuple(key[:axis]) + (m,) + tuple(key[axis + 1:])] = h[m]
                box = new
                pos[axis] = 2 * pos[axis] + o[axis]
        got = dict(root)
        for axis in range(3):
            new = {}
            for key in got:
                if key[axis] != 0:
                    continue
                line = [got[tuple(key[:axis]) + (m,) + tuple(key[axis + 1:])] for m in range(3)]
                c = closed_form(line, d, pos[axis])
                for m in range(3):
                    new[tuple(key[:axis]) + (m,) + tuple(key[axis + 1:])] = c[m]
            got = new
        assert got == box
