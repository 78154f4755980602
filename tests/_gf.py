"""Independent GF(2^p) arithmetic for the tests: shift-and-add multiplication
reduced by the field polynomial, one bit at a time (no tables)."""

POLY = {1: 0x3, 2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x89, 8: 0x11D}


def mul(a: int, b: int, p: int, poly: int | None = None) -> int:
    poly = POLY[p] if poly is None else poly
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> p:
            a ^= poly
    return r


def table(q: int, poly: int | None = None):
    p = q.bit_length() - 1
    return [[mul(a, b, p, poly) for b in range(q)] for a in range(q)]


def syndrome(rows, cols, vals, M, x, q):
    p = q.bit_length() - 1
    z = [0] * M
    for r, c, h in zip(rows, cols, vals):
        z[int(r)] ^= mul(int(h), int(x[int(c)]), p)
    return z
