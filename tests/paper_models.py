"""The paper's three worked examples (Sec. V) written with the library's
front end (paper_2407_19987_gb300.model), for the front-end tests."""
from paper_2407_19987_gb300.model import Model


def seating():
    """Sec. V.A: 5x5 seats; -1 per occupied seat, +10 per three consecutive
    occupied seats in a row or a column."""
    m = Model()
    q = m.binary("q", (5, 5))
    H = -sum(q[i, j] for i in range(5) for j in range(5))
    for i in range(5):
        for j in range(3):
            H = H + 10 * q[i, j] * q[i, j + 1] * q[i, j + 2]
            H = H + 10 * q[j, i] * q[j + 1, i] * q[j + 2, i]
    return m, m.compile(H)


def pythagorean():
    """Sec. V.B: 4-bit integers x, y, z (least significant bit first);
    (x^2 + y^2 - z^2)^2 plus 10 for each integer that is zero."""
    m = Model()
    ints = [m.integer(n, 4) for n in ("x", "y", "z")]
    x, y, z = ints
    H = (x * x + y * y - z * z) ** 2
    for n in ("x", "y", "z"):
        zero = 1
        for b in m.bits(n):
            zero = zero * (1 - b)
        H = H + 10 * zero
    return m, m.compile(H)


def tsp():
    """Sec. V.C: 2-bit integers xB, xC, xD (most significant bit first);
    10 * (xB * xC * xD - 6)^2."""
    m = Model()
    xB, xC, xD = (m.integer(n, 2, msb_first=True) for n in ("xB", "xC", "xD"))
    return m, m.compile(10 * (xB * xC * xD - 6) ** 2)

