"""Prints the polynomial coefficients of the FP64 sine and cosine in
bh_common.cuh (d_sincos): Chebyshev fits, at 40 digits, of
  g(x) = (sin(sqrt x) / sqrt x - 1) / x      (sin r = r + r^3 g(r^2)),
  h(x) = (cos(sqrt x) - 1 + x / 2) / x^2     (cos r = 1 - r^2 / 2 + r^4 h(r^2)),
on 0 <= x <= (pi/4)^2, the range left by the reduction by multiples of pi/2;
six terms each, highest degree first, with their bound on the result.
    python fit_sincos.py
"""
import mpmath as mp


def main():
    mp.mp.dps = 40
    X = (mp.pi / 4) ** 2

    def g(x):
        if x == 0:
            return mp.mpf(-1) / 6
        r = mp.sqrt(x)
        return (mp.sin(r) / r - 1) / x

    def h(x):
        if x == 0:
            return mp.mpf(1) / 24
        r = mp.sqrt(x)
        return (mp.cos(r) - 1 + x / 2) / (x * x)

    for name, f, scale in (("sin: g", g, X), ("cos: h", h, X * X)):
        poly, err = mp.chebyfit(f, [0, X], 6, error=True)
        print(f"{name}, |error| in the result <= {mp.nstr(err * scale, 3)}")
        for c in poly:
            print(f"  {float(c)!r}")


if __name__ == "__main__":
    main()
