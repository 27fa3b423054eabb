"""Prints the tables of the FP64 log(1 + x) in bh_common.cuh (d_log1p).

For m in [1, 2) the six leading fraction bits pick j = floor(64 (m - 1)) and
a factor r_j close to 1/m, so that z = m r_j - 1 is small and
    log m = s_j ln 2 + T_j + log(1 + z),   T_j = -log(r_j) - s_j ln 2,
with s_j = 1 for j >= 32 (there log m is near ln 2, and the ln 2 is moved
into the exponent's multiple so that log u for u just below 1 does not
cancel) and s_j = 0 below.
  j = 0:        r = 1 exactly, T = 0 (z = m - 1 exact, 0 <= z < 1/64);
  1 <= j <= 62: r_j = the double nearest 1 / (1 + (j + 1/2) / 64),
                |z| <= 1/128;
  j = 63:       r = 1/2 exactly, T = 0 (z = m/2 - 1 exact, -1/128 <= z < 0).
T_j is printed as hi + lo, each a double, at 40 digits of working precision.
    python gen_log_table.py
"""
import mpmath as mp


def tables():
    mp.mp.dps = 40
    r, hi, lo = [], [], []
    for j in range(64):
        if j == 0:
            rj = 1.0
        elif j == 63:
            rj = 0.5
        else:
            rj = float(1 / (1 + (mp.mpf(j) + mp.mpf(1) / 2) / 64))
        s = 1 if j >= 32 else 0
        t = -mp.log(mp.mpf(rj)) - s * mp.log(2)
        th = float(t)
        tl = float(t - mp.mpf(th))
        r.append(rj)
        hi.append(th)
        lo.append(tl)
    return r, hi, lo


def main():
    for name, vals in zip(("kLogR", "kLogTHi", "kLogTLo"), tables()):
        print(f"static __device__ const double {name}[64] = {{")
        for i in range(0, 64, 4):
            print("    " + ", ".join(repr(v) for v in vals[i:i + 4]) + ",")
        print("};")


if __name__ == "__main__":
    main()
