"""Write twiddles.h: cos(2 pi k / 192) for k = 0..191 as double literals.

192 = 2^6 * 3 covers every FFT length the kernels use (N divides 192).  Values
are taken from the first octant (k <= 24) with the host libm and extended by
the exact symmetries of cosine, so cos(pi/2) = 0 and cos(pi/3) = 1/2 exactly.
Run from this directory: python gen_twiddles.py
"""
import math

N = 192


def first_octant(k):
    # 0 <= k <= N/8: direct evaluation
    return math.cos(2.0 * math.pi * k / N), math.sin(2.0 * math.pi * k / N)


def cos_exact(k):
    k %= N
    q = N // 4
    # reduce to [0, N/4] with sign
    sign = 1.0
    if k > N // 2:
        k = N - k
    if k > q:
        k = N // 2 - k
        sign = -1.0
    if k == q:
        return 0.0
    if k <= N // 8:
        return sign * first_octant(k)[0]
    return sign * first_octant(q - k)[1]


vals = [cos_exact(k) for k in range(N)]
vals[32] = 0.5   # cos(pi/3)
vals[160] = 0.5
vals[64] = -0.5  # cos(2 pi/3)
vals[128] = -0.5
rows = []
for i in range(0, N, 4):
    rows.append("    " + ", ".join(repr(v) for v in vals[i:i + 4]) + ",")
with open("twiddles.h", "w") as f:
    f.write("// Generated by gen_twiddles.py: cos(2 pi k / 192), k = 0..191.\n")
    f.write("#pragma once\n")
    f.write("#define WZ_TW_N 192\n")
    f.write("#define WZ_TW_TABLE \\\n")
    f.write(" \\\n".join(rows) + "\n")
