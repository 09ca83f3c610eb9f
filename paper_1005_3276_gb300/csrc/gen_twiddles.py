"""Write twiddles.h: cos(2 pi k / 384) for k = 0..383 as double literals.

384 = 2^7 * 3 covers every FFT length the kernels use (N divides 384) and the
antiperiodic time momenta pi (2n + 1) / T up to T = 64 (2 T divides 384).
Values are taken from the first octant (k <= 48) with the host libm and
extended by the exact symmetries of cosine, so cos(pi/2) = 0 and
cos(pi/3) = 1/2 exactly.  The angle 2 pi k / 384 is the same double as
2 pi (k/2) / 192 for even k, so the entries of a shorter table are unchanged.
Run from this directory: python gen_twiddles.py
"""
import math

N = 384


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
vals[N // 6] = 0.5       # cos(pi/3)
vals[5 * N // 6] = 0.5
vals[N // 3] = -0.5      # cos(2 pi/3)
vals[2 * N // 3] = -0.5
rows = []
for i in range(0, N, 4):
    rows.append("    " + ", ".join(repr(v) for v in vals[i:i + 4]) + ",")
with open("twiddles.h", "w") as f:
    f.write(f"// Generated by gen_twiddles.py: cos(2 pi k / {N}), k = 0..{N - 1}.\n")
    f.write("#pragma once\n")
    f.write(f"#define WZ_TW_N {N}\n")
    f.write("#define WZ_TW_TABLE \\\n")
    f.write(" \\\n".join(rows) + "\n")
