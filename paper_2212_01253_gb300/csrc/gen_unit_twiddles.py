"""Writes the FP32 twiddle constants of the in-register radix stages
(kTwC / kTwS in mslice_device.cuh).

The radix-2 networks apply exp(-+ 2 pi i e / 32), e = 0..15.  Correctly
rounded FP32 cos/sin pairs all have c^2 + s^2 < 1 (by 1.5e-8 to 5.8e-8 here),
so every forward + inverse transform loses a little energy, the same amount in
every slice of the multislice loop.  Here e = 0 and e = 8 are exact and the
other pairs are chosen, within six ulps of the correctly rounded values and a
phase deviation of at most 2e-7 rad, so that the first-order energy drift of
a whole transform of length 64 ... 1024 (a 32-point network followed by an
N/32-point one; the drift is the sum of c^2 + s^2 - 1 over the twiddles an
output passes) is as close to zero as the FP32 grid allows.
The four symmetry classes {1,7,9,15}, {2,6,10,14}, {3,5,11,13}, {4,12} share
one magnitude each; a network of R points applies class k with the weights
computed below.  Run: python gen_unit_twiddles.py"""
import itertools
import math

import numpy as np


def candidates(e, span=6, max_dev=2e-7):
    C, S = math.cos(math.pi * e / 16), math.sin(math.pi * e / 16)
    c0, s0 = np.float32(C), np.float32(S)
    out = {}
    for dc in range(-span, span + 1):
        c = c0
        for _ in range(abs(dc)):
            c = np.nextafter(c, np.float32(math.copysign(np.inf, dc)))
        for ds in range(-span, span + 1):
            s = s0
            for _ in range(abs(ds)):
                s = np.nextafter(s, np.float32(math.copysign(np.inf, ds)))
            dev = abs(float(c) * S - float(s) * C)
            if dev > max_dev:
                continue
            m = float(c) * float(c) + float(s) * float(s) - 1.0
            key = round(m * 1e13)
            if key not in out or dev < out[key][1]:
                out[key] = (m, dev, c, s)
    return sorted(out.values(), key=lambda x: abs(x[0]))[:10]


def class_weights(R):
    """Fraction of the R outputs of a radix-2 DIF network that pass each
    twiddle class, summed over the stages (first-order energy drift weights)."""
    w = {1: 0.0, 2: 0.0, 3: 0.0, 4: 0.0}
    half = R // 2
    while half >= 1:
        for blk in range(0, R, 2 * half):
            for k in range(half):
                e = k * (32 // (2 * half))
                cls = {1: 1, 7: 1, 9: 1, 15: 1, 2: 2, 6: 2, 10: 2, 14: 2, 3: 3, 5: 3, 11: 3, 13: 3, 4: 4, 12: 4}.get(e)
                if cls:
                    w[cls] += 1.0 / R
        half //= 2
    return w


def choose():
    """Class representatives minimising the worst first-order energy drift of
    a whole length-N transform, N = 64 ... 1024 (a 32-point network followed by
    an N/32-point one), ties broken by the largest phase deviation."""
    cl = {k: sorted(candidates(k), key=lambda x: abs(x[0]))[:12] for k in (1, 2, 3, 4)}
    w = {R: class_weights(R) for R in (32, 16, 8, 4, 2)}
    best = None
    for pick in itertools.product(*[cl[k] for k in (1, 2, 3, 4)]):
        m = {k: pick[k - 1][0] for k in (1, 2, 3, 4)}
        d = {R: sum(w[R][k] * m[k] for k in m) for R in w}
        drift = max(abs(d[32] + d[N // 32]) for N in (64, 128, 256, 512, 1024))
        score = (drift, max(p[1] for p in pick))
        if best is None or score < best[0]:
            best = (score, pick)
    return best


def table(pick):
    """(c, s) for e = 0..15 from the class representatives e = 1..4."""
    base = {1: pick[0], 2: pick[1], 3: pick[2], 4: pick[3]}
    cs = {0: (np.float32(1), np.float32(0)), 8: (np.float32(0), np.float32(1))}
    for e in (1, 2, 3, 4):
        c, s = base[e][2], base[e][3]
        cs[e] = (c, s)
        if e != 4:
            cs[8 - e] = (s, c)                          # cos((8-e) pi/16) = sin(e pi/16)
    for e in range(9, 16):
        c, s = cs[e - 8]
        cs[e] = (np.float32(-s), c)                    # rotation by pi/2
    return [cs[e] for e in range(16)]


def main():
    (drift, _), pick = choose()
    cs = table(pick)
    for name, idx in (("kTwC", 0), ("kTwS", 1)):
        print("__host__ __device__ __forceinline__ constexpr float %s(int e) {" % name)
        print("    switch (e) {")
        for e, pair in enumerate(cs):
            v = float(pair[idx])
            lit = "%sf" % float.hex(v) if v != 0 else "0.0f"
            print(("        case %d: return %s;" % (e, lit)) if e < 15 else ("        default: return %s;" % lit))
        print("    }")
        print("}")
    print("// worst first-order energy drift of a length 64..1024 transform: %.2e" % drift)
    for e, (c, s) in enumerate(cs):
        print("// e=%2d |w|^2-1 = %+.3e  phase dev %.1e" % (
            e, float(c) ** 2 + float(s) ** 2 - 1,
            abs(float(c) * math.sin(math.pi * e / 16) - float(s) * math.cos(math.pi * e / 16))))


if __name__ == "__main__":
    main()
