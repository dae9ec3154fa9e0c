"""Generate straight-line in-register DFT codelets for the CUDA kernels.

``python gen_dft.py OUT.cuh`` writes ``DFT<N, SIGN>::run(float2* v)`` for every
size in ``SIZES``: an in-place DFT of ``N`` complex values held in registers,
``X_k = sum_n x_n exp(SIGN * 2 pi i n k / N)`` (unnormalised, natural order in
and out).  Composite sizes are split recursively down to radix-2/3/4/5
butterflies written from the DFT definition: sizes with coprime factors by the
Good-Thomas prime-factor mapping (no twiddle factors between the stages),
prime powers by mixed-radix Cooley-Tukey (``n = n1 + N1 n2``, ``k = k2 + N2
k1``) with twiddle factors as numeric literals computed here in double
precision.

Every emitted codelet is executed symbolically in float64 during generation
and compared with a direct DFT; generation fails if any differs.
"""
from __future__ import annotations

import math
import re
import sys
from types import SimpleNamespace

import numpy as np

SIZES = [2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30, 32]
ZERO_TAIL = [(8, 4), (16, 8)]   # (N, non-zero leading inputs) for zero-padded transforms


def flit(v: float) -> str:
    return repr(float(v)) + "f"


ZERO = "ZERO"   # an input known to be zero; ops on it are folded away


class Gen:
    def __init__(self, rng):
        self.lines: list[str] = []
        self.n = 0
        self.val: dict[str, complex] = {ZERO: 0j}
        self.flops = 0

    def fresh(self, value: complex) -> str:
        self.n += 1
        name = f"t{self.n}"
        self.val[name] = value
        return name

    # ---- primitive ops (each emits one CUDA statement and tracks the value) ----
    def add(self, a, b):
        if a == ZERO:
            return b
        if b == ZERO:
            return a
        r = self.fresh(self.val[a] + self.val[b])
        self.lines.append(f"const float2 {r} = make_float2({a}.x + {b}.x, {a}.y + {b}.y);")
        self.flops += 2
        return r

    def sub(self, a, b):
        if b == ZERO:
            return a
        if a == ZERO:
            return self.neg(b)
        r = self.fresh(self.val[a] - self.val[b])
        self.lines.append(f"const float2 {r} = make_float2({a}.x - {b}.x, {a}.y - {b}.y);")
        self.flops += 2
        return r

    def scale(self, a, c):
        if a == ZERO:
            return ZERO
        r = self.fresh(self.val[a] * c)
        self.lines.append(f"const float2 {r} = make_float2({flit(c)} * {a}.x, {flit(c)} * {a}.y);")
        self.flops += 2
        return r

    def mulj(self, a, s):
        """``a * (s * i)`` with ``s = +-1`` (no arithmetic, a swap and a negation)."""
        if a == ZERO:
            return ZERO
        r = self.fresh(self.val[a] * 1j * s)
        if s > 0:
            self.lines.append(f"const float2 {r} = make_float2(-{a}.y, {a}.x);")
        else:
            self.lines.append(f"const float2 {r} = make_float2({a}.y, -{a}.x);")
        return r

    def neg(self, a):
        if a == ZERO:
            return ZERO
        r = self.fresh(-self.val[a])
        self.lines.append(f"const float2 {r} = make_float2(-{a}.x, -{a}.y);")
        return r

    def fma_add(self, a, b, c):
        """``a + c * b`` for a real constant ``c``."""
        if b == ZERO:
            return a
        if a == ZERO:
            return self.scale(b, c)
        r = self.fresh(self.val[a] + c * self.val[b])
        self.lines.append(
            f"const float2 {r} = make_float2(fmaf({flit(c)}, {b}.x, {a}.x), fmaf({flit(c)}, {b}.y, {a}.y));")
        self.flops += 4
        return r

    def twiddle(self, a, e: int, N: int, sign: int):
        """``a * exp(sign * 2 pi i e / N)``."""
        if a == ZERO:
            return ZERO
        e %= N
        if e == 0:
            return a
        if (4 * e) % N == 0:
            q = (4 * e) // N          # multiple of a quarter turn
            if q == 2:
                return self.neg(a)
            return self.mulj(a, sign if q == 1 else -sign)
        ang = sign * 2 * math.pi * e / N
        c, s = math.cos(ang), math.sin(ang)
        if (8 * e) % N == 0:
            # (+-1 +- i)/sqrt(2): two adds and two multiplies
            h = math.sqrt(0.5)
            sc, ss = (1 if c > 0 else -1), (1 if s > 0 else -1)
            r = self.fresh(self.val[a] * complex(c, s))
            xr = f"({a}.x {'-' if ss * sc > 0 else '+'} {a}.y)"
            yr = f"({a}.y {'+' if ss * sc > 0 else '-'} {a}.x)"
            # re = c*ax - s*ay = sc*h*(ax - (ss/sc) ay); im = s*ax + c*ay = sc*h*(ay + (ss/sc) ax)
            self.lines.append(f"const float2 {r} = make_float2({flit(sc * h)} * {xr}, {flit(sc * h)} * {yr});")
            self.flops += 4
            return r
        r = self.fresh(self.val[a] * complex(c, s))
        self.lines.append(
            f"const float2 {r} = make_float2(fmaf({flit(c)}, {a}.x, {flit(-s)} * {a}.y), "
            f"fmaf({flit(s)}, {a}.x, {flit(c)} * {a}.y));")
        self.flops += 6
        return r

    # ---- butterflies from the DFT definition ----
    def bf2(self, x, sign):
        return [self.add(x[0], x[1]), self.sub(x[0], x[1])]

    def bf3(self, x, sign):
        # W = exp(sign 2 pi i / 3) = -1/2 + sign i sqrt(3)/2
        a, b, c = x
        t1 = self.add(b, c)
        t2 = self.fma_add(a, t1, -0.5)
        d = self.sub(b, c)
        t3 = self.scale(d, math.sqrt(3) / 2)
        t3 = self.mulj(t3, sign)
        return [self.add(a, t1), self.add(t2, t3), self.sub(t2, t3)]

    def bf4(self, x, sign):
        a, b, c, d = x
        s0, d0 = self.add(a, c), self.sub(a, c)
        s1, d1 = self.add(b, d), self.sub(b, d)
        j1 = self.mulj(d1, sign)
        return [self.add(s0, s1), self.add(d0, j1), self.sub(s0, s1), self.sub(d0, j1)]

    def bf5(self, x, sign):
        x0, x1, x2, x3, x4 = x
        c1, c2 = math.cos(2 * math.pi / 5), math.cos(4 * math.pi / 5)
        s1, s2 = math.sin(2 * math.pi / 5), math.sin(4 * math.pi / 5)
        t1, t2 = self.add(x1, x4), self.add(x2, x3)
        t3, t4 = self.sub(x1, x4), self.sub(x2, x3)
        X0 = self.add(self.add(x0, t1), t2)
        a1 = self.fma_add(self.fma_add(x0, t1, c1), t2, c2)
        a2 = self.fma_add(self.fma_add(x0, t1, c2), t2, c1)
        b1 = self.fma_add(self.scale(t3, s1), t4, s2)
        b2 = self.fma_add(self.scale(t3, s2), t4, -s1)
        jb1, jb2 = self.mulj(b1, sign), self.mulj(b2, sign)
        return [X0, self.add(a1, jb1), self.add(a2, jb2), self.sub(a2, jb2), self.sub(a1, jb1)]

    def dft(self, x, sign):
        N = len(x)
        if N == 1:
            return list(x)
        if N in (2, 3, 4, 5):
            return {2: self.bf2, 3: self.bf3, 4: self.bf4, 5: self.bf5}[N](x, sign)
        split = coprime_split(N)
        if split:
            return self.dft_pfa(x, sign, *split)
        N1 = next(r for r in (4, 2, 3, 5) if N % r == 0)   # outer radix
        N2 = N // N1
        Y = []
        for n1 in range(N1):
            y = self.dft([x[n1 + N1 * n2] for n2 in range(N2)], sign)
            Y.append([self.twiddle(y[k2], n1 * k2, N, sign) for k2 in range(N2)])
        X = [None] * N
        for k2 in range(N2):
            z = self.dft([Y[n1][k2] for n1 in range(N1)], sign)
            for k1 in range(N1):
                X[k2 + N2 * k1] = z[k1]
        return X


def coprime_split(N: int):
    """(N1, N2) with N = N1 N2, gcd(N1, N2) = 1, N1 the power-of-two part (or
    the smallest prime-power factor), or None for a prime power."""
    f = 1
    while N % (2 * f) == 0:
        f *= 2
    if f == 1:
        p = next(q for q in range(3, N + 1) if N % q == 0)
        f = p
        while N % (f * p) == 0:
            f *= p
    return (f, N // f) if 1 < f < N else None


def _dft_pfa(self, x, sign, N1, N2):
    """Good-Thomas prime-factor split for coprime N1, N2: input n = (n1 N2 +
    n2 N1) mod N, output k = the number with k = k1 (mod N1) and k = k2 (mod
    N2) (Chinese remainder theorem); the exponent n k / N then separates into
    n1 k1 / N1 + n2 k2 / N2, so no twiddle factors appear between the stages."""
    N = N1 * N2
    Y = [self.dft([x[(n1 * N2 + n2 * N1) % N] for n2 in range(N2)], sign) for n1 in range(N1)]
    X = [None] * N
    for k2 in range(N2):
        z = self.dft([Y[n1][k2] for n1 in range(N1)], sign)
        for k1 in range(N1):
            k = next(kk for kk in range(k2, N, N2) if kk % N1 == k1)
            X[k] = z[k1]
    return X


Gen.dft_pfa = _dft_pfa


def codelet(N: int, sign: int, rng, nz: int | None = None) -> tuple[str, int]:
    """DFT of N inputs of which only the first ``nz`` may be non-zero."""
    nz = N if nz is None else nz
    g = Gen(rng)
    vals = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    vals[nz:] = 0
    ins = []
    for i in range(N):
        name = f"i{i}" if i < nz else ZERO
        if i < nz:
            g.val[name] = vals[i]
        ins.append(name)
    outs = g.dft(ins, sign)
    n = np.arange(N)
    want = np.exp(sign * 2j * np.pi * np.outer(n, n) / N) @ vals
    got = np.array([g.val[o] for o in outs])
    if not np.allclose(got, want, rtol=1e-12, atol=1e-12):
        raise AssertionError(f"codelet N={N} sign={sign} is wrong")
    # execute the emitted statements themselves (not the tracked values)
    env = {"make_float2": lambda a, b: SimpleNamespace(x=a, y=b), "fmaf": lambda a, b, c: a * b + c,
           ZERO: SimpleNamespace(x=0.0, y=0.0)}
    for i in range(nz):
        env[f"i{i}"] = SimpleNamespace(x=vals[i].real, y=vals[i].imag)
    for line in g.lines:
        m = re.fullmatch(r"const float2 (t\d+) = (.*);", line)
        expr = re.sub(r"(\d)f\b", r"\1", m.group(2))
        env[m.group(1)] = eval(expr, env)
    got2 = np.array([env[o].x + 1j * env[o].y for o in outs])
    if not np.allclose(got2, want, rtol=1e-12, atol=1e-12):
        raise AssertionError(f"emitted code for N={N} sign={sign} is wrong")
    body = [f"    const float2 i{i} = v[{i}];" for i in range(nz)]
    body += ["    " + l for l in g.lines]
    body += [f"    v[{k}] = {'make_float2(0.f, 0.f)' if outs[k] == ZERO else outs[k]};" for k in range(N)]
    return "\n".join(body), g.flops


def main(out_path: str):
    rng = np.random.default_rng(12345)
    parts = [
        "// Generated by gen_dft.py -- in-register DFT codelets (do not edit).",
        "#pragma once",
        "#include <cuda_runtime.h>",
        "namespace pico {",
        "template <int N, int SIGN> struct DFT;",
        "template <int SIGN> struct DFT<1, SIGN> { static __device__ __forceinline__ void run(float2*) {} };",
    ]
    table = []
    for N in SIZES:
        for sign in (-1, 1):
            body, flops = codelet(N, sign, rng)
            parts.append(f"template <> struct DFT<{N}, {sign}> {{")
            parts.append("  static __device__ __forceinline__ void run(float2* v) {")
            parts.append(body)
            parts.append("  }")
            parts.append(f"  static constexpr int flops = {flops};")
            parts.append("};")
            table.append((N, sign, flops))
    # zero-tail variants: DFTZ<N, SIGN, NZ> treats inputs NZ..N-1 as zero
    parts.append("template <int N, int SIGN, int NZ> struct DFTZ;")
    for N, nz in ZERO_TAIL:
        for sign in (-1, 1):
            body, flops = codelet(N, sign, rng, nz)
            parts.append(f"template <> struct DFTZ<{N}, {sign}, {nz}> {{")
            parts.append("  static __device__ __forceinline__ void run(float2* v) {")
            parts.append(body)
            parts.append("  }")
            parts.append(f"  static constexpr int flops = {flops};")
            parts.append("};")
    parts.append("}  // namespace pico")
    with open(out_path, "w") as f:
        f.write("\n".join(parts) + "\n")
    return table


if __name__ == "__main__":
    t = main(sys.argv[1])
    for N, s, fl in t:
        if s < 0:
            print(f"N={N:3d} flops={fl:5d} ({fl / N:.1f}/pt, 5NlogN={5 * N * math.log2(N):.0f})")
