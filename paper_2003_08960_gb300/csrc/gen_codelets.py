#!/usr/bin/env python3
"""Writes fft_codelets.cuh: straight-line in-register DFTs for the CUDA kernels.

Build step of the library (run by the package's build script).  For each size R
in SIZES and each sign, it emits

    template<> struct Dft<R, SIGN> {
      template<int ST, int OFF> static __host__ __device__ __forceinline__ void run(float2* x);
    };

which replaces x[OFF + k*ST], k = 0..R-1, by sum_j x[OFF + j*ST] exp(SIGN 2 pi i j k / R)
(unnormalised, natural order in and out).  Indices are compile-time constants, so
a register array passed in stays in registers.

Power-of-two sizes use split-radix decimation in time (Duhamel and Hollmann,
1984) with the trivial twiddles (1, +-i, (+-1 +- i)/sqrt 2) expanded into
additions; sizes 3 and 5 use the
direct real/imaginary symmetric form; composite sizes with a factor 3 or 5 use
one mixed-radix (Cooley-Tukey) split.  Twiddle constants are computed here in
float64 and rounded once to float32.
"""

import math
import os
import sys

SIZES = [2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 25, 32, 40]


def f32(v: float) -> str:
    import struct
    r = struct.unpack("f", struct.pack("f", v))[0]
    s = repr(float(r))
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


class Gen:
    def __init__(self):
        self.lines = []
        self.n = 0

    def var(self):
        self.n += 1
        return f"v{self.n}"

    def emit(self, s):
        self.lines.append("    " + s)

    # complex helpers producing new SSA names ---------------------------------
    def add(self, a, b):
        v = self.var()
        self.emit(f"const float2 {v} = make_float2({a}.x + {b}.x, {a}.y + {b}.y);")
        return v

    def sub(self, a, b):
        v = self.var()
        self.emit(f"const float2 {v} = make_float2({a}.x - {b}.x, {a}.y - {b}.y);")
        return v

    def twiddle(self, a, k, n, sign):
        """a * exp(sign 2 pi i k / n), with the trivial cases expanded."""
        k %= n
        if k == 0:
            return a
        g = math.gcd(k, n)
        kk, nn = k // g, n // g
        v = self.var()
        s = sign
        if nn == 2:
            self.emit(f"const float2 {v} = make_float2(-{a}.x, -{a}.y);")
        elif nn == 4:
            # exp(s i pi/2 * kk): kk = 1 -> s i ; kk = 3 -> -s i
            q = s if kk == 1 else -s
            if q > 0:
                self.emit(f"const float2 {v} = make_float2(-{a}.y, {a}.x);")
            else:
                self.emit(f"const float2 {v} = make_float2({a}.y, -{a}.x);")
        elif nn == 8:
            r = f32(math.sqrt(0.5))
            c = math.cos(2 * math.pi * kk / 8)
            sn = s * math.sin(2 * math.pi * kk / 8)
            cs = "+" if c > 0 else "-"
            # (a.x + i a.y)(c + i sn) with |c| = |sn| = r
            if sn > 0:
                re = f"{cs}{a}.x - {a}.y"
                im = f"{cs}{a}.y + {a}.x"
            else:
                re = f"{cs}{a}.x + {a}.y"
                im = f"{cs}{a}.y - {a}.x"
            re = re.lstrip("+")
            im = im.lstrip("+")
            self.emit(f"const float2 {v} = make_float2(({re}) * {r}, ({im}) * {r});")
        else:
            c = f32(math.cos(2 * math.pi * kk / nn))
            sn = f32(s * math.sin(2 * math.pi * kk / nn))
            self.emit(f"const float2 {v} = make_float2(fmaf({a}.x, {c}, -{a}.y * {sn}), "
                      f"fmaf({a}.x, {sn}, {a}.y * {c}));")
        return v

    # DFTs ---------------------------------------------------------------------
    def dft(self, xs, sign):
        n = len(xs)
        if n == 1:
            return list(xs)
        if n == 2:
            return [self.add(xs[0], xs[1]), self.sub(xs[0], xs[1])]
        if n == 3:
            return self.dft3(xs, sign)
        if n == 5:
            return self.dft5(xs, sign)
        if n % 4 == 0 and (n & (n - 1)) == 0:
            return self.split_radix(xs, sign)
        # mixed radix: n = p * m with p the smallest prime factor in {2,3,5}
        for p in (2, 3, 5):
            if n % p == 0:
                break
        else:
            raise ValueError(n)
        m = n // p
        # decimation in time: x[j] with j = p*j2 + j1 ... use x[j1 + p*j2]
        sub_out = [self.dft(xs[j1::p], sign) for j1 in range(p)]   # each length m, index k2
        out = [None] * n
        for k2 in range(m):
            col = [self.twiddle(sub_out[j1][k2], j1 * k2, n, sign) for j1 in range(p)]
            res = self.dft(col, sign)                               # length p, index k1
            for k1 in range(p):
                out[k2 + m * k1] = res[k1]
        return out

    def mul_i(self, a, s):
        """a * (s i), s = +-1: a swap and a negation, no arithmetic."""
        v = self.var()
        if s > 0:
            self.emit(f"const float2 {v} = make_float2(-{a}.y, {a}.x);")
        else:
            self.emit(f"const float2 {v} = make_float2({a}.y, -{a}.x);")
        return v

    def fma2(self, a, c, b):
        """b + c * a for a real constant c (two FMAs)."""
        v = self.var()
        cs = f32(c)
        self.emit(f"const float2 {v} = make_float2(fmaf({a}.x, {cs}, {b}.x), fmaf({a}.y, {cs}, {b}.y));")
        return v

    def rot(self, a, k, n, sign):
        """a * exp(sign 2 pi i k / n) as (r, c) with the product equal to c * r.
        W = C + iS is written C (1 + i S/C) when |C| >= |S|, else S (C/S + i),
        so r costs two FMAs (or nothing / two additions for the trivial
        twiddles) and |c| >= 1/sqrt 2; the scale c is folded into the FMAs of
        the butterflies that use the product."""
        k %= n
        if k == 0:
            return a, 1.0
        g = math.gcd(k, n)
        kk, nn = k // g, n // g
        if nn == 2:
            return a, -1.0
        if nn == 4:
            return self.mul_i(a, sign if kk == 1 else -sign), 1.0
        ang = 2 * math.pi * kk / nn
        C, S = math.cos(ang), sign * math.sin(ang)
        v = self.var()
        if nn == 8:
            # (+-1 +- i) / sqrt 2: r = a (C' + i S') with C', S' = +-1, two additions
            cx, sx = (1 if C > 0 else -1), (1 if S > 0 else -1)
            re = f"{'' if cx > 0 else '-'}{a}.x {'-' if sx > 0 else '+'} {a}.y"
            im = f"{'' if cx > 0 else '-'}{a}.y {'+' if sx > 0 else '-'} {a}.x"
            self.emit(f"const float2 {v} = make_float2({re}, {im});")
            return v, math.sqrt(0.5)
        if abs(C) >= abs(S):
            t = f32(S / C)
            self.emit(f"const float2 {v} = make_float2(fmaf(-{a}.y, {t}, {a}.x), fmaf({a}.x, {t}, {a}.y));")
            return v, C
        t = f32(C / S)
        self.emit(f"const float2 {v} = make_float2(fmaf({a}.x, {t}, -{a}.y), fmaf({a}.y, {t}, {a}.x));")
        return v, S

    def split_radix(self, xs, sign):
        """Split-radix decimation in time (Duhamel and Hollmann, 1984), n a power
        of two >= 4: U = DFT_{n/2} of the even samples, Z and Z' = DFT_{n/4} of
        the samples 4m+1 and 4m+3.  With W = exp(sign 2 pi i / n),
        t1 = W^k Z[k], t2 = W^{3k} Z'[k], s = t1 + t2, d = t1 - t2:
            X[k]        = U[k] + s          X[k + n/2]  = U[k] - s
            X[k + n/4]  = U[k + n/4] + sign i d
            X[k + 3n/4] = U[k + n/4] - sign i d        (k = 0 .. n/4 - 1).
        The twiddle products are kept scaled (t1 = c1 r1, t2 = c3 r3), so that
        s = c1 (r1 + (c3/c1) r3) and the outputs are fused multiply-adds with
        c1: four FMAs per twiddle pair instead of the multiplications of the
        plain form."""
        n = len(xs)
        u = self.dft(xs[0::2], sign)
        z1 = self.dft(xs[1::4], sign)
        z3 = self.dft(xs[3::4], sign)
        out = [None] * n
        q = n // 4
        for k in range(q):
            r1, c1 = self.rot(z1[k], k, n, sign)
            r3, c3 = self.rot(z3[k], 3 * k, n, sign)
            rho = c3 / c1
            if abs(rho - 1.0) < 1e-12:
                sm, df = self.add(r1, r3), self.sub(r1, r3)
            elif abs(rho + 1.0) < 1e-12:
                sm, df = self.sub(r1, r3), self.add(r1, r3)
            else:
                sm, df = self.fma2(r3, rho, r1), self.fma2(r3, -rho, r1)
            df = self.mul_i(df, sign)
            if abs(c1 - 1.0) < 1e-12:
                out[k], out[k + 2 * q] = self.add(u[k], sm), self.sub(u[k], sm)
                out[k + q], out[k + 3 * q] = self.add(u[k + q], df), self.sub(u[k + q], df)
            elif abs(c1 + 1.0) < 1e-12:
                out[k], out[k + 2 * q] = self.sub(u[k], sm), self.add(u[k], sm)
                out[k + q], out[k + 3 * q] = self.sub(u[k + q], df), self.add(u[k + q], df)
            else:
                out[k], out[k + 2 * q] = self.fma2(sm, c1, u[k]), self.fma2(sm, -c1, u[k])
                out[k + q], out[k + 3 * q] = self.fma2(df, c1, u[k + q]), self.fma2(df, -c1, u[k + q])
        return out

    def dft3(self, xs, sign):
        a, b, c = xs
        s = self.add(b, c)
        d = self.sub(b, c)
        y0 = self.add(a, s)
        # y1 = a - s/2 + sign * i * (sqrt3/2) * (b - c);  y2 = a - s/2 - ...
        h = self.var()
        self.emit(f"const float2 {h} = make_float2(fmaf({s}.x, -0.5f, {a}.x), fmaf({s}.y, -0.5f, {a}.y));")
        r = f32(sign * math.sqrt(3.0) / 2.0)
        y1 = self.var()
        y2 = self.var()
        self.emit(f"const float2 {y1} = make_float2(fmaf(-{d}.y, {r}, {h}.x), fmaf({d}.x, {r}, {h}.y));")
        self.emit(f"const float2 {y2} = make_float2(fmaf({d}.y, {r}, {h}.x), fmaf(-{d}.x, {r}, {h}.y));")
        return [y0, y1, y2]

    def dft5(self, xs, sign):
        x0, x1, x2, x3, x4 = xs
        s1 = self.add(x1, x4)
        d1 = self.sub(x1, x4)
        s2 = self.add(x2, x3)
        d2 = self.sub(x2, x3)
        y0 = self.var()
        self.emit(f"const float2 {y0} = make_float2({x0}.x + {s1}.x + {s2}.x, {x0}.y + {s1}.y + {s2}.y);")
        c1, c2 = math.cos(2 * math.pi / 5), math.cos(4 * math.pi / 5)
        n1, n2 = sign * math.sin(2 * math.pi / 5), sign * math.sin(4 * math.pi / 5)
        # y_k = x0 + s1 cos(2pi k/5) + s2 cos(4pi k/5) + i [d1 sin(2pi k/5) + d2 sin(4pi k/5)] * sign
        outs = [y0]
        coef = {1: (c1, c2, n1, n2), 2: (c2, c1, n2, -n1)}
        tmp = {}
        for k in (1, 2):
            ca, cb, sa, sb = coef[k]
            re = self.var()
            im = self.var()
            self.emit(f"const float2 {re} = make_float2(fmaf({s1}.x, {f32(ca)}, fmaf({s2}.x, {f32(cb)}, {x0}.x)), "
                      f"fmaf({s1}.y, {f32(ca)}, fmaf({s2}.y, {f32(cb)}, {x0}.y)));")
            self.emit(f"const float2 {im} = make_float2(fmaf({d1}.x, {f32(sa)}, {d2}.x * {f32(sb)}), "
                      f"fmaf({d1}.y, {f32(sa)}, {d2}.y * {f32(sb)}));")
            tmp[k] = (re, im)
        # multiply im-part by i: i*(u) = (-u.y, u.x)
        for k in (1, 2):
            re, im = tmp[k]
            v = self.var()
            self.emit(f"const float2 {v} = make_float2({re}.x - {im}.y, {re}.y + {im}.x);")
            tmp[k] = tmp[k] + (v,)
        for k in (3, 4):
            re, im = tmp[5 - k][:2]
            v = self.var()
            self.emit(f"const float2 {v} = make_float2({re}.x + {im}.y, {re}.y - {im}.x);")
            tmp[k] = (None, None, v)
        return [y0, tmp[1][2], tmp[2][2], tmp[3][2], tmp[4][2]]


def codelet(n, sign):
    g = Gen()
    ins = []
    for k in range(n):
        v = f"x{k}"
        g.emit(f"const float2 {v} = x[OFF + {k} * ST];")
        ins.append(v)
    outs = g.dft(ins, sign)
    for k, v in enumerate(outs):
        g.emit(f"x[OFF + {k} * ST] = {v};")
    body = "\n".join(g.lines)
    return (f"template <> struct Dft<{n}, {sign}> {{\n"
            f"  template <int ST, int OFF>\n"
            f"  static __host__ __device__ __forceinline__ void run(float2* x) {{\n{body}\n  }}\n}};\n")


def main(out_path):
    parts = [
        "// Generated by gen_codelets.py: straight-line in-register DFTs.  Do not edit.\n"
        "// The build rewrites this file; the copy kept in the tree must equal the\n"
        "// generator's output (checked by tests/test_codelets_host.py).\n",
        "#pragma once\n#include <cuda_runtime.h>\n\nnamespace ssoct {\n",
        "template <int N, int SIGN> struct Dft;\n",
        "template <int SIGN> struct Dft<1, SIGN> {\n  template <int ST, int OFF>\n"
        "  static __host__ __device__ __forceinline__ void run(float2*) {}\n};\n",
    ]
    for n in SIZES:
        for sign in (1, -1):
            parts.append(codelet(n, sign))
    parts.append("}  // namespace ssoct\n")
    text = "\n".join(parts)
    if os.path.exists(out_path) and open(out_path).read() == text:
        return
    with open(out_path, "w") as f:
        f.write(text)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "fft_codelets.cuh"))
