"""Writes fastmath_tables.cuh: the tables of the table-driven fp64 exp and log in
fastmath.cuh (the method of P. T. P. Tang, ACM TOMS 15 (1989) 144 and 16 (1990) 378).
Values are computed with Python's decimal module at 50 digits and rounded to the nearest
double (float(Decimal) rounds correctly).  Run: python gen_fastmath_tables.py"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 50
HERE = os.path.dirname(os.path.abspath(__file__))
LN2 = Decimal(2).ln()


def d(x: Decimal) -> str:
    return float(x).hex()


def main():
    lines = ["// fastmath_tables.cuh -- written by gen_fastmath_tables.py; do not edit.", "#pragma once", "",
             "namespace mdk {", ""]
    # exp: 2^(j/256), j = 0..255
    lines.append("// 2^(j/256), j = 0..255, rounded to double")
    vals = [d((LN2 * j / 256).exp()) for j in range(256)]
    lines.append("__device__ const double kExp2Tab[256] = {")
    lines += [f"    {v}," for v in vals]
    lines.append("};")
    # ln2/256 split into a head and a tail (head rounded to 32 significant bits so that
    # k * head is exact for |k| < 2^21)
    l64 = LN2 / 256
    head = float(l64)
    # keep 32 significant bits of the head
    import math
    m, e = math.frexp(head)
    head = math.ldexp(math.floor(m * 2 ** 32) / 2 ** 32, e)
    tail = float(l64 - Decimal(head))
    lines.append(f"constexpr double kLn2o256Hi = {head.hex()};   // ln2/256, 32 leading bits")
    lines.append(f"constexpr double kLn2o256Lo = {tail.hex()};   // ln2/256 - kLn2o256Hi")
    lines.append(f"constexpr double kInvLn2o256 = {d(256 / LN2)};   // 256/ln2")
    # ln2 split for the log
    h2 = float(LN2)
    m, e = math.frexp(h2)
    h2 = math.ldexp(math.floor(m * 2 ** 32) / 2 ** 32, e)
    t2 = float(LN2 - Decimal(h2))
    lines.append(f"constexpr double kLn2Hi = {h2.hex()};   // ln2, 32 leading bits")
    lines.append(f"constexpr double kLn2Lo = {t2.hex()};   // ln2 - kLn2Hi")
    lines.append("")
    # log: for the mantissa interval j (m in [1 + j/256, 1 + (j+1)/256)), c_j = 1 + (j + 1/2)/256,
    # inv_j = RN(1/c_j) and minus the logarithm of inv_j (exactly the inv used)
    inv, lg = [], []
    for j in range(256):
        c = 1 + (Decimal(j) + Decimal("0.5")) / 256
        iv = float(Decimal(1) / c)
        inv.append(iv.hex())
        lg.append(d(-Decimal(iv).ln()))
    lines.append("// 1/c_j rounded to double, c_j = 1 + (j + 1/2)/256, j = 0..255")
    lines.append("__device__ const double kLogInvTab[256] = {")
    lines += [f"    {v}," for v in inv]
    lines.append("};")
    lines.append("// -log(kLogInvTab[j]) rounded to double")
    lines.append("__device__ const double kLogTab[256] = {")
    lines += [f"    {v}," for v in lg]
    lines.append("};")
    # float-float routines: the reduction constants and polynomial coefficients as pairs of
    # floats (head rounded to float, tail = the rest rounded to float)
    def fpair(x: Decimal):
        import struct
        h = struct.unpack("f", struct.pack("f", float(x)))[0]
        t = struct.unpack("f", struct.pack("f", float(x - Decimal(h))))[0]
        return h, t
    lines.append("")
    lines.append("// ln2/256 - kLn2o256Hi as a float pair (head, tail)")
    ch, ct = fpair(l64 - Decimal(head))
    lines.append(f"constexpr float kLn2o256LoF[2] = {{{ch.hex()}f, {ct.hex()}f}};".replace("0x", "0x"))
    for name, val in (("kThirdF", Decimal(1) / 3), ("kSixthF", Decimal(1) / 6)):
        h, t = fpair(val)
        lines.append(f"constexpr float {name}[2] = {{{h.hex()}f, {t.hex()}f}};   // {name[1:-1].lower()} as a float pair")
    lines.append(f"constexpr float kLn2LoF[2] = {{{fpair(LN2 - Decimal(h2))[0].hex()}f, {fpair(LN2 - Decimal(h2))[1].hex()}f}};"
                 "   // ln2 - kLn2Hi as a float pair")
    # log with a float reciprocal: i_j = RN_float(1/c_j) and -log(i_j) (of that float) in double
    import struct
    invf, lgf = [], []
    for j in range(256):
        c = 1 + (Decimal(j) + Decimal("0.5")) / 256
        iv = struct.unpack("f", struct.pack("f", float(Decimal(1) / c)))[0]
        invf.append(iv.hex())
        lgf.append(d(-Decimal(iv).ln()))
    lines.append("// 1/c_j rounded to float, c_j = 1 + (j + 1/2)/256, j = 0..255")
    lines.append("__device__ const float kLogInvTabF[256] = {")
    lines += [f"    {v}f," for v in invf]
    lines.append("};")
    lines.append("// -log(kLogInvTabF[j]) rounded to double")
    lines.append("__device__ const double kLogTabF[256] = {")
    lines += [f"    {v}," for v in lgf]
    lines.append("};")
    # all-fp32 routines (exp_f2, log_f2): ln2/256 and ln2 as three floats each, the head cut to
    # few significant bits so that k * head is exact in fp32 (ln2/256: 9 bits, |k| < 2^15;
    # ln2: 16 bits, |e| < 2^8), the middle rounded to float, the tail = the rest rounded
    def f32(x: Decimal) -> float:
        return struct.unpack("f", struct.pack("f", float(x)))[0]

    def three(x: Decimal, head_bits: int):
        m, e = math.frexp(float(x))
        h = math.ldexp(math.floor(m * 2 ** head_bits) / 2 ** head_bits, e)
        mid = f32(x - Decimal(h))
        tail = f32(x - Decimal(h) - Decimal(mid))
        return h, mid, tail
    for name, val, bits, what in (("kLn2o256F3", l64, 9, "ln2/256"), ("kLn2F3", LN2, 16, "ln2")):
        a, b, c = three(val, bits)
        lines.append(f"constexpr float {name}[3] = {{{a.hex()}f, {b.hex()}f, {c.hex()}f}};   // {what}, head {bits} bits")
    lines += ["", "}  // namespace mdk", ""]
    with open(os.path.join(HERE, "fastmath_tables.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
