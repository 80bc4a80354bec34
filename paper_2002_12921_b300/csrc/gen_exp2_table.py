"""Write exp2_table.h: the 64 values 2^(j/64), j = 0..63, each rounded to the
nearest double (computed with 200-bit mpmath), for the table-driven double
exponential of fp64_exp.cuh.  Usage: python gen_exp2_table.py > exp2_table.h"""
import mpmath

mpmath.mp.prec = 200


def table():
    return [float(mpmath.mpf(2) ** (mpmath.mpf(j) / 64)) for j in range(64)]


def main():
    print("// 2^(j/64), j = 0..63, rounded to nearest double (written by gen_exp2_table.py).")
    print("#pragma once")
    print()
    print("namespace vegas {")
    print()
    print("__device__ const double kExp2Over64[64] = {")
    vals = table()
    for i in range(0, 64, 2):
        print(f"    {vals[i].hex()}, {vals[i + 1].hex()},")
    print("};")
    print()
    print("}  // namespace vegas")


if __name__ == "__main__":
    main()
