"""Write exp2_table.h: the 256 values 2^(j/256), j = 0..255, each rounded to
the nearest double (computed with 200-bit mpmath), for the table-driven double
exponential of fp64_exp.cuh.  Usage: python gen_exp2_table.py > exp2_table.h"""
import mpmath

mpmath.mp.prec = 200

ENTRIES = 256


def table():
    return [float(mpmath.mpf(2) ** (mpmath.mpf(j) / ENTRIES)) for j in range(ENTRIES)]


def main():
    print(f"// 2^(j/{ENTRIES}), j = 0..{ENTRIES - 1}, rounded to nearest double "
          "(written by gen_exp2_table.py).")
    print("#pragma once")
    print()
    print("namespace vegas {")
    print()
    print(f"__device__ const double kExp2Table[{ENTRIES}] = {{")
    vals = table()
    for i in range(0, ENTRIES, 2):
        print(f"    {vals[i].hex()}, {vals[i + 1].hex()},")
    print("};")
    print()
    print("}  // namespace vegas")


if __name__ == "__main__":
    main()
