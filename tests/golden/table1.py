"""Reader for the paper's Table 1 values stored in paper_table1.txt."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def rows():
    out = []
    with open(os.path.join(HERE, "paper_table1.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, dim, impl, val, err, t = line.split()
            out.append(dict(integrand=name, dim=int(dim), impl=impl, value=float(val),
                            error=float(err), time_s=None if t == "-" else float(t)))
    return out


def row(integrand, dim, impl):
    for r in rows():
        if r["integrand"] == integrand and r["dim"] == dim and r["impl"] == impl:
            return r
    raise KeyError((integrand, dim, impl))
