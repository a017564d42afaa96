"""Precision study of the neighbour decision (Tables 1 and 2 of arXiv
2401.08586) on the GPU: wrong-decision counts of FP16 / FP32 absolute
coordinates and of FP16 cell-relative coordinates alone, next to this
library's tiered decision.  Run: ``python -m paper_2401_08586_gb300.study``.

Table 1 set-up: a centre particle and 60 particles at distance kh (1 +- dR)
in random directions (kh = 1, centre at the origin); only the centre's 60
decisions are counted.  Table 2 set-up: N random particles in the unit square
with spacing ds = N^(-1/2), h = 1.2 ds, kh = 2h (the paper does not state h);
the percentage is wrong decisions over true neighbour pairs.
"""
import json
import sys

PAPER_T1 = {"fp32": [0, 0, 0, 0, 0, 39], "fp16": [0, 0, 1, 34, 53, 57]}
T1_DR = [1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-8]
PAPER_T2 = {"all-list / link-list": [0, 0.028, 0.17, 1.2, 3.3, 31], "RCLL": [0, 0, 0, 0, 0, 0]}
T2_DS = [0.01, 0.005, 0.002, 0.00125, 0.001, 0.0005]


def table1(sph, torch, count=60, seed=0):
    from . import workloads as W
    rows = []
    for dR in T1_DR:
        xyz = W.circle_pairs(1.0, dR, count, dim=2, seed=seed, center=(0.0, 0.0))
        g = sph.Grid(torch.from_numpy(xyz).cuda(), 0.5, 1.0)
        c = sph.sph_precision_study(g.handle, 0, 1)
        g.close()
        rows.append(dict(dR=dR, **c))
    return rows


def table2(sph, torch, ds_list=T2_DS, seed=1):
    from . import workloads as W
    rows = []
    for ds in ds_list:
        n = int(round(1.0 / ds ** 2))
        xyz = W.random_uniform(n, 2, seed)
        h = 1.2 * ds
        g = sph.Grid(torch.from_numpy(xyz).cuda(), h, 2 * h)
        c = sph.sph_precision_study(g.handle)
        g.close()
        pct = {k: 100.0 * c[k] / max(c["neighbours"], 1) for k in
               ("wrong_fp16_abs", "wrong_fp32_abs", "wrong_fp16_rcll", "wrong_tiered")}
        rows.append(dict(ds=ds, n=n, **c, pct=pct))
    return rows


def main():
    import torch
    from . import sph
    sph.load()
    t1 = table1(sph, torch)
    t2 = table2(sph, torch)
    print("Table 1 (centre particle, 60 on the circle): wrong decisions")
    print("%-8s %8s %8s %8s %8s | paper FP32 FP16" % ("dR", "fp16abs", "fp32abs", "fp16rcll", "tiered"))
    for k, r in enumerate(t1):
        print("%-8.0e %8d %8d %8d %8d | %5d %5d" % (r["dR"], r["wrong_fp16_abs"], r["wrong_fp32_abs"],
                                                     r["wrong_fp16_rcll"], r["wrong_tiered"],
                                                     PAPER_T1["fp32"][k], PAPER_T1["fp16"][k]))
    print("Table 2 (random unit square): wrong decisions, % of neighbour pairs")
    print("%-8s %9s %9s %9s %9s %9s | paper list RCLL" % ("ds", "N", "fp16abs", "fp32abs", "fp16rcll", "tiered"))
    for k, r in enumerate(t2):
        p = r["pct"]
        print("%-8g %9d %9.4f %9.4f %9.4f %9.4f | %6g %4g" % (r["ds"], r["n"], p["wrong_fp16_abs"],
                                                             p["wrong_fp32_abs"], p["wrong_fp16_rcll"],
                                                             p["wrong_tiered"], PAPER_T2["all-list / link-list"][k],
                                                             PAPER_T2["RCLL"][k]))
    if "--json" in sys.argv:
        print(json.dumps({"table1": t1, "table2": t2}))


if __name__ == "__main__":
    main()
