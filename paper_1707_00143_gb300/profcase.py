"""Small, self-contained workloads for kernel profiling (one kernel family per
case, a few GB of device memory at most), run as

    python -m paper_1707_00143_gb300.profcase search --n 300000 --nq 2000 --L 150 --prec 0
    python -m paper_1707_00143_gb300.profcase knn --n 262144 --K 100
    python -m paper_1707_00143_gb300.profcase build --n 300000

`search` builds an index (K=100, L=40, R=50, C=500) on an n-row SIFT-shaped
synthetic base and runs `--reps` searches of nq queries with top-k 100 at
pool size L in the given precision form (0 FP32, 1 BF16, 2 FP8, 3 U8);
`knn` runs one brute-force kNN graph construction; `build` one full index
construction.  Each prints one line when it finishes."""
import argparse
import sys

import torch

from . import build as B, capi, datagen


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["search", "knn", "build"])
    p.add_argument("--n", type=int, default=300000)
    p.add_argument("--nq", type=int, default=2000)
    p.add_argument("--L", type=int, default=150)
    p.add_argument("--K", type=int, default=100)
    p.add_argument("--prec", type=int, default=0)
    p.add_argument("--reps", type=int, default=2)
    a = p.parse_args(argv)
    B.build()
    torch.cuda.set_device(0)
    base, q = datagen.workload("sift", n=a.n, nq=a.nq)
    bt, qt = torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda()
    if a.case == "knn":
        capi.nsg_knn_init(bt, a.K, with_d2=False)
        torch.cuda.synchronize()
        print(f"knn n={a.n} K={a.K} done")
        return 0
    idx = capi.nsg_build(bt, a.K, 40, 50, 500)
    if a.case == "build":
        torch.cuda.synchronize()
        print(f"build n={a.n} done: {idx.info()}")
        return 0
    if a.prec:
        idx.prepare(a.prec)
    for _ in range(a.reps):
        idx.search_ex(qt, 100, a.L, params=capi.SearchParams(0, 0, a.prec), counters=False)
    torch.cuda.synchronize()
    print(f"search n={a.n} nq={a.nq} L={a.L} prec={a.prec} done")
    return 0


if __name__ == "__main__":
    sys.exit(main())
