"""Writes ``rmat24_ef16_truss.txt``: the trussness of every edge of the
R-MAT scale-24 workload (edge factor 16, a/b/c/d = .57/.19/.19/.05, seed 4),
reduced to SHA-256 digests, computed by the CPU oracle alone.

The oracle's serial peel (Algorithm 1, §II) needs several hours on one core
for this graph (Σ min(d(u), d(v)) ≈ 2.7e11 row entries), far too long for a
test, so it is run once by this script and its result stored as:

* the SHA-256 of the canonical edge list (int32 u then int32 v, little
  endian, canonical order: (min, max) lexicographic) — identifies the input;
* the SHA-256 of the trussness array (int32, little endian, canonical order);
* m, the largest trussness and the number of edges of each trussness.

A GPU test hashes the device's edge list and trussness the same way and
compares them with these digests, which fixes every edge.  The R-MAT draws
use only an exact integer-to-double scaling and comparisons, so the raw
edge list is the same bits on every host architecture.

Run: ``python tests/golden/make_rmat24_digest.py`` (about 8 GB of host
memory; it calls only ``graphgen`` for the input and ``oracle`` for every
result).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(_HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(_HERE, "rmat24_ef16_truss.txt")


def digest_i32(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def main() -> None:
    t0 = time.time()
    g = graphgen.workload("rmat24_ef16")
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    del g
    t1 = time.time()
    print(f"canonical: m = {eu.shape[0]} ({t1 - t0:.0f} s)", flush=True)
    tau = oracle.truss(1 << 24, eu, ev)
    t2 = time.time()
    print(f"oracle trussness: {t2 - t1:.0f} s", flush=True)
    hist = np.bincount(tau)
    lines = [
        "# Trussness of the R-MAT scale-24 workload (edge factor 16, a/b/c/d = .57/.19/.19/.05,",
        "# seed 4, 2^28 raw samples, self-loops and repeats dropped), computed by the CPU",
        "# oracle's serial peel (Algorithm 1; trussness as defined in §II) and written by",
        "# make_rmat24_digest.py.  Digests are SHA-256 over int32 little-endian arrays in",
        "# canonical edge order ((min, max) lexicographic): edges = u array then v array.",
        f"# oracle time on the writing host: {t2 - t1:.0f} s (one core)",
        "n 16777216",
        f"m {eu.shape[0]}",
        f"edges_sha256 {digest_i32(eu, ev)}",
        f"truss_sha256 {digest_i32(tau)}",
        f"truss_max {int(tau.max()) if tau.size else 0}",
        "# trussness count",
    ]
    lines += [f"hist {k} {int(c)}" for k, c in enumerate(hist) if c]
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(tmp, OUT)
    print(f"wrote {OUT}", flush=True)


if __name__ == "__main__":
    main()
