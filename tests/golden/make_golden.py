"""Writes tests/golden/chaingen_digest.txt: SHA-256 digests of small seeded
melts, used to check that the generator produces identical bits on every
platform.  Calls only the input generator (no product code, no oracle)."""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import chaingen  # noqa: E402

CASES = [(2, 1), (10, 1), (50, 5)]


def digest(n_chains, seed):
    m = chaingen.melt(n_chains, seed=seed)
    h = hashlib.sha256()
    h.update(m["pos"].tobytes()); h.update(m["vel"].tobytes())
    h.update(repr(m["L"]).encode())
    return h.hexdigest()


if __name__ == "__main__":
    with open(os.path.join(HERE, "chaingen_digest.txt"), "w") as f:
        f.write("# n_chains seed sha256(pos||vel||repr(L)); written by make_golden.py\n")
        for n, s in CASES:
            f.write(f"{n} {s} {digest(n, s)}\n")
