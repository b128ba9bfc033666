"""Writes the stored oracle values used by the GPU parity tests at full size.

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing here
touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py diamond64    # 64-atom diamond, DZP-like (~ minutes)

Output: tests/golden/oracle_<name>.json with E_K = tr(PK), per-class counts of kept
canonical quartets, norms of K and a seeded sample of K blocks.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_03559_gb300 import inputs  # noqa: E402

CASES = {
    "diamond64": lambda: inputs.config1(64),
}


def main(name):
    s, P = CASES[name]()
    B = oracle.Basis(s)
    t0 = time.time()
    S = oracle.Screen(B)
    counts = S.count_quartets()
    K, ek = S.build_K(P, "sym")
    dt = time.time() - t0
    rng = np.random.default_rng(20240)
    off, nb = s.shell_offset, s.shell_nbf
    blocks = []
    for _ in range(96):
        I, J = (int(x) for x in rng.integers(0, s.n_shells, 2))
        blk = K[off[I]:off[I] + nb[I], off[J]:off[J] + nb[J]]
        blocks.append({"I": I, "J": J, "K": blk.tolist()})
    out = {
        "case": name, "n_atoms": s.n_atoms, "n_shells": s.n_shells, "n_bf": s.n_bf,
        "seed": s.seed, "tau": s.tau, "rcut": s.rcut, "omega": s.omega,
        "E_K": ek, "K_max_abs": float(np.abs(K).max()), "K_fro": float(np.linalg.norm(K)),
        "n_quartets": int(counts[21]), "n_quartets_class": [int(c) for c in counts[:21]],
        "oracle_seconds": dt, "oracle_threads": oracle.max_threads(), "blocks": blocks,
        "written_by": "tests/golden/make_golden.py (CPU oracle only)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, ek, dt)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "diamond64")
