"""Writes the stored oracle values used by the GPU parity tests at full size.

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing here
touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py diamond64    # 64-atom diamond, DZP-like (~ 20 min)
    python tests/golden/make_golden.py diamond96    # 96-atom piece of the 216-atom diamond (~ 1 h)
    python tests/golden/make_golden.py diamond216   # 216-atom diamond: K blocks only (~ 3 min)
    python tests/golden/make_golden.py batch32      # the 32-system batch: K blocks only (~ 8 min)

Output: tests/golden/oracle_<name>.json.  diamond64 and diamond96: E_K = tr(PK), per-class
counts of kept canonical quartets, norms of K and a seeded sample of K blocks of the full
oracle K (diamond96 is the first 96 sites of the 216-atom workload's generator, the largest
piece of it whose full oracle K a CPU finishes in about an hour).
diamond216 and batch32 are too large for a full oracle K on a CPU; they store per-class
counts and K blocks computed one by one (oracle K_block: the sum over all kept quartets
(I J|K L) P_JL for one shell pair I, K), half of them between shells on nearby atoms,
where K is largest, half between random shells.
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
    "diamond96": lambda: inputs.config3(96),
}


def sample_pairs(s, rng, n_near, n_rand, near_bohr=4.5):
    """Shell pairs (I, K): n_near with atoms closer than near_bohr, n_rand uniform."""
    xyz, atom = s.xyz, s.shell_atom
    out = []
    while len(out) < n_near:
        I = int(rng.integers(0, s.n_shells))
        d = np.linalg.norm(xyz[atom] - xyz[atom[I]], axis=1)
        cand = np.nonzero(d < near_bohr)[0]
        out.append((I, int(rng.choice(cand))))
    for _ in range(n_rand):
        out.append((int(rng.integers(0, s.n_shells)), int(rng.integers(0, s.n_shells))))
    return out


def blocks_only(name, systems, n_near, n_rand, seed):
    t0 = time.time()
    rng = np.random.default_rng(seed)
    out_sys = []
    for s, P in systems:
        S = oracle.Screen(oracle.Basis(s))
        counts = S.count_quartets()
        blocks = [{"I": I, "J": K, "K": S.K_block(P, I, K).tolist()}
                  for I, K in sample_pairs(s, rng, n_near, n_rand)]
        out_sys.append({"n_atoms": s.n_atoms, "n_bf": s.n_bf, "kind": s.kind, "seed": s.seed,
                        "n_quartets": int(counts[21]), "n_quartets_class": [int(c) for c in counts[:21]],
                        "blocks": blocks})
        print(name, s.n_atoms, s.n_bf, int(counts[21]), f"{time.time() - t0:.0f}s", flush=True)
    out = {"case": name, "systems": out_sys, "oracle_seconds": time.time() - t0,
           "written_by": "tests/golden/make_golden.py (CPU oracle only)"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path)


def main(name):
    if name == "diamond216":
        return blocks_only(name, [inputs.config3()], 24, 24, 21600)
    if name == "batch32":
        return blocks_only(name, inputs.config2_systems(), 4, 4, 3200)
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
