"""The generated recurrence tables, run on the CPU the way the kernels decode them, against the
oracle's primitive integrals: no GPU involved.

For every class and every generated warp-schedule variant (k = 1, 2, 4 streams) the schedule's
32-entry iterations are decoded field by field as the warp kernel decodes them (destination and
source slots, coefficient indices from the direction, n-factors, the bra/ket base and the
fold/add flags, the stream of each entry) and executed on k coefficient sets of k primitive
quartets (same centres, different exponents), with all reads of an iteration done before its
writes; then the streams' accumulators are summed and the post-contraction ops (HGP horizontal
recurrences and the Cartesian -> spherical steps, the generator's uint4 words) run on the block.
The result must equal the sum of the oracle's primitive Cartesian integrals [ab|cd] over the k
primitive quartets (spherical components for d shells taken with the tables' coefficients).
The base values G_m come from the oracle's attenuated Boys function, the prefactor
sqrt(2) pi^{5/4} exp(-ab/p |AB|^2) / p per pair (weight 1).  The same run with every write done
at once (sequentially) must give the same numbers: no entry reads a slot that an entry of the
same iteration writes.  The thread kernel's tables (VRR levels with folded accumulations and
the accumulator adds) are run the same way, one primitive quartet after another."""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location(
    "gen_eri_tables", os.path.join(ROOT, "paper_2009_03559_gb300", "csrc", "gen_eri_tables.py"))
gen = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(gen)

CF, NCOEF, KET_BASE = gen.CF, gen.NCOEF, gen.KET_BASE


def pair(a, b, A, B):
    p = a + b
    P = (a * A + b * B) / p
    C = math.sqrt(2.0) * math.pi ** 1.25 * math.exp(-a * b / p * float(np.dot(A - B, A - B))) / p
    return p, P, C


def coef_set(ex, cen, Lt, omega):
    """The 39 coefficients of one primitive quartet (layout of the kernels' sets)."""
    a, b, c, d = ex
    A, B, Cc, D = cen
    p, P, Cab = pair(a, b, A, B)
    q, Q, Ccd = pair(c, d, Cc, D)
    s = p + q
    rho = p * q / s
    PQ = P - Q
    T = rho * float(PQ @ PQ)
    kap = omega ** 2 / (omega ** 2 + rho) if omega > 0 else 0.0
    G = Cab * Ccd / math.sqrt(s) * (oracle.gboys(Lt, T, kap) if omega > 0 else oracle.boys(Lt, T))
    cf = np.zeros(NCOEF)
    cf[CF["PA"]:CF["PA"] + 3] = P - A
    cf[CF["WP"]:CF["WP"] + 3] = -(q / s) * PQ
    cf[CF["CA"] + 1], cf[CF["CA"] + 2], cf[CF["CA"] + 3] = 1 / (2 * p), 1 / p, 3 / (2 * p)
    cf[CF["RP"]] = -q / s
    cf[CF["QC"]:CF["QC"] + 3] = Q - Cc
    cf[CF["WQ"]:CF["WQ"] + 3] = (p / s) * PQ
    cf[CF["CK"] + 1], cf[CF["CK"] + 2], cf[CF["CK"] + 3] = 1 / (2 * q), 1 / q, 3 / (2 * q)
    cf[CF["RQ"]] = -p / s
    for n in range(1, 5):
        cf[CF["CB"] + n] = n / (2 * s)
    cf[CF["ONE"]] = 1.0
    cf[CF["G"]:CF["G"] + Lt + 1] = G
    return cf


def run_schedule(c, ws, sets, parallel=True, dtype=np.float64):
    k, rsz = ws.k, ws.rsz
    S = np.zeros(k * rsz, dtype=dtype)
    sets = [np.asarray(cf, dtype=dtype) for cf in sets]
    for u in range(k):
        S[u * rsz + c.n_acc:u * rsz + c.n_acc + c.Lt + 1] = sets[u][CF["G"]:CF["G"] + c.Lt + 1]
    words = np.array(ws.words(), dtype=np.uint64).reshape(-1, 4)
    for t in range(len(ws.iters)):
        writes = []
        for x, y, z, w in words[32 * t:32 * (t + 1)].tolist():
            if not (w >> 10) & 1:
                continue
            u = (w >> 13) & 7
            X, cf = u * rsz, sets[u]
            base = KET_BASE if (w >> 7) & 1 else 0
            d, add, fold = w & 3, (w >> 9) & 1, (w >> 8) & 1
            i1 = CF["ONE"] if add else base + CF["PA"] + d
            i2 = CF["ZERO"] if add else base + CF["WP"] + d
            dst, s1, s2, s3, s4, s5 = x & 0xFFFF, x >> 16, y & 0xFFFF, y >> 16, z & 0xFFFF, z >> 16
            s0 = dst if fold else ws.zero
            v = cf[i1] * S[X + s1] + S[X + s0]
            v = cf[i2] * S[X + s2] + v
            if (w >> 11) & 1:
                v = cf[base + CF["CA"] + ((w >> 2) & 3)] * (cf[base + CF["RP"]] * S[X + s4] + S[X + s3]) + v
            if (w >> 12) & 1:
                v = cf[CF["CB"] + ((w >> 4) & 7)] * S[X + s5] + v
            if parallel:
                writes.append((X + dst, v))
            else:
                S[X + dst] = v
        for i, v in writes:
            S[i] = v
    acc = sum(S[u * rsz:u * rsz + c.n_acc].astype(np.float64) for u in range(k))
    return acc


def run_post(c, acc, AB, CD):
    p_type, p_rel, p_n, words, out_base = gen.post_words_of(c)
    T, _ = c.layout()
    S = np.zeros(max(T, c.n_acc) + 1)
    S[:c.n_acc] = acc
    W = np.array(words, dtype=np.uint64).reshape(-1, 4).tolist()
    for st in range(len(p_type)):
        for x, y, z, _ in W[p_rel[st]:p_rel[st] + p_n[st]]:
            dst, s1, s2, s3 = x & 0xFFFF, x >> 16, y & 0xFFFF, y >> 16
            if p_type[st] == 2:
                c0, c1, c2 = z & 15, (z >> 4) & 15, (z >> 8) & 15
                v = gen.SPH_COEF[c0] * S[s1]
                if c1:
                    v += gen.SPH_COEF[c1] * S[s2]
                if c2:
                    v += gen.SPH_COEF[c2] * S[s3]
            else:
                i = (z >> 12) & 3
                v = (AB if p_type[st] == 0 else CD)[i] * S[s2] + S[s1]
            S[dst] = v
    n = int(np.prod(c.final_dims))
    return S[out_base:out_base + n].reshape(c.final_dims)


def expected(c, exps, cen, omega):
    ls = (c.la, c.lb, c.lc, c.ld)
    cart = sum(oracle.prim_cart(ls, e, cen, omega) for e in exps)
    # d shells: the spherical components as the tables define them (rows of Cartesian weights)
    M = np.zeros((5, 6))
    for m, row in enumerate(gen.SPH_D):
        for cc, ci in row:
            M[m, cc] = gen.SPH_COEF[ci]
    for ax, l in enumerate(ls):
        if l == 2:
            cart = np.moveaxis(np.tensordot(M, np.moveaxis(cart, ax, 0), axes=(1, 0)), 0, ax)
    return cart


CLASSES = gen.all_classes()


@pytest.mark.parametrize("ci", range(len(CLASSES)), ids=[c.name() for c in CLASSES])
def test_schedules_and_post_ops_reproduce_oracle_integrals(ci):
    c = CLASSES[ci]
    rng = np.random.default_rng(100 + ci)
    cen = rng.uniform(-1.5, 1.5, (4, 3))
    omega = 0.11 if ci % 5 else 0.0  # every fifth class with the Coulomb kernel
    variants = gen.warp_schedules(c)
    assert 1 in variants
    for k, ws in variants.items():
        exps = [rng.uniform(0.2, 3.0, 4) for _ in range(k)]
        sets = [coef_set(e, cen, c.Lt, omega) for e in exps]
        acc = run_schedule(c, ws, sets)
        assert np.array_equal(acc, run_schedule(c, ws, sets, parallel=False))
        got = run_post(c, acc, cen[0] - cen[1], cen[2] - cen[3])
        ref = expected(c, exps, cen, omega)
        scale = np.abs(ref).max()
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * scale), (c.name(), k, np.abs(got - ref).max(), scale)


def run_levels(c, sets):
    """The thread kernel's tables: VRR levels (packed ops, folded accumulations) and the
    accumulator adds, one primitive quartet after another on one set of slots."""
    S = np.zeros(c.n_acc)
    for cf in sets:
        V = np.zeros(c.n_vrr_slots)
        V[:c.Lt + 1] = cf[CF["G"]:CF["G"] + c.Lt + 1]
        nb = len(c.bra_ops)
        for li, lvl in enumerate(c.bra_ops + c.ket_ops):
            ket = li >= nb
            base = KET_BASE if ket else 0
            for o in lvl:
                x, y, z, w = gen.pack_vrr(o)
                dst, s1, s2, s3, s4, s5 = x & 0xFFFF, x >> 16, y & 0xFFFF, y >> 16, z & 0xFFFF, z >> 16
                i, nA, nB, acc = w & 3, (w >> 2) & 7, (w >> 5) & 7, (w >> 8) & 1
                v = cf[base + CF["PA"] + i] * V[s1] + (S[dst] if acc else 0.0)
                v = cf[base + CF["WP"] + i] * V[s2] + v
                if nA:
                    v = cf[base + CF["CA"] + nA] * (cf[base + CF["RP"]] * V[s4] + V[s3]) + v
                if ket and nB:
                    v = cf[CF["CB"] + nB] * V[s5] + v
                if acc:
                    S[dst] = v
                else:
                    V[dst] = v
        for a, sl in c.acc_src:
            S[a] += V[sl]
    return S


@pytest.mark.parametrize("ci", range(len(CLASSES)), ids=[c.name() for c in CLASSES])
def test_thread_tables_reproduce_oracle_integrals(ci):
    c = CLASSES[ci]
    rng = np.random.default_rng(300 + ci)
    cen = rng.uniform(-1.5, 1.5, (4, 3))
    exps = [rng.uniform(0.2, 3.0, 4) for _ in range(3)]
    sets = [coef_set(e, cen, c.Lt, 0.11) for e in exps]
    got = run_post(c, run_levels(c, sets), cen[0] - cen[1], cen[2] - cen[3])
    ref = expected(c, exps, cen, 0.11)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), c.name()


def test_fp32_recurrence_error_by_class():
    """The schedules run in float32 on far-apart quartets (the kind that qualify for FP32),
    horizontal recurrences in FP64: the error relative to the quartet's largest integral grows
    with the total angular momentum, and (dd|dd) (L = 8) has the largest of all classes: the
    class the default FP32 mask leaves in FP64."""
    errs = {}
    for ci, c in enumerate(CLASSES):
        ws = gen.warp_schedules(c)[1]
        rng = np.random.default_rng(7 + ci)
        worst = 0.0
        for _ in range(6):
            A = rng.uniform(-1, 1, 3)
            B = A + rng.uniform(-2, 2, 3)
            shift = rng.normal(size=3)
            shift *= rng.uniform(9, 12) / np.linalg.norm(shift)
            Cc = shift + rng.uniform(-1, 1, 3)
            D = Cc + rng.uniform(-2, 2, 3)
            cf = coef_set(rng.uniform(0.1, 3.0, 4), np.array([A, B, Cc, D]), c.Lt, 0.11)
            o64 = run_post(c, run_schedule(c, ws, [cf]), A - B, Cc - D)
            o32 = run_post(c, run_schedule(c, ws, [cf], dtype=np.float32), A - B, Cc - D)
            worst = max(worst, np.abs(o32 - o64).max() / np.abs(o64).max())
        errs[c.name()] = worst
    assert max(errs.values()) == errs["dddd"]
    assert errs["dddd"] > 3 * max(v for k, v in errs.items() if k != "dddd")
    assert max(errs[n] for n in ("ssss", "psss", "psps", "ppss", "ppps")) < 1e-6
