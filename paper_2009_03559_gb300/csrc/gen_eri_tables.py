#!/usr/bin/env python3
"""Generate the per-class recurrence tables of the table-driven ERI engine.

For every shell-quartet class (la lb | lc ld) with la >= lb, lc >= ld and bra pair
class >= ket pair class (21 classes for s, p, d shells) this emits:

* the vertical recurrence (Obara-Saika, in the Head-Gordon-Pople arrangement) as
  levels of independent ops over shared-memory slots:
      bra  [e+1_i 0|00]^(m) = PA_i [e]^(m) + WP_i [e]^(m+1)
                              + e_i/(2p) ([e-1_i]^(m) - rho/p [e-1_i]^(m+1))
      ket  [e0|f+1_i 0]^(m) = QC_i [e|f]^(m) + WQ_i [e|f]^(m+1)
                              + f_i/(2q) ([e|f-1_i]^(m) - rho/q [e|f-1_i]^(m+1))
                              + e_i/(2(p+q)) [e-1_i|f]^(m+1)
  pruned to what the targets [e0|f0]^(0), e in [la, la+lb], f in [lc, lc+ld], need;
* the contraction list (VRR slot -> accumulator);
* the horizontal recurrence (Head-Gordon-Pople) on bra then ket:
      (a, b+1_i| = (a+1_i, b| + AB_i (a, b|,   |c, d+1_i) = |c+1_i, d) + CD_i |c, d);
* the Cartesian -> spherical step for d shells, real solid harmonics in the order
  xy, yz, 3z^2-r^2, xz, x^2-y^2 with the relative factors 1, 1, 1/(2 sqrt 3), 1, 1/2
  (all five then share one radial normalisation);
* FP64 operation counts per primitive quartet and per contracted quartet.

The output is a C header consumed by the CUDA library (``eri_tables.inc``).  Run:
    python gen_eri_tables.py > eri_tables.inc
"""
from __future__ import annotations

import json
import math
import os
import sys

PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
FOLD = "--no-fold" not in sys.argv
# classes whose group scratch fits in this many doubles run one quartet per thread
# (the kernels read this limit from the generated header); only those fold their
# accumulation into the VRR ops, which measured faster there and slower for warp groups
G1_MAX_SCRATCH = int(os.environ.get("HFX_G1_MAX_SCRATCH", "100"))


def monos(l):
    """Cartesian monomials of degree l in the order xx, xy, xz, yy, yz, zz (for l = 2)."""
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def ncart(l):
    return (l + 1) * (l + 2) // 2


def sub1(v, i):
    w = list(v)
    w[i] -= 1
    return tuple(w)


def add1(v, i):
    w = list(v)
    w[i] += 1
    return tuple(w)


def deg(v):
    return v[0] + v[1] + v[2]


def vrr_dir(v):
    """Axis with the smallest positive power: avoids the (e-1_i) term where possible."""
    best = None
    for i in range(3):
        if v[i] > 0 and (best is None or v[i] < v[best]):
            best = i
    return best


def hrr_dir(v):
    for i in range(3):
        if v[i] > 0:
            return i
    return None


# coefficient table for the Cartesian -> spherical step (indices into SPH_COEF)
S3 = 1.0 / (2.0 * math.sqrt(3.0))
SPH_COEF = [0.0, 1.0, -S3, 2.0 * S3, 0.5, -0.5]
# rows: spherical component; entries: (cartesian index in monos(2), coefficient index)
SPH_D = [
    [(1, 1)],                       # xy
    [(4, 1)],                       # yz
    [(5, 3), (0, 2), (3, 2)],       # (2zz - xx - yy) / (2 sqrt 3)
    [(2, 1)],                       # xz
    [(0, 4), (3, 5)],               # (xx - yy) / 2
]


def nsph(l):
    return 2 * l + 1


class ClassTables:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.E, self.F = la + lb, lc + ld
        self.Lt = self.E + self.F
        self.fold = False
        self.build()
        T, _ = self.layout()
        if FOLD and T <= G1_MAX_SCRATCH:   # folding leaves the layout unchanged
            self.fold = True
            self.build()

    # ------------------------------------------------------------------ VRR
    def build(self):
        la, lb, lc, ld, E, F, Lt = self.la, self.lb, self.lc, self.ld, self.E, self.F, self.Lt
        targets = [(e, f, 0) for de in range(la, E + 1) for e in monos(de)
                   for df in range(lc, F + 1) for f in monos(df)]
        need = set()
        stack = list(targets)
        deps = {}
        while stack:
            k = stack.pop()
            if k in need:
                continue
            need.add(k)
            e, f, m = k
            d = []
            if deg(f) > 0:
                i = vrr_dir(f)
                f1 = sub1(f, i)
                d += [(e, f1, m), (e, f1, m + 1)]
                if f1[i] > 0:
                    f2 = sub1(f1, i)
                    d += [(e, f2, m), (e, f2, m + 1)]
                if e[i] > 0:
                    d += [(sub1(e, i), f1, m + 1)]
            elif deg(e) > 0:
                i = vrr_dir(e)
                e1 = sub1(e, i)
                d += [(e1, f, m), (e1, f, m + 1)]
                if e1[i] > 0:
                    e2 = sub1(e1, i)
                    d += [(e2, f, m), (e2, f, m + 1)]
            deps[k] = d
            stack.extend(d)
        z = (0, 0, 0)
        # base slots: [00|00]^(m) for m = 0..Lt (all of them, filled by the Boys step)
        slot = {}
        for m in range(Lt + 1):
            slot[(z, z, m)] = m
        nslot = Lt + 1
        bra_levels, ket_levels = [], []
        for de in range(1, E + 1):
            lvl = sorted([k for k in need if deg(k[1]) == 0 and deg(k[0]) == de],
                         key=lambda k: (monos(de).index(k[0]), k[2]))
            for k in lvl:
                slot[k] = nslot
                nslot += 1
            bra_levels.append(lvl)
        for df in range(1, F + 1):
            lvl = sorted([k for k in need if deg(k[1]) == df],
                         key=lambda k: (deg(k[0]), k[0], k[1], k[2]))
            for k in lvl:
                slot[k] = nslot
                nslot += 1
            ket_levels.append(lvl)
        self.n_vrr_slots = nslot
        self.slot = slot
        # ops
        self.bra_ops = []
        for lvl in bra_levels:
            ops = []
            for k in lvl:
                e, f, m = k
                i = vrr_dir(e)
                e1 = sub1(e, i)
                n = e1[i]
                s1, s2 = slot[(e1, f, m)], slot[(e1, f, m + 1)]
                s3 = s4 = 0
                if n > 0:
                    e2 = sub1(e1, i)
                    s3, s4 = slot[(e2, f, m)], slot[(e2, f, m + 1)]
                ops.append(dict(dst=slot[k], s=[s1, s2, s3, s4, 0], dir=i, nA=n, nB=0))
            ops.sort(key=lambda o: (o["nA"] > 0, o["dst"]))
            self.bra_ops.append(ops)
        self.ket_ops = []
        for lvl in ket_levels:
            ops = []
            for k in lvl:
                e, f, m = k
                i = vrr_dir(f)
                f1 = sub1(f, i)
                n = f1[i]
                s1, s2 = slot[(e, f1, m)], slot[(e, f1, m + 1)]
                s3 = s4 = s5 = 0
                if n > 0:
                    f2 = sub1(f1, i)
                    s3, s4 = slot[(e, f2, m)], slot[(e, f2, m + 1)]
                nB = e[i]
                if nB > 0:
                    s5 = slot[(sub1(e, i), f1, m + 1)]
                ops.append(dict(dst=slot[k], s=[s1, s2, s3, s4, s5], dir=i, nA=n, nB=nB))
            ops.sort(key=lambda o: (o["nA"] > 0, o["nB"] > 0, o["dst"]))
            self.ket_ops.append(ops)
        # accumulators: e over degrees la..E (ordered), f over lc..F
        self.e_list = [e for de in range(la, E + 1) for e in monos(de)]
        self.f_list = [f for df in range(lc, F + 1) for f in monos(df)]
        self.n_acc = len(self.e_list) * len(self.f_list)
        # contraction: a target that no op reads is accumulated by the op that makes it
        # (the op ends its FMA chain on the accumulator: one FP64 add saved per target);
        # the others are added from their slot after the last level
        read = set()
        for lvl in self.bra_ops + self.ket_ops:
            for o in lvl:
                read.update(o["s"][:2])
                if o["nA"]:
                    read.update(o["s"][2:4])
                if o["nB"]:
                    read.add(o["s"][4])
        writer = {o["dst"]: o for lvl in self.bra_ops + self.ket_ops for o in lvl}
        self.acc_src = []      # (acc index, slot) added after the levels
        self.n_folded = 0
        a = 0
        for e in self.e_list:
            for f in self.f_list:
                sl = slot[(e, f, 0)]
                if self.fold and sl in writer and sl not in read:
                    writer[sl]["acc"] = a
                    self.n_folded += 1
                else:
                    self.acc_src.append((a, sl))
                a += 1
        self.build_hrr()

    # ------------------------------------------------------------------ HRR + sph
    def build_hrr(self):
        """Post-contraction stages, each reading only the previous stage's block:
        bra HRR levels -> sph(a) -> sph(b) -> ket HRR levels -> sph(c) -> sph(d).
        A stage is a list of (dst_index, [(src_index, kind_or_coef)], dir); indices
        are positions in the previous / current stage's block."""
        la, lb, lc, ld, E, F = self.la, self.lb, self.lc, self.ld, self.E, self.F
        z = (0, 0, 0)
        # stage 0: the accumulator block, keys (a, b, f) with b = 0
        cur_keys = [(e, z, f) for e in self.e_list for f in self.f_list]
        self.stages = []       # each: dict(type, ops=[(dst, srcs, dir)]) with srcs indices into prev block
        self.stage_sizes = [len(cur_keys)]

        def add_stage(kind, new_keys, make_srcs):
            nonlocal cur_keys
            idx = {k: i for i, k in enumerate(cur_keys)}
            ops = []
            for j, k in enumerate(new_keys):
                srcs, d = make_srcs(k)
                ops.append((j, [(idx[sk], c) for sk, c in srcs], d))
            self.stages.append(dict(type=kind, ops=ops))
            self.stage_sizes.append(len(new_keys))
            cur_keys = new_keys

        # bra HRR: (a, b + 1_i | f) = (a + 1_i, b | f) + AB_i (a, b | f)
        for db in range(1, lb + 1):
            new = [(a, b, f) for da in range(la, E - db + 1) for a in monos(da)
                   for b in monos(db) for f in self.f_list]

            def mk(k):
                a, b, f = k
                i = hrr_dir(b)
                b1 = sub1(b, i)
                return [((add1(a, i), b1, f), 1), ((a, b1, f), 2)], i
            add_stage("hrr_bra", new, mk)
        # keys are now (a, b, f) with deg a = la, deg b = lb; move to spherical a, b
        # representation: key (ka, kb, f) where ka/kb are Cartesian tuples or ("s", m)
        ls = [la, lb]
        for t in range(2):
            if ls[t] != 2:
                continue
            old = cur_keys
            comps = []
            for k in old:
                kk = list(k)
                kk[t] = None
                comps.append(tuple(kk))
            seen = []
            for c in comps:
                if c not in seen:
                    seen.append(c)
            new = []
            for c in seen:
                for m in range(5):
                    kk = list(c)
                    kk[t] = ("s", m)
                    new.append(tuple(kk))
            # order: row-major over (a, b, f)
            new = self._order3(new)

            def mk(k, t=t):
                m = k[t][1]
                srcs = []
                for (cc, ci) in SPH_D[m]:
                    kk = list(k)
                    kk[t] = monos(2)[cc]
                    srcs.append((tuple(kk), ci))
                return srcs, 0
            add_stage("sph", new, mk)
        # ket HRR on f: |c, d + 1_i) = |c + 1_i, d) + CD_i |c, d); keys become (a, b, c, d)
        cur_keys = [(a, b, f, z) for (a, b, f) in cur_keys]
        AB_keys = []
        for (a, b, f, d) in cur_keys:
            if (a, b) not in AB_keys:
                AB_keys.append((a, b))
        for dd in range(1, ld + 1):
            new = [(a, b, c, d) for (a, b) in AB_keys for dc in range(lc, F - dd + 1)
                   for c in monos(dc) for d in monos(dd)]

            def mk(k):
                a, b, c, d = k
                i = hrr_dir(d)
                d1 = sub1(d, i)
                return [((a, b, add1(c, i), d1), 1), ((a, b, c, d1), 2)], i
            add_stage("hrr_ket", new, mk)
        ls2 = [lc, ld]
        for t in (2, 3):
            if ls2[t - 2] != 2:
                continue
            old = cur_keys
            seen = []
            for k in old:
                kk = list(k)
                kk[t] = None
                kk = tuple(kk)
                if kk not in seen:
                    seen.append(kk)
            new = []
            for c in seen:
                for m in range(5):
                    kk = list(c)
                    kk[t] = ("s", m)
                    new.append(tuple(kk))
            new = sorted(new, key=lambda k: tuple(self._comp_order(k[u]) for u in range(4)))

            def mk(k, t=t):
                m = k[t][1]
                srcs = []
                for (cc, ci) in SPH_D[m]:
                    kk = list(k)
                    kk[t] = monos(2)[cc]
                    srcs.append((tuple(kk), ci))
                return srcs, 0
            add_stage("sph", new, mk)
        if len(cur_keys[0]) == 3:
            cur_keys = [(a, b, f, z) for (a, b, f) in cur_keys]
        # final block must be row-major (a, b, c, d) over the final components
        self.final_dims = [nsph(la) if la == 2 else ncart(la), nsph(lb) if lb == 2 else ncart(lb),
                           nsph(lc) if lc == 2 else ncart(lc), nsph(ld) if ld == 2 else ncart(ld)]
        n = 1
        for d in self.final_dims:
            n *= d
        assert len(cur_keys) == n, (self.name(), len(cur_keys), n)
        self._check_row_major(cur_keys)

    @staticmethod
    def _comp_order(c, l_hint=None):
        if isinstance(c, tuple) and len(c) == 2 and c[0] == "s":
            return (1, c[1])
        return (0, monos(deg(c)).index(c))

    def _order3(self, keys):
        # keep the f order of self.f_list
        fpos = {f: i for i, f in enumerate(self.f_list)}
        return sorted(keys, key=lambda k: (self._comp_order(k[0]), self._comp_order(k[1]), fpos[k[2]]))

    def _check_row_major(self, keys):
        orders = [sorted({self._comp_order(k[t]) for k in keys}) for t in range(4)]
        exp = []
        for a in orders[0]:
            for b in orders[1]:
                for c in orders[2]:
                    for d in orders[3]:
                        exp.append((a, b, c, d))
        got = [tuple(self._comp_order(k[t]) for t in range(4)) for k in keys]
        assert got == exp, self.name()

    def name(self):
        L = "spd"
        return f"{L[self.la]}{L[self.lb]}{L[self.lc]}{L[self.ld]}"

    # ------------------------------------------------------------------ counts
    def flops(self):
        """FP64 flops (fma = 2) of the recurrence parts."""
        vrr = 0
        for lvl in self.bra_ops:
            for o in lvl:
                vrr += 3 + (4 if o["nA"] else 0)            # mul+fma [+ fma + fma]
        for lvl in self.ket_ops:
            for o in lvl:
                vrr += 3 + (4 if o["nA"] else 0) + (2 if o["nB"] else 0)
        acc = self.n_acc          # one add per accumulator (inside an FMA when folded)
        hrr = sph = 0
        for st in self.stages:
            for _, srcs, _ in st["ops"]:
                if st["type"] == "sph":
                    sph += 2 * len(srcs) - 1
                else:
                    hrr += 2
        nout = 1
        for d in self.final_dims:
            nout *= d
        na, nb, nc, nd = self.final_dims
        digest = 2 * nout * 4 + (na * nc + na * nd + nb * nc + nb * nd)
        return dict(vrr=vrr, acc=acc, hrr=hrr, sph=sph, digest=digest, nout=nout)

    # ------------------------------------------------------------------ layout
    def layout(self):
        """Group scratch (doubles): acc block at 0 and the VRR slots after it while the
        primitive loop runs; afterwards the stages alternate between the bottom (offset
        0) and the top (ending at the scratch size) of the same scratch."""
        T, bases = self.post_layout()
        return max(T, self.n_acc + self.n_vrr_slots), bases

    def post_layout(self):
        """Scratch of the post-contraction stages alone: the largest two consecutive stage
        blocks (the first being the accumulators at offset 0), and the stage offsets."""
        sizes = self.stage_sizes
        T = sizes[0]
        for k in range(1, len(sizes)):
            T = max(T, sizes[k - 1] + sizes[k])
        bases = [0]
        for k in range(1, len(sizes)):
            bases.append(T - sizes[k] if k % 2 == 1 else 0)
        return T, bases


# ---------------------------------------------------------------------------------------
# Warp schedules.  A warp runs k primitive quartets ("streams") of one contracted quartet at
# a time; each stream owns a region of group scratch: [accumulators | VRR slots | a zero
# slot].  The VRR ops of all streams, and one add per accumulator whose target another op
# reads, are list-scheduled into iterations of at most 32 ops (one per lane).  The FP64
# pipe of this part charges every warp instruction in full whatever the number of active
# lanes, and an iteration costs the union of its lanes' instruction sequences, so the
# scheduler packs each iteration with ops of one shape:
#   2 instructions (leading FMA from the accumulator or the zero slot, then the W term),
#   +2 with the n/(2p) (V3 - rho/p V4) term, +1 with the e_i/(2(p+q)) V5 term.
# Targets that no op reads accumulate in their producing op (its first FMA starts from the
# accumulator), so the contraction costs no separate add for them.
# Coefficient-set layout (per primitive quartet, doubles or floats):
CF = dict(PA=0, WP=3, CA=6, RP=10, QC=11, WQ=14, CK=17, RQ=21, CB=22, ONE=27, ZERO=28, G=29)
NCOEF = 39            # 38 used; odd so that the lanes' sets start in different banks
KET_BASE = CF["QC"] - CF["PA"]
SCHED_KS = (1, 2, 4)
SCHED_MAX_REGION_DOUBLES = 3600   # k * region limit for a variant to be generated


def shape_cost(a, b):
    return 2 + 2 * a + b


class WarpSchedule:
    def __init__(self, c, k):
        self.c, self.k = c, k
        n_acc, nvs = c.n_acc, c.n_vrr_slots
        self.zero = n_acc + nvs   # before slot assignment: a slot past the VRR slots
        nb = len(c.bra_ops)
        ops = []             # (dst_region, fold, s1..s5 region, dir, nA, nB, ket, add, deps(op ids), level)
        writer = {}
        lv_all = c.bra_ops + c.ket_ops
        for li, lv in enumerate(lv_all):
            for o in lv:
                writer[o["dst"]] = len(writer)
        # read set of VRR slots
        read = set()
        for li, lv in enumerate(lv_all):
            ket = li >= nb
            for o in lv:
                read.update(o["s"][:2])
                if o["nA"]:
                    read.update(o["s"][2:4])
                if ket and o["nB"]:
                    read.add(o["s"][4])
        acc_of = {}
        for a, (e, f) in enumerate((e, f) for e in c.e_list for f in c.f_list):
            acc_of[c.slot[(e, f, 0)]] = a
        opid = {}
        for li, lv in enumerate(lv_all):
            ket = li >= nb
            for o in lv:
                d = o["dst"]
                fold = d in acc_of and d not in read
                srcs = [o["s"][0], o["s"][1]]
                srcs += [o["s"][2], o["s"][3]] if o["nA"] else [None, None]
                srcs += [o["s"][4]] if (ket and o["nB"]) else [None]
                deps = set(opid[s] for s in srcs if s is not None and s in opid)
                reg = [n_acc + s if s is not None else self.zero for s in srcs]
                opid[d] = len(ops)
                ops.append(dict(dst=acc_of[d] if fold else n_acc + d, fold=fold, s=reg, dir=o["dir"],
                                nA=o["nA"], nB=o["nB"] if ket else 0, ket=int(ket), add=0, deps=deps,
                                A=int(o["nA"] > 0), B=int(ket and o["nB"] > 0)))
        # adds for accumulators whose target is read (or is a base slot)
        for sl, a in sorted(acc_of.items(), key=lambda t: t[1]):
            if sl in opid and ops[opid[sl]]["fold"]:
                continue
            deps = {opid[sl]} if sl in opid else set()
            ops.append(dict(dst=a, fold=True, s=[n_acc + sl, self.zero, self.zero, self.zero, self.zero],
                            dir=0, nA=0, nB=0, ket=0, add=1, deps=deps, A=0, B=0))
        self.ops = ops
        # longest path to a sink (critical-path priority)
        h = [0] * len(ops)
        succ = [[] for _ in ops]
        for i, o in enumerate(ops):
            for d in o["deps"]:
                succ[d].append(i)
        for i in reversed(range(len(ops))):
            h[i] = 1 + max((h[j] for j in succ[i]), default=0)
        self.height = h
        self.schedule()

    def schedule(self):
        ops, k = self.ops, self.k
        n = len(ops)
        ndep = [[len(o["deps"]) for o in ops] for _ in range(k)]
        succ = [[] for _ in ops]
        for i, o in enumerate(ops):
            for d in o["deps"]:
                succ[d].append(i)
        ready = [(u, i) for u in range(k) for i in range(n) if ndep[u][i] == 0]
        iters = []
        cost = 0
        left = k * n
        while left:
            best = None
            for cap in ((0, 0), (1, 0), (0, 1), (1, 1)):
                cand = [t for t in ready if ops[t[1]]["A"] <= cap[0] and ops[t[1]]["B"] <= cap[1]]
                if not cand:
                    continue
                cand.sort(key=lambda t: (-self.height[t[1]], t[0], t[1]))
                cand = cand[:32]
                ea = max(ops[t[1]]["A"] for t in cand)
                eb = max(ops[t[1]]["B"] for t in cand)
                score = len(cand) / shape_cost(ea, eb)
                if best is None or score > best[0] + 1e-12:
                    best = (score, cand, ea, eb)
            _, it, ea, eb = best
            cost += shape_cost(ea, eb)
            iters.append((it, ea, eb))
            sel = set(it)
            ready = [t for t in ready if t not in sel]
            for (u, i) in it:
                for j in succ[i]:
                    ndep[u][j] -= 1
                    if ndep[u][j] == 0:
                        ready.append((u, j))
            left -= len(it)
        self.iters = iters
        self.cost = cost
        self.assign_slots()
        # every stream's accumulators: each written by exactly one entry per stream
        seen = set()
        for it, _, _ in iters:
            for (u, i) in it:
                o = ops[i]
                if o["fold"]:
                    key = (u, o["dst"])
                    assert key not in seen
                    seen.add(key)
        assert len(seen) == k * self.c.n_acc, (self.c.name(), k)

    def assign_slots(self):
        """Physical slots of each stream's region: accumulators [0, n_acc), the base values
        G_m [n_acc, n_acc + Lt + 1), the zero slot, then the VRR values, each holding a slot
        from the iteration that writes it to the last iteration that reads it (a slot freed
        by the reads of iteration t is written again at t + 1 at the earliest)."""
        c, k = self.c, self.k
        n_acc, nbase = c.n_acc, c.Lt + 1
        zero = n_acc + nbase
        first = zero + 1
        base_old = {n_acc + m: n_acc + m for m in range(nbase)}
        old_zero = self.zero
        # last reading iteration of each (stream, old slot)
        last = {}
        for t, (it, ea, eb) in enumerate(self.iters):
            for (u, i) in it:
                o = self.ops[i]
                for sl in o["s"]:
                    if sl >= n_acc and sl != old_zero and sl not in base_old:
                        last[(u, sl)] = t
        phys = {}           # (u, old slot) -> physical slot
        free = [[] for _ in range(k)]
        top = [first] * k
        release = {}        # iteration -> [(u, phys)]
        mapped = []         # per iteration: entries (u, i, dst, srcs)
        for t, (it, ea, eb) in enumerate(self.iters):
            for (u, p) in release.pop(t - 1, []):
                free[u].append(p)
            for u in range(k):
                free[u].sort(reverse=True)
            row = []
            for (u, i) in it:
                o = self.ops[i]
                src = []
                for sl in o["s"]:
                    if sl == old_zero:
                        src.append(zero)
                    elif sl < n_acc or sl in base_old:
                        src.append(sl)
                    else:
                        src.append(phys[(u, sl)])
                row.append((u, i, src))
            for (u, i, src) in row:
                o = self.ops[i]
                if o["fold"]:
                    dst = o["dst"]
                else:
                    key = (u, o["dst"])
                    if free[u]:
                        dst = free[u].pop()
                    else:
                        dst = top[u]
                        top[u] += 1
                    phys[key] = dst
                    lt = last.get(key, t)
                    release.setdefault(lt, []).append((u, dst))
                mapped.append((t, u, i, dst, src))
        self.mapped = mapped
        self.zero = zero
        T, _ = c.post_layout()
        rsz = max(top)
        if rsz % 2 == 0:
            rsz += 1
        self.rsz = rsz
        self.group = max(k * rsz, T)    # the post-contraction stages use the first T doubles

    def words(self):
        out = []
        by_iter = {}
        for (t, u, i, dst, src) in self.mapped:
            by_iter.setdefault(t, []).append((u, i, dst, src))
        for t, (it, ea, eb) in enumerate(self.iters):
            ents = by_iter.get(t, [])
            for lane in range(32):
                if lane < len(ents):
                    u, i, dst, s = ents[lane]
                    o = self.ops[i]
                    w = (o["dir"] | (o["nA"] << 2) | (o["nB"] << 4) | (o["ket"] << 7) | (int(o["fold"]) << 8)
                         | (o["add"] << 9) | (1 << 10) | (ea << 11) | (eb << 12) | (u << 13))
                    out += [dst | (s[0] << 16), s[1] | (s[2] << 16), s[3] | (s[4] << 16), w]
                else:
                    out += [0, 0, 0, (ea << 11) | (eb << 12)]
        return out


def warp_schedules(c):
    """The generated variants (k = 1, 2, 4 streams) whose scratch stays within the limit."""
    out = {}
    for k in SCHED_KS:
        ws = WarpSchedule(c, k)
        if k == 1 or ws.group <= SCHED_MAX_REGION_DOUBLES:
            out[k] = ws
    return out


def pack_vrr(o):
    """uint4 op: dst|s1, s2|s3, s4|s5 (16 bits each), dir | nA << 2 | nB << 5 | acc << 8.
    With the acc flag, dst is an accumulator index (group scratch slot) and the op adds
    its value there instead of storing a VRR slot."""
    s = o["s"]
    acc = "acc" in o
    dst = o["acc"] if acc else o["dst"]
    return [(dst & 0xFFFF) | ((s[0] & 0xFFFF) << 16),
            (s[1] & 0xFFFF) | ((s[2] & 0xFFFF) << 16),
            (s[3] & 0xFFFF) | ((s[4] & 0xFFFF) << 16),
            o["dir"] | (o["nA"] << 2) | (o["nB"] << 5) | (int(acc) << 8)]


def all_classes():
    out = []
    for hi in range(6):
        for lo in range(hi + 1):
            la, lb = PAIR_CLASSES[hi]
            lc, ld = PAIR_CLASSES[lo]
            out.append(ClassTables(la, lb, lc, ld))
    return out


STAGE_TYPE = {"hrr_bra": 0, "hrr_ket": 1, "sph": 2}


def post_words_of(c):
    """The post-contraction stages of a class as uint4 ops (dst | s1, s2 | s3, spherical
    coefficient indices | direction << 12, 0), slots in the group scratch: per stage its type,
    first op (relative) and op count, the words, and where the final block starts."""
    T, bases = c.layout()
    p_type, p_rel, p_n, words = [], [], [], []
    for k, st in enumerate(c.stages):
        src_base = bases[k]
        dst_base = bases[k + 1]
        p_type.append(STAGE_TYPE[st["type"]])
        p_rel.append(len(words) // 4)
        p_n.append(len(st["ops"]))
        for (dst, srcs, d) in st["ops"]:
            sl = [src_base + s for s, _ in srcs] + [0] * (3 - len(srcs))
            cs = [cc for _, cc in srcs] + [0] * (3 - len(srcs))
            if st["type"] != "sph":
                cs = [0, 0, 0]
            words.extend([((dst_base + dst) & 0xFFFF) | ((sl[0] & 0xFFFF) << 16),
                          (sl[1] & 0xFFFF) | ((sl[2] & 0xFFFF) << 16),
                          cs[0] | (cs[1] << 4) | (cs[2] << 8) | (d << 12),
                          0])
    return p_type, p_rel, p_n, words, bases[len(c.stages)]


def emit(classes, f=sys.stdout):
    w = f.write
    w("// Generated by gen_eri_tables.py -- do not edit by hand.\n")
    w("// Per-class Obara-Saika / Head-Gordon-Pople recurrence tables for the FP64 engine.\n")
    w("#pragma once\n\n")
    vrr_words, post_words, acc_words = [], [], []
    rows = []
    for c in classes:
        T, bases = c.layout()
        work_base = c.n_acc
        lv_off, lv_n = [], []
        for lvl in c.bra_ops + c.ket_ops:
            lv_off.append(len(vrr_words) // 4)
            lv_n.append(len(lvl))
            for o in lvl:
                vrr_words.extend(pack_vrr(o))
        acc_off = len(acc_words)
        acc_words.extend([(a & 0xFFFF) | ((sl & 0xFFFF) << 16) for a, sl in c.acc_src])
        p_type, p_rel, p_n, words, out_base = post_words_of(c)
        p_off = [len(post_words) // 4 + r for r in p_rel]
        post_words.extend(words)
        fl = c.flops()
        rows.append(dict(c=c, T=T, work_base=work_base, lv_off=lv_off, lv_n=lv_n, acc_off=acc_off,
                         p_type=p_type, p_off=p_off, p_n=p_n, out_base=out_base, fl=fl))

    def arr(name, words, per_line=8):
        w(f"HFX_TABLE_QUAL uint32_t {name}[{max(len(words), 4)}] = {{\n")
        ws = words if words else [0, 0, 0, 0]
        for i in range(0, len(ws), per_line):
            w("  " + ", ".join(f"{x}u" for x in ws[i:i + per_line]) + ",\n")
        w("};\n\n")

    w(f"#define HFX_N_CLASSES {len(classes)}\n")
    w(f"#define HFX_G1_MAX_SCRATCH {G1_MAX_SCRATCH}\n\n")
    w("static const double kSphCoefHost[6] = {" + ", ".join(repr(x) for x in SPH_COEF) + "};\n\n")
    arr("kVrrOps", vrr_words)
    arr("kPostOps", post_words)
    arr("kAccSrc", acc_words)

    def lst(v, n):
        v = list(v) + [0] * (n - len(v))
        assert len(v) == n
        return "{" + ", ".join(str(x) for x in v) + "}"
    w("static const EriClassInfo kClassInfo[HFX_N_CLASSES] = {\n")
    for r in rows:
        c, fl = r["c"], r["fl"]
        w(f"  // ({c.name()}) vrr {fl['vrr']} flop/prim + acc {fl['acc']}; per quartet hrr {fl['hrr']}, "
          f"sph {fl['sph']}, digest {fl['digest']}; scratch {r['T']} doubles\n")
        w("  {" + ", ".join([
            str(c.la), str(c.lb), str(c.lc), str(c.ld), str(c.E), str(c.F), str(c.Lt),
            str(c.n_acc), str(r["work_base"]), str(r["T"]),
            str(len(c.bra_ops)), str(len(c.ket_ops)),
            lst(r["lv_off"], 8), lst(r["lv_n"], 8), str(r["acc_off"]), str(len(c.acc_src)),
            str(len(c.stages)), lst(r["p_type"], 8), lst(r["p_off"], 8), lst(r["p_n"], 8),
            str(r["out_base"]), lst(c.final_dims, 4),
            str(fl["vrr"] + fl["acc"]), str(fl["hrr"] + fl["sph"] + fl["digest"]), str(fl["digest"]),
        ]) + "},\n")
    w("};\n\n")
    # warp schedules
    w("// Coefficient set of one primitive quartet (group scratch of the warp kernel)\n")
    for name, v in CF.items():
        w(f"#define HFX_CF_{name} {v}\n")
    w(f"#define HFX_NCOEF {NCOEF}\n")
    w(f"#define HFX_CF_KET_BASE {KET_BASE}\n\n")
    sched_words, info = [], []
    for c in classes:
        row = []
        ws = warp_schedules(c)
        for k in SCHED_KS:
            if k in ws:
                v = ws[k]
                row.append((k, v.rsz, v.zero, len(v.iters), len(sched_words) // 4, v.group, v.cost))
                sched_words.extend(v.words())
            else:
                row.append((0, 0, 0, 0, 0, 0, 0))
        info.append((c, row))
    w("// Warp schedules: per entry (uint4) dst | s1 << 16, s2 | s3 << 16, s4 | s5 << 16, flags\n")
    w("// (dir | nA << 2 | nB << 4 | ket << 7 | fold << 8 | add << 9 | valid << 10 | shapeA << 11 |\n")
    w("//  shapeB << 12 | stream << 13); 32 entries per iteration.\n")
    sched_words.extend([0] * (32 * 4))   # padding iteration: the warp kernel prefetches one past the end
    w(f"HFX_TABLE_QUAL uint32_t kSched[{len(sched_words)}] = {{\n")
    for i in range(0, len(sched_words), 8):
        w("  " + ", ".join(f"0x{x:x}u" for x in sched_words[i:i + 8]) + ",\n")
    w("};\n\n")
    w(f"static const SchedVariant kSchedInfo[HFX_N_CLASSES][{len(SCHED_KS)}] = {{\n")
    for c, row in info:
        costs = ", ".join(f"k{r[0]} {r[6] / max(r[0], 1):.1f}" for r in row if r[0])
        w(f"  // ({c.name()}) FP64 warp instructions per primitive quartet: {costs}\n")
        w("  {" + ", ".join("{" + ", ".join(str(x) for x in r[:6]) + "}" for r in row) + "},\n")
    w("};\n")


if __name__ == "__main__":
    cl = all_classes()
    if len(sys.argv) > 1 and sys.argv[1] == "--summary":
        for c in cl:
            fl = c.flops()
            T, bases = c.layout()
            print(f"{c.name()}: vrr_slots {c.n_vrr_slots} acc {c.n_acc} scratch {T} "
                  f"stages {[st['type'] for st in c.stages]} sizes {c.stage_sizes} "
                  f"levels {[len(l) for l in c.bra_ops + c.ket_ops]} flops {json.dumps(fl)}")
    else:
        emit(cl)
