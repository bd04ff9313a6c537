"""Oracle of the population search of Fig. 2 (test infrastructure only: the
tests, the smoke check and the benchmark's CPU-baseline leg may use it).

Written from the search's definition, independently of the library's
implementation; the two share only the uniform draw stream, passed in, and
consume it in the same order:

  1. probe: `probe` genes, each component lo + u (hi - lo); f_el = the
     (probe // 10 + 1)-th smallest probe fitness; viable means f < f_el;
  2. batches of `batch` random genes until `elite` viable genes (in draw
     order, probe first) or `max_batches` batches;
  3. per generation, `pop` children: parent A then parent B by roulette over
     the elite (weights 1/f, cumulative in elite order, first cumulative
     weight above u times the total), then per component three draws:
     crossover (A if u < 1/2), mutation gate (u < p_mut), mutation amount
     (v + (2u - 1) mut_scale (hi - lo), clipped to the box);
  4. if the best child is worse than the best elite, the elite is kept;
     otherwise the elite is the best `elite` of elite + children (ties: elite
     first, then children in order).

Fitness: Euclidean distance of P = [log M(1,1), log M(1,0)] per (plane, beam)
to P0, the moments (Eq. 8) of the FP64 oracle march; +inf when it blew up.
"""
import math

import numpy as np

from . import march as _march
from . import moment as _moment


def roulette(fs, x):
    """Index picked by the uniform draw x with probability proportional to 1/f."""
    ws = []
    for f in fs:
        ws.append(1.0 / f if f > 0.0 else 1e300)
    tot = 0.0
    for w in ws:
        tot += w
    lim = x * tot
    run = 0.0
    for i in range(len(ws)):
        run += ws[i]
        if run > lim:
            return i
    return len(ws) - 1


def search(fitness, lo, hi, draws, elite=5, pop=10, probe=20, batch=10, max_batches=50, generations=4,
           p_mut=0.2, mut_scale=0.1):
    u = list(np.asarray(draws, dtype=np.float64))
    pos = [0]

    def take():
        x = float(u[pos[0]])
        pos[0] += 1
        return x

    d = len(lo)

    def draw_gene():
        g = []
        for j in range(d):
            x = take()
            g.append(float(lo[j]) + x * (float(hi[j]) - float(lo[j])))
        return g

    probe_genes = [draw_gene() for _ in range(probe)]
    probe_f = list(fitness(probe_genes))
    level = sorted(probe_f)[probe // 10]
    kept = []
    for g, f in zip(probe_genes, probe_f):
        if f < level:
            kept.append((g, float(f)))
    nb = 0
    while len(kept) < elite and nb < max_batches:
        gs = [draw_gene() for _ in range(batch)]
        for g, f in zip(gs, fitness(gs)):
            if f < level:
                kept.append((g, float(f)))
        nb += 1
    el = kept[:elite]
    best_hist = [min(f for _, f in el)]

    def pick(x):
        return roulette([f for _, f in el], x)

    for _ in range(generations):
        kids = []
        for _k in range(pop):
            A = el[pick(take())][0]
            B = el[pick(take())][0]
            kid = []
            for j in range(d):
                xc = take()
                xm = take()
                xa = take()
                v = A[j] if xc < 0.5 else B[j]
                if xm < p_mut:
                    v = v + (2.0 * xa - 1.0) * mut_scale * (float(hi[j]) - float(lo[j]))
                    if v < float(lo[j]):
                        v = float(lo[j])
                    if v > float(hi[j]):
                        v = float(hi[j])
                kid.append(v)
            kids.append(kid)
        kf = [float(f) for f in fitness(kids)]
        if min(kf) <= min(f for _, f in el):
            pool = el + list(zip(kids, kf))
            idx = list(range(len(pool)))
            idx.sort(key=lambda i: (pool[i][1], i))
            el = [pool[i] for i in idx[:elite]]
        best_hist.append(min(f for _, f in el))
    ib = 0
    for i in range(1, len(el)):
        if el[i][1] < el[ib][1]:
            ib = i
    return dict(gene=el[ib][0], fitness=el[ib][1], f_el=level, history=best_hist, elite=el, draws_used=pos[0])


def _log(x):
    """log, with -inf at 0 and nan for negative or nan input (a blown-up march)."""
    if x > 0.0:
        return math.log(x)
    return -math.inf if x == 0.0 else math.nan


def p_vectors(genes, cfgs, fields, steps, samples):
    """P of each gene: [log M(1,1), log M(1,0)] per (plane, beam) from the FP64 march."""
    k = steps // samples
    out = []
    for g in genes:
        per_beam = []
        for c, U0 in zip(cfgs, fields):
            cg = dict(c, theta=tuple(g))
            U = np.asarray(U0, dtype=np.complex128)
            planes = []
            for _ in range(samples):
                U, _, _ = _march(U, cg, k, record=False)
                planes.append((_moment(U, c["L"], 1, 1), _moment(U, c["L"], 1, 0)))
            per_beam.append(planes)
        v = []
        for s in range(samples):
            for b in range(len(cfgs)):
                q1, pw = per_beam[b][s]
                v += [_log(q1), _log(pw)]
        out.append(np.array(v))
    return out


class OracleFitness:
    def __init__(self, cfgs, fields, steps, samples, target_gene):
        self.cfgs, self.fields, self.steps, self.samples = cfgs, fields, steps, samples
        self.P0 = p_vectors([target_gene], cfgs, fields, steps, samples)[0]

    def __call__(self, genes):
        fs = []
        for v in p_vectors(genes, self.cfgs, self.fields, self.steps, self.samples):
            f = float(np.linalg.norm(v - self.P0))
            if not math.isfinite(f):
                f = math.inf
            fs.append(f)
        return fs
