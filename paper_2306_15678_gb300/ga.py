"""Population (genetic) search over screen genes, the fit loop of Fig. 2,
with the fitness of Eq. 8's moment measure evaluated by the batched march.

The search (host logic; every march and moment runs in the library's kernels):

  elite generation  genes drawn uniformly in the box [lo, hi]; a probe of
                    `probe` random genes sets the viability level f_el to its
                    (probe // 10 + 1)-th smallest fitness, so that about one in
                    ten random genes is viable (f < f_el); batches of `batch`
                    random genes are drawn until `elite` viable genes are found;
  evolution         each generation breeds `pop` children: two parents picked
                    by roulette (probability proportional to 1/f), uniform
                    crossover, and with probability p_mut per component a
                    uniform mutation of up to mut_scale of the box; if the best
                    child is worse than the best elite, the children are
                    discarded and the elite generation is kept (the paper's
                    "destruction of degenerative descendants"); otherwise the
                    elite becomes the `elite` best of elite and children.

Every random choice reads the next value of one uniform stream (``draws``,
see beams.ga_draws) in a fixed order: a gene takes d values; a child takes
2 (parents) + 3 per component (crossover, mutation gate, mutation amount).

Fitness (Fig. 2, Eq. 8): the Euclidean distance between the vector P of a
gene and the target vector P0 (+inf when a march blew up), P = [log Q^1, log P] of every test beam at
every sample plane, Q^1 = M(1, 1) = int I r^2 (Eq. 8 with m = 1) and P the
power M(1, 0).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import beams, configs
from .batch import Batch
from .grid import Grid

DEFAULTS = dict(elite=5, pop=10, probe=20, batch=10, max_batches=50, generations=4, p_mut=0.2, mut_scale=0.1)


class _Stream:
    def __init__(self, draws):
        self.u = np.asarray(draws, dtype=np.float64)
        self.c = 0

    def next(self) -> float:
        if self.c >= self.u.size:
            raise RuntimeError("genetic search: the draw stream is exhausted")
        v = float(self.u[self.c])
        self.c += 1
        return v


def _roulette(fs, u: float) -> int:
    w = [1.0 / f if f > 0.0 else 1e300 for f in fs]
    total = 0.0
    for x in w:
        total += x
    t = u * total
    acc = 0.0
    for i, x in enumerate(w):
        acc += x
        if acc > t:
            return i
    return len(w) - 1


def search(fitness, lo, hi, draws, **kw) -> dict:
    """Run the search.  fitness(list of genes) -> sequence of fitness values."""
    o = dict(DEFAULTS, **kw)
    lo = [float(v) for v in lo]
    hi = [float(v) for v in hi]
    d = len(lo)
    s = _Stream(draws)

    def random_genes(k):
        return [[lo[j] + s.next() * (hi[j] - lo[j]) for j in range(d)] for _ in range(k)]

    probe = random_genes(o["probe"])
    fp = [float(f) for f in fitness(probe)]
    f_el = sorted(fp)[o["probe"] // 10]
    viable = [(g, f) for g, f in zip(probe, fp) if f < f_el]
    batches = 0
    while len(viable) < o["elite"] and batches < o["max_batches"]:
        genes = random_genes(o["batch"])
        fb = [float(f) for f in fitness(genes)]
        viable += [(g, f) for g, f in zip(genes, fb) if f < f_el]
        batches += 1
    if not viable:
        raise RuntimeError("genetic search: no viable gene")
    elite = viable[: o["elite"]]
    history = [min(f for _, f in elite)]
    restored = []
    for _ in range(o["generations"]):
        fs = [f for _, f in elite]
        children = []
        for _k in range(o["pop"]):
            a = elite[_roulette(fs, s.next())][0]
            b = elite[_roulette(fs, s.next())][0]
            child = []
            for j in range(d):
                uc, um, ua = s.next(), s.next(), s.next()
                v = a[j] if uc < 0.5 else b[j]
                if um < o["p_mut"]:
                    v = v + (2.0 * ua - 1.0) * o["mut_scale"] * (hi[j] - lo[j])
                    v = min(max(v, lo[j]), hi[j])
                child.append(v)
            children.append(child)
        fc = [float(f) for f in fitness(children)]
        if min(fc) > min(fs):
            restored.append(True)
        else:
            restored.append(False)
            pool = list(elite) + list(zip(children, fc))
            order = sorted(range(len(pool)), key=lambda i: (pool[i][1], i))
            elite = [pool[i] for i in order[: o["elite"]]]
        history.append(min(f for _, f in elite))
    best = min(range(len(elite)), key=lambda i: (elite[i][1], i))
    return dict(gene=elite[best][0], fitness=elite[best][1], f_el=f_el, history=history, restored=restored,
                elite=elite, draws_used=s.c)


# ------------------------------------------------ fitness by the batched march

def fit_cfgs(n: int = 256, count: int = 2, steps: int = 20, length: float = 15.0) -> list:
    """Workload dicts of the Eq. 7 test beams: full screen, FP32 batch, marched
    over `length` cm (15 cm keeps the narrowest, 3 P_cr beam short of its
    collapse for every gene of the box used in the tests)."""
    out = []
    for (r, pp, L) in beams.fit_beam_set(n, count):
        c = configs.physics(n, L, length / steps, configs.ALL_TERMS)
        c["beam"] = dict(w0=r, P=pp * configs.critical_power())
        out.append(c)
    return out


def p_vector(moments_per_plane) -> np.ndarray:
    """[log Q^1, log P] for every (beam, plane) pair, in order."""
    v = []
    for q1, pw in moments_per_plane:
        v += [q1, pw]
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.log(np.array(v, dtype=np.float64))  # non-finite for a march that blew up


class BatchFitness:
    """Fitness of a list of genes: every (gene, test beam) pair is one beam of
    one batched march; the fields are read at `samples` planes and their Eq. 8
    moments taken on the device."""

    def __init__(self, cfgs: list, steps: int, samples: int, target_gene, device=None):
        self.cfgs = cfgs
        self.steps = steps
        self.samples = samples
        self.device = torch.device(device or "cuda")
        self.fields = [torch.from_numpy(beams.make_field(c).astype(np.complex64)).to(self.device) for c in cfgs]
        self._grids = {}
        self.P0 = self.vectors([target_gene])[0]

    def _grid(self, c):
        # one helper grid per (n, L): it only holds a field for its moments
        key = (c["n"], c["L"])
        if key not in self._grids:
            self._grids[key] = Grid(dict(c, theta=(1, 0, 1, 0, 1, 0)), precision="fp32", device=self.device)
        return self._grids[key]

    def vectors(self, genes) -> list:
        cfgs = [dict(c, theta=tuple(g)) for g in genes for c in self.cfgs]
        b = Batch(cfgs, device=self.device)
        try:
            for i in range(len(cfgs)):
                b.load(i, self.fields[i % len(self.cfgs)])
            per = [[] for _ in cfgs]
            k = self.steps // self.samples
            for _ in range(self.samples):
                b.step(k)
                if b.status() != 0:
                    raise RuntimeError("batched march failed")
                for i, c in enumerate(cfgs):
                    g = self._grid(c)
                    g.load(b.field(i, device=True))
                    q1, pw = g.moments([(1, 1), (1, 0)])
                    per[i].append((q1, pw))
        finally:
            b.close()
        nb = len(self.cfgs)
        out = []
        for gi in range(len(genes)):
            planes = []
            for s in range(self.samples):
                for bi in range(nb):
                    planes.append(per[gi * nb + bi][s])
            out.append(p_vector(planes))
        return out

    def __call__(self, genes) -> list:
        out = []
        for v in self.vectors(genes):
            f = float(np.linalg.norm(v - self.P0))
            out.append(f if math.isfinite(f) else math.inf)  # a march that blew up is never viable
        return out

    def close(self):
        for g in self._grids.values():
            g.close()
        self._grids = {}
