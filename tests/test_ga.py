"""Population search of Fig. 2 on the CPU: the oracle's search pinned by its
invariants and by analytic fitness functions, and the library's search (host
logic) against the oracle's on the same draw stream."""
import numpy as np
import pytest

from oracle import ga as oga
from paper_2306_15678_gb300 import beams, ga

LO = [0.0, -1.0, 2.0]
HI = [1.0, 1.0, 5.0]
TARGET = np.array([0.3, -0.2, 4.1])


def sphere(genes):
    return [float(np.linalg.norm(np.asarray(g) - TARGET)) + 1e-3 for g in genes]


def test_roulette_frequencies_follow_inverse_fitness():
    """Roulette with weights 1/f: over a fine grid of draws each index is
    picked with frequency w_i / sum w (to the grid spacing)."""
    fs = [1.0, 2.0, 4.0, 0.5]
    w = np.array([1 / f for f in fs])
    u = (np.arange(100000) + 0.5) / 100000
    picks = np.bincount([oga.roulette(fs, x) for x in u], minlength=4)
    assert np.max(np.abs(picks / u.size - w / w.sum())) < 2e-5
    assert oga.roulette(fs, 0.0) == 0 and oga.roulette(fs, 0.999999999) == 3


def test_oracle_search_invariants_and_convergence():
    """Probe level: exactly probe // 10 probe genes are viable when the probe
    fitness values are distinct; every elite gene is viable; elitism makes
    the best fitness non-increasing; the draws consumed follow the protocol;
    on a sphere the search closes in on the minimum."""
    d = len(LO)
    draws = beams.ga_draws(5, 20000)
    r = oga.search(sphere, LO, HI, draws, generations=12)
    probe = [[LO[j] + draws[i * d + j] * (HI[j] - LO[j]) for j in range(d)] for i in range(20)]
    pf = sphere(probe)
    assert r["f_el"] == sorted(pf)[2]
    assert sum(f < r["f_el"] for f in pf) == 2
    assert r["history"][0] < r["f_el"]  # the elite generation is viable
    h = r["history"]
    assert all(h[i + 1] <= h[i] for i in range(len(h) - 1))
    nb = (r["draws_used"] - 20 * d - 12 * 10 * (2 + 3 * d)) // d
    assert r["draws_used"] == 20 * d + nb * d + 12 * 10 * (2 + 3 * d)
    assert nb % 10 == 0
    assert r["fitness"] < 0.5 * h[0]
    assert all(LO[j] <= r["gene"][j] <= HI[j] for j in range(d))


def test_oracle_search_one_dimensional_brute_force():
    """One gene, fitness |g - 0.3| + 1e-3: the search ends within the mutation
    reach of the minimum (brute force over the box gives 0.3)."""
    r = oga.search(lambda gs: [abs(g[0] - 0.3) + 1e-3 for g in gs], [0.0], [1.0], beams.ga_draws(9, 20000),
                   generations=20)
    assert abs(r["gene"][0] - 0.3) < 0.02


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_library_search_equals_oracle_search(seed):
    """Same draws, same fitness function: the library's search and the oracle's
    make the same choices and return the same gene, bit for bit."""
    draws = beams.ga_draws(seed, 20000)
    kw = dict(generations=6, pop=8, elite=5)
    a = ga.search(sphere, LO, HI, draws, **kw)
    b = oga.search(sphere, LO, HI, draws, **kw)
    assert a["gene"] == b["gene"] and a["fitness"] == b["fitness"]
    assert a["history"] == b["history"] and a["draws_used"] == b["draws_used"]
    assert [g for g, _ in a["elite"]] == [g for g, _ in b["elite"]]


def test_exhausted_stream_raises():
    with pytest.raises(RuntimeError):
        ga.search(sphere, LO, HI, beams.ga_draws(1, 50))
