"""Host logic of the batched form (no GPU): the packer behind fdtdbath_batch_plan.

Every cavity must land whole in one cluster; every cell in exactly one CTA; no CTA above its
shared-memory budget; the per-CTA work close to the cluster-level optimum; bad cavities are
rejected with the cavity named."""
import numpy as np
import pytest

from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl


def test_sweep_plan_covers_and_fits():
    probs = wl.batch_sweep(steps=10)
    cap = 200 * 1024
    r = fb.batch_plan(probs, 32, cluster_ctas=8, nclusters=19, smem_per_cta=cap)
    L = np.array([p["n"][2] for p in probs])
    assert r["work"].size == 8 * 19
    assert int(r["cells"].sum()) == int(L.sum())
    assert np.all(r["smem"] <= cap)
    assert set(np.unique(r["cluster"])) <= set(range(19))
    # cells of the cavities of each cluster add up to that cluster's CTAs
    for k in range(19):
        assert int(r["cells"][8 * k:8 * k + 8].sum()) == int(L[r["cluster"] == k].sum())
    # balance: the worst CTA within 25% of the ideal over all CTAs
    ideal = r["work"].sum() / r["work"].size
    assert r["work"].max() <= 1.25 * ideal, (r["work"].max(), ideal)


def test_single_cta_clusters_hold_whole_cavities():
    probs = wl.batch_small(seed=0, steps=10)
    r = fb.batch_plan(probs, 64, cluster_ctas=1, nclusters=3, smem_per_cta=200 * 1024)
    assert r["work"].size == 3
    L = np.array([p["n"][2] for p in probs])
    for k in range(3):
        assert int(r["cells"][k]) == int(L[r["cluster"] == k].sum())


def test_shared_memory_budget_is_enforced():
    probs = wl.batch_sweep(n=4, steps=10, lmin=7000, lmax=8000)
    with pytest.raises(fb.FdtdBathError) as e:
        fb.batch_plan(probs, 32, cluster_ctas=1, nclusters=4, smem_per_cta=64 * 1024)
    assert e.value.code == fb.ERR_UNSUPPORTED
    r = fb.batch_plan(probs, 32, cluster_ctas=16, nclusters=4, smem_per_cta=64 * 1024)
    assert np.all(r["smem"] <= 64 * 1024)


def test_bad_cavities_are_named():
    p = wl.batch_cavity(1000, rabi=0.1, num_bath=4, steps=10)
    bad = dict(p, sources=[dict(p["sources"][0], component=2)])
    with pytest.raises(fb.FdtdBathError) as e:
        fb.batch_plan([p, bad], 32, cluster_ctas=2, nclusters=2, smem_per_cta=100000)
    assert e.value.code == fb.ERR_ARG and "cavity 1" in str(e.value)
    short = wl.slab_cavity(1, 1, (8, 10, 2, 10, 2, 10), 100.0, num_bath=0, sigma=0.01,
                           phase_seed=None, nfreq=2, steps=10)
    with pytest.raises(fb.FdtdBathError) as e:
        fb.batch_plan([short], 32, cluster_ctas=1, nclusters=1, smem_per_cta=100000)
    assert e.value.code == fb.ERR_ARG and "nz" in str(e.value)
    hot = wl.batch_cavity(1000, rabi=0.1, num_bath=4, steps=10, resolution=2.0)
    with pytest.raises(fb.FdtdBathError) as e:
        fb.batch_plan([hot], 32, cluster_ctas=1, nclusters=1, smem_per_cta=100000)
    assert e.value.code == fb.ERR_CFL


def _cell_work(p):
    """Work units of every cell of a batch cavity, the packer's calibration: 4 per cell, 2 per
    CPML memory (E: the first and last npml cells, H: one more on the right), 8 per Lorentz /
    Drude cell, 8 + 4 N_b per Lorentz-Bath cell."""
    L = p["n"][2]
    w = np.full(L, 4, np.int64)
    pml = int(p["pml"])
    w[:pml] += 4
    w[L - pml:] += 4
    w[L - pml - 1] += 2
    for m in p["materials"]:
        z0, z1 = m["z"]
        nb = len(m.get("bath_frequencies", ()))
        w[z0:z1] += 8 + 4 * nb if nb else (8 if m["kind"] != "vacuum" else 0)
    return w


def _busiest_thread(probs, r, C, T):
    """Largest per-thread work of a plan: the cells of a cluster's cavities (in index order) cut
    into its CTAs by their cell counts, cell l of a CTA on thread l mod T."""
    worst = 0
    for k in range(r["work"].size // C):
        ids = np.nonzero(r["cluster"] == k)[0]
        if ids.size == 0:
            continue
        w = np.concatenate([_cell_work(probs[i]) for i in sorted(ids)])
        off = 0
        for c in range(C):
            n = int(r["cells"][k * C + c])
            pad = np.zeros(-(-max(n, 1) // T) * T, np.int64)
            pad[:n] = w[off:off + n]
            off += n
            worst = max(worst, int(pad.reshape(-1, T).sum(0).max()))
        assert off == w.size
    return worst


@pytest.mark.parametrize("C,T", [(4, 768), (8, 512)])
def test_plan_bounds_the_busiest_thread(C, T):
    """Cells are dealt round-robin over a CTA's threads, so a Lorentz-Bath run's remainder lands
    on some threads only; the plan for T threads bounds the busiest thread, which the whole-CTA
    balance (block_threads = 1) leaves up to twice the mean on the sweep."""
    probs = wl.batch_sweep(steps=10)
    cap = 220 * 1024
    kw = dict(cluster_ctas=C, nclusters=152 // C, smem_per_cta=cap)
    flat = fb.batch_plan(probs, 32, **kw)
    aware = fb.batch_plan(probs, 32, block_threads=T, **kw)
    L = np.array([p["n"][2] for p in probs])
    assert int(aware["cells"].sum()) == int(L.sum())
    assert np.all(aware["smem"] <= cap)
    b_flat = _busiest_thread(probs, flat, C, T)
    b_aware = _busiest_thread(probs, aware, C, T)
    one_cell = 4 + 8 + 4 * 32          # an N_b = 32 bath cell: no thread can carry less
    mean = int(aware["work"].sum()) / (aware["work"].size * T)
    print(f"\nC={C} T={T}: busiest thread {b_flat} (whole-CTA balance) -> {b_aware}; mean {mean:.0f}")
    assert b_aware <= 0.75 * b_flat
    assert b_aware <= max(2 * mean, 1.25 * one_cell)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("C,T", [(1, 128), (2, 384), (4, 896), (16, 1024)])
def test_random_batches_are_covered(seed, C, T):
    """Seeded random batches (lengths 200..3000, N_b in {0, 4, 32, 100}; a cavity is at most as
    long as its bath state, 8 N_b B per layer cell in FP32, lets it fit 80% of a cluster's shared
    memory) in several launch shapes: every cavity in one cluster, every cell in exactly one CTA,
    no CTA above its budget."""
    cap = 200 * 1024
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(int(rng.integers(3, 20))):
        nb = int(rng.choice([0, 4, 32, 100]))
        lmax = min(3000, int(0.8 * C * cap / (0.4 * 8 * nb + 40)))
        L = int(rng.integers(200, lmax + 1))
        p = wl.batch_cavity(L, rabi=float(rng.uniform(0.01, 0.2)), num_bath=4, steps=10)
        m = dict(p["materials"][1])
        if nb == 0:   # plain Lorentz layer
            m["kind"] = "lorentz"
            for k in ("bath_frequencies", "bath_gammas", "bath_couplings"):
                m.pop(k, None)
        elif nb > 4:
            m["bath_frequencies"] = np.linspace(0.8, 1.2, nb)
            m["bath_gammas"] = np.full(nb, 4e-4)
            m["bath_couplings"] = np.full(nb, 0.002)
        p["materials"] = [p["materials"][0], m, p["materials"][2]]
        probs.append(p)
    ncl = max(1, 152 // C)
    r = fb.batch_plan(probs, 32, cluster_ctas=C, nclusters=ncl, smem_per_cta=cap, block_threads=T)
    L = np.array([p["n"][2] for p in probs])
    assert r["work"].size % C == 0
    assert np.all(r["cells"] >= 0) and np.all(r["smem"] <= cap)
    for k in range(r["work"].size // C):
        assert int(r["cells"][C * k:C * k + C].sum()) == int(L[r["cluster"] == k].sum())
    assert int(r["cells"].sum()) == int(L.sum())
