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
