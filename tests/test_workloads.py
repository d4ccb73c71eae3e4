"""The seeded workload generators: deterministic, and shaped as the measured workloads are
described (grid, layer layout, bath size, seeds).  No method arithmetic lives in them; these
checks keep the stated input recipes and the generated inputs in step."""
import numpy as np

from paper_2505_23963_gb300 import workloads as wl


def layers(p):
    return [(m["kind"], m["z"], len(m.get("bath_frequencies", ()))) for m in p["materials"]]


def test_slab_3d_recipe():
    p = wl.slab_3d(steps=10)
    assert p["n"] == (256, 256, 256) and p["resolution"] == 32.0 and p["pml"] == 16
    assert layers(p) == [("drude", (88, 96), 0), ("lorentz_bath", (96, 160), 8), ("drude", (160, 168), 0)]
    assert p["sources"][0]["z"] == 24 and p["sources"][0]["component"] == 0
    assert p["sources"][0]["phase"].shape == (256, 256)
    assert p["monitors"][0]["z"] == 232 and p["monitors"][0]["freqs"].size == 256
    assert np.array_equal(p["sources"][0]["phase"], wl.slab_3d(steps=10)["sources"][0]["phase"])


def test_precision_and_adjoint_recipes():
    p = wl.precision_3d(steps=10)
    assert p["n"] == (512, 512, 384)
    assert [l[2] for l in layers(p)] == [0, 16, 0] and layers(p)[1][1] == (144, 240)
    a = wl.adjoint_2d(steps=10)
    assert a["n"] == (2048, 1, 2048) and a["sources"][0]["component"] == 1
    assert layers(a)[1] == ("lorentz_bath", (776, 1288), 8)
    assert a["monitors"][0]["freqs"].size == 128


def test_batch_sweep_recipe():
    probs = wl.batch_sweep(steps=10)
    L = np.array([p["n"][2] for p in probs])
    nb = np.array([layers(p)[1][2] for p in probs])
    assert len(probs) == 64
    assert np.array_equal(L, np.random.default_rng(0).integers(1000, 8001, size=64))
    assert np.array_equal(nb, np.random.default_rng(1).choice([4, 8, 16, 32], size=64))
    for p, n in zip(probs, L):
        (k0, m1, _), (k1, lay, _), (k2, m2, _) = layers(p)
        assert (k0, k1, k2) == ("drude", "lorentz_bath", "drude")
        assert lay[1] - lay[0] == round(0.4 * n) and m1[1] - m1[0] == 20 and m2[1] - m2[0] == 20
        assert p["energy_box"] == lay and p["pml"] == 16
    sig = np.array([p["materials"][1]["sigma"] for p in probs])
    assert np.allclose(np.sqrt(sig), np.linspace(0.01, 0.2, 64))
