"""The seeded synthetic inputs: the batch generator keeps its stated ranges and separations and is
reproducible; the small batch and the named configurations are well formed."""

import numpy as np

import workloads as W


def _min_image_distance(frac, abc):
    best = np.inf
    for i in range(len(frac)):
        for j in range(i):
            d = np.asarray(frac[i]) - np.asarray(frac[j])
            d -= np.round(d)
            best = min(best, float(np.linalg.norm(d * abc)))
    return best


def test_batch_generator_ranges_and_reproducibility():
    cells = W.batch_cells()
    again = W.batch_cells()
    assert len(cells) == 16
    for c, c2 in zip(cells, again):
        assert c["atoms"] == c2["atoms"] and c["ecutwfc"] == c2["ecutwfc"]
        abc = np.array([c["cell"][0][0], c["cell"][1][1], c["cell"][2][2]])
        assert np.all((abc >= 7.0) & (abc <= 12.0))
        assert 2 <= len(c["atoms"]) <= 12
        kinds = [s for s, _ in c["atoms"]]
        assert 0 in kinds  # at least one H
        assert _min_image_distance([p for _, p in c["atoms"]], abc) >= 3.5
        assert 25.0 <= c["ecutwfc"] <= 45.0
        assert all(k in (2, 3, 4) for k in c["kmesh"])
        assert all(q in (1, 2) and k % q == 0 for k, q in zip(c["kmesh"], c["qmesh"]))
    sizes = {len(c["atoms"]) for c in cells}
    assert len(sizes) > 3  # uneven
    other = W.batch_cells(seed=1)
    assert any(a["atoms"] != b["atoms"] for a, b in zip(cells, other))


def test_small_batch_and_configs_well_formed():
    for w in W.batch_small() + [f() for f in W.CONFIGS.values()]:
        assert w["nelec"] > 0 and w["nelec"] % 2 == 0
        assert w["nspin"] in (1, 2)
        assert len(w["kmesh"]) == 3 and len(w["qmesh"]) == 3
        if w["nspin"] == 2:
            assert w["moments"] is not None and len(w["moments"]) == len(w["atoms"])
