"""Several independent cells at once (hp_batch_run): each cell on its own CUDA stream and host
thread gives the same chi_0, chi and U/V as the same cell run alone (every kernel reduces in a fixed
order, so to rounding identity), and the batch finishes."""

import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2203_15684_gb300")
torch = pytest.importorskip("torch")


def _cells():
    return [W.tiny_q(ecut=8.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 1, 1)),
            W.tiny_lowcut(ecut=10.0, grid=(12, 12, 12), kmesh=(2, 2, 2), qmesh=(2, 2, 1)),
            W.medium_small(ecut=6.0, grid=(16, 16, 16), kmesh=(2, 1, 1), qmesh=(2, 1, 1))]


def _ready(w, precision):
    stream = torch.cuda.Stream()
    ctx = P.Context.from_workload(w, cuda_stream=stream.cuda_stream, precision=precision)
    ctx.ground_state(w["nelec"], w["nspin"], w.get("moments"))
    return ctx, stream


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_cells_alone(precision):
    cells = _cells()
    alone = []
    t0 = time.perf_counter()
    for w in cells:
        ctx, _ = _ready(w, precision)
        atoms, _ = ctx.hubbard_atoms()
        for J in atoms:
            for iq in range(ctx.query_sizes()["nq"]):
                ctx.response(iq, int(J))
        alone.append(ctx.hubbard())
    t_alone = time.perf_counter() - t0
    ready = [_ready(w, precision) for w in cells]
    t0 = time.perf_counter()
    batch = P.batch_run([c for c, _ in ready])
    t_batch = time.perf_counter() - t0
    print("batch of %d cells: %.2f s (alone, with ground states: %.2f s)" % (len(cells), t_batch, t_alone))
    for (a0, a1, a2), (b0, b1, b2) in zip(alone, batch):
        for a, b in ((a0, b0), (a1, b1), (a2, b2)):
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_seeded_cells_electron_rule_and_batch():
    """Two cells of the seeded batch of 16 cells: the library's bare spectrum at the first and the last
    k point equals the oracle's dense diagonalisation of T + V_loc + V_NL (1e-9 Ha); the electron-count
    rule (largest gap over the k mesh among band counts n_H + n_L .. 5 n_H + 3 n_L) gives a ground
    state with a gap; the two cells at once equal the cells alone (mixed form)."""
    from oracle.groundstate import eigensolve
    from oracle.model import Model

    cells = [c for c in W.batch_cells() if c["name"] in ("batch03", "batch07")]
    ready, alone = [], []
    for w in cells:
        stream = torch.cuda.Stream()
        ctx = P.Context.from_workload(w, cuda_stream=stream.cuda_stream, precision=1)
        nH = sum(1 for s, _ in w["atoms"] if s == 0)
        n = 5 * nH + 3 * (len(w["atoms"]) - nH) + 1
        m = Model(w)
        for ik in (0, len(m.kpts) - 1):
            lev = ctx.bare_levels(n, ik)
            ref, _ = eigensolve(m, m.kdata(m.kpts[ik]), m.vloc_r(), n)
            assert np.abs(lev - ref).max() < 1e-9
        nelec = P.batch_electron_count(ctx, w)
        assert nelec % 2 == 0 and 2 * (len(w["atoms"])) <= nelec <= 2 * (n - 1)
        gs = ctx.ground_state(nelec, 1)
        assert gs["gap"] > 1e-4
        atoms, _ = ctx.hubbard_atoms()
        for J in atoms:
            for iq in range(ctx.query_sizes()["nq"]):
                ctx.response(iq, int(J))
        alone.append(ctx.hubbard())
        ready.append((ctx, stream))
    batch = P.batch_run([c for c, _ in ready])
    for (a0, a1, a2), (b0, b1, b2) in zip(alone, batch):
        for a, b in ((a0, b0), (a1, b1), (a2, b2)):
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())
