"""Uneven-length batches (64/128/256/512 bp, Table 1 steps): the grouped
launch of all four length groups in clusters of two CTAs (or one launch per
group on its own stream), CUDA-graph replay of step chunks, and the
chains-per-tile autotuner.  None of them may change a trajectory."""
import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu

DT = {64: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def mixed(C, seed=3):
    rng = np.random.default_rng(seed)
    lengths = rng.choice([64, 128, 256, 512], size=C)
    return [{"n_beads": int(M), "dtau": DT[int(M)], "job_id": i,
             "shear_rate_per_s": 0.0 if i % 3 else 5e7} for i, M in enumerate(lengths)]


def run(chains, steps, graph=False, autotune=False, grouped=True, precision=sfp.SFP_FP32):
    b = sfp.Batch(chains, seed=7, precision=precision)
    b.set_grouped(grouped)
    b.init_equilibrium(0)
    tiles = None
    if autotune:
        before = [x.copy() for x in b.modes()]
        tiles = b.autotune(5)
        after = b.modes()
        assert all(np.array_equal(x, y) for x, y in zip(before, after))
        assert np.all(b.observe(sfp.SFP_OBS_STEP) == 0)
    if graph:
        b.set_graph(True)
    for k in (37, 100, 63):
        b.step(k)
    out = b.modes(), b.observe(sfp.SFP_OBS_COM), b.observe(sfp.SFP_OBS_STEP), b.info()["launches"]
    b.close()
    return out, tiles


def test_graph_replay_and_autotune_leave_trajectories_unchanged():
    chains = mixed(600)
    (ref, _) = run(chains, 200)
    (gr, _) = run(chains, 200, graph=True)
    (at, tiles) = run(chains, 200, autotune=True)
    for (a, b) in ((ref, gr), (ref, at)):
        assert all(np.array_equal(x, y) for x, y in zip(a[0], b[0]))
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.all(ref[2] == 200)
    # a replay counts the kernels it runs: all four length groups are one
    # grouped launch (clusters of two CTAs), so a chunk is one launch with or
    # without graphs
    assert gr[3] == ref[3]
    assert len(tiles) == 4 and all(4 <= t <= 40 and t % 4 == 0 for t in tiles)


@pytest.mark.parametrize("precision", [sfp.SFP_FP32, sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_BF16_2],
                         ids=["tf32x3", "bf16x3", "bf16x2"])
def test_grouped_launch_equals_one_launch_per_group(precision):
    """The grouped launch (clusters of two CTAs: a 512-bp tile per cluster, or two
    tiles of the other lengths) computes each tile exactly as the launch of its
    own group does: the same trajectories bit for bit, with and without graph
    replay, and one launch instead of four per chunk of steps."""
    chains = mixed(700, seed=5)
    (grp, _) = run(chains, 200, grouped=True, precision=precision)
    (sep, _) = run(chains, 200, grouped=False, precision=precision)
    (grg, _) = run(chains, 200, grouped=True, graph=True, precision=precision)
    for other in (sep, grg):
        assert all(np.array_equal(x, y) for x, y in zip(grp[0], other[0]))
        assert np.array_equal(grp[1], other[1]) and np.array_equal(grp[2], other[2])
    assert np.all(grp[2] == 200)
    assert sep[3] - grp[3] == 3 * 3        # three calls, three launches fewer each


def test_concurrent_groups_match_the_oracle():
    chains = mixed(40, seed=11)
    b = sfp.Batch(chains, seed=7)
    starts = [O.Model(c["n_beads"], dtau=c["dtau"]).equilibrium_start(7, c["job_id"]) for c in chains]
    b.set_modes(starts)
    b.set_graph(True)
    b.step(90)
    G = b.modes()
    for i in (0, 7, 13, 22, 39):
        c = chains[i]
        m = O.Model(c["n_beads"], dtau=c["dtau"])
        ref = m.run_modes(starts[i][None], 7, [c["job_id"]], 0, 90, shear=shear_tau(c["shear_rate_per_s"]))[0]
        err = np.linalg.norm(G[i][:, 1:] - ref[:, 1:]) / np.linalg.norm(ref[:, 1:])
        assert err < 1e-5, (i, err)
