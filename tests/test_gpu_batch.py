"""Batched form: many independent 1-D/2-D problems in one persistent,
graph-captured kernel per stage.  Each problem must evolve exactly as it does
alone, whatever the launch configuration."""
import numpy as np
import pytest

from paper_2404_08247_gb300 import inputs as I
from parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def R():
    from paper_2404_08247_gb300 import build as B
    B.build()
    from paper_2404_08247_gb300 import rhd
    rhd.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return rhd


def small_batch(n=10, seed=5):
    return I.batched_problems(nprob=n, seed=seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_each_problem_alone(R, precision):
    problems = small_batch()
    nsteps = 4
    with R.RHDBatch([p for p, _ in problems], precision) as b:
        for i, (_, U) in enumerate(problems):
            b.set_state(i, U)
        info = b.step(nsteps)
        assert info["steps_done"] == nsteps
        got = [b.get_state(i) for i in range(len(problems))]
    for i, (p, U) in enumerate(problems):
        with R.RHDContext(p, precision) as ctx:
            ctx.set_state(U)
            ctx.step(nsteps)
            want = ctx.get_state()
        assert_parity(got[i], want, TOL, "problem %d" % i)


def test_batch_fp64_matches_oracle(R, oracle_mod):
    problems = []
    for k, (ndim, n) in enumerate([(1, [300]), (2, [40, 24]), (1, [77]), (2, [17, 33])]):
        prob = I.base_problem(ndim, n, [1.0 / v for v in n], c=1e3, chat=1e2)
        problems.append((prob, I.random_state(prob, seed=50 + k, beta_max=1e-2)))
    with R.RHDBatch([p for p, _ in problems], "fp64") as b:
        for i, (_, U) in enumerate(problems):
            b.set_state(i, U)
        b.step(3)
        got = [b.get_state(i) for i in range(len(problems))]
    for i, (p, U) in enumerate(problems):
        Uo = U.copy()
        oracle_mod.step(p, Uo, nsteps=3)
        assert_parity(got[i], Uo, TOL, "problem %d" % i)


def test_every_launch_configuration_gives_the_same_bits(R):
    problems = small_batch(8, seed=9)
    results = {}
    for tile2d in (0, 1, 2):
        for bps in (1, 2):
            with R.RHDBatch([p for p, _ in problems], "mixed") as b:
                b.configure(tile2d, bps)
                for i, (_, U) in enumerate(problems):
                    b.set_state(i, U)
                b.step(3)
                results[(tile2d, bps)] = [b.get_state(i) for i in range(len(problems))]
    ref = results[(0, 2)]
    for cfg, res in results.items():
        for i in range(len(problems)):
            assert np.array_equal(res[i], ref[i]), (cfg, i)


def test_graph_replays_compose(R):
    """step(2) twice (one graph replayed) equals step(4) (another graph)."""
    problems = small_batch(6, seed=13)
    out = []
    for plan in ([2, 2], [4], [1, 3]):
        with R.RHDBatch([p for p, _ in problems], "mixed") as b:
            for i, (_, U) in enumerate(problems):
                b.set_state(i, U)
            for n in plan:
                b.step(n)
            out.append([b.get_state(i) for i in range(len(problems))])
    for res in out[1:]:
        for i in range(len(problems)):
            assert np.array_equal(res[i], out[0][i])


def test_failure_is_located_and_state_kept(R):
    problems = small_batch(6, seed=17)
    probs = [dict(p) for p, _ in problems]
    probs[3]["newton_max_iter"] = 1
    with R.RHDBatch(probs, "fp64") as b:
        for i, (_, U) in enumerate(problems):
            b.set_state(i, U)
        info = b.step(2, raise_on_error=False)
        assert info["status"] == R.RHD_ERR_NEWTON and info["steps_done"] == 0
        p, cell = b.locate(info["fail_cell"])
        assert p == 3 and 0 <= cell < b.cells(3)
        for i, (_, U) in enumerate(problems):
            assert np.array_equal(b.get_state(i), U)


def test_autotuner_picks_and_caches(R, tmp_path):
    from paper_2404_08247_gb300 import autotune
    problems = small_batch(6, seed=21)
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(problems, "mixed", nsteps=2, cache_path=cache)
    assert not res["cached"]
    assert (res["tile2d"], res["blocks_per_sm"]) in autotune.CANDIDATES
    assert len(res["timings_ms"]) == len(autotune.CANDIDATES)
    again = autotune.tune(problems, "mixed", nsteps=2, cache_path=cache)
    assert again["cached"] and again["tile2d"] == res["tile2d"]


def test_batch_mixed_workload_subset_matches_oracle(R, oracle_mod):
    """The batched workload as the benchmark runs it (mixed precision, the
    persistent graph-captured kernel): its first 16 problems (the generator
    draws problems in sequence, so these are the 512-problem workload's
    first 16: 1-D up to 4096 cells and 2-D up to 256^2, log10 tau_cell iid
    U[-3, 3], |v|/c up to 1e-3) over 50 steps, each against the FP64 oracle
    to the mixed-precision bound 1e-5 per field."""
    problems = I.batched_problems(nprob=16, seed=11)
    nsteps = 50
    with R.RHDBatch([p for p, _ in problems], "mixed") as b:
        for i, (_, U) in enumerate(problems):
            b.set_state(i, U)
        info = b.step(nsteps)
        assert info["steps_done"] == nsteps
        got = [b.get_state(i) for i in range(len(problems))]
    worst = 0.0
    for i, (p, U) in enumerate(problems):
        Uo = U.copy()
        oracle_mod.step(p, Uo, nsteps=nsteps)
        errs = assert_parity(got[i], Uo, 1e-5, "problem %d (%s cells)" % (i, p["n"]))
        worst = max(worst, max(errs.values()))
    print("worst per-field error over the 16 problems: %.2e" % worst)


def test_direct_launches_equal_graph_replays(R):
    """rhd_batch_use_graphs(0) enqueues each step's launches directly: the
    same bits as the captured graphs."""
    problems = small_batch(6, seed=23)
    out = []
    for graphs in (True, False):
        with R.RHDBatch([p for p, _ in problems], "mixed") as b:
            b.use_graphs(graphs)
            for i, (_, U) in enumerate(problems):
                b.set_state(i, U)
            b.step(3)
            out.append([b.get_state(i) for i in range(len(problems))])
    for i in range(len(problems)):
        assert np.array_equal(out[0][i], out[1][i]), i
