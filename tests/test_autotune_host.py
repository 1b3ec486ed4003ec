"""The autotuner's host logic on the CPU, with a stand-in context whose step
time is a known function of the knobs: coordinate descent finds the minimum,
every candidate starts from the restored snapshot, and the space is pruned by
what the context runs (one system: no balance; the resident solver: no block
budget, which the general one-system solver keeps; a plain Jacobi form keeps
its degree)."""
import pytest

from paper_1906_08125_gb300 import autotune


class FakeCtx:
    def __init__(self, n_rep=1, resident=1, cheb=6, cost=None):
        self._info = {"n_rep": n_rep, "pcg_resident": resident, "n_tets": 1000}
        self.params = {"precision": 1, "pcg_cheb_degree": cheb}
        self.knobs = {"particle_blocks_per_sm": 8, "walk_form": 1, "pcg_blocks_per_sm": 0,
                      "pcg_cheb_degree": cheb, "pcg_balance": 1}
        self.cost = cost or (lambda k: 1.0)
        self.restores = 0
        self.step_index = 0
        self.clock = 0.0

    def info(self):
        return self._info

    def tuning(self):
        return dict(self.knobs)

    def set_tuning(self, **kw):
        self.knobs.update(kw)

    def potential(self):
        return "phi"

    def particles(self):
        return ("r", "v", "cell", "pid")

    def set_potential(self, phi):
        self.restores += 1

    def set_particles(self, *parts):
        pass

    def num_particles(self):
        return 1000

    def step(self, n, stats=True):
        self.clock += n * self.cost(self.knobs) * 1e-3

    def sync(self):
        pass


@pytest.fixture
def fake_clock(monkeypatch):
    ctxs = []
    monkeypatch.setattr(autotune.time, "perf_counter", lambda: ctxs[0].clock if ctxs else 0.0)
    monkeypatch.setattr(autotune, "signature", lambda ctx: "stand-in")   # names a device
    return ctxs


def test_descent_finds_the_minimum_and_restores(fake_clock):
    best = {"particle_blocks_per_sm": 24, "walk_form": 2}
    cost = lambda k: (1.0 + abs(k["particle_blocks_per_sm"] - best["particle_blocks_per_sm"]) / 8
                      + (0.5 if k["walk_form"] != best["walk_form"] else 0.0))
    c = FakeCtx(cost=cost)
    fake_clock.append(c)
    knobs, ms, trials = autotune.tune(c, steps=2, warmup=1, use_cache=False,
                                      space={"particle_blocks_per_sm": (4, 8, 16, 24, 32),
                                             "walk_form": (1, 2, 3)})
    assert knobs["particle_blocks_per_sm"] == 24 and knobs["walk_form"] == 2
    assert ms == pytest.approx(1.0)
    assert c.restores >= 2 * len(trials)        # every candidate from the snapshot
    assert c.knobs["particle_blocks_per_sm"] == 24


@pytest.mark.parametrize("n_rep,resident,cheb,kept,dropped", [
    (1, 1, 6, [], ["pcg_blocks_per_sm", "pcg_balance"]),
    (1, 0, 6, ["pcg_blocks_per_sm"], ["pcg_balance"]),
    (4, 0, 6, ["pcg_blocks_per_sm", "pcg_balance"], []),
    (1, 1, 0, [], ["pcg_cheb_degree"]),
])
def test_space_follows_the_solver_in_use(fake_clock, n_rep, resident, cheb, kept, dropped):
    c = FakeCtx(n_rep=n_rep, resident=resident, cheb=cheb)
    fake_clock.append(c)
    _, _, trials = autotune.tune(c, steps=1, warmup=0, use_cache=False)
    tried = set()
    for knobs, _ in trials:
        tried.update(k for k, v in knobs.items() if v != FakeCtx(cheb=cheb).knobs.get(k))
    for k in kept:
        assert k in tried, k
    for k in dropped:
        assert k not in tried, k
