"""Evolutionary search for error-inducing launch configurations (Sec. 3.3, Algorithms 1 and 2).

A solution is a launch of a parametric model kernel: grid and block dimensions
and real-valued arguments (converted to integers, truncating toward zero, when
the kernel is simulated). Its fitness is Eq. 1's F = sum g / sum f over the
trace the launch records (1: no two threads share an address; smaller: more
sharing), computed for a whole population at once by one batched device call
(simulee_model_traces + simulee_fitness_batch); the secondary fitness R =
end - start of the accessed range breaks the ranking only when the best F is 1.

Algorithm 1: an initial random population is scored and ranked; every
generation each solution yields two children (Algorithm 2: the arguments plus a
standard normal step in one child and a standard Cauchy step in the other; the
dimensions plus a random vector of -1, 0, 1 in each child), parents and
children are ranked together and the best `population` survive; the search
stops as soon as the best solution is acceptable (F < 0.3) or after
`generations` generations. The accepted launch then goes to the check
(simulee_check) for the bug report.

The random draws come from one seeded numpy generator, so a run is reproducible
and any scorer that computes the same fitness gives the same trajectory.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import simulee

# dimension limits per model: (grid_x, grid_y, block_x, block_y) lower and upper bounds
LIMITS = {
    simulee.MODEL_COPY2D: ((1, 1, 1, 1), (16, 16, 32, 32)),
    simulee.MODEL_STENCIL: ((1, 1, 1, 1), (64, 1, 1024, 1)),
}
ARG_BOUND = float(1 << 20)   # arguments stay within int32 after conversion


@dataclasses.dataclass
class Solution:
    model: int
    dims: tuple       # (grid_x, grid_y, block_x, block_y)
    args: tuple       # (arg0, arg1), real
    F: float = math.nan
    R: int = 0

    def launch(self):
        gx, gy, bx, by = self.dims
        return (self.model, (gx, gy), (bx, by), tuple(int(a) for a in self.args))


def scores(fit: dict) -> tuple[float, int]:
    """(F, R) of one fitness result: F = n_addresses / n_pairs (1 for an empty trace); R = the widest
    accessed range over the two spaces."""
    F = fit["n_addresses"] / fit["n_pairs"] if fit["n_pairs"] else 1.0
    R = 0
    for lo, hi in ((fit["shared_lo"], fit["shared_hi"]), (fit["global_lo"], fit["global_hi"])):
        if lo <= hi:
            R = max(R, hi - lo)
    return F, R


def rank(pop: list[Solution]) -> list[Solution]:
    """Order by F; when the best F is 1 (no sharing anywhere), order by R instead (stable sorts)."""
    pop = sorted(pop, key=lambda s: s.F)
    if pop and pop[0].F >= 1.0:
        pop = sorted(pop, key=lambda s: s.R)
    return pop


class DeviceScorer:
    """Scores a population on the GPU: one generator launch and one batched fitness call."""

    def __init__(self, checker: simulee.Checker):
        self.chk = checker

    def __call__(self, sols: list[Solution]) -> list[dict]:
        dts = self.chk.model_traces([s.launch() for s in sols])
        return self.chk.fitness_batch(dts)


class Evolution:
    def __init__(self, model: int, scorer, population: int = 50, generations: int = 3, acceptable: float = 0.3,
                 seed: int = 1905018330, init_arg_range: float = 64.0, limits=None):
        self.model = model
        self.scorer = scorer
        self.population = population
        self.generations = generations
        self.acceptable = acceptable
        self.rng = np.random.default_rng(seed)
        self.lo, self.hi = (np.array(v) for v in (limits or LIMITS[model]))
        self.init_arg_range = init_arg_range

    def _clamp_dims(self, d) -> tuple:
        d = np.minimum(np.maximum(np.asarray(d, dtype=np.int64), self.lo), self.hi)
        gx, gy, bx, by = (int(v) for v in d)
        while bx * by > 1024:          # a block holds at most 1024 threads
            if by > 1:
                by -= 1
            else:
                bx -= 1
        return (gx, gy, bx, by)

    def _clamp_args(self, a) -> tuple:
        return tuple(float(min(max(v, -ARG_BOUND), ARG_BOUND)) for v in a)

    def initial(self) -> Solution:
        dims = self.rng.integers(self.lo, self.hi + 1)
        args = self.rng.uniform(0.0, self.init_arg_range, size=2)
        return Solution(self.model, self._clamp_dims(dims), self._clamp_args(args))

    def mutate(self, parent: Solution) -> list[Solution]:
        """Algorithm 2 for the arguments (normal and Cauchy steps), -1/0/1 steps for the dimensions."""
        children = []
        for draw in (self.rng.standard_normal, self.rng.standard_cauchy):   # per child: its step, then its dims
            step = draw(2)
            dims = np.asarray(parent.dims) + self.rng.integers(-1, 2, size=4)
            args = np.asarray(parent.args) + step
            children.append(Solution(self.model, self._clamp_dims(dims), self._clamp_args(args)))
        return children

    def score(self, sols: list[Solution]) -> None:
        for s, fit in zip(sols, self.scorer(sols)):
            if fit["status"] != simulee.OK:
                raise RuntimeError(f"fitness failed with status {fit['status']}")
            s.F, s.R = scores(fit)

    def run(self) -> dict:
        pop = [self.initial() for _ in range(self.population)]
        self.score(pop)
        pop = rank(pop)
        history = [(pop[0].F, pop[0].R)]
        gens = 0
        for _ in range(self.generations):
            gens += 1
            children = [c for s in pop for c in self.mutate(s)]
            self.score(children)
            pop = rank(pop + children)[:self.population]
            history.append((pop[0].F, pop[0].R))
            if pop[0].F < self.acceptable:
                break
        return dict(best=pop[0], population=pop, history=history, generations=gens,
                    accepted=pop[0].F < self.acceptable)


def detect(checker: simulee.Checker, sol: Solution) -> dict:
    """Run the check on the trace of one launch (the bug report for an accepted solution)."""
    dt = checker.model_traces([sol.launch()])[0]
    return checker.check(dt)
