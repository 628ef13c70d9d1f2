"""Ensembles of independent 2D Model B instances, sharded over ranks.

An ensemble of noise realisations or a parameter sweep (section "Adding
noise": every realisation is an independent run of the same equations) is
a list of instances, each with its own lattice side, Philox seed and
coefficient a.  A single system does not shard without an all-to-all
transpose per FFT pass; an ensemble does, instance by instance, with no
exchange while it runs.  The one collective is at the end: the per-instance
radially binned S(q) (FP64 bin means, 64 bins) are gathered and averaged per
lattice size in instance order, so the merged result does not depend on how
the instances were spread over ranks.

* ``recipe`` draws the 512-instance workload (sides uniform over
  {64, 128, 256, 512}, seeds base + i, a ~ U[-1.5, -0.5]).
* ``partition`` splits instances over ranks by cost (sites x steps), longest
  first onto the least-loaded rank (ties: lower index, lower rank).
* ``build_systems`` makes one batched system per lattice size for a share of
  the instances (launches through the library's C ABI).
* ``structure_factors`` reads every instance's S(q) from its system.
* ``merge`` averages per-instance S(q) per lattice size in instance order;
  ``gather`` brings every rank's per-instance S(q) together first
  (torch.distributed, any backend).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

SIZES = (64, 128, 256, 512)


@dataclass
class Spec:
    """The instances of an ensemble: side[i] (square lattice), seed[i], a[i]; shared Model B
    coefficients b, K, D, time step dt, initial field U[lo, hi), steps, S(q) bins."""

    side: List[int]
    seed: List[int]
    a: List[float]
    b: float = 1.0
    K: float = 1.0
    D: float = 0.01
    dt: float = 0.01
    lo: float = -0.1
    hi: float = 0.1
    steps: int = 1000
    nbins: int = 64
    extra: dict = field(default_factory=dict)

    def __len__(self) -> int:
        return len(self.side)

    def cost(self, i: int) -> int:
        """Sites x steps of instance i."""
        return int(self.side[i]) ** 2 * int(self.steps)


def recipe(n: int = 512, gen_seed: int = 2405, base_seed: int = 10000, steps: int = 1000,
           sizes: Sequence[int] = SIZES) -> Spec:
    """The ensemble workload: n instances, sides drawn uniformly from `sizes` with numpy's
    default_rng(gen_seed), seeds base_seed + i, a ~ U[-1.5, -0.5] from the same generator."""
    g = np.random.default_rng(gen_seed)
    side = g.choice(list(sizes), size=n)
    a = g.uniform(-1.5, -0.5, size=n)
    return Spec(side=[int(x) for x in side], seed=[base_seed + i for i in range(n)], a=[float(x) for x in a],
                steps=steps)


def partition(costs: Sequence[int], world: int) -> List[List[int]]:
    """Instances (by index) per rank: longest processing time first onto the rank with the least
    cost so far; ties go to the lower instance index and the lower rank, so every rank computes
    the same split.  Each rank's list is in increasing instance order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-int(costs[i]), i))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(costs[i])
    return [sorted(x) for x in out]


def share(spec: Spec, rank: int, world: int) -> List[int]:
    """This rank's instances."""
    return partition([spec.cost(i) for i in range(len(spec))], world)[rank]


def build_systems(pss, spec: Spec, indices: Sequence[int], precision: str = "f32"):
    """One batched system per lattice side for the given instances (each initialised from its own
    seed): returns [(side, system, [instance indices in batch order])]."""
    out = []
    for sz in sorted({spec.side[i] for i in indices}):
        idx = [i for i in indices if spec.side[i] == sz]
        s = pss.System((sz, sz), dt=spec.dt, batch=len(idx), seeds=[spec.seed[i] for i in idx], precision=precision)
        pss.add_model_b_field(s, a=-1.0, b=spec.b, K=spec.K, D=spec.D)
        s.set_param_batch(0, np.array([spec.a[i] for i in idx], dtype=np.float64))
        for j in range(len(idx)):
            s.select_instance(j)
            s.init_uniform(0, spec.lo, spec.hi)
        s.select_instance(0)
        out.append((sz, s, idx))
    return out


def structure_factors(groups, nbins: int = 64) -> Dict[int, np.ndarray]:
    """Per-instance S(q) bin means {instance: S[nbins]} of systems made by build_systems."""
    out = {}
    for _, s, idx in groups:
        for j, i in enumerate(idx):
            s.select_instance(j)
            S, _, _ = s.structure_factor(0, nbins)
            out[int(i)] = np.asarray(S, dtype=np.float64)
        s.select_instance(0)
    return out


def merge(spec: Spec, per_instance: Dict[int, np.ndarray]) -> Dict[int, np.ndarray]:
    """Ensemble-averaged S(q) per lattice side: the instances' bin means added in increasing
    instance order (FP64), divided by their number."""
    out = {}
    for sz in sorted(set(spec.side)):
        idx = [i for i in range(len(spec)) if spec.side[i] == sz]
        if not all(i in per_instance for i in idx):
            missing = [i for i in idx if i not in per_instance]
            raise KeyError(f"S(q) of instances {missing[:8]} missing")
        acc = np.zeros_like(per_instance[idx[0]])
        for i in idx:
            acc = acc + per_instance[i]
        out[sz] = acc / len(idx)
    return out


def gather(local: Dict[int, np.ndarray], world: int) -> Dict[int, np.ndarray]:
    """Every rank's per-instance S(q), on every rank (torch.distributed all_gather_object; with
    world == 1 the local dict itself)."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    parts: List[Optional[dict]] = [None] * world
    dist.all_gather_object(parts, {int(k): np.asarray(v).tolist() for k, v in local.items()})
    out: Dict[int, np.ndarray] = {}
    for p in parts:
        for k, v in p.items():
            if int(k) in out:
                raise ValueError(f"instance {k} ran on two ranks")
            out[int(k)] = np.asarray(v, dtype=np.float64)
    return out


def run_sharded(spec: Spec, rank: int, world: int, runner: Callable[[Spec, List[int]], Dict[int, np.ndarray]]):
    """This rank's share through `runner(spec, indices) -> {instance: S[nbins]}`, then the
    gathered, merged ensemble average on every rank: (merged, this rank's indices)."""
    idx = share(spec, rank, world)
    local = runner(spec, idx) if idx else {}
    return merge(spec, gather(local, world)), idx
