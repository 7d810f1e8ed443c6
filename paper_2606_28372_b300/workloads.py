"""Seeded synthetic inputs: search-space definitions, fitness tables, candidate tuples.

This module only *describes* inputs.  It holds none of the method's arithmetic:
it never decodes Cartesian indices, evaluates constraints, packs keys, looks up
ranks or repairs candidates.  Both the CUDA path and the CPU oracle receive the
objects built here and do all of that themselves.

Spaces follow the CSP statement of Section IV-A (variables, finite domains,
constraints as predicates over a scope).  Constraints are strings in a small
integer expression language (Python syntax): integer literals, parameter names,
``+ - * // %`` (C semantics: ``//`` and ``%`` truncate toward zero), unary
minus, ``min(a, b)``, ``max(a, b)``, comparisons (chains allowed),
``and``/``or``/``not``.  Arithmetic is 64-bit two's complement.  A division or
modulo by zero poisons the sub-expression: a comparison with a poisoned operand
is false, and a poisoned value at the top of a constraint makes it false.

The shapes imitate the benchmark spaces of Table III (parameter counts, value
list lengths, densities from ~1.4 % to ~56 %); the BAT suite itself is not used.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

POW2 = lambda lo, hi: [1 << k for k in range(lo, hi + 1)]  # noqa: E731


@dataclass(frozen=True)
class SpaceDef:
    """A tuning space: ordered parameters with value lists, plus constraints."""

    name: str
    params: tuple  # tuple of (name, tuple(values))
    constraints: tuple  # tuple of constraint strings
    note: str = ""

    @property
    def names(self):
        return [p[0] for p in self.params]

    @property
    def values(self):
        return [list(p[1]) for p in self.params]

    @property
    def n_values(self):
        return [len(p[1]) for p in self.params]

    @property
    def cartesian_size(self):
        s = 1
        for p in self.params:
            s *= len(p[1])
        return s


def _space(name, params, constraints, note=""):
    return SpaceDef(name, tuple((n, tuple(int(v) for v in vals)) for n, vals in params),
                    tuple(constraints), note)


def tiny_space() -> SpaceDef:
    """4 parameters, 1,296 Cartesian points; the GEMM-style block constraint of Section II."""
    return _space(
        "tiny",
        [("bx", POW2(5, 10)), ("by", POW2(0, 5)), ("tile", POW2(0, 5)), ("unroll", POW2(0, 5))],
        ["bx*by<=1024", "bx%tile==0", "4*bx*tile<=49152"],
        "hand count: 122 (bx,by,tile) triples x 6 unroll values = 732 valid",
    )


def medium_space() -> SpaceDef:
    """10 parameters, 9,408,000 Cartesian points, 8 constraints (density near Hotspot's)."""
    return _space(
        "medium",
        [("bx", POW2(4, 10)), ("by", POW2(0, 6)), ("tx", POW2(0, 4)), ("ty", POW2(0, 4)),
         ("unroll", POW2(0, 4)), ("vec", POW2(0, 3)), ("stages", range(1, 7)), ("pad", [0, 1]),
         ("splitk", [1, 2, 3, 4, 6, 8, 12, 16]), ("ro", [0, 1, 2, 3])],
        ["64<=bx*by<=1024", "bx%(tx*vec)==0", "by*ty<=16",
         "4*(bx*tx+pad)*(by*ty)*stages<=49152", "unroll*vec<=tx*ty",
         "splitk<=2 or stages>=4", "vec*tx<=8", "ro==0 or pad==0"],
    )


_LARGE_A = (
    [("wgx", POW2(3, 9)), ("wgy", POW2(0, 5)), ("tpx", POW2(0, 4)), ("tpy", POW2(0, 4)),
     ("vw", POW2(0, 3)), ("kwg", POW2(4, 7)), ("kwi", POW2(0, 4)), ("sa", [0, 1, 2])],
    ["64<=wgx*wgy<=1024", "kwg%kwi==0", "(wgx*tpx)%vw==0",
     "4*kwg*(wgx*tpx+wgy*tpy)*(1+sa)<=49152", "tpx*tpy<=64", "vw<=tpx"],
)
_LARGE_B = (
    [("mdimc", POW2(3, 6)), ("ndimc", POW2(3, 6)), ("mwg", POW2(4, 8)), ("nwg", POW2(4, 8)),
     ("vwm", POW2(0, 3)), ("vwn", POW2(0, 3)), ("strm", range(0, 4)), ("strn", range(0, 8))],
    ["mwg%mdimc==0", "nwg%ndimc==0", "(mwg//mdimc)%vwm==0", "(nwg//ndimc)%vwn==0",
     "mdimc*ndimc<=512", "strm+strn<=3 or mwg==nwg"],
)


def large_group_a() -> SpaceDef:
    return _space("large_a", *_LARGE_A)


def large_group_b() -> SpaceDef:
    return _space("large_b", *_LARGE_B)


def large_space() -> SpaceDef:
    """16 parameters, 51,609,600,000 Cartesian points (needs an int64 index), 12 constraints.

    It is the product of two independent 8-parameter groups (no constraint spans both),
    so |V| = |V_A| * |V_B| — a closed form that pins the full-size count.
    """
    return _space("large", _LARGE_A[0] + _LARGE_B[0], _LARGE_A[1] + _LARGE_B[1],
                  "|V| = |V(large_a)| * |V(large_b)|")


def large_slice_space() -> SpaceDef:
    """The large space with wgx restricted to {64, 128}: 146,321,600 valid keys (1.17 GB), the
    same constraint structure and key layout widths; a smaller case of the same kernels for
    hardware-counter captures."""
    params = list(_LARGE_A[0] + _LARGE_B[0])
    params[0] = ("wgx", [64, 128])
    return _space("large_slice", params, _LARGE_A[1] + _LARGE_B[1])


def batched_space(s: int) -> SpaceDef:
    """Space ``s`` (0..31) of the batched workload: the medium template with resized value lists.

    A fixed deterministic recipe shrinks or grows value lists so that valid sizes spread
    roughly log-uniformly over 1e3..1e6; the exact count of each is whatever enumeration
    yields.  The constraints are the medium space's.
    """
    rng = np.random.Generator(np.random.Philox(key=0xBA7C4 + s))
    scale = (10.0 ** (3.0 + 3.0 * s / 31.0)) / 139604.0
    lens = {"bx": 7, "by": 7, "tx": 5, "ty": 5, "unroll": 5, "vec": 4, "stages": 6, "pad": 2,
            "splitk": 8, "ro": 4}
    lo = {"bx": 3, "by": 3, "tx": 2, "ty": 2, "unroll": 1, "vec": 1, "stages": 1, "pad": 1,
          "splitk": 1, "ro": 1}
    hi = {"bx": 7, "by": 7, "tx": 5, "ty": 5, "unroll": 7, "vec": 4, "stages": 12, "pad": 2,
          "splitk": 16, "ro": 8}
    order = ["ro", "splitk", "unroll", "stages", "pad", "vec", "ty", "tx", "by", "bx"]
    rng.shuffle(order)
    for name in order * 3:
        cur = lens[name]
        if scale < 0.8 and cur > lo[name]:
            new = min(cur - 1, max(lo[name], int(round(cur * max(scale, 0.4)))))
        elif scale > 1.25 and cur < hi[name]:
            new = max(cur + 1, min(hi[name], int(round(cur * min(scale, 2.0)))))
        else:
            continue
        scale /= new / cur
        lens[name] = new
    vals = {
        "bx": POW2(4, 10)[-lens["bx"]:],
        "by": POW2(0, 6)[: lens["by"]],
        "tx": POW2(0, 4)[: lens["tx"]],
        "ty": POW2(0, 4)[: lens["ty"]],
        "unroll": POW2(0, 6)[: lens["unroll"]],
        "vec": POW2(0, 3)[: lens["vec"]],
        "stages": list(range(1, lens["stages"] + 1)),
        "pad": [0, 1][: lens["pad"]],
        "splitk": list(range(1, lens["splitk"] + 1)),
        "ro": list(range(0, lens["ro"])),
    }
    names = ["bx", "by", "tx", "ty", "unroll", "vec", "stages", "pad", "splitk", "ro"]
    return _space(f"batched_{s}", [(n, vals[n]) for n in names], medium_space().constraints)


# medium constraints in the order they are dropped to raise the density (the first is implied
# by the others: bx >= 16 is a power of two and tx*vec <= 8 divides it)
_DENSITY_DROP = ["bx%(tx*vec)==0", "64<=bx*by<=1024", "by*ty<=16", "ro==0 or pad==0", "vec*tx<=8",
                 "splitk<=2 or stages>=4", "unroll*vec<=tx*ty", "4*(bx*tx+pad)*(by*ty)*stages<=49152"]


def density_space(j: int) -> SpaceDef:
    """Space ``j`` (0..7) of the density ladder: the medium parameters under fewer and fewer of
    its constraints, so that the density climbs from ~1.5 % (all eight, Hotspot-like) through
    ~2.1, 2.9, 4.4, 6.9, 13 and 29 % to 100 % (none), spanning the densities of Table III."""
    if not 0 <= j <= 7:
        raise ValueError("density ladder index is 0..7")
    sd = medium_space()
    keep = _DENSITY_DROP[j + 1 if j else 0:]
    return _space(f"density_{j}", sd.params, [c for c in sd.constraints if c in keep])


SPACES = {"tiny": tiny_space, "medium": medium_space, "large": large_space,
          "large_a": large_group_a, "large_b": large_group_b, "large_slice": large_slice_space}


# ---------------------------------------------------------------------------------------
# fitness tables (the synthetic stand-in for measured kernel runtimes; lower is better)
# ---------------------------------------------------------------------------------------

def lognormal_table(n_valid: int, seed: int = 0, sigma: float = 1.0) -> np.ndarray:
    """t[rank] = float32(exp(sigma * z)), z standard normal from a Philox-seeded generator."""
    g = np.random.Generator(np.random.Philox(key=seed))
    z = g.standard_normal(n_valid)
    return np.exp(sigma * z).astype(np.float32)


def smooth_table(space: SpaceDef, idx_tuples: np.ndarray, seed: int = 0,
                 noise: float = 0.1) -> np.ndarray:
    """Smooth bowl plus lognormal noise over the valid tuples given in rank order.

    ``idx_tuples`` is an (|V|, n) array of value indices (row = valid configuration, in
    increasing key order).  t = float32((1 + sum_k a_k (u_k - c_k)^2) * exp(noise * z)),
    u_k = idx_k / (r_k - 1), with a_k ~ U[0.5, 2], c_k ~ U[0, 1] per seed.
    """
    idx_tuples = np.asarray(idx_tuples)
    n = len(space.params)
    g = np.random.Generator(np.random.Philox(key=0x5EED0000 + seed))
    a = g.uniform(0.5, 2.0, size=n)
    c = g.uniform(0.0, 1.0, size=n)
    r = np.array(space.n_values, dtype=np.float64)
    den = np.where(r > 1, r - 1, 1.0)
    u = idx_tuples.astype(np.float64) / den
    bowl = 1.0 + ((u - c) ** 2 * a).sum(axis=1)
    z = g.standard_normal(len(idx_tuples))
    return (bowl * np.exp(noise * z)).astype(np.float32)


def smooth_table_device(space: SpaceDef, idx_tuples, seed: int = 0, noise: float = 0.1, generator=None):
    """Device form of smooth_table for spaces too large for host memory: the same bowl (a_k,
    c_k drawn exactly as smooth_table draws them) over a torch int32 tensor of value indices
    [n, N] on the device, times exp(noise * z) with z standard normal from ``generator`` (a
    torch.Generator on that device, consumed in order; so the noise differs from smooth_table's
    numpy draws).  Returns a float32 tensor of n entries."""
    import torch
    n = len(space.params)
    g = np.random.Generator(np.random.Philox(key=0x5EED0000 + seed))
    a = g.uniform(0.5, 2.0, size=n)
    c = g.uniform(0.0, 1.0, size=n)
    r = np.array(space.n_values, dtype=np.float64)
    den = np.where(r > 1, r - 1, 1.0)
    dev = idx_tuples.device
    u = idx_tuples.to(torch.float64) / torch.tensor(den, dtype=torch.float64, device=dev)
    bowl = 1.0 + ((u - torch.tensor(c, dtype=torch.float64, device=dev)) ** 2
                  * torch.tensor(a, dtype=torch.float64, device=dev)).sum(dim=1)
    z = torch.randn(len(idx_tuples), generator=generator, device=dev, dtype=torch.float64)
    return (bowl * torch.exp(noise * z)).to(torch.float32)


def eval_cost_table(table: np.ndarray, seed: int = 0, compile_s: float = 1.5, sigma: float = 0.25,
                    repeats: int = 7) -> np.ndarray:
    """Simulated time, in whole microseconds (uint32), of evaluating each valid configuration:
    a compile time lognormal around ``compile_s`` seconds plus ``repeats`` runs of the kernel,
    reading the fitness table as kernel runtimes in milliseconds."""
    g = np.random.Generator(np.random.Philox(key=0xC0575EED + seed))
    compile_us = 1e6 * compile_s * np.exp(sigma * g.standard_normal(len(table)))
    return np.rint(compile_us + repeats * 1e3 * np.asarray(table, np.float64)).astype(np.uint32)


# ---------------------------------------------------------------------------------------
# candidate tuples for repair workloads (value-index tuples; packing is each side's job)
# ---------------------------------------------------------------------------------------

def uniform_tuples(space: SpaceDef, count: int, seed: int) -> np.ndarray:
    """Uniform random value-index tuples over the Cartesian product (worst case for repair)."""
    g = np.random.Generator(np.random.Philox(key=0xC0FFEE + seed))
    r = np.array(space.n_values, dtype=np.int64)
    return (g.random((count, len(r))) * r).astype(np.int64)


def perturbed_tuples(space: SpaceDef, base: np.ndarray, seed: int, frac: float = 0.6,
                     scale: float = 0.7) -> np.ndarray:
    """DE-like perturbations of valid tuples: each field, with probability ``frac``, moves by
    round(scale * (a - b)) for two random indices a, b of that parameter (clipped)."""
    g = np.random.Generator(np.random.Philox(key=0xDE0000 + seed))
    base = np.asarray(base, dtype=np.int64)
    r = np.array(space.n_values, dtype=np.int64)
    a = (g.random(base.shape) * r).astype(np.int64)
    b = (g.random(base.shape) * r).astype(np.int64)
    move = np.rint(scale * (a - b)).astype(np.int64)
    take = g.random(base.shape) < frac
    out = np.where(take, base + move, base)
    return np.clip(out, 0, r - 1)


def random_ranks(n_valid: int, count: int, seed: int) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=0x4A4E + seed))
    return (g.random(count) * n_valid).astype(np.int64)
