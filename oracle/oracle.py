"""CPU oracle — TEST INFRASTRUCTURE ONLY (tests, the smoke check, the benchmark's CPU leg).

Thin ctypes front-end over ``oracle.c``: parses constraint strings into the oracle's own
expression trees and calls the plain C implementation.  Nothing here is shared with, or
imported by, the CUDA library.

Follows: Section IV-A (CSP P=(X,D,C), full resolution of the valid space, validity
query, neighbour rules), Algorithm 1 and Section IV-B (DE), Section IV-C (PSO, Firefly),
Section IV-D and Algorithm 3 (GA), Table IV (hyper-parameters).  Repair uses the Hamming
metric on value indices with ties to the smallest key (the hot path's repair rule).
"""
from __future__ import annotations

import ast
import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

N_CONST, N_PARAM, N_ADD, N_SUB, N_MUL, N_DIV, N_MOD, N_NEG, N_MIN, N_MAX = range(10)
N_LT, N_LE, N_GT, N_GE, N_EQ, N_NE, N_AND, N_OR, N_NOT = range(10, 19)
KIND = {"de": 0, "pso": 1, "firefly": 2, "ga": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE binary32 semantics (no contraction, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Node(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("pad", C.c_int32),
                ("imm", C.c_int64)]


class _Params(C.Structure):
    _fields_ = [("de_F", C.c_float), ("de_CR", C.c_float), ("pso_w", C.c_float),
                ("pso_c1", C.c_float), ("pso_c2", C.c_float), ("fa_beta0", C.c_float),
                ("fa_gamma", C.c_float), ("fa_alpha", C.c_float), ("ga_pmut", C.c_float),
                ("target", C.c_float), ("repair_rule", C.c_int), ("constraint_aware", C.c_int),
                ("de_mutation", C.c_int), ("de_crossover", C.c_int), ("ga_crossover", C.c_int),
                ("cost", C.c_void_p)]


class _Surr(C.Structure):
    _fields_ = [("pool", C.c_int), ("H", C.c_int), ("batch", C.c_int), ("steps", C.c_int), ("warm_mult", C.c_int),
                ("lr", C.c_float), ("mu", C.c_float), ("mae_ratio", C.c_float), ("logt", C.c_void_p)]


class _STrace(C.Structure):
    _fields_ = [("used", C.c_void_p), ("mae", C.c_void_p), ("tau", C.c_void_p), ("n_e", C.c_void_p),
                ("params", C.c_void_p)]


class _Trace(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("cand", "rep", "evalk", "fit", "popk", "popf", "pos", "best_key", "best_fit",
                 "n_unique", "hit", "cost", "ev_gen", "ev_idx", "ev_clock", "ev_fit", "ev_n")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        p = C.c_void_p
        L.or_key_layout.restype = C.c_int
        L.or_enumerate.restype = C.c_int64
        L.or_enumerate.argtypes = [C.c_int, p, p, p, p, p, C.c_int, C.c_int64, C.c_int64, p, C.c_int64]
        L.or_check_tuples.argtypes = [C.c_int, p, p, p, p, p, C.c_int, p, C.c_int64, p]
        L.or_lookup.argtypes = [p, C.c_int64, p, C.c_int64, p]
        L.or_repair.restype = C.c_int
        L.or_repair.argtypes = [C.c_int, p, p, C.c_int64, p, C.c_int64, p, p]
        L.or_philox4x32_10.argtypes = [p, p, p]
        L.or_rng_word.restype = C.c_uint32
        L.or_rng_word.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_exp_ct.restype = C.c_float
        L.or_exp_ct.argtypes = [C.c_float]
        L.or_beta_pick.restype = C.c_uint32
        L.or_beta_pick.argtypes = [C.c_uint32, C.c_uint32]
        L.or_u01.restype = C.c_float
        L.or_u01.argtypes = [C.c_uint32]
        L.or_run.restype = C.c_int
        L.or_run.argtypes = [C.c_int, C.c_int, p, p, C.c_int64, p, C.c_int, C.c_int, C.c_uint64,
                             C.POINTER(_Params), C.POINTER(_Trace), C.c_void_p, C.c_void_p]
        L.or_mlp_param_count.restype = C.c_int64
        L.or_mlp_param_count.argtypes = [C.c_int, C.c_int]
        L.or_mlp_init.argtypes = [C.c_int, C.c_int, C.c_uint64, p]
        L.or_mlp_forward.argtypes = [p, C.c_int, C.c_int, C.c_int, p, C.c_int, p, p]
        L.or_mlp_grad.argtypes = [p, C.c_int, C.c_int, C.c_int, p, p, C.c_int, p]
        L.or_mlp_sgd.argtypes = [p, p, p, C.c_int64, C.c_float, C.c_float]
        L.or_mlp_loss64.restype = C.c_double
        L.or_mlp_loss64.argtypes = [p, C.c_int, C.c_int, C.c_int, p, p, C.c_int, p]
        L.or_repair_paper.argtypes = [C.c_int, C.c_int, p, p, C.c_int64, p, C.c_int64, p, C.c_float, p, p]
        L.or_bf16_round.restype = C.c_float
        L.or_bf16_round.argtypes = [C.c_float]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------------------------
# constraint strings -> expression trees (the oracle's own parser)
# ------------------------------------------------------------------------------------
class _TreeBuilder:
    BIN = {ast.Add: N_ADD, ast.Sub: N_SUB, ast.Mult: N_MUL, ast.FloorDiv: N_DIV, ast.Mod: N_MOD}
    CMP = {ast.Lt: N_LT, ast.LtE: N_LE, ast.Gt: N_GT, ast.GtE: N_GE, ast.Eq: N_EQ, ast.NotEq: N_NE}

    def __init__(self, names):
        self.names = {n: i for i, n in enumerate(names)}
        self.nodes = []

    def add(self, op, a=-1, b=-1, imm=0):
        self.nodes.append((op, a, b, imm))
        return len(self.nodes) - 1

    def visit(self, e):
        if isinstance(e, ast.Constant) and isinstance(e.value, (int, bool)):
            return self.add(N_CONST, imm=int(e.value))
        if isinstance(e, ast.Name):
            if e.id not in self.names:
                raise ValueError(f"unknown parameter {e.id!r}")
            return self.add(N_PARAM, a=self.names[e.id])
        if isinstance(e, ast.UnaryOp):
            x = self.visit(e.operand)
            if isinstance(e.op, ast.USub):
                return self.add(N_NEG, a=x)
            if isinstance(e.op, ast.UAdd):
                return x
            if isinstance(e.op, ast.Not):
                return self.add(N_NOT, a=x)
        if isinstance(e, ast.BinOp) and type(e.op) in self.BIN:
            return self.add(self.BIN[type(e.op)], self.visit(e.left), self.visit(e.right))
        if isinstance(e, ast.BoolOp):
            op = N_AND if isinstance(e.op, ast.And) else N_OR
            acc = self.visit(e.values[0])
            for v in e.values[1:]:
                acc = self.add(op, acc, self.visit(v))
            return acc
        if isinstance(e, ast.Compare):
            left = self.visit(e.left)
            acc = None
            for op, comp in zip(e.ops, e.comparators):
                right = self.visit(comp)
                c = self.add(self.CMP[type(op)], left, right)
                acc = c if acc is None else self.add(N_AND, acc, c)
                left = right
            return acc
        if isinstance(e, ast.Call) and isinstance(e.func, ast.Name) and e.func.id in ("min", "max"):
            op = N_MIN if e.func.id == "min" else N_MAX
            acc = self.visit(e.args[0])
            for a in e.args[1:]:
                acc = self.add(op, acc, self.visit(a))
            return acc
        raise ValueError(f"unsupported constraint syntax: {ast.dump(e)}")


@dataclass
class OracleSpace:
    n: int
    r: np.ndarray
    values: np.ndarray
    vstart: np.ndarray
    nodes: np.ndarray
    roots: np.ndarray
    m: int
    cartesian: int


def make_space(names, value_lists, constraints) -> OracleSpace:
    tb = _TreeBuilder(names)
    roots = [tb.visit(ast.parse(c, mode="eval").body) for c in constraints]
    nodes = (_Node * max(1, len(tb.nodes)))()
    for i, (op, a, b, imm) in enumerate(tb.nodes):
        nodes[i].op, nodes[i].a, nodes[i].b, nodes[i].imm = op, a, b, imm
    arr = np.frombuffer(bytes(nodes), dtype=np.uint8).copy()
    r = np.array([len(v) for v in value_lists], dtype=np.int32)
    vstart = np.concatenate([[0], np.cumsum(r)[:-1]]).astype(np.int32)
    values = np.array([x for v in value_lists for x in v], dtype=np.int64)
    cart = 1
    for x in r:
        cart *= int(x)
    return OracleSpace(len(r), r, values, vstart, arr, np.array(roots, dtype=np.int32),
                       len(roots), cart)


def from_def(sd) -> OracleSpace:
    return make_space(sd.names, sd.values, sd.constraints)


def key_layout(sp: OracleSpace):
    w = np.zeros(sp.n, np.int32)
    o = np.zeros(sp.n, np.int32)
    bits = lib().or_key_layout(C.c_int(sp.n), _ptr(sp.r), _ptr(w), _ptr(o))
    return w, o, bits


def pack(sp: OracleSpace, tuples) -> np.ndarray:
    w, o, _ = key_layout(sp)
    t = np.asarray(tuples, dtype=np.uint64).reshape(-1, sp.n)
    return (t << o.astype(np.uint64)).sum(axis=1, dtype=np.uint64) if sp.n else np.zeros(len(t), np.uint64)


def unpack(sp: OracleSpace, keys) -> np.ndarray:
    w, o, _ = key_layout(sp)
    k = np.asarray(keys, dtype=np.uint64).reshape(-1, 1)
    mask = ((np.uint64(1) << w.astype(np.uint64)) - np.uint64(1)).astype(np.uint64)
    return ((k >> o.astype(np.uint64)) & mask).astype(np.int64)


def enumerate_range(sp: OracleSpace, c_lo: int = 0, c_hi: int | None = None, count_only=False):
    """Valid keys of Cartesian indices [c_lo, c_hi) in order (brute force)."""
    c_hi = sp.cartesian if c_hi is None else c_hi
    L = lib()
    args = (C.c_int(sp.n), _ptr(sp.r), _ptr(sp.values), _ptr(sp.vstart), _ptr(sp.nodes),
            _ptr(sp.roots), C.c_int(sp.m), C.c_int64(c_lo), C.c_int64(c_hi))
    if count_only:
        return int(L.or_enumerate(*args, None, C.c_int64(0)))
    cnt = int(L.or_enumerate(*args, None, C.c_int64(0)))
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    got = int(L.or_enumerate(*args, _ptr(out), C.c_int64(cnt)))
    assert got == cnt
    return out[:cnt]


def valid_keys(sp: OracleSpace) -> np.ndarray:
    return enumerate_range(sp)


def check_tuples(sp: OracleSpace, tuples) -> np.ndarray:
    t = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32).reshape(-1, sp.n))
    out = np.zeros(len(t), dtype=np.uint8)
    lib().or_check_tuples(C.c_int(sp.n), _ptr(sp.r), _ptr(sp.values), _ptr(sp.vstart),
                          _ptr(sp.nodes), _ptr(sp.roots), C.c_int(sp.m), _ptr(t),
                          C.c_int64(len(t)), _ptr(out))
    return out.astype(bool)


def lookup(keys: np.ndarray, cand) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cand = np.ascontiguousarray(cand, dtype=np.uint64)
    out = np.zeros(len(cand), dtype=np.int64)
    lib().or_lookup(_ptr(keys), C.c_int64(len(keys)), _ptr(cand), C.c_int64(len(cand)), _ptr(out))
    return out


def repair(sp: OracleSpace, keys: np.ndarray, cand):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cand = np.ascontiguousarray(cand, dtype=np.uint64)
    out = np.zeros(len(cand), dtype=np.uint64)
    dist = np.zeros(len(cand), dtype=np.uint8)
    rc = lib().or_repair(C.c_int(sp.n), _ptr(sp.r), _ptr(keys), C.c_int64(len(keys)), _ptr(cand),
                         C.c_int64(len(cand)), _ptr(out), _ptr(dist))
    if rc == -1:
        raise ValueError("candidate outside the Cartesian domain")
    if rc == -2:
        raise ValueError("empty valid space")
    return out, dist


def repair_paper(rule, sp: OracleSpace, keys, cand, pos=None, eps=0.0, words=None):
    """The paper's repairs: 1 = index distance (DE), 2 = Algorithm 2 (PSO/Firefly, positions
    pos), 3 = Algorithm 3 (GA, one RNG word per candidate)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cand = np.ascontiguousarray(cand, dtype=np.uint64)
    out = np.zeros(len(cand), np.uint64)
    pos = np.ascontiguousarray(pos if pos is not None else np.zeros((len(cand), sp.n)), dtype=np.float32)
    words = np.ascontiguousarray(words if words is not None else np.zeros(len(cand)), dtype=np.uint32)
    lib().or_repair_paper(rule, sp.n, _ptr(sp.r), _ptr(keys), C.c_int64(len(keys)), _ptr(cand),
                          C.c_int64(len(cand)), _ptr(pos), C.c_float(eps), _ptr(words), _ptr(out))
    return out


def philox(ctr, key):
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def rng_word(seed, indiv, gen, purpose, t):
    return int(lib().or_rng_word(seed, indiv, gen, purpose, t))


def exp_ct(x: float) -> float:
    return float(lib().or_exp_ct(C.c_float(x)))


def beta_pick(w: int, P: int) -> int:
    return int(lib().or_beta_pick(w, P))


DEFAULTS = dict(de_F=0.7, de_CR=0.6, pso_w=0.5, pso_c1=3.0, pso_c2=0.5, fa_beta0=1.0, fa_gamma=1.0,
                fa_alpha=0.2, ga_pmut=0.2, target=-np.inf, repair_rule=0, constraint_aware=1,
                de_mutation="best1", de_crossover="bin", ga_crossover="single_point")
DE_MUTATIONS = ["best1", "rand1", "rand2", "best2", "currenttobest1", "randtobest1"]
DE_CROSSOVERS = ["bin", "exp"]
GA_CROSSOVERS = ["single_point", "two_point", "uniform", "disruptive_uniform"]
_ENUMS = {"de_mutation": DE_MUTATIONS, "de_crossover": DE_CROSSOVERS, "ga_crossover": GA_CROSSOVERS}


SURROGATE_DEFAULTS = dict(pool=16, H=256, batch=256, steps=8, warm_mult=4, lr=1e-2, mu=0.9, mae_ratio=1.0)


def run(kind: str, sp: OracleSpace, keys: np.ndarray, table: np.ndarray, pop: int, gens: int,
        seed: int, surrogate=None, log_table=None, cost=None, **params):
    """One optimizer run: generation 0 (initial sample) plus ``gens`` generations.

    With ``surrogate`` (a dict overriding SURROGATE_DEFAULTS) and ``log_table`` (log-fitness per
    valid rank), DE and GA proposals are screened by the MLP surrogate.  Returns a dict of
    per-generation arrays (rows = generations 0..gens)."""
    prm = dict(DEFAULTS)
    prm.update(params)
    P, G, n = pop, gens, sp.n
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    table = np.ascontiguousarray(table, dtype=np.float32)
    T = {
        "cand": np.zeros((G + 1, P), np.uint64), "rep": np.zeros((G + 1, P), np.uint64),
        "evalk": np.zeros((G + 1, P), np.uint64), "fit": np.zeros((G + 1, P), np.float32),
        "popk": np.zeros((G + 1, P), np.uint64), "popf": np.zeros((G + 1, P), np.float32),
        "pos": np.zeros((G + 1, P, n), np.float32), "best_key": np.zeros(G + 1, np.uint64),
        "best_fit": np.zeros(G + 1, np.float32), "n_unique": np.zeros(G + 1, np.uint64),
        "hit": np.zeros(2, np.int64), "cost": np.zeros(G + 1, np.uint64),
        "ev_gen": np.zeros(P * (G + 1), np.int32), "ev_idx": np.zeros(P * (G + 1), np.int32),
        "ev_clock": np.zeros(P * (G + 1), np.uint64), "ev_fit": np.zeros(P * (G + 1), np.float32),
        "ev_n": np.zeros(1, np.int64),
    }
    tr = _Trace(*[T[f].ctypes.data for f, _ in _Trace._fields_])
    cost_arr = None if cost is None else np.ascontiguousarray(cost, dtype=np.uint32)
    if cost_arr is not None:
        assert len(cost_arr) == len(keys)
    vals = {}
    for f, _ in _Params._fields_:
        if f == "cost":
            vals[f] = None if cost_arr is None else cost_arr.ctypes.data
        elif f in _ENUMS:
            v = prm[f]
            vals[f] = _ENUMS[f].index(v) if isinstance(v, str) else int(v)
        elif f in ("repair_rule", "constraint_aware"):
            vals[f] = int(prm[f])
        else:
            vals[f] = float(np.float32(prm[f]))
    pr = _Params(**vals)
    sg = st = None
    if surrogate is not None:
        cfg = dict(SURROGATE_DEFAULTS)
        cfg.update(surrogate)
        logt = np.ascontiguousarray(log_table, dtype=np.float32)
        D = int(sp.r.sum())
        T["logt_ref"] = logt
        T["s_used"] = np.zeros(G + 1, np.int8)
        T["s_mae"] = np.zeros(G + 1, np.float32)
        T["s_tau"] = np.zeros(G + 1, np.float32)
        T["s_ne"] = np.zeros(G + 1, np.int64)
        T["s_params"] = np.zeros(int(lib().or_mlp_param_count(D, cfg["H"])), np.float32)
        sg = _Surr(cfg["pool"], cfg["H"], cfg["batch"], cfg["steps"], cfg["warm_mult"], float(np.float32(cfg["lr"])),
                   float(np.float32(cfg["mu"])), float(np.float32(cfg["mae_ratio"])), logt.ctypes.data)
        st = _STrace(T["s_used"].ctypes.data, T["s_mae"].ctypes.data, T["s_tau"].ctypes.data, T["s_ne"].ctypes.data,
                     T["s_params"].ctypes.data)
    rc = lib().or_run(KIND[kind], n, _ptr(sp.r), _ptr(keys), C.c_int64(len(keys)), _ptr(table),
                      P, G, C.c_uint64(seed), C.byref(pr), C.byref(tr),
                      C.cast(C.byref(sg), C.c_void_p) if sg else None, C.cast(C.byref(st), C.c_void_p) if st else None)
    if rc != 0:
        raise ValueError(f"oracle run rejected its arguments (code {rc})")
    T.pop("logt_ref", None)
    ne = int(T.pop("ev_n")[0])
    for f in ("ev_gen", "ev_idx", "ev_clock", "ev_fit"):
        T[f] = T[f][:ne]
    return T


# ------------------------------------------------------------------------------------
# MLP surrogate pieces
# ------------------------------------------------------------------------------------
def mlp_param_count(D, H):
    return int(lib().or_mlp_param_count(D, H))


def mlp_init(D, H, seed):
    p = np.zeros(mlp_param_count(D, H), np.float32)
    lib().or_mlp_init(D, H, C.c_uint64(seed), _ptr(p))
    return p


def mlp_forward(params, D, H, feats):
    feats = np.ascontiguousarray(feats, dtype=np.int32)
    B, N = feats.shape
    out = np.zeros(B, np.float32)
    lib().or_mlp_forward(_ptr(np.ascontiguousarray(params, np.float32)), D, H, N, _ptr(feats), B, _ptr(out), None)
    return out


def mlp_grad(params, D, H, feats, y):
    feats = np.ascontiguousarray(feats, dtype=np.int32)
    B, N = feats.shape
    g = np.zeros(mlp_param_count(D, H), np.float32)
    lib().or_mlp_grad(_ptr(np.ascontiguousarray(params, np.float32)), D, H, N, _ptr(feats),
                      _ptr(np.ascontiguousarray(y, np.float32)), B, _ptr(g))
    return g


def mlp_sgd(params, mom, grad, lr=1e-3, mu=0.9):
    lib().or_mlp_sgd(_ptr(params), _ptr(mom), _ptr(np.ascontiguousarray(grad, np.float32)), C.c_int64(len(params)),
                     C.c_float(lr), C.c_float(mu))


def mlp_loss64(params, D, H, feats, y, want_grad=True):
    feats = np.ascontiguousarray(feats, dtype=np.int32)
    B, N = feats.shape
    p = np.ascontiguousarray(params, np.float64)
    g = np.zeros(len(p), np.float64) if want_grad else None
    loss = lib().or_mlp_loss64(_ptr(p), D, H, N, _ptr(feats), _ptr(np.ascontiguousarray(y, np.float64)), B,
                               _ptr(g) if g is not None else None)
    return loss, g


def bf16_round(x):
    return float(lib().or_bf16_round(C.c_float(x)))


def features(sp: OracleSpace, keys):
    """One-hot feature indices (ascending) of keys: base_k + idx_k."""
    idx = unpack(sp, keys)
    base = np.concatenate([[0], np.cumsum(sp.r)[:-1]]).astype(np.int64)
    return (idx + base).astype(np.int32)
