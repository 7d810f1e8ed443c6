"""Python binding of libcatune.so: the C-ABI calls under the same names, argument marshalling only.

Device buffers are torch CUDA tensors (PyTorch supplies device memory and streams); every step
of the hot path runs in the library's kernels.  There is no fallback: importing this module on a
machine without the built library raises.
"""
from __future__ import annotations

import ast
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcatune.so")

CT_OK, CT_ERR_INVALID_ARG, CT_ERR_KEY_OVERFLOW, CT_ERR_EMPTY_SPACE = 0, 1, 2, 3
CT_ERR_OOM, CT_ERR_CUDA, CT_ERR_TIMEOUT, CT_ERR_STATE, CT_ERR_LIMIT = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "KEY_OVERFLOW", 3: "EMPTY_SPACE", 4: "OOM", 5: "CUDA",
                6: "TIMEOUT", 7: "STATE", 8: "LIMIT"}
KINDS = {"de": 0, "pso": 1, "firefly": 2, "ga": 3}

OP = dict(END=0, PARAM=1, CONST=2, ADD=3, SUB=4, MUL=5, DIV=6, MOD=7, NEG=8, MIN=9, MAX=10, LT=11, LE=12,
          GT=13, GE=14, EQ=15, NE=16, AND=17, OR=18, NOT=19)
MAX_PARAMS = 32
REPAIR_NOALLOC_MAX = 16384


class CatuneError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ct_instr(C.Structure):
    _fields_ = [("op", C.c_int32), ("arg", C.c_int32), ("imm", C.c_int64)]


class ct_space_info(C.Structure):
    _fields_ = [("n_params", C.c_int32), ("n_constraints", C.c_int32), ("key_bits", C.c_int32),
                ("n_blocks", C.c_int32), ("width", C.c_int32 * MAX_PARAMS), ("offset", C.c_int32 * MAX_PARAMS),
                ("n_values", C.c_int32 * MAX_PARAMS), ("cartesian", C.c_uint64), ("n_valid", C.c_uint64),
                ("built", C.c_int32)]


class ct_build_stats(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("timed", C.c_int32), ("parents", C.c_uint64 * MAX_PARAMS),
                ("children", C.c_uint64 * MAX_PARAMS), ("count_ms", C.c_float * MAX_PARAMS),
                ("emit_ms", C.c_float * MAX_PARAMS), ("host_setup_ms", C.c_float), ("host_levels_ms", C.c_float),
                ("host_balls_ms", C.c_float), ("host_total_ms", C.c_float), ("hinted", C.c_int32)]


class ct_surrogate_params(C.Structure):
    _fields_ = [("pool", C.c_int32), ("hidden", C.c_int32), ("batch", C.c_int32), ("steps", C.c_int32),
                ("warmup_mult", C.c_int32), ("lr", C.c_float), ("momentum", C.c_float), ("mae_ratio", C.c_float)]


class ct_opt_params(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("de_F", "de_CR", "pso_w", "pso_c1", "pso_c2", "fa_beta0",
                                         "fa_gamma", "fa_alpha", "ga_pmut", "target")] + [("repair_rule", C.c_int32),
                                                                                          ("constraint_aware", C.c_int32),
                                                                                          ("de_mutation", C.c_int32),
                                                                                          ("de_crossover", C.c_int32),
                                                                                          ("ga_crossover", C.c_int32)]
DE_MUTATIONS = ["best1", "rand1", "rand2", "best2", "currenttobest1", "randtobest1"]
DE_CROSSOVERS = ["bin", "exp"]
GA_CROSSOVERS = ["single_point", "two_point", "uniform", "disruptive_uniform"]
_ENUMS = {"de_mutation": DE_MUTATIONS, "de_crossover": DE_CROSSOVERS, "ga_crossover": GA_CROSSOVERS}


_lib = None
_SIGS = {
    "ct_define_space": [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)],
    "ct_space_destroy": [C.c_void_p],
    "ct_space_info_get": [C.c_void_p, C.POINTER(ct_space_info)],
    "ct_pack_keys": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "ct_unpack_keys": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "ct_unpack_keys_device": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "ct_build_valid_space": [C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64)],
    "ct_space_keys": [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint64)],
    "ct_set_fitness": [C.c_void_p, C.c_void_p, C.c_uint64],
    "ct_set_eval_cost": [C.c_void_p, C.c_void_p, C.c_uint64],
    "ct_lookup": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "ct_repair": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_set_repair_mode": [C.c_void_p, C.c_int32, C.c_int32],
    "ct_repair_noalloc": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_repair_paper": [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                        C.c_void_p],
    "ct_evaluate": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_space_status": [C.c_void_p, C.c_void_p],
    "ct_opt_params_default": [C.POINTER(ct_opt_params)],
    "ct_opt_create": [C.c_void_p, C.c_int32, C.POINTER(ct_opt_params), C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)],
    "ct_opt_destroy": [C.c_void_p],
    "ct_propose_population": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p],
    "ct_opt_post_repair": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p],
    "ct_opt_select": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_opt_step": [C.c_void_p, C.c_uint32, C.c_void_p],
    "ct_opt_run_graph": [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p],
    "ct_opt_best": [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_float), C.POINTER(C.c_uint64),
                    C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_void_p],
    "ct_opt_state": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_opt_cost": [C.c_void_p, C.POINTER(C.c_uint64), C.c_void_p],
    "ct_opt_save": [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t), C.c_void_p],
    "ct_opt_load": [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p],
    "ct_batch_create": [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(ct_opt_params), C.POINTER(C.c_void_p)],
    "ct_batch_destroy": [C.c_void_p],
    "ct_batch_step": [C.c_void_p, C.c_void_p],
    "ct_batch_run_graph": [C.c_void_p, C.c_uint32, C.c_void_p],
    "ct_batch_results": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_batch_run_state": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_batch_reset": [C.c_void_p],
    "ct_batch_set_trace": [C.c_void_p, C.c_int32, C.c_int32],
    "ct_batch_events": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_batch_trace": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_batch_set_launch": [C.c_void_p, C.c_int32, C.c_int32],
    "ct_batch_set_gens_per_launch": [C.c_void_p, C.c_int32],
    "ct_batch_autotune": [C.c_void_p, C.c_char_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                          C.POINTER(C.c_float), C.c_void_p],
    "ct_opt_last_generation": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_surrogate_params_default": [C.c_void_p],
    "ct_opt_set_surrogate": [C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_opt_surrogate_info": [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_float),
                              C.POINTER(C.c_float), C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p],
    "ct_mlp_param_count": [C.c_int32, C.c_int32],
    "ct_mlp_init": [C.c_int32, C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p],
    "ct_mlp_workspace_bytes": [C.c_int32, C.c_int32, C.c_int32],
    "ct_mlp_forward": [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                       C.c_void_p],
    "ct_mlp_grad": [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                    C.c_void_p, C.c_void_p, C.c_void_p],
    "ct_mlp_sgd": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_void_p],
    "ct_space_set_timing": [C.c_void_p, C.c_int32],
    "ct_space_build_stats": [C.c_void_p, C.c_void_p],
    "ct_measure_int_peak": [C.POINTER(C.c_double), C.c_void_p],
    "ct_measure_fp32_peak": [C.POINTER(C.c_double), C.c_void_p],
    "ct_measure_smem_peak": [C.POINTER(C.c_double), C.c_void_p],
    "ct_launch_count": [],
    "ct_alloc_count": [],
    "ct_trim_cache": [],
    "ct_last_error": [],
    "ct_version": [],
}


def lib():
    """The loaded C library.  Raises if it has not been built — there is no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcatune.so not built ({LIB_PATH}); run paper_2606_28372_b300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.ct_last_error.restype = C.c_char_p
        L.ct_version.restype = C.c_char_p
        L.ct_space_destroy.restype = None
        L.ct_opt_destroy.restype = None
        L.ct_batch_destroy.restype = None
        L.ct_surrogate_params_default.restype = None
        L.ct_mlp_param_count.restype = C.c_int64
        L.ct_mlp_workspace_bytes.restype = C.c_size_t
        L.ct_opt_params_default.restype = None
        L.ct_launch_count.restype = C.c_uint64
        L.ct_alloc_count.restype = C.c_uint64
        L.ct_trim_cache.restype = None
        _lib = L
    return _lib


def check(status):
    if status != CT_OK:
        raise CatuneError(status, lib().ct_last_error().decode())
    return status


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ------------------------------------------------------------------------------------------
# constraint strings -> postfix programs
# ------------------------------------------------------------------------------------------
class _Postfix:
    BIN = {ast.Add: "ADD", ast.Sub: "SUB", ast.Mult: "MUL", ast.FloorDiv: "DIV", ast.Mod: "MOD"}
    CMP = {ast.Lt: "LT", ast.LtE: "LE", ast.Gt: "GT", ast.GtE: "GE", ast.Eq: "EQ", ast.NotEq: "NE"}

    def __init__(self, names):
        self.idx = {n: i for i, n in enumerate(names)}
        self.code = []

    def emit(self, op, arg=0, imm=0):
        self.code.append((OP[op], arg, imm))

    def gen(self, e):
        if isinstance(e, ast.Constant) and isinstance(e.value, (int, bool)):
            return self.emit("CONST", imm=int(e.value))
        if isinstance(e, ast.Name):
            if e.id not in self.idx:
                raise ValueError(f"unknown parameter {e.id!r}")
            return self.emit("PARAM", arg=self.idx[e.id])
        if isinstance(e, ast.UnaryOp):
            self.gen(e.operand)
            if isinstance(e.op, ast.USub):
                return self.emit("NEG")
            if isinstance(e.op, ast.Not):
                return self.emit("NOT")
            if isinstance(e.op, ast.UAdd):
                return None
        if isinstance(e, ast.BinOp) and type(e.op) in self.BIN:
            self.gen(e.left)
            self.gen(e.right)
            return self.emit(self.BIN[type(e.op)])
        if isinstance(e, ast.BoolOp):
            op = "AND" if isinstance(e.op, ast.And) else "OR"
            self.gen(e.values[0])
            for v in e.values[1:]:
                self.gen(v)
                self.emit(op)
            return None
        if isinstance(e, ast.Compare):
            operands = [e.left] + list(e.comparators)
            for i, op in enumerate(e.ops):
                self.gen(operands[i])
                self.gen(operands[i + 1])
                self.emit(self.CMP[type(op)])
                if i:
                    self.emit("AND")
            return None
        if isinstance(e, ast.Call) and isinstance(e.func, ast.Name) and e.func.id in ("min", "max"):
            self.gen(e.args[0])
            for a in e.args[1:]:
                self.gen(a)
                self.emit("MIN" if e.func.id == "min" else "MAX")
            return None
        raise ValueError(f"unsupported constraint syntax: {ast.dump(e)}")


_COMPILED = {}


def compile_constraints(names, constraints):
    """Constraint strings -> concatenated postfix program (ct_instr array); memoised."""
    key = (tuple(names), tuple(constraints))
    if key in _COMPILED:
        return _COMPILED[key]
    pf = _Postfix(names)
    for c in constraints:
        pf.gen(ast.parse(c, mode="eval").body)
        pf.emit("END")
    arr = (ct_instr * max(1, len(pf.code)))()
    for i, (op, arg, imm) in enumerate(pf.code):
        arr[i].op, arr[i].arg, arr[i].imm = op, arg, imm
    if len(_COMPILED) < 4096:
        _COMPILED[key] = (arr, len(pf.code))
    return arr, len(pf.code)


# ------------------------------------------------------------------------------------------
# handles
# ------------------------------------------------------------------------------------------
class Space:
    """ct_space: a tuning space P = (X, D, C) and, once built, its sorted valid keys."""

    def __init__(self, names, value_lists, constraints):
        L = lib()
        self.names = list(names)
        nv = np.array([len(v) for v in value_lists], dtype=np.int32)
        vals = np.array([int(x) for v in value_lists for x in v], dtype=np.int64)
        prog, n_instr = compile_constraints(names, constraints)
        h = C.c_void_p()
        check(L.ct_define_space(len(nv), nv.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p),
                                C.cast(prog, C.c_void_p), n_instr, C.byref(h)))
        self.h = h
        self._fit = None

    @classmethod
    def from_def(cls, sd):
        return cls(sd.names, sd.values, sd.constraints)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ct_space_destroy(self.h)
            self.h = None

    def info(self):
        inf = ct_space_info()
        check(lib().ct_space_info_get(self.h, C.byref(inf)))
        return inf

    def pack(self, idx):
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, self.info().n_params))
        out = np.zeros(len(idx), dtype=np.uint64)
        check(lib().ct_pack_keys(self.h, idx.ctypes.data_as(C.c_void_p), len(idx), out.ctypes.data_as(C.c_void_p)))
        return out

    def unpack(self, keys):
        keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
        out = np.zeros((len(keys), self.info().n_params), dtype=np.int32)
        check(lib().ct_unpack_keys(self.h, keys.ctypes.data_as(C.c_void_p), len(keys), out.ctypes.data_as(C.c_void_p)))
        return out

    def unpack_device(self, keys, out, stream=None):
        """Value indices of device keys into a device int32 tensor of shape [n, n_params]."""
        check(lib().ct_unpack_keys_device(self.h, _ptr(keys), keys.numel(), _ptr(out), _stream(stream)))

    def build(self, stream=None, allow_empty=False):
        n = C.c_uint64()
        st = lib().ct_build_valid_space(self.h, _stream(stream), C.byref(n))
        if st == CT_ERR_EMPTY_SPACE and allow_empty:
            return 0
        check(st)
        return int(n.value)

    def keys(self):
        """Borrowed view of the device keys as an int64 torch tensor (bit pattern of uint64)."""
        import torch
        p, n = C.c_void_p(), C.c_uint64()
        check(lib().ct_space_keys(self.h, C.byref(p), C.byref(n)))
        n = int(n.value)
        if n == 0:
            return torch.zeros(0, dtype=torch.int64, device="cuda")
        holder = _CudaArray(p.value, n)
        return torch.as_tensor(holder, device="cuda")

    def set_fitness(self, table):
        check(lib().ct_set_fitness(self.h, _ptr(table), table.numel()))
        self._fit = table

    def set_eval_cost(self, cost):
        """Simulated evaluation time per valid rank (device int32 tensor read as uint32 microseconds;
        None removes it)."""
        check(lib().ct_set_eval_cost(self.h, _ptr(cost), 0 if cost is None else cost.numel()))
        self._cost = cost

    def lookup(self, cand, rank, stream=None):
        check(lib().ct_lookup(self.h, _ptr(cand), cand.numel(), _ptr(rank), _stream(stream)))

    def repair(self, cand, out, dist=None, stream=None):
        check(lib().ct_repair(self.h, _ptr(cand), cand.numel(), _ptr(out), _ptr(dist), _stream(stream)))

    def repair_noalloc(self, cand, out, dist=None, stream=None):
        """ct_repair without device allocations (fixed in-library scratch; at most
        REPAIR_NOALLOC_MAX candidates per call; calls must not overlap on the GPU)."""
        check(lib().ct_repair_noalloc(self.h, _ptr(cand), cand.numel(), _ptr(out), _ptr(dist), _stream(stream)))

    def repair_paper(self, rule, cand, out, pos=None, eps=0.0, words=None, stream=None):
        """The paper's repair rules: 1 index distance (DE), 2 Algorithm 2 (PSO/Firefly), 3 Algorithm 3 (GA)."""
        check(lib().ct_repair_paper(self.h, rule, _ptr(cand), cand.numel(), _ptr(pos), C.c_float(eps), _ptr(words),
                                    _ptr(out), _stream(stream)))

    def set_repair_mode(self, mode, max_radius=0):
        check(lib().ct_set_repair_mode(self.h, mode, max_radius))

    def evaluate(self, keys, fit, rank=None, opt=None, stream=None):
        check(lib().ct_evaluate(self.h, opt.h if opt is not None else None, _ptr(keys), keys.numel(), _ptr(fit),
                                _ptr(rank), _stream(stream)))

    def status(self, stream=None):
        return lib().ct_space_status(self.h, _stream(stream))

    def set_timing(self, enable=True):
        check(lib().ct_space_set_timing(self.h, 1 if enable else 0))

    def build_stats(self):
        st = ct_build_stats()
        check(lib().ct_space_build_stats(self.h, C.byref(st)))
        n = st.n_levels
        return dict(levels=n, timed=bool(st.timed), parents=list(st.parents[:n]), children=list(st.children[:n]),
                    count_ms=list(st.count_ms[:n]), emit_ms=list(st.emit_ms[:n]),
                    host_ms=dict(setup=st.host_setup_ms, levels=st.host_levels_ms, balls=st.host_balls_ms,
                                 total=st.host_total_ms), hinted=bool(st.hinted))


def launch_count():
    return int(lib().ct_launch_count())


def alloc_count():
    """Device blocks the library has taken so far (from its cache or the driver)."""
    return int(lib().ct_alloc_count())


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for a borrowed device pointer."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False), "version": 3}


def measure_int_peak(stream=None):
    """Population counts per second of the library's integer microbenchmark (32-bit xor/popc/add
    chains, bound by the population-count pipe like the key scans)."""
    v = C.c_double()
    check(lib().ct_measure_int_peak(C.byref(v), _stream(stream)))
    return float(v.value)


def measure_fp32_peak(stream=None):
    """fp32 operations per second of the library's fused multiply-add microbenchmark (the
    denominator of the surrogate's CUDA-core products)."""
    v = C.c_double()
    check(lib().ct_measure_fp32_peak(C.byref(v), _stream(stream)))
    return float(v.value)


def measure_smem_peak(stream=None):
    """Shared-memory wavefronts per second of the library's 16-byte shared-load microbenchmark
    (the denominator of the distance-table scan)."""
    v = C.c_double()
    check(lib().ct_measure_smem_peak(C.byref(v), _stream(stream)))
    return float(v.value)


def default_params(**over):
    p = ct_opt_params()
    lib().ct_opt_params_default(C.byref(p))
    for k, v in over.items():
        if k in _ENUMS:
            setattr(p, k, _ENUMS[k].index(v) if isinstance(v, str) else int(v))
        else:
            setattr(p, k, int(v) if k in ("repair_rule", "constraint_aware") else float(np.float32(v)))
    return p


class Opt:
    """ct_opt: one optimizer run on a built space with a fitness table.

    params: any field of ct_opt_params (F, CR, ..., repair_rule, constraint_aware, and the
    operators by name: de_mutation in DE_MUTATIONS, de_crossover in DE_CROSSOVERS, ga_crossover
    in GA_CROSSOVERS)."""

    def __init__(self, space, kind, pop, seed, **params):
        self.space = space
        self.pop = pop
        self.kind = kind
        self.params = default_params(**params)
        h = C.c_void_p()
        check(lib().ct_opt_create(space.h, KINDS[kind], C.byref(self.params), pop, seed, C.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ct_opt_destroy(self.h)
            self.h = None

    def propose(self, gen, cand, stream=None):
        check(lib().ct_propose_population(self.h, gen, _ptr(cand), _stream(stream)))

    def post_repair(self, gen, keys, stream=None):
        check(lib().ct_opt_post_repair(self.h, gen, _ptr(keys), _stream(stream)))

    def select(self, gen, keys, fit, stream=None):
        check(lib().ct_opt_select(self.h, gen, _ptr(keys), _ptr(fit), _stream(stream)))

    def step(self, gen, stream=None):
        check(lib().ct_opt_step(self.h, gen, _stream(stream)))

    def run_graph(self, first, count, stream=None):
        check(lib().ct_opt_run_graph(self.h, first, count, _stream(stream)))

    def best(self, stream=None):
        k, f, u = C.c_uint64(), C.c_float(), C.c_uint64()
        hg, he = C.c_int64(), C.c_int64()
        check(lib().ct_opt_best(self.h, C.byref(k), C.byref(f), C.byref(u), C.byref(hg), C.byref(he), _stream(stream)))
        return dict(best_key=int(k.value), best_fit=float(f.value), n_unique=int(u.value), hit_gen=int(hg.value),
                    hit_evals=int(he.value))

    def cost(self, stream=None):
        c = C.c_uint64()
        check(lib().ct_opt_cost(self.h, C.byref(c), _stream(stream)))
        return int(c.value)

    def set_surrogate(self, log_table, **cfg):
        """Screen DE/GA proposals with the MLP surrogate (before generation 0)."""
        p = ct_surrogate_params()
        lib().ct_surrogate_params_default(C.byref(p))
        for k, v in cfg.items():
            setattr(p, k, v)
        self._logt = log_table
        check(lib().ct_opt_set_surrogate(self.h, C.byref(p), _ptr(log_table)))

    def surrogate_info(self, params=None, stream=None):
        sc, un, mae, tau, ne = C.c_int32(), C.c_int32(), C.c_float(), C.c_float(), C.c_uint64()
        check(lib().ct_opt_surrogate_info(self.h, C.byref(sc), C.byref(un), C.byref(mae), C.byref(tau), C.byref(ne),
                                          _ptr(params), _stream(stream)))
        return dict(screened=sc.value, use_next=un.value, mae=mae.value, tau=tau.value, n_e=int(ne.value))

    def last_generation(self, cand=None, rep=None, evk=None, fit=None, stream=None):
        check(lib().ct_opt_last_generation(self.h, _ptr(cand), _ptr(rep), _ptr(evk), _ptr(fit), _stream(stream)))

    def state(self, keys=None, fit=None, pos=None, stream=None):
        check(lib().ct_opt_state(self.h, _ptr(keys), _ptr(fit), _ptr(pos), _stream(stream)))

    def save(self, stream=None):
        n = C.c_size_t()
        check(lib().ct_opt_save(self.h, None, C.byref(n), _stream(stream)))
        buf = (C.c_char * n.value)()
        check(lib().ct_opt_save(self.h, C.cast(buf, C.c_void_p), C.byref(n), _stream(stream)))
        return bytes(buf)

    def load(self, blob, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        check(lib().ct_opt_load(self.h, C.cast(buf, C.c_void_p), len(blob), _stream(stream)))


class ct_batch_run(C.Structure):
    _fields_ = [("space", C.c_int32), ("kind", C.c_int32), ("pop", C.c_int32), ("pad", C.c_int32),
                ("seed", C.c_uint64), ("target", C.c_float), ("pad2", C.c_int32)]


class Batch:
    """ct_batch: many independent runs over several spaces, one persistent launch per generation.

    runs: list of (space_index, kind, pop, seed, target); params: shared ct_opt_params fields as
    for Opt (repair_rule must stay 0)."""

    def __init__(self, spaces, runs, **params):
        self.spaces = list(spaces)
        self.n = len(runs)
        arr = (ct_batch_run * self.n)()
        for i, (si, kind, pop, seed, target) in enumerate(runs):
            arr[i].space, arr[i].kind, arr[i].pop, arr[i].seed = si, KINDS[kind], pop, seed
            arr[i].target = float(np.float32(target))
        hs = (C.c_void_p * len(self.spaces))(*[s.h.value for s in self.spaces])
        self.params = default_params(**params)
        h = C.c_void_p()
        check(lib().ct_batch_create(C.cast(hs, C.c_void_p), len(self.spaces), C.cast(arr, C.c_void_p), self.n,
                                    C.byref(self.params), C.byref(h)))
        self.h = h
        self.runs = runs

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ct_batch_destroy(self.h)
            self.h = None

    def step(self, stream=None):
        check(lib().ct_batch_step(self.h, _stream(stream)))

    def run_graph(self, count, stream=None):
        check(lib().ct_batch_run_graph(self.h, count, _stream(stream)))

    def reset(self):
        check(lib().ct_batch_reset(self.h))

    def set_gens_per_launch(self, gens):
        check(lib().ct_batch_set_gens_per_launch(self.h, gens))

    def set_launch(self, threads, ctas_per_sm):
        check(lib().ct_batch_set_launch(self.h, threads, ctas_per_sm))

    def autotune(self, cache_path=None, gens=5, stream=None):
        t, c, ms = C.c_int32(), C.c_int32(), C.c_float()
        check(lib().ct_batch_autotune(self.h, cache_path.encode() if cache_path else None, gens, C.byref(t),
                                      C.byref(c), C.byref(ms), _stream(stream)))
        return int(t.value), int(c.value), float(ms.value)

    def results(self, stream=None):
        bk = np.zeros(self.n, np.uint64)
        bf = np.zeros(self.n, np.float32)
        nu = np.zeros(self.n, np.uint64)
        hg = np.zeros(self.n, np.int64)
        he = np.zeros(self.n, np.int64)
        check(lib().ct_batch_results(self.h, *[a.ctypes.data_as(C.c_void_p) for a in (bk, bf, nu, hg, he)],
                                     _stream(stream)))
        return dict(best_key=bk, best_fit=bf, n_unique=nu, hit_gen=hg, hit_evals=he)

    def run_state(self, run, keys=None, fit=None, pos=None, stream=None):
        check(lib().ct_batch_run_state(self.h, run, _ptr(keys), _ptr(fit), _ptr(pos), _stream(stream)))

    def set_trace(self, gens, events=0):
        check(lib().ct_batch_set_trace(self.h, gens, events))
        self.trace_gens = gens
        self.event_cap = events

    def events(self, stream=None):
        """Per run, the improvements of its best in evaluation order: (generation, index,
        simulated time, best) arrays; raises if a run overflowed the capacity."""
        cap = self.event_cap
        cnt = np.zeros(self.n, np.uint32)
        gen = np.zeros((self.n, cap), np.int32)
        idx = np.zeros((self.n, cap), np.int32)
        clk = np.zeros((self.n, cap), np.uint64)
        fit = np.zeros((self.n, cap), np.float32)
        check(lib().ct_batch_events(self.h, *[a.ctypes.data_as(C.c_void_p) for a in (cnt, gen, idx, clk, fit)],
                                    _stream(stream)))
        if (cnt > cap).any():
            raise CatuneError(CT_ERR_LIMIT, f"event log overflow: {int(cnt.max())} events, capacity {cap}")
        return [(gen[r, :c], idx[r, :c], clk[r, :c], fit[r, :c]) for r, c in enumerate(cnt)]

    def trace(self, stream=None):
        """Per-run, per-generation best fitness, simulated time and unique evaluations
        (arrays of shape [runs, gens])."""
        g = self.trace_gens
        bf = np.zeros((self.n, g), np.float32)
        co = np.zeros((self.n, g), np.uint64)
        nu = np.zeros((self.n, g), np.uint64)
        check(lib().ct_batch_trace(self.h, *[a.ctypes.data_as(C.c_void_p) for a in (bf, co, nu)], _stream(stream)))
        return dict(best_fit=bf, cost=co, n_unique=nu)


def u64(t):
    """View an int64 torch tensor holding uint64 bit patterns as a numpy uint64 array (host copy)."""
    return t.cpu().numpy().view(np.uint64)
