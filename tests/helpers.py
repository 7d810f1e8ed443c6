"""Shared test helpers: build both sides from the same seeded inputs."""
import numpy as np

from paper_2606_28372_b300 import workloads as W


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def to_dev_u64(arr):
    import torch
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint64))
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def from_dev_u64(t):
    return t.cpu().numpy().view(np.uint64)


class Pair:
    """A space built on the GPU and in the oracle from one definition."""

    def __init__(self, sd, O, table="auto", seed=0):
        import torch
        from paper_2606_28372_b300 import catune as ct
        self.sd = sd
        self.O = O
        self.osp = O.from_def(sd)
        self.okeys = O.valid_keys(self.osp)
        self.sp = ct.Space.from_def(sd)
        self.nv = self.sp.build(allow_empty=True)
        self.table = None
        if table is not None and len(self.okeys):
            if table == "auto":
                table = "lognormal" if sd.name == "tiny" else "smooth"
            if table == "lognormal":
                t = W.lognormal_table(len(self.okeys), seed=seed)
            else:
                t = W.smooth_table(sd, O.unpack(self.osp, self.okeys), seed=seed)
            self.table = t
            self.dtable = torch.from_numpy(t).cuda()
            self.sp.set_fitness(self.dtable)

    def gkeys(self):
        return from_dev_u64(self.sp.keys())
