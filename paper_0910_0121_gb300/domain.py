"""Several processes on one periodic box: the paper's parallel step (Sec. 2.2 steps 3-5 and
7; Sec. 2.3.1) around the library's single-process calls.

Each process owns the particles of one domain box, and one step of the short-range force
runs as the paper describes it:

1. Decomposition (Sec. 2.3.1).  Every process samples n_samp particles (Eq. 3-5,
   greem_sample_count: its share of the measured force time, with the lower limit of
   Eq. 5) and takes their finest cells (greem_cell_index); the samples of all processes
   are gathered, and greem_domain_boxes cuts them into px*py*pz boxes by recursive
   multisection, identically on every process.
2. Redistribution (step 7).  greem_domain_pack orders the particles by destination box
   and one all-to-all-v moves them.
3. LET (steps 3-4).  Each process builds the tree of its particles and exports to every
   other box the items that box needs (greem_let_export); one all-to-all-v delivers them.
4. Force (step 5).  The tree of the process's particles and the items it received
   (greem_short_force_ex over both), of which the process keeps its own particles'
   accelerations.

The per-process computation goes through an object with the calls ``cells``, ``pack``,
``let_export`` and ``short_force`` (``GpuCompute``: the library on this process's GPU);
the data movement goes through a communicator with ``allgather_float``,
``allgather_rows`` and ``alltoallv`` (``TorchComm``: torch.distributed, NCCL for device
tensors or gloo for host tensors).  No step computes anything in Python: the arithmetic
is the library's.
"""
from __future__ import annotations

import numpy as np

from . import greem


class TorchComm:
    """torch.distributed (already initialised) as the communicator.  Collective buffers
    live on ``device`` (a CUDA device for NCCL, the CPU for gloo); results come back on
    the device of the tensor that was sent."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.device = torch.device("cpu") if device is None else torch.device(device)

    def allgather_float(self, x: float) -> list:
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t)
        return [float(o.item()) for o in out]

    def allgather_rows(self, t):
        """The row blocks of every process, concatenated in rank order (sizes may differ)."""
        import torch
        src = t.to(self.device)
        n = torch.tensor([src.shape[0]], dtype=torch.int64, device=self.device)
        sizes = [torch.empty_like(n) for _ in range(self.size)]
        self.dist.all_gather(sizes, n)
        sizes = [int(s.item()) for s in sizes]
        pad = torch.zeros((max(max(sizes), 1),) + tuple(src.shape[1:]), dtype=src.dtype, device=self.device)
        pad[: src.shape[0]].copy_(src)
        outs = [torch.empty_like(pad) for _ in range(self.size)]
        self.dist.all_gather(outs, pad)
        return torch.cat([o[:s] for o, s in zip(outs, sizes)]).to(t.device)

    def alltoallv(self, send, counts):
        """Rows [sum counts[:d], sum counts[:d+1]) of send go to process d; returns (the rows
        received, in rank order, and the count from each process)."""
        import torch
        src = send.to(self.device).contiguous()
        sc = torch.tensor([int(c) for c in counts], dtype=torch.int64, device=self.device)
        rc = torch.empty_like(sc)
        self.dist.all_to_all_single(rc, sc)
        rcl = [int(x) for x in rc.tolist()]
        out = torch.empty((sum(rcl),) + tuple(src.shape[1:]), dtype=src.dtype, device=self.device)
        self.dist.all_to_all_single(out, src, output_split_sizes=rcl, input_split_sizes=[int(c) for c in counts])
        return out.to(send.device), rcl


class GpuCompute:
    """The library's calls on this process's CUDA device (one greem.Context)."""

    def __init__(self, ctx: "greem.Context"):
        self.ctx = ctx

    def cells(self, pos, idx, L):
        import torch
        return self.ctx.cell_index(pos, L, torch.from_numpy(np.ascontiguousarray(idx, np.int64)).to(pos.device))

    def pack(self, pos, mass, ids, L, boxes):
        return self.ctx.domain_pack(pos, mass, ids, L, boxes)

    def let_export(self, pos, mass, prm, boxes, self_index):
        self.ctx.build_tree(pos, mass, greem.params(**prm))
        po, mo, _, counts = self.ctx.let_export(boxes, self_index)
        return po, mo, counts

    def short_force(self, pos, mass, prm):
        """(acc, milliseconds of the call on the device)."""
        import torch
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        acc = self.ctx.short_force(pos, mass, greem.params(**prm))
        b.record()
        b.synchronize()
        return acc, a.elapsed_time(b)


def _concat(a, b):
    """a then b along the rows, by two copies into a new tensor."""
    import torch
    out = torch.empty((a.shape[0] + b.shape[0],) + tuple(a.shape[1:]), dtype=a.dtype, device=a.device)
    out[: a.shape[0]].copy_(a)
    out[a.shape[0]:].copy_(b)
    return out


class DomainStep:
    """The parallel short-range force of one process (see the module docstring).

    prm: the force parameters as keywords of greem.params (L, r_cut, theta, n_crit, n_leaf,
    ...).  grid: (px, py, pz) with px*py*pz = the number of processes.  rate: the global
    sampling rate R of Eq. 3 (the paper uses 4e-4); alpha: Eq. 5's limit on the particles of
    one process (alpha < 0: no limit)."""

    ITEM_BYTES = 28  # an exported item: FP64 position and FP32 mass (Eq. 10 counts 16)

    def __init__(self, comm, compute, prm: dict, grid, rate: float = 4e-4, alpha: float = 0.2, seed: int = 0):
        px, py, pz = (int(g) for g in grid)
        if px * py * pz != comm.size:
            raise ValueError(f"grid {grid} does not give one box per process ({comm.size})")
        self.comm, self.compute, self.prm = comm, compute, dict(prm)
        self.grid, self.rate, self.alpha, self.seed = (px, py, pz), float(rate), float(alpha), int(seed)
        self.boxes = None
        self.t_last = None     # this process's last measured force time (Eq. 4)
        self.n_decomp = 0
        self.info = {}

    def decompose(self, pos, mass, ids, n_total: int):
        """New boxes from sampled particles (Sec. 2.3.1), then the particles moved to the
        process of their box (step 7).  Before any force time is measured, a process's
        particle count stands in for its time in Eq. 4.  Returns this process's (pos, mass,
        ids)."""
        comm = self.comm
        n_local = int(pos.shape[0])
        t = self.t_last if self.t_last is not None else float(n_local)
        times = comm.allgather_float(t)
        ns = greem.sample_count(n_total, n_local, comm.size, self.rate, t, sum(times), self.alpha)
        rng = np.random.default_rng([self.seed, comm.rank, self.n_decomp])
        idx = np.sort(rng.choice(n_local, size=ns, replace=False)) if ns else np.zeros(0, np.int64)
        cells = self.compute.cells(pos, idx, self.prm["L"])
        allc = comm.allgather_rows(cells)
        self.boxes = greem.domain_boxes(allc.cpu().numpy(), self.grid)
        self.n_decomp += 1
        po, mo, io, counts = self.compute.pack(pos, mass, ids, self.prm["L"], self.boxes)
        pos_l, _ = comm.alltoallv(po, counts)
        mass_l, _ = comm.alltoallv(mo, counts)
        ids_l, _ = comm.alltoallv(io, counts)
        self.info.update(samples=ns, samples_total=int(allc.shape[0]), n_local=int(pos_l.shape[0]))
        return pos_l, mass_l, ids_l

    def force(self, pos, mass):
        """The short-range acceleration of this process's particles (steps 3-5): the LET
        exchange, then the force over the process's particles and the items received.
        Returns acc [n_local, 3]; self.info gets the counts and the force time."""
        if self.boxes is None:
            raise RuntimeError("decompose() first")
        comm, n = self.comm, int(pos.shape[0])
        if n:
            ip, im, counts = self.compute.let_export(pos, mass, self.prm, self.boxes, comm.rank)
        else:
            import torch
            ip = torch.zeros((0, 3), dtype=torch.float64, device=pos.device)
            im = torch.zeros((0,), dtype=torch.float32, device=pos.device)
            counts = np.zeros(comm.size, np.int64)
        rp, rcount = comm.alltoallv(ip, counts)
        rm, _ = comm.alltoallv(im, counts)
        if n:
            acc, ms = self.compute.short_force(_concat(pos, rp), _concat(mass, rm), self.prm)
            acc = acc[:n]
        else:
            import torch
            acc, ms = torch.zeros((0, 3), dtype=torch.float32, device=pos.device), 0.0
        self.t_last = ms
        self.info.update(n_local=n, n_import=int(sum(rcount)), n_export=int(np.sum(counts)),
                         let_bytes_sent=self.ITEM_BYTES * int(np.sum(counts)), force_ms=ms)
        return acc
