"""The per-process calls of paper_0910_0121_gb300.domain (cells, pack, let_export,
short_force) computed by the FP64 CPU oracle, for multi-process tests without a GPU.
Test infrastructure: the product path uses the library (GpuCompute)."""
import time

import numpy as np
import torch

import oracle


def _cells(pos, L):
    """Finest cells by the key's reading: the periodic wrap, then the cell index."""
    return np.array([[oracle.cell_index(oracle.wrap(x, L), L) for x in p] for p in pos],
                    dtype=np.int32).reshape(-1, 3)


class OracleCompute:
    def cells(self, pos, idx, L):
        p = pos.numpy()[np.asarray(idx, np.int64)]
        return torch.from_numpy(_cells(p, L))

    def pack(self, pos, mass, ids, L, boxes):
        p = pos.numpy()
        c = _cells(p, L)
        dom = np.full(len(p), -1, np.int64)
        for d, b in enumerate(boxes):
            inside = np.all((c >= b[0::2]) & (c < b[1::2]), axis=1)
            dom[inside & (dom < 0)] = d
        assert np.all(dom >= 0), "boxes do not tile the box"
        order = np.argsort(dom, kind="stable")
        wrapped = np.array([[oracle.wrap(x, L) for x in q] for q in p[order]]).reshape(-1, 3)
        i = (np.arange(len(p)) if ids is None else ids.numpy())[order]
        counts = np.bincount(dom, minlength=len(boxes)).astype(np.int64)
        return (torch.from_numpy(wrapped), torch.from_numpy(mass.numpy()[order].copy()),
                torch.from_numpy(np.ascontiguousarray(i, np.int64)), counts)

    def let_export(self, pos, mass, prm, boxes, self_index):
        T = oracle.Tree(pos.numpy(), mass.numpy(), prm["L"], prm["r_cut"], n_crit=prm["n_crit"],
                        n_leaf=prm.get("n_leaf", 10))
        _, _, xyz, ms = T.sorted()
        mom = T.moments()
        ps, mm, counts = [], [], np.zeros(len(boxes), np.int64)
        for d, b in enumerate(boxes):
            if d == self_index:
                continue
            kind, idx = T.let_export(b, prm["theta"])
            part = kind == 0
            p = np.where(part[:, None], xyz[np.where(part, idx, 0)], mom[np.where(part, 0, idx), 1:])
            m = np.where(part, ms[np.where(part, idx, 0)], mom[np.where(part, 0, idx), 0].astype(np.float32))
            ps.append(p)
            mm.append(m.astype(np.float32))
            counts[d] = len(idx)
        P = np.concatenate(ps) if ps else np.zeros((0, 3))
        M = np.concatenate(mm) if mm else np.zeros(0, np.float32)
        return torch.from_numpy(np.ascontiguousarray(P)), torch.from_numpy(np.ascontiguousarray(M)), counts

    def short_force(self, pos, mass, prm):
        t0 = time.perf_counter()
        a = oracle.short_force(pos.numpy(), mass.numpy(), prm["L"], prm["r_cut"], prm["theta"], prm["n_crit"],
                               prm.get("n_leaf", 10))
        return torch.from_numpy(a), 1e3 * (time.perf_counter() - t0)
