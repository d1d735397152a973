"""A communicator for processes emulated as threads of one process on one GPU (tests only):
a shared table and a barrier.  Each rank publishes what it sends after synchronising its
stream, every rank copies what it receives, synchronises, and only then may the senders
go on; no kernel of one rank ever waits on another's."""
import threading

import torch


class World:
    def __init__(self, size):
        self.size = size
        self.barrier = threading.Barrier(size, timeout=600)
        self.slots = [None] * size

    def comm(self, rank):
        return ThreadComm(self, rank)


class ThreadComm:
    def __init__(self, world, rank):
        self.w, self.rank, self.size = world, rank, world.size

    def _exchange(self, item):
        torch.cuda.current_stream().synchronize()
        self.w.slots[self.rank] = item
        self.w.barrier.wait()
        got = list(self.w.slots)
        return got

    def _done(self):
        torch.cuda.current_stream().synchronize()
        self.w.barrier.wait()

    def allgather_float(self, x):
        got = self._exchange(float(x))
        self._done()
        return got

    def allgather_rows(self, t):
        got = self._exchange(t)
        out = torch.cat([g.to(t.device) for g in got])
        self._done()
        return out

    def alltoallv(self, send, counts):
        off = [0]
        for c in counts:
            off.append(off[-1] + int(c))
        got = self._exchange((send, off))
        parts = [s[o[self.rank]:o[self.rank + 1]] for s, o in got]
        out = torch.cat([p.to(send.device) for p in parts]) if parts else send[:0]
        rc = [int(p.shape[0]) for p in parts]
        self._done()
        return out, rc
