"""Dynamic-setting oracle (TEST INFRASTRUCTURE ONLY; see oracle/__init__).

The paper makes the structure dynamic by keeping the pairs (pi(p), p) in a B-tree multimap
(Sec. 2.1, "Dynamic implementation"; experiments of Sec. 3.3).  Whatever the container, the
state after a batch of updates is fully defined by the live point set, so this oracle keeps
only that set (coordinates by id, a liveness flag, the next id) and rebuilds the sorted array
from scratch after every batch with the static oracle.

Batch semantics (the paper applies single-element updates and leaves ids unspecified):
deletes are applied before inserts; inserted points get ids next_id, next_id + 1, ...; ids
are never reused; a batch that deletes an id that is not live, or the same id twice, is
rejected whole and changes nothing.
"""
from __future__ import annotations

import numpy as np

from . import OMEGA, Index, build, query


class NotFound(Exception):
    pass


class DynamicOracle:
    def __init__(self, xy: np.ndarray, w: int = OMEGA, curve="z"):
        xy = np.ascontiguousarray(xy, np.int32).reshape(-1, 2)
        self.w, self.curve = w, curve
        self.xy_by_id = xy.copy()
        self.alive = np.ones(xy.shape[0], dtype=bool)
        self.next_id = xy.shape[0]
        self.index = None
        self.rebuild()

    def apply(self, inserts: np.ndarray, delete_ids: np.ndarray) -> int:
        """Applies one batch; returns the first id given to the inserts."""
        inserts = np.ascontiguousarray(inserts, np.int32).reshape(-1, 2)
        d = np.asarray(delete_ids, dtype=np.int64).reshape(-1)
        if d.size:
            if d.min() < 0 or d.max() >= self.next_id:
                raise NotFound("delete of an id that was never issued")
            if np.unique(d).size != d.size:
                raise NotFound("duplicate delete id")
            if not self.alive[d].all():
                raise NotFound("delete of an id that is not live")
            self.alive[d] = False
        first = self.next_id
        k = inserts.shape[0]
        if k:
            self.xy_by_id = np.concatenate([self.xy_by_id, inserts])
            self.alive = np.concatenate([self.alive, np.ones(k, dtype=bool)])
            self.next_id += k
        self.rebuild()
        return first

    def rebuild(self):
        live = np.nonzero(self.alive)[0]
        idx = build(self.xy_by_id[live], self.w, self.curve)
        # build() numbers points by their position in the live list; positions follow
        # ascending id, so (key, position) order equals (key, id) order.
        self.index = Index(idx.keys, live[idx.ids].astype(np.uint32), idx.xy, idx.w, idx.curve)

    @property
    def n(self) -> int:
        return self.index.n

    def query(self, q, delta, threads: int = 1):
        return query(self.index, q, delta, threads=threads)
