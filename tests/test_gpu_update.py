"""GPU dynamic setting (Sec. 2.1 "Dynamic implementation", Sec. 3.3): after every batch the
sorted arrays and the query answers equal those of the oracle rebuilt from scratch over the
live set, bit for bit; rejected batches change nothing."""
import numpy as np
import pytest
import torch

import oracle
from oracle.dynamic import DynamicOracle, NotFound
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def check_same(idx, dyn, qs, d, dev):
    keys, ids, xy = sfc.sfc_get_sorted(idx)
    assert np.array_equal(u64(keys), dyn.index.keys)
    assert np.array_equal(u32(ids), dyn.index.ids)
    assert np.array_equal(xy.cpu().numpy(), dyn.index.xy)
    off, out = sfc.query(idx, to_dev(qs, dev), to_dev(d, dev))
    roff, rids = dyn.query(qs, d)
    assert np.array_equal(u64(off), roff)
    assert np.array_equal(u32(out), rids)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("bounds", ["binary", "learned"])
def test_rounds_vs_rebuilt_oracle(cuda, curve, bounds):
    dwl = W.dynamic_5e7(scale=0.002, rounds=5)
    base = dwl.base
    idx = sfc.sfc_build(to_dev(base, cuda), curve, bounds=bounds, leaves=256)
    dyn = DynamicOracle(base, curve=curve)
    cluster = dwl.meta["base_cluster"]
    for r, rd in enumerate(dwl.rounds):
        live = np.nonzero(dyn.alive)[0]
        dels = live[rd["delete_rank"]].astype(np.uint32)
        first = sfc.sfc_update(idx, to_dev(rd["inserts"], cuda), to_dev(dels.view(np.int32), cuda))
        rfirst = dyn.apply(rd["inserts"], dels)
        assert first == rfirst
        cluster = np.concatenate([cluster, rd["insert_cluster"]])
        live = np.nonzero(dyn.alive)[0]
        qs, d = W.dynamic_round_queries(dwl, r, dyn.xy_by_id[live], cluster[live])
        check_same(idx, dyn, qs, d, cuda)
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_rejected_batches_change_nothing(cuda):
    pts, qs, d = W.tiny_dense(21, 3000, 300, 12, 50)
    idx = sfc.sfc_build(to_dev(pts, cuda), "z")
    dyn = DynamicOracle(pts)
    sfc.sfc_update(idx, None, to_dev(np.array([5, 6], np.int32), cuda))
    dyn.apply(np.zeros((0, 2), np.int32), np.array([5, 6]))
    before = [t.clone() for t in sfc.sfc_get_sorted(idx)]
    ins = to_dev(np.array([[1, 1]], np.int32), cuda)
    for bad in ([5], [7, 7], [3000], [100, 6]):
        with pytest.raises(sfc.SfcError) as e:
            sfc.sfc_update(idx, ins, to_dev(np.array(bad, np.int32), cuda))
        assert e.value.status == sfc.SFC_ERR_NOT_FOUND
        after = sfc.sfc_get_sorted(idx)
        assert all(torch.equal(a, b) for a, b in zip(before, after))
    # the index still works and ids continue from where they were
    first = sfc.sfc_update(idx, ins, None)
    assert first == 3000 == dyn.apply(np.array([[1, 1]], np.int32), np.zeros(0, np.int64))
    check_same(idx, dyn, qs, d, cuda)


def test_delete_everything_then_insert(cuda):
    pts, qs, d = W.tiny_dense(22, 500, 100, 8, 20)
    idx = sfc.sfc_build(to_dev(pts, cuda), "h")
    dyn = DynamicOracle(pts, curve="h")
    all_ids = np.arange(500, dtype=np.uint32)
    sfc.sfc_update(idx, None, to_dev(all_ids.view(np.int32), cuda))
    dyn.apply(np.zeros((0, 2), np.int32), all_ids)
    check_same(idx, dyn, qs, d, cuda)
    ins = np.random.default_rng(3).integers(0, 256, size=(700, 2)).astype(np.int32)
    assert sfc.sfc_update(idx, to_dev(ins, cuda), None) == 500 == dyn.apply(ins, np.zeros(0, np.int64))
    check_same(idx, dyn, qs, d, cuda)


def test_insert_into_empty_index(cuda):
    idx = sfc.sfc_build(torch.empty((0, 2), dtype=torch.int32, device=cuda), "z")
    dyn = DynamicOracle(np.zeros((0, 2), np.int32))
    pts, qs, d = W.tiny_dense(23, 900, 100, 10, 40)
    assert sfc.sfc_update(idx, to_dev(pts, cuda), None) == 0 == dyn.apply(pts, np.zeros(0, np.int64))
    check_same(idx, dyn, qs, d, cuda)
