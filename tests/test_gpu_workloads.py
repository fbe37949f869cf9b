"""The batched workload at its full size, as the benchmark runs it: 64
independent relocalizations (mixed map sizes, beam counts, FoVs, hypothesis
counts and K) in one batch.  Every result equals the same request run alone,
and the first request's SMAD numerators (Eq. 19), survivors and sampled TAM
scores (Eq. 31) equal the oracle's."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


@pytest.fixture(scope="module")
def instances():
    return workloads.batched_instances()


def test_batched_workload_equals_alone_and_oracle(relo, instances):
    import torch
    ctx = relo.Relo(n_orient=360, topk=1024, batch=1024, local_topk=20, early_stop=0)
    items = []
    for it in instances:
        mid = ctx.load_map(it.grid, it.res)
        ctx.set_hypotheses(mid, workloads.cell_centres(it.hyps, it.res))
        items.append((mid, it.ranges, it.angles, it.max_range, it.topk))
    batch = ctx.relocalize_batch(items)
    assert len(batch) == len(items) and all(b.status == 0 for b in batch)

    # the first request against the oracle
    it = instances[0]
    K = min(it.topk, len(it.hyps))
    num = ctx.stage(relo.STAGE_SMAD_NUM, torch.empty(len(it.hyps), dtype=torch.int64, device="cuda")).cpu().numpy()
    surv = ctx.stage(relo.STAGE_SURVIVORS, torch.empty(K, dtype=torch.int32, device="cuda")).cpu().numpy()
    T = ctx.stage(relo.STAGE_TAM, torch.empty(K * 360, dtype=torch.float32, device="cuda")).cpu().numpy()
    prm = oracle.Params(n_orient=360, topk=it.topk, batch=1024, local_topk=20)
    pl = oracle.plan(it.ranges, it.angles, it.max_range, it.res, prm)
    want_num, _ = oracle.coarse(it.grid, it.hyps, pl, prm)
    assert np.array_equal(num, want_num)
    assert np.array_equal(surv, oracle.rank(want_num, K))
    rows = np.unique(np.concatenate([[0], np.random.default_rng(3).choice(K, 5, replace=False)]))
    want_T = oracle.tam_grid(it.grid, it.hyps, surv[rows], pl, prm, it.res, oracle.edt(it.grid))
    got_T = T.reshape(K, 360)[rows].astype(np.float64)
    err = np.abs(got_T - want_T)
    assert np.all((err <= RTOL * np.abs(want_T)) | ((want_T == 0) & (np.abs(got_T) <= 1e-7)))

    # every request alone gives the same result
    for item, b in zip(items, batch):
        assert ctx.relocalize_batch([item])[0].as_dict() == b.as_dict()
    ctx.close()
