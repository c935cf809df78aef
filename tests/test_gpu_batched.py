"""GPU parity of the batched path: several wings of different sizes in one
cooperative greedy launch and one volume launch, checked problem by problem
against the oracle, and replayed from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu
SIZES = [(6, 30), (10, 50), (16, 125), (8, 40), (12, 90)]


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.fixture(scope="module")
def batch():
    cases, probs = [], []
    for k, (ns, ncn) in enumerate(SIZES):
        c = synth.wing_case(ns, ncn, 3000 + 500 * k, vol_seed=100 + k, radius=2.0,
                            tol_rel=1e-3)
        c["d_xb"], c["d_db"], c["d_xv"] = cuda(c["xb"]), cuda(c["db"]), cuda(c["xv"])
        c["estar"] = oracle.tolerance(c["db"], c["tol_rel"])
        c["m"] = [1, 3, 5, 2, 7][k]
        cases.append(c)
        probs.append(dict(xb=c["d_xb"], db=c["d_db"], radius=2.0, tol=c["estar"], tol_mode=0,
                          m=c["m"], seed=1 + k, nc_max=min(len(c["xb"]), 1000)))
    gb = P.GreedyBatch(probs)
    gb.run()
    res = gb.results()
    vprobs = [dict(xv=c["d_xv"], xb=c["d_xb"], idx=gb.idx[i], w=gb.w[i],
                   nc_ptr=gb.nc_ptr + 8 * i, radius=2.0) for i, c in enumerate(cases)]
    vb = P.VolumeBatch(vprobs)
    vb.run()
    torch.cuda.synchronize()
    return cases, gb, res, vb


def test_batched_greedy_each_problem_certified(batch):
    cases, gb, res, _ = batch
    for i, c in enumerate(cases):
        r = res[i]
        assert r["status"] == 0
        nc = r["nc"]
        idx = gb.idx[i][:nc].cpu().numpy()
        o = oracle.greedy(c["xb"], c["db"], 2.0, c["estar"], m=c["m"], seed=1 + i,
                          history=False)
        assert idx.tolist() == o["idx"].tolist(), i
        assert r["final_max"] <= c["estar"]
        Wo, _, _ = oracle.solve_weights(c["xb"], c["db"], idx, 2.0)
        assert np.abs(gb.w[i][:nc].cpu().numpy() - Wo).max() <= 1e-5 * np.abs(c["db"]).max()


def test_batched_volume_matches_oracle(batch):
    cases, gb, res, vb = batch
    for i, c in enumerate(cases):
        nc = res[i]["nc"]
        idx = gb.idx[i][:nc].cpu().numpy()
        W = gb.w[i][:nc].cpu().numpy()
        ref = oracle.rbf_sum(c["xv"], c["xb"], idx, W, 2.0)
        got = vb.dv[i].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11
    info = vb.info()
    assert info["threads"] in (128, 256) and info["points_per_thread"] in (1, 2)


def test_batched_graph_replay_is_identical(batch):
    cases, gb, res, vb = batch
    before = [d.clone() for d in vb.dv]
    idx_before = [t.clone() for t in gb.idx]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        gb.run()
        vb.run()
    for d in vb.dv:
        d.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(cases)):
        nc = res[i]["nc"]
        assert torch.equal(gb.idx[i][:nc], idx_before[i][:nc])
        assert torch.equal(vb.dv[i], before[i])


# ---- configuration 4a's problem sizes: the eight smallest of its 64 wings
# (N_b from PCG64(seed) ~ U[5000, 100000], seeds 100-163, 5.4k-23k nodes),
# tolerance 1e-4, m = round(1.5 N_b / N_c) from a plain-greedy batch; every
# decision of every problem replayed by the oracle's follow mode ----
CONFIG4A_SEEDS = [108, 123, 157, 147, 148, 107, 114, 112]


def _config4a_case(seed, nv):
    import math
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = int(rng.integers(5000, 100001))
    ns = max(2, int(round(math.sqrt(nb / 5))))
    nch = int(round(nb / ns))
    return synth.wing_case(ns, nch, nv, vol_seed=seed, vol_kind="box", radius=2.0,
                           tol_rel=1e-4)


def test_batched_config4a_sizes_follow_oracle():
    from _follow import check_follow
    cases = [_config4a_case(s, 20_000) for s in CONFIG4A_SEEDS]
    base = []
    for s, c in zip(CONFIG4A_SEEDS, cases):
        c["d_xb"], c["d_db"], c["d_xv"] = cuda(c["xb"]), cuda(c["db"]), cuda(c["xv"])
        c["estar"] = oracle.tolerance(c["db"], c["tol_rel"])
        base.append(dict(xb=c["d_xb"], db=c["d_db"], radius=2.0, tol=c["estar"], tol_mode=0,
                         seed=s, nc_max=1024))
    cal = P.GreedyBatch([dict(q, m=1) for q in base])
    cal.run()
    ms = [max(1, int(round(1.5 * len(c["xb"]) / r["nc"])))
          for c, r in zip(cases, cal.results())]
    gb = P.GreedyBatch([dict(q, m=m) for q, m in zip(base, ms)])
    gb.run()
    res = gb.results()
    vb = P.VolumeBatch([dict(xv=c["d_xv"], xb=c["d_xb"], idx=gb.idx[i], w=gb.w[i],
                             nc_ptr=gb.nc_ptr + 8 * i, radius=2.0)
                        for i, c in enumerate(cases)])
    vb.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    for i, (s, c, m) in enumerate(zip(CONFIG4A_SEEDS, cases, ms)):
        r = res[i]
        assert r["status"] == 0, (s, r["status"])
        nc = r["nc"]
        idx = gb.idx[i][:nc].cpu().numpy()
        it = gb.iter[i][:nc].cpu().numpy()
        f = oracle.greedy(c["xb"], c["db"], 2.0, c["estar"], m=m, seed=s, follow=(idx, it),
                          tie_rel=1e-6, history=False)
        check_follow(f, f"batched wing seed {s}, N_b {len(c['xb'])}, m={m}, N_c {nc}")
        assert f["nc"] == nc and f["stats"]["iterations"] == r["iterations"]
        assert r["final_max"] <= c["estar"]
        dmax = np.abs(c["db"]).max()
        Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], idx, 2.0)
        assert st == 0
        assert np.abs(gb.w[i][:nc].cpu().numpy() - Wo).max() <= 1e-5 * dmax
        sample = np.sort(rng.choice(len(c["xv"]), 1000, replace=False))
        ref = oracle.rbf_sum(c["xv"][sample], c["xb"], idx, Wo, 2.0)
        got = vb.dv[i].cpu().numpy()[sample]
        assert np.abs(got - ref).max() <= 1e-5 * dmax


def test_batched_config4a_full_batch_certified():
    """The whole 64-wing batch at the sizes and settings the benchmark times
    (N_b 5.4k-99k, 200,000 volume points each, tol 1e-4 relative, m = 1.5
    N_b / N_c from a plain-greedy batch): every problem ends certified, i.e.
    the oracle's FP64 error of every boundary node with weights solved on the
    selected set is at most E* (the stopping rule of Sec. 3); weights and
    sampled volume displacements match the oracle; the two largest problems'
    selections are replayed by the oracle's follow mode."""
    from _follow import check_follow
    seeds = list(range(100, 164))
    cases = [_config4a_case(s, 200_000) for s in seeds]
    base = []
    for s, c in zip(seeds, cases):
        c["d_xb"], c["d_db"], c["d_xv"] = cuda(c["xb"]), cuda(c["db"]), cuda(c["xv"])
        base.append(dict(xb=c["d_xb"], db=c["d_db"], radius=2.0, tol=c["tol_rel"], tol_mode=1,
                         seed=s, nc_max=1024))
    cal = P.GreedyBatch([dict(q, m=1) for q in base])
    cal.run()
    ms = [max(1, int(round(1.5 * len(c["xb"]) / r["nc"])))
          for c, r in zip(cases, cal.results())]
    del cal
    gb = P.GreedyBatch([dict(q, m=m) for q, m in zip(base, ms)])
    gb.run()
    res = gb.results()
    vb = P.VolumeBatch([dict(xv=c["d_xv"], xb=c["d_xb"], idx=gb.idx[i], w=gb.w[i],
                             nc_ptr=gb.nc_ptr + 8 * i, radius=2.0)
                        for i, c in enumerate(cases)])
    vb.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for i, (s, c) in enumerate(zip(seeds, cases)):
        r = res[i]
        assert r["status"] == 0, (s, r["status"])
        nc = r["nc"]
        idx = gb.idx[i][:nc].cpu().numpy()
        assert len(np.unique(idx)) == nc
        estar = oracle.tolerance(c["db"], c["tol_rel"])
        assert r["final_max"] <= estar * (1.0 + 1e-12), (s, r["final_max"], estar)
        dmax = np.abs(c["db"]).max()
        Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], idx, 2.0)
        assert st == 0
        assert np.abs(gb.w[i][:nc].cpu().numpy() - Wo).max() <= 1e-5 * dmax, s
        # every node within E*: the certificate of the stopping rule
        E = np.linalg.norm(c["db"] - oracle.rbf_sum(c["xb"], c["xb"], idx, Wo, 2.0), axis=1)
        assert E.max() <= estar * (1.0 + 1e-6), (s, E.max(), estar)
        sample = np.sort(rng.choice(len(c["xv"]), 200, replace=False))
        ref = oracle.rbf_sum(c["xv"][sample], c["xb"], idx, Wo, 2.0)
        got = vb.dv[i].cpu().numpy()[sample]
        assert np.abs(got - ref).max() <= 1e-5 * dmax, s
    for i in sorted(range(len(cases)), key=lambda k: -len(cases[k]["xb"]))[:2]:
        c, r = cases[i], res[i]
        nc = r["nc"]
        idx = gb.idx[i][:nc].cpu().numpy()
        it = gb.iter[i][:nc].cpu().numpy()
        estar = oracle.tolerance(c["db"], c["tol_rel"])
        f = oracle.greedy(c["xb"], c["db"], 2.0, estar, m=ms[i], seed=seeds[i], follow=(idx, it),
                          tie_rel=1e-6, history=False)
        check_follow(f, f"64-wing batch, seed {seeds[i]}, N_b {len(c['xb'])}, m={ms[i]}, N_c {nc}")
        assert f["nc"] == nc and f["stats"]["iterations"] == r["iterations"]
