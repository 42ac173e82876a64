"""Spatial decomposition (slabs + ghost imports): every rank's owned outputs equal those of the
whole step, and the step sums are the sum over ranks of the owned particles' terms.  Checked
with the oracle on the CPU, in one process and with two gloo ranks that allreduce the sums."""
import os
import socket

import numpy as np
import pytest

from oracle import units
from oracle.expect import expected_dm
from oracle.pairs import pairs_bruteforce
from oracle.step import oracle_step
from paper_2603_24688_gb300 import partition as PT
from paper_2603_24688_gb300 import workloads as W


def _open():
    return W.galaxy_workload(1800, 1300, seed=W.SEED_BASE + 77, n=-2)


def _periodic():
    return W.box_workload(n_dm=900, n_gas=800, seed=78, n=0, bulk_dm=(80.0, 0.0, 0.0))


def _owned_sums(out, dm, gas, params, dt, own_d, own_g):
    """The 16 step sums restricted to the owned particles (the terms of oracle_step's sums)."""
    Mi, Mj = dm["mass"], gas["mass"]
    v0, v1 = dm["vel"], out["mc"]["vel_new"]
    u_old = units.u_from_T(gas["T"], gas["mu"])
    pi, pj = out["pairs"]
    _, E_dE, _ = expected_dm(dm, gas, pi, pj, params, dt, out["g"])
    s = np.zeros(16)
    s[0:3] = np.sum((Mi[:, None] * (v1 - v0))[own_d], axis=0)
    s[3:6] = np.sum((Mj[:, None] * out["acc"] * dt)[own_g], axis=0)
    s[6] = np.sum((0.5 * Mi * (np.sum(v1 * v1, 1) - np.sum(v0 * v0, 1)))[own_d])
    s[7] = np.sum((Mj * (0.5 * (np.sum(out["V_new"] ** 2, 1) - np.sum(gas["vel"] ** 2, 1))
                         + out["u_new"] - u_old))[own_g])
    s[8] = np.sum(E_dE[own_d])
    s[9] = np.count_nonzero(out["mc"]["scattered"][own_d])
    s[10] = np.count_nonzero(out["mc"]["clamped"][own_d])
    s[11] = np.count_nonzero((out["u_new"] == 0.0)[own_g] & (u_old[own_g] > 0.0))
    s[12] = np.count_nonzero(own_g[pj])
    s[13] = np.sum(out["mc"]["C_total"][own_d])
    s[14] = out["mc"]["p_ratio_max"][own_d].max() if own_d.any() else 0.0
    return s


def _rank_result(w, edges, r):
    prm = w["params"]
    v = PT.rank_view(w["dm"], w["gas"], edges, r, prm["periodic"], prm["box"])
    dm, gas = PT.subset(w["dm"], v["dm"]), PT.subset(w["gas"], v["gas"])
    out = oracle_step(dm, gas, prm, 5, w["dt"])
    return v, out, _owned_sums(out, dm, gas, prm, w["dt"], v["dm_owned"], v["gas_owned"])


@pytest.mark.parametrize("which,nparts", [("open", 2), ("open", 3), ("periodic", 2), ("periodic", 3)])
def test_owned_outputs_equal_the_whole_step(which, nparts):
    w = _open() if which == "open" else _periodic()
    prm = w["params"]
    full = oracle_step(w["dm"], w["gas"], prm, 5, w["dt"])
    x = np.concatenate([w["dm"]["pos"][:, 0], w["gas"]["pos"][:, 0]])
    if prm["periodic"]:
        x = np.mod(x, prm["box"][0])
    edges = PT.slab_edges(x, nparts)
    seen_d = np.zeros(len(w["dm"]["h"]), int)
    seen_g = np.zeros(len(w["gas"]["h"]), int)
    tot = np.zeros(16)
    for r in range(nparts):
        v, out, s = _rank_result(w, edges, r)
        od, og = v["dm"][v["dm_owned"]], v["gas"][v["gas_owned"]]
        seen_d[od] += 1
        seen_g[og] += 1
        # the Monte Carlo: the same draws, partners and velocities
        assert np.array_equal(out["mc"]["vel_new"][v["dm_owned"]], full["mc"]["vel_new"][od])
        assert np.array_equal(out["mc"]["scattered"][v["dm_owned"]], full["mc"]["scattered"][od])
        assert np.array_equal(out["mc"]["partner"][v["dm_owned"]], full["mc"]["partner"][od])
        # the mean field: the same partners in the same order
        np.testing.assert_allclose(out["acc"][v["gas_owned"]], full["acc"][og], rtol=1e-13, atol=0)
        np.testing.assert_allclose(out["dudt"][v["gas_owned"]], full["dudt"][og], rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(out["T_new"][v["gas_owned"]], full["T_new"][og], rtol=1e-13)
        tot[:14] += s[:14]
        tot[14] = max(tot[14], s[14])
    assert np.all(seen_d == 1) and np.all(seen_g == 1)          # every particle owned exactly once
    ref = full["sums"]
    assert tot[9] == ref[9] and tot[10] == ref[10] and tot[11] == ref[11] and tot[12] == ref[12]
    assert tot[14] == ref[14]
    for k in (0, 1, 2, 3, 4, 5, 6, 7, 8, 13):
        assert abs(tot[k] - ref[k]) <= 1e-11 * (abs(ref[k]) + 1e-12 * np.abs(ref[:9]).max()), k


def test_ghost_zone_holds_every_partner():
    w = _open()
    prm = w["params"]
    x = np.concatenate([w["dm"]["pos"][:, 0], w["gas"]["pos"][:, 0]])
    edges = PT.slab_edges(x, 4)
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], False, None)
    for r in range(4):
        v = PT.rank_view(w["dm"], w["gas"], edges, r)
        own_g = np.zeros(len(w["gas"]["h"]), bool)
        own_g[v["gas"][v["gas_owned"]]] = True
        local_d = np.zeros(len(w["dm"]["h"]), bool)
        local_d[v["dm"]] = True
        assert np.all(local_d[pi[own_g[pj]]])                  # partners of owned gas are local
        own_d = np.zeros(len(w["dm"]["h"]), bool)
        own_d[v["dm"][v["dm_owned"]]] = True
        local_g = np.zeros(len(w["gas"]["h"]), bool)
        local_g[v["gas"]] = True
        assert np.all(local_g[pj[own_d[pi]]])                  # partners of owned DM are local


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _periodic()
    x = np.mod(np.concatenate([w["dm"]["pos"][:, 0], w["gas"]["pos"][:, 0]]), w["params"]["box"][0])
    edges = PT.slab_edges(x, world)
    _, _, s = _rank_result(w, edges, rank)
    t = torch.tensor(s[:14], dtype=torch.float64)
    m = torch.tensor([s[14]], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    q.put((rank, np.concatenate([t.numpy(), m.numpy()])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_allreduce_the_step_sums():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = _periodic()
    ref = oracle_step(w["dm"], w["gas"], w["params"], 5, w["dt"])["sums"]
    for _, s in got:
        assert s[9] == ref[9] and s[12] == ref[12] and s[14] == ref[14]
        for k in (0, 1, 2, 3, 4, 5, 6, 7, 8, 13):
            assert abs(s[k] - ref[k]) <= 1e-11 * (abs(ref[k]) + 1e-12 * np.abs(ref[:9]).max()), k
