"""Spatial-domain split of one system over two ranks (gloo, CPU), with the
oracle as each rank's evaluator: the multi-GPU design for a single large
system (the paper's MPI layout, Sec. 4 and 6) checked on the host.

Rank r owns the sites whose x lies in its half of the periodic box.  The
exchanges of the design, in order:
  1. a halo of (q, sigma, x) from the other rank: every remote site within
     2 r_list of the rank's slab (periodic in x).  r_list covers the owned
     sites' neighbours; the second r_list gives those neighbours complete
     neighbourhoods, so their embedding coefficients (a, b) -- which the
     owned sites' forces and chemical potentials read -- come out right
     without a separate exchange of (a, b);
  2. the owned sites' excess chemical potentials, gathered before the Euler
     step (the bonds that cross the boundary read the other side's mu);
  3. one all-reduce of the FIRE scalars (P = f.v, |v|^2, |f|^2 and the
     largest force norm);
  4. the bond fluxes that cross the boundary are evaluated by both sides,
     each for its own sites, so the total mass is conserved without an
     exchange of fluxes.
Every owned result must equal the single-domain oracle's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    from paper_1910_01235_gb300 import workloads as W
    s = W.config_binary_alloy(cells=4)
    # 14 x 4 x 4 cells (L_x = 50.4 A, r_list ~ 5.5 A): a slab of 25.2 A plus
    # a halo of 2 r_list on each side leaves part of the box out of each rank
    q = W.fcc_positions(14, 4, 4, s.a)
    n = q.shape[1]
    rng = np.random.default_rng(77)
    t = s.copy()
    t.L = np.array([14 * s.a, 4 * s.a, 4 * s.a])
    t.q = q + rng.uniform(-0.05, 0.05, q.shape)
    t.sigma = 0.1 + rng.uniform(-0.02, 0.02, n)
    xa = rng.uniform(0.85, 0.95, n)
    t.x = np.vstack([xa, 0.995 - xa])
    t.T = np.full(n, 1000.0)
    t.sublattice = np.zeros(n, np.uint8)
    return t


def _slab_distance(xs, lo, hi, L):
    """Periodic distance of coordinates xs from the interval [lo, hi)."""
    inside = (xs >= lo) & (xs < hi)
    d = np.minimum(np.mod(lo - xs, L), np.mod(xs - hi, L))
    return np.where(inside, 0.0, d)


def _all_gather_columns(a, world):
    """Concatenate every rank's [rows, k_r] block (row 0: global site ids).
    Gloo gathers equal shapes, so each block is padded with id -1 columns."""
    k = torch.tensor([a.shape[1]])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, k)
    kmax = int(max(x.item() for x in sizes))
    pad = np.full((a.shape[0], kmax), -1.0)
    pad[:, : a.shape[1]] = a
    bufs = [torch.zeros((a.shape[0], kmax), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, torch.from_numpy(pad))
    g = torch.cat(bufs, dim=1).numpy()
    return g[:, g[0] >= 0]


def _rank(rank, world, port, out):
    try:
        _rank_body(rank, world, port, out)
    except BaseException as e:  # report to the parent instead of leaving it waiting
        out.put((rank, repr(e)))
        raise


def _rank_body(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    try:
        s = _system()
        n, S, L = s.n, s.S, s.L
        r_list = O.r_list_for(s)
        r_bond = 0.5 * (s.a / np.sqrt(2.0) + s.a)
        xs = np.mod(s.q[0], L[0])
        lo, hi = rank * L[0] / world, (rank + 1) * L[0] / world
        owned = np.nonzero((xs >= lo) & (xs < hi))[0]
        # 1. halo of (q, sigma, x): each rank publishes its owned sites
        glob = _all_gather_columns(np.vstack([owned[None, :].astype(float), s.q[:, owned], s.sigma[None, owned],
                                              s.x[:, owned]]), world)
        gid = glob[0].astype(int)
        order = np.argsort(gid)
        gid, glob = gid[order], glob[:, order]
        assert np.array_equal(gid, np.arange(n))          # every site owned once
        gq, gsig, gx = glob[1:4], glob[4], glob[5:5 + S]
        near = _slab_distance(np.mod(gq[0], L[0]), lo, hi, L[0]) < 2.0 * r_list
        local = np.nonzero(near)[0]                         # owned + halo, global order
        assert owned.size < local.size < n                  # a real halo, and a real split
        t = s.copy()
        t.q, t.sigma, t.x, t.T = gq[:, local], gsig[local], gx[:, local], s.T[local]
        t.sublattice = s.sublattice[local]
        st, off, idx = O.neighbors(t.q, t.L, r_list)
        assert st == O.OK
        fe = O.free_energy(t, (off, idx))
        assert fe["status"] == O.OK
        pos = np.searchsorted(local, owned)                 # owned sites in the local numbering
        res = {"owned": owned, "gq": fe["gq"][:, pos], "gs": fe["gs"][pos], "mu_ex": fe["mu_ex"][:, pos]}
        # 2. the owned chemical potentials, gathered for the bonds across the boundary
        mg = _all_gather_columns(np.vstack([owned[None, :].astype(float), res["mu_ex"]]), world)
        mu_all = np.zeros((S, n))
        mu_all[:, mg[0].astype(int)] = mg[1:]
        boff, bidx = O.bonds(t, r_bond, off, idx)
        dt = s.dt_default()
        # 4. the Euler step of the local set with the exchanged mu; only the
        # owned sites' new fractions are kept (bonds across the boundary are
        # evaluated by both sides, each for its own site)
        st, x1 = O.diffuse_step(t, mu_all[:, local], (boff, bidx), dt)
        assert st == O.OK
        res["x1"] = x1[:, pos]
        # 3. FIRE scalars from the owned sites (v = -g dt, one kick from rest)
        f = -res["gq"]
        fs = -res["gs"]
        v, vs = 0.02 * f, 0.02 * fs
        loc = torch.tensor([np.sum(f * v) + np.sum(fs * vs), np.sum(v * v) + np.sum(vs * vs),
                            np.sum(f * f) + np.sum(fs * fs)], dtype=torch.float64)
        dist.all_reduce(loc)
        fmax = torch.tensor([max(np.sqrt((f * f).sum(0)).max(), np.abs(fs).max())], dtype=torch.float64)
        dist.all_reduce(fmax, op=dist.ReduceOp.MAX)
        res["scalars"] = np.concatenate([loc.numpy(), fmax.numpy()])
        res["dmass"] = (res["x1"] - s.x[:, owned]).sum(axis=1)
        out.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_domain_split_matches_single_domain():
    import oracle as O
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for r in range(world):
        assert isinstance(res[r], dict), f"rank {r} failed: {res[r]}"
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = _system()
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, 0.5 * (s.a / np.sqrt(2.0) + s.a), off, idx)
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), s.dt_default())
    assert st == O.OK
    assert np.abs(x1 - s.x).max() > 1e-9
    for r in range(world):
        o = res[r]["owned"]
        assert 0 < o.size < s.n
        np.testing.assert_allclose(res[r]["gq"], fe["gq"][:, o], rtol=0, atol=1e-11)
        np.testing.assert_allclose(res[r]["gs"], fe["gs"][o], rtol=0, atol=1e-11)
        np.testing.assert_allclose(res[r]["mu_ex"], fe["mu_ex"][:, o], rtol=0, atol=1e-11)
        np.testing.assert_allclose(res[r]["x1"], x1[:, o], rtol=0, atol=1e-14)
    # the all-reduced FIRE scalars are the global ones; both ranks hold them
    f, fs = -fe["gq"], -fe["gs"]
    v, vs = 0.02 * f, 0.02 * fs
    ref = np.array([np.sum(f * v) + np.sum(fs * vs), np.sum(v * v) + np.sum(vs * vs), np.sum(f * f) + np.sum(fs * fs),
                    max(np.sqrt((f * f).sum(0)).max(), np.abs(fs).max())])
    for r in range(world):
        np.testing.assert_allclose(res[r]["scalars"], ref, rtol=1e-12)
    # mass: the two sides' changes cancel (each boundary bond seen from both ends)
    total = res[0]["dmass"] + res[1]["dmass"]
    assert np.abs(total).max() <= 1e-13
