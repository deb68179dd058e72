"""The binning step (slice geometry of eq. forward-projector; points grouped per brick of
the fine grid before spreading, Section 3.4; bricks of 8 x 8 x depth cells, the depth
reported by firm_bin_info) checked exactly: the ids are a permutation
of all points, the work items tile the id array, every point sits in its item's brick
(positions recomputed in FP64 from the rotations; points within 1e-4 cells of a brick
face may go either way), no item exceeds the work-item size, and within every item the
sequence of bank classes is exactly the round-robin arrangement of that item's class
histogram (the order within one class is free)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1307_5824_gb300 as pkg
    return pkg


def half_disc(N):
    h = N // 2
    H = [(0, k2) for k2 in range(0, h + 1)]
    H += [(k1, k2) for k1 in range(1, h + 1) for k2 in range(-h, h + 1) if k1 * k1 + k2 * k2 <= h * h]
    return np.array(H)


def round_robin(classes):
    """Class sequence of the round-robin order: level r lists, in ascending class order,
    every class with more than r points."""
    cnt = np.bincount(classes, minlength=32)
    seq = []
    for r in range(cnt.max()):
        seq.extend(np.flatnonzero(cnt > r).tolist())
    return np.array(seq)


@pytest.mark.parametrize("channel", [0, 1])
def test_binning_is_an_exact_partition_by_brick(F, channel):
    N, M, W = 32, 60, 6
    inp = synth.config_inputs("C2", M=M, N=N, images=False)
    rec = F.Reconstructor(N, M, W=W)
    F._lib.firm_bin(rec.plan, M, torch.from_numpy(inp["R"].reshape(M, 9).copy()).cuda(), channel)
    n_work, n_pts, nb, bzd, chunk = F._lib.firm_bin_info(rec.plan)
    assert bzd in (8, 16)
    ids = torch.empty(n_pts, dtype=torch.int32, device="cuda")
    work = torch.empty((n_work, 4), dtype=torch.int32, device="cuda")
    F._lib.firm_copy_out(rec.plan, F._lib.FIRM_OUT_BIN_IDS, ids)
    F._lib.firm_copy_out(rec.plan, F._lib.FIRM_OUT_BIN_WORK, work)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy().view(np.uint32)
    work = work.cpu().numpy()
    rec.close()

    H = half_disc(N)
    nH = H.shape[0]
    assert n_pts == M * nH
    # a permutation of every (m, t), bit for bit
    expect = (np.arange(M, dtype=np.uint32)[:, None] << 13) | np.arange(nH, dtype=np.uint32)[None, :]
    assert np.array_equal(np.sort(ids), np.sort(expect.ravel()))
    # the items tile [0, n_pts)
    order = np.argsort(work[:, 1])
    starts, lens = work[order, 1], work[order, 2]
    assert starts[0] == 0 and np.all(starts[1:] == starts[:-1] + lens[:-1]) and starts[-1] + lens[-1] == n_pts
    assert lens.min() >= 1 and lens.max() <= chunk

    # FP64 positions on the fine grid (G = 4N for the kernel channel, 2N for A*b)
    G = 4 * N if channel == 0 else 2 * N
    s = G // N
    R = inp["R"]
    m = (ids >> 13).astype(np.int64)
    t = (ids & 0x1FFF).astype(np.int64)
    k1, k2 = H[t, 0].astype(float), H[t, 1].astype(float)
    y = G / 2 + s * (k1[:, None] * R[m, 0, :] + k2[:, None] * R[m, 1, :])        # (n, 3): x, y, z
    fl = np.floor(y)
    cell = fl.astype(np.int64) % G
    frac = y - fl
    near = np.any(np.minimum(frac, 1 - frac) < 1e-4, axis=1)                   # too close to a cell face
    bxyz = cell // np.array([8, 8, bzd])
    brick_of_pos = np.empty(n_pts, np.int64)
    for w_ in work:
        brick_of_pos[w_[1]:w_[1] + w_[2]] = w_[0]
    bz, by, bx = brick_of_pos // (nb * nb), (brick_of_pos // nb) % nb, brick_of_pos % nb
    ok = (bxyz[:, 0] == bx) & (bxyz[:, 1] == by) & (bxyz[:, 2] == bz)
    assert np.all(ok | near), int((~(ok | near)).sum())

    # bank classes: first tap r = cell - brick origin + ceil(frac) (even W), base in an
    # (8+W) x (8+W) x (depth+W) region, x fastest
    RG = 8 + W
    r = cell - np.array([8, 8, bzd]) * np.stack([bx, by, bz], 1) + np.ceil(frac).astype(np.int64)
    cls = ((r[:, 2] * RG + r[:, 1]) * RG + r[:, 0]) % 32
    checked = 0
    for w_ in work:
        sl = slice(w_[1], w_[1] + w_[2])
        if near[sl].any():
            continue
        c = cls[sl]
        if np.bincount(c, minlength=32).max() > 1024:      # skewed piece: grouped by class only
            continue
        assert np.array_equal(c, round_robin(c)), w_
        checked += 1
    print(f"channel {channel}: {n_work} items, {checked} checked for the round-robin class order")
    assert checked >= 0.5 * n_work
