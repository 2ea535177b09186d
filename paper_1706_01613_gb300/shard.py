"""Element-range sharding of one validation problem across ranks.

Elements are independent (the verdict of a hexahedron depends on its own 8
nodes only), so a mesh splits into contiguous element ranges with no
exchange between ranks: each rank validates its range and the per-element
outputs of the ranks, concatenated in rank order, are those of one rank
validating the whole mesh.  An indexed mesh ships to each rank only the
nodes its range touches, renumbered in increasing global id.

Host-side logic only (numpy); the data path has no collective.
"""
import numpy as np


def element_range(n, rank, world):
    """[lo, hi) of rank `rank` among `world`: contiguous, sizes differing by
    at most one, ranks in order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_soa(corners, rank, world):
    """The rank's slice of SoA corner planes (8, 3, n) (a copy, contiguous)
    and its element range."""
    lo, hi = element_range(corners.shape[2], rank, world)
    return np.ascontiguousarray(corners[:, :, lo:hi]), (lo, hi)


def shard_indexed(nodes, conn, rank, world):
    """The rank's part of an indexed mesh: (local nodes, local conn, (lo, hi),
    global ids of the local nodes).  Local node i is global node ids[i]
    (ids ascending); local conn row e is global row lo + e with its entries
    renumbered.  Entries outside [0, len(nodes)) are kept out of range
    (mapped to len(local nodes)) so that the rank reports them as the whole
    mesh would."""
    lo, hi = element_range(conn.shape[0], rank, world)
    part = conn[lo:hi]
    ok = (part >= 0) & (part < nodes.shape[0])
    ids = np.unique(part[ok])
    local = np.searchsorted(ids, np.where(ok, part, 0)).astype(np.int32)
    local[~ok] = len(ids)
    return np.ascontiguousarray(nodes[ids]), np.ascontiguousarray(local), (lo, hi), ids
