"""Seeded synthetic inputs for the linear-hexahedron validity test.

This module only draws coordinates and connectivity; it contains none of the
validity method's arithmetic.  Both the CUDA path and the CPU oracle are fed
from it, so the same bytes reach both.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.

The paper measures on hex sets built from two tetrahedral meshes (Sec. 7,
Fusee_1 and FT47 from hextreme.eu); those sets are not available, so the
generators below stand in for them with the same mix of mostly valid, some
invalid and some barely valid elements.

Layouts (node order of Appendix A):
  * SoA: float64 (8, 3, n) -- plane [k][d] holds coordinate d of node k;
  * indexed: nodes float64 (n_nodes, 3), conn int32 (n_hex, 8).
"""
import math

import numpy as np

# Appendix A reference corners (unit cube), nodes 1..8.
REF_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.float64)

SEED_BASE = 20170000


def rng_for(config_id, seed=None):
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id if seed is None else seed))


def perturbed_cubes(n, noise=0.3, seed=None):
    """Unit-cube corners with every coordinate perturbed by i.i.d. U[-noise, noise].
    (10,000 of these, seed 20170001, is the small CPU-sized workload.)"""
    rng = rng_for(1, seed)
    X = np.broadcast_to(REF_CORNERS[:, :, None], (8, 3, n)).copy()
    X += rng.uniform(-noise, noise, size=(8, 3, n))
    return X


def structured_grid(nx=128, ny=None, nz=None, sigma=0.15, seed=None):
    """(nx+1)(ny+1)(nz+1) nodes of spacing 1; interior nodes displaced by
    i.i.d. N(0, sigma^2) per axis, boundary nodes fixed.  Node id
    i + (nx+1)(j + (ny+1)k); hex (i,j,k) has index i + nx(j + ny k) and its
    corners in Appendix A order.  Returns (nodes (n_nodes,3) f64, conn (n,8) i32)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = rng_for(2, seed)
    px, py, pz = nx + 1, ny + 1, nz + 1
    k, j, i = np.meshgrid(np.arange(pz), np.arange(py), np.arange(px), indexing="ij")
    nodes = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(np.float64)
    disp = rng.normal(0.0, sigma, size=nodes.shape)
    ii, jj, kk = i.reshape(-1), j.reshape(-1), k.reshape(-1)
    interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz))
    nodes[interior] += disp[interior]
    hk, hj, hi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    hi, hj, hk = hi.reshape(-1), hj.reshape(-1), hk.reshape(-1)

    def nid(a, b, c):
        return a + px * (b + py * c)

    conn = np.stack([
        nid(hi, hj, hk), nid(hi + 1, hj, hk), nid(hi + 1, hj + 1, hk), nid(hi, hj + 1, hk),
        nid(hi, hj, hk + 1), nid(hi + 1, hj, hk + 1), nid(hi + 1, hj + 1, hk + 1),
        nid(hi, hj + 1, hk + 1)], axis=1).astype(np.int32)
    return nodes, conn


def _for_chunks(fn, n, chunk=1 << 18):
    """fn(slice) over consecutive chunks of range(n) on the host's cores (fn
    writes its own part of the output; the random numbers are drawn
    beforehand, so the result does not depend on the chunking)."""
    import concurrent.futures as cf
    import os
    parts = [slice(i, min(n, i + chunk)) for i in range(0, n, chunk)]
    if len(parts) <= 1:
        for sl in parts:
            fn(sl)
        return
    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(fn, parts))


def _rotations_from(G):
    """Proper rotations from Gaussian matrices (QR with the diagonal of R made
    positive, then one column flipped where the determinant is negative)."""
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    Q = Q * d[:, None, :]
    # orientation of the orthogonal Q (det = +-1): sign of the triple product
    det = np.einsum("ni,ni->n", Q[:, :, 0], np.cross(Q[:, :, 1], Q[:, :, 2]))
    Q[det < 0, :, 0] *= -1.0  # proper rotations only
    return Q


def affine_mixture(n, seed=None, frac_degenerate=0.05, frac_inverted=0.05, r_max=1e-6):
    """Precision-stress mixture.  90%: random affine images A C + t of the unit
    cube, A = R S D (R a rotation, S unit upper triangular with U[-1,1]
    shears, D = diag(exp(ln(delta)/3 + u_i)) with centred u_i ~ U[-1,1] and
    delta log-uniform in [1e-3, 1e3]), t ~ U[-10,10]^3.  5%: the same with one
    random corner k moved, in reference space, towards the centre by
    2 s (centre - C_k), s = (1 - r)/3, r ~ U[-r_max, r_max], so that
    min J / max |J| = r.  5%: one random corner reflected, in reference space,
    through the plane of its three edge neighbours.
    Returns (corners (8,3,n) f64, kind (n,) int8: 0 affine, 1 near-degenerate,
    2 inverted, r (n,) f64 for the near-degenerate ones, else 0)."""
    rng = rng_for(3, seed)
    # every random number first, in a fixed order; then the elements chunk by
    # chunk straight into the output planes (bounded host memory)
    G = rng.normal(size=(n, 3, 3))
    shear = [rng.uniform(-1, 1, n) for _ in range(3)]
    log_delta = rng.uniform(math.log(1e-3), math.log(1e3), n)
    u = rng.uniform(-1, 1, size=(n, 3))
    t = rng.uniform(-10, 10, size=(n, 3))
    kind = np.zeros(n, np.int8)
    pick = rng.uniform(size=n)
    kind[pick < frac_degenerate + frac_inverted] = 2
    kind[pick < frac_degenerate] = 1
    corner = rng.integers(0, 8, n)
    r = np.where(kind == 1, rng.uniform(-r_max, r_max, n), 0.0)
    out = np.empty((8, 3, n))
    centre = np.full(3, 0.5)

    def chunk(sl):
        m = sl.stop - sl.start
        R = _rotations_from(G[sl])
        S = np.tile(np.eye(3), (m, 1, 1))
        S[:, 0, 1], S[:, 0, 2], S[:, 1, 2] = shear[0][sl], shear[1][sl], shear[2][sl]
        uc = u[sl] - u[sl].mean(axis=1, keepdims=True)
        D = np.exp(log_delta[sl, None] / 3.0 + uc)
        A = R @ S * D[:, None, :]
        ref = np.broadcast_to(REF_CORNERS[None], (m, 8, 3)).copy()
        kc, cc, rc = kind[sl], corner[sl], r[sl]
        idx = np.nonzero(kc == 1)[0]
        s_ = (1.0 - rc[idx]) / 3.0
        ck = REF_CORNERS[cc[idx]]
        ref[idx, cc[idx]] = ck + 2.0 * s_[:, None] * (centre - ck)
        idx = np.nonzero(kc == 2)[0]
        ck = REF_CORNERS[cc[idx]]
        # the three edge neighbours of corner C_k differ from it in one
        # coordinate; their plane is sum_d |x_d - C_kd| = 1, and the mirror
        # image of C_k in it is C_k + (4/3) (centre - C_k)
        ref[idx, cc[idx]] = ck + (4.0 / 3.0) * (centre - ck)
        X = np.einsum("nij,nkj->nki", A, ref) + t[sl, None, :]
        out[:, :, sl] = X.transpose(1, 2, 0)

    _for_chunks(chunk, n)
    return out, kind, r


def twisted_layers(n, seed=None, theta_max_deg=120.0, ar_max=1e3, noise=0.01):
    """Boundary-layer elements: bottom face (+-1/2, +-1/2, 0); top face the
    same rotated by theta ~ U[0, theta_max] about the z axis and lifted to
    z = t, t = 1/AR with AR log-uniform in [1, ar_max]; then i.i.d.
    U[-noise t, noise t] on every coordinate.  Returns (8, 3, n) f64."""
    rng = rng_for(4, seed)
    base = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
    theta = np.deg2rad(rng.uniform(0.0, theta_max_deg, n))
    t = 1.0 / np.exp(rng.uniform(0.0, math.log(ar_max), n))
    X = np.zeros((8, 3, n))
    X[0:4, 0, :] = base[:, 0:1]
    X[0:4, 1, :] = base[:, 1:2]
    cs, sn = np.cos(theta), np.sin(theta)
    X[4:8, 0, :] = base[:, 0:1] * cs - base[:, 1:2] * sn
    X[4:8, 1, :] = base[:, 0:1] * sn + base[:, 1:2] * cs
    X[4:8, 2, :] = t
    X += rng.uniform(-1.0, 1.0, size=(8, 3, n)) * (noise * t)
    return X


def soa_from_indexed(nodes, conn):
    """Gather an indexed mesh into SoA corner planes (8, 3, n)."""
    return np.ascontiguousarray(nodes[conn].transpose(1, 2, 0))


def request_stream(n_requests, seed=None, size_min=100, size_max=10_000_000):
    """Serving workload: per request a size n log-uniform in [size_min,
    size_max], a generator kind (1 perturbed cubes, 2 structured grid,
    3 affine mixture) and a per-request seed 20175000 + request id.
    Returns a list of dicts (no arrays; inputs are built on demand with
    ``request_inputs``)."""
    rng = rng_for(5, seed)
    sizes = np.exp(rng.uniform(math.log(size_min), math.log(size_max), n_requests))
    kinds = rng.integers(1, 4, n_requests)
    return [dict(id=i, size=int(sizes[i]), kind=int(kinds[i]), seed=20175000 + i)
            for i in range(n_requests)]


def request_inputs(req):
    """Inputs of one serving request: ('soa', corners) or ('indexed', nodes, conn)."""
    n, kind, seed = req["size"], req["kind"], req["seed"]
    if kind == 1:
        return ("soa", perturbed_cubes(n, seed=seed))
    if kind == 2:
        a = max(1, int(math.floor(n ** (1.0 / 3.0) + 1e-9)))
        b = max(1, -(-n // (a * a)))
        nodes, conn = structured_grid(a, a, b, seed=seed)
        return ("indexed", nodes, conn)
    X, _, _ = affine_mixture(n, seed=seed)
    return ("soa", X)


# ------------------------------------------------------------ quadrangles --
# Layouts: SoA float64 (4, 2, n) (plane [k][d] = coordinate d of node k,
# nodes 1..4 at reference (0,0), (1,0), (1,1), (0,1)); indexed: nodes
# float64 (n_nodes, 2), conn int32 (n, 4).
REF_SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)


def perturbed_squares(n, noise=0.3, seed=None):
    """Unit-square corners with every coordinate perturbed by i.i.d.
    U[-noise, noise] (seed 20170006 by default)."""
    rng = rng_for(6, seed)
    X = np.broadcast_to(REF_SQUARE[:, :, None], (4, 2, n)).copy()
    X += rng.uniform(-noise, noise, size=(4, 2, n))
    return X


def structured_grid_2d(nx=4096, ny=None, sigma=0.15, seed=None):
    """(nx+1)(ny+1) nodes of spacing 1, interior nodes displaced by i.i.d.
    N(0, sigma^2) per axis (seed 20170007 by default).  Node id i + (nx+1) j;
    quad (i, j) has index i + nx j.  Returns (nodes (n_nodes, 2) f64,
    conn (n, 4) i32)."""
    ny = nx if ny is None else ny
    rng = rng_for(7, seed)
    px, py = nx + 1, ny + 1
    j, i = np.meshgrid(np.arange(py), np.arange(px), indexing="ij")
    nodes = np.stack([i, j], axis=-1).reshape(-1, 2).astype(np.float64)
    disp = rng.normal(0.0, sigma, size=nodes.shape)
    ii, jj = i.reshape(-1), j.reshape(-1)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    nodes[interior] += disp[interior]
    qj, qi = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    qi, qj = qi.reshape(-1), qj.reshape(-1)
    conn = np.stack([qi + px * qj, qi + 1 + px * qj, qi + 1 + px * (qj + 1), qi + px * (qj + 1)],
                    axis=1).astype(np.int32)
    return nodes, conn


# ------------------------------------------------------ candidate sets ------

def cube_symmetries():
    """The 48 symmetries of the reference cube as permutations of the corner
    labels (Appendix A order), with +1 for the 24 rotations and -1 for the 24
    orientation-reversing ones.  Returns (perm (48, 8) int, sign (48,) int)."""
    import itertools
    ref = REF_CORNERS - 0.5
    perms, signs = [], []
    for p in itertools.permutations(range(3)):
        for s in itertools.product((1.0, -1.0), repeat=3):
            S = np.zeros((3, 3))
            for i in range(3):
                S[i, p[i]] = s[i]
            img = ref @ S.T
            perm = [int(np.nonzero(np.all(np.isclose(ref, img[k]), axis=1))[0][0]) for k in range(8)]
            perms.append(perm)
            signs.append(int(round(np.linalg.det(S))))
    return np.array(perms), np.array(signs)


def hex_candidates(nx=64, per_node=40, sigma=0.15, seed=None):
    """A candidate set over one node array, the shape of indirect hex-dominant
    meshing input (many more candidates than vertices): the nodes of an
    (nx+1)^3 structured grid with N(0, sigma^2) interior noise, and
    per_node x n_nodes candidate hexahedra, each a random cell of the grid
    with its corners relabelled by a random cube symmetry (a rotation keeps
    the cell's validity, a reflection inverts it).  Seed 20170008 by default.
    Returns (nodes, conn (n_cand, 8) int32, cell (n_cand,), sym (n_cand,))."""
    nodes, cells = structured_grid(nx, sigma=sigma, seed=(SEED_BASE + 8) if seed is None else seed)
    rng = rng_for(8, seed)
    n = per_node * nodes.shape[0]
    cell = rng.integers(0, cells.shape[0], size=n)
    sym = rng.integers(0, 48, size=n)
    perm, _ = cube_symmetries()
    conn = np.take_along_axis(cells[cell], perm[sym], axis=1).astype(np.int32)
    return nodes, conn, cell, sym
