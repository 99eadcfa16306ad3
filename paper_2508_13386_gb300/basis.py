"""Host-side construction of the sparse material-aware (SMS) basis.

This is the untimed precompute whose output the library uploads with
``mls_upload_basis``.  It follows the paper's construction:

1. Partitioning (Sec. 3.6): K-means by Lloyd relaxation under a stiffness-
   weighted geodesic distance, seeded by kmeans++ with the same distance;
   elements touching a material boundary get a small "jump penalty"
   stiffness (0.1-0.5 x the softest material, Sec. 3.6.2; 0.25 here), and
   every 10 iterations clusters whose volume is below median/1.75 become
   candidates and the 5 smallest are deleted (Sec. 3.6.3), starting from a
   denser sampling of 1.25 x the target handle count.
   Distances: the paper uses heat-method geodesics with a stiffness-weighted
   Laplacian (diffusion coefficient ~ stiffness).  Heat travel time over an
   edge of length l with diffusivity k scales as l^2 / k, i.e. the metric is
   ds / sqrt(k).  Two realisations of that metric: the default computes its
   graph geodesic on the tet edge graph (multi-source Dijkstra), which gives
   the labels of a whole Lloyd assignment step in one pass; ``distance="heat"``
   uses the heat method itself (``HeatDistance``: heat flow with the
   stiffness-weighted Laplacian, then a Poisson fit to the unit flow direction
   scaled by the slowness 1/sqrt(k)), one pair of sparse solves per centre.
2. Handles (Sec. 3.5): one per partition, at the mesh vertex of the partition
   nearest its volume-weighted centroid.
3. Weights (Sec. 3.5): for partition i, the subdomain T_i is the partition
   plus its face-sharing neighbour partitions; solve K u = 0 on T_i with
   K = L_E^T M^{-1} L_E (stiffness-weighted bilaplacian; L_E the P1 stiffness
   matrix with per-tet weight E_e / E_min, M the lumped volume mass), with
   u = 1 at the own handle vertex, u = 0 at neighbour handle vertices, u = 0
   on the internal boundary of T_i (boundary of T_i that is not boundary of
   the mesh) and, with Dirichlet conditions, u = 0 at Dirichlet vertices.
   Clip u_pos = max(u, 0).
4. Dirichlet basis (Sec. 3.5.1): u_DBC solved the same way on the partitions
   holding Dirichlet vertices and their neighbours, u = 1 at Dirichlet
   vertices and u = 0 at those partitions' handle vertices.
5. Partition of unity: phi_i = u_pos,i / (sum_j u_pos,j + u_DBC).  A vertex
   with a zero denominator takes phi = 1 for its own partition's handle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

JUMP_PENALTY = 0.25
PRUNE_RATIO = 1.75
PRUNE_EVERY = 10
PRUNE_COUNT = 5
OVERSAMPLE = 1.25


def _rest(X, tets):
    D = np.stack([X[tets[:, k]] - X[tets[:, 0]] for k in (1, 2, 3)], axis=-1)
    vol = np.linalg.det(D) / 6.0
    Dinv = np.linalg.inv(D)
    return vol, Dinv


def _edges(tets):
    pairs = np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)], axis=0)
    pairs.sort(axis=1)
    return pairs


def stiffness_weights(tets, E, jump=JUMP_PENALTY):
    """Per-tet relative stiffness E_e / E_min, with the jump penalty applied to
    tets incident to a vertex that touches more than one material."""
    E = np.asarray(E, dtype=np.float64)
    n = int(tets.max()) + 1
    emin = np.full(n, np.inf)
    emax = np.full(n, -np.inf)
    np.minimum.at(emin, tets.ravel(), np.repeat(E, 4))
    np.maximum.at(emax, tets.ravel(), np.repeat(E, 4))
    mixed_v = emax > emin * (1 + 1e-12)
    w = E / E.min()
    w_geo = w.copy()
    w_geo[mixed_v[tets].any(axis=1)] = jump
    return w, w_geo


def geodesic_graph(X, tets, w_geo):
    """Edge graph with lengths l / sqrt(k_edge), k_edge the mean weight of the
    tets containing the edge."""
    n = X.shape[0]
    pairs = _edges(tets)
    kw = np.tile(w_geo, 6)
    key = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
    uk, inv = np.unique(key, return_inverse=True)
    ksum = np.bincount(inv, weights=kw)
    kcnt = np.bincount(inv)
    i = (uk // n).astype(np.int64)
    j = (uk % n).astype(np.int64)
    length = np.linalg.norm(X[i] - X[j], axis=1) / np.sqrt(ksum / kcnt)
    G = sp.coo_matrix((np.concatenate([length, length]), (np.concatenate([i, j]), np.concatenate([j, i]))),
                      shape=(n, n)).tocsr()
    return G


class HeatDistance:
    """Heat-method geodesic distances (Sec. 3.6, after Crane et al.'s heat
    method) for the stiffness metric ds / sqrt(k) that ``geodesic_graph``
    uses on edges.

    For a source vertex s:
      1. heat flow: (M + t L_k) u = e_s, with L_k the P1 stiffness matrix
         weighted by k (diffusion faster in stiff tets), M the lumped volume
         mass, t = (mean edge length)^2;
      2. per tet, the unit direction X = -grad u / |grad u|, scaled by the
         local slowness: Y = X / sqrt(k);
      3. Poisson: the phi whose gradient fits Y in the k-weighted least-squares
         sense, L_k phi = sum_e k_e vol_e G_e^T Y_e (G_e the P1 gradients);
      4. shift so that phi(s) = 0 and clip at 0.
    Step 3 fixes phi up to one constant per connected piece of the mesh; one
    vertex per piece is pinned, and the shift of step 4 removes the constant
    of the source's piece (vertices in other pieces get +inf).  Both systems
    are factored once; sources are solved in chunks of ``chunk`` right-hand
    sides."""

    def __init__(self, X, tets, w_geo, chunk=16):
        X = np.asarray(X, dtype=np.float64)
        tets = np.asarray(tets, dtype=np.int64)
        self.n = n = X.shape[0]
        self.tets = tets
        vol, Dinv = _rest(X, tets)
        self.grads = np.concatenate([-Dinv.sum(axis=1, keepdims=True), Dinv], axis=1)   # [t, 4, 3]
        self.w = np.asarray(w_geo, dtype=np.float64)
        self.kvol = self.w * vol
        L, Mv = p1_stiffness(X, tets, self.w)
        pairs = _edges(tets)
        t_heat = float(np.mean(np.linalg.norm(X[pairs[:, 0]] - X[pairs[:, 1]], axis=1))) ** 2
        self.heat = spla.splu((sp.diags(Mv) + t_heat * L).tocsc())
        adj = sp.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
        _, self.piece = csg.connected_components(adj, directed=False)
        first = np.unique(self.piece, return_index=True)[1]
        self.free = np.setdiff1d(np.arange(n), first)
        self.poisson = spla.splu(L[self.free][:, self.free].tocsc())
        self.chunk = chunk

    def __call__(self, sources):
        """Distances [n, len(sources)] from each source vertex."""
        sources = np.atleast_1d(np.asarray(sources, dtype=np.int64))
        out = np.empty((self.n, len(sources)))
        for c0 in range(0, len(sources), self.chunk):
            src = sources[c0:c0 + self.chunk]
            rhs = np.zeros((self.n, len(src)))
            rhs[src, np.arange(len(src))] = 1.0
            u = self.heat.solve(rhs)                                           # [n, c]
            gu = np.einsum("tac,tas->tcs", self.grads, u[self.tets])           # [t, 3, c]
            mag = np.linalg.norm(gu, axis=1, keepdims=True)
            Y = -gu / np.where(mag > 0, mag, 1.0) / np.sqrt(self.w)[:, None, None]
            nodal = np.einsum("tac,tcs->tas", self.grads, Y) * self.kvol[:, None, None]
            b = np.zeros((self.n, len(src)))
            np.add.at(b, self.tets.ravel(), nodal.reshape(-1, len(src)))
            phi = np.zeros((self.n, len(src)))
            phi[self.free] = self.poisson.solve(np.ascontiguousarray(b[self.free]))
            phi -= phi[src, np.arange(len(src))][None, :]
            phi = np.maximum(phi, 0.0)
            phi[self.piece[:, None] != self.piece[src][None, :]] = np.inf
            out[:, c0:c0 + len(src)] = phi
        return out


def _vertex_volume(n, tets, vol):
    vv = np.zeros(n)
    np.add.at(vv, tets.ravel(), np.repeat(vol / 4.0, 4))
    return vv


def kmeans_partition(X, tets, E, m_target, seed=0, max_iter=40, distance="graph"):
    """Stiffness-aware geodesic K-means on vertices; returns vertex labels
    (0..k-1) and the centre vertex of each cluster.  ``distance``: "graph"
    (edge-graph geodesics of the metric ds / sqrt(k), the default) or "heat"
    (heat-method geodesics of the same metric, ``HeatDistance``)."""
    n = X.shape[0]
    vol, _ = _rest(X, tets)
    vv = _vertex_volume(n, tets, vol)
    _, w_geo = stiffness_weights(tets, E)
    if distance == "graph":
        G = geodesic_graph(X, tets, w_geo)
    elif distance == "heat":
        heat = HeatDistance(X, tets, w_geo)
    else:
        raise ValueError(f"unknown distance {distance!r}")

    def nearest(centers):
        """Index into ``centers`` of each vertex's nearest centre (-1: unreachable)."""
        if distance == "graph":
            _, _, src = csg.dijkstra(G, indices=centers, min_only=True, return_predecessors=True)
            pos = {int(c): k for k, c in enumerate(centers)}
            return np.array([pos.get(int(s), -1) for s in src])
        best = np.full(n, np.inf)
        lab = np.full(n, -1)
        for c0 in range(0, len(centers), heat.chunk):
            D = heat(centers[c0:c0 + heat.chunk])
            j = np.argmin(D, axis=1)
            d = D[np.arange(n), j]
            better = d < best
            best[better] = d[better]
            lab[better] = c0 + j[better]
        return lab

    rng = np.random.default_rng(seed)
    k0 = int(np.ceil(OVERSAMPLE * m_target))
    k0 = max(1, min(k0, n))
    # kmeans++ seeding with the same distance
    centers = [int(rng.integers(n))]
    D = csg.dijkstra(G, indices=centers[0]) if distance == "graph" else heat([centers[0]])[:, 0]
    for _ in range(1, k0):
        p = vv * D ** 2
        s = p.sum()
        if not np.isfinite(s) or s <= 0:
            break
        c = int(rng.choice(n, p=p / s))
        centers.append(c)
        if distance == "graph":
            D = np.minimum(D, csg.dijkstra(G, indices=c, limit=float(D.max())))
        else:
            D = np.minimum(D, heat([c])[:, 0])
    centers = np.array(centers)
    labels = None
    for it in range(max_iter):
        new_labels = nearest(centers)
        # unreachable vertices (disconnected pieces) join the nearest centre in space
        bad = new_labels < 0
        if bad.any():
            d2 = ((X[bad, None, :] - X[centers][None, :, :]) ** 2).sum(-1)
            new_labels[bad] = np.argmin(d2, axis=1)
        k = len(centers)
        cvol = np.bincount(new_labels, weights=vv, minlength=k)
        # pruning of small clusters
        if (it + 1) % PRUNE_EVERY == 0 and k > m_target:
            med = np.median(cvol)
            cand = np.nonzero(med / np.maximum(cvol, 1e-300) > PRUNE_RATIO)[0]
            if len(cand):
                drop = cand[np.argsort(cvol[cand])][:min(PRUNE_COUNT, k - m_target)]
                keep = np.setdiff1d(np.arange(k), drop)
                centers = centers[keep]
                labels = None
                continue
        # centre update: vertex of the cluster nearest its volume-weighted centroid
        new_centers = centers.copy()
        for c in range(k):
            idx = np.nonzero(new_labels == c)[0]
            if len(idx) == 0:
                continue
            g = (vv[idx, None] * X[idx]).sum(0) / vv[idx].sum()
            new_centers[c] = idx[np.argmin(((X[idx] - g) ** 2).sum(1))]
        converged = labels is not None and np.array_equal(new_labels, labels) and \
            np.array_equal(new_centers, centers)
        labels = new_labels
        centers = new_centers
        if converged:
            break
    if labels is None:
        labels = np.maximum(nearest(centers), 0)
    # while the sampling is still denser than the target, merge the smallest
    # clusters into their neighbours by dropping their centres
    while len(centers) > m_target:
        k = len(centers)
        cvol = np.bincount(labels, weights=vv, minlength=k)
        drop = np.argsort(cvol)[:min(PRUNE_COUNT, k - m_target)]
        centers = np.delete(centers, drop)
        labels = np.maximum(nearest(centers), 0)
    return labels, centers


def tet_partition(tets, vlabels):
    """Partition of tets: the label held by most of a tet's vertices (ties:
    the smallest label)."""
    L = np.sort(vlabels[tets], axis=1)
    cnt = (L[:, :, None] == L[:, None, :]).sum(axis=2)     # multiplicity of each entry
    best = cnt.max(axis=1, keepdims=True)
    cand = np.where(cnt == best, L, np.iinfo(np.int64).max)
    return cand.min(axis=1)


def _faces(tets):
    f = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0)
    owner = np.tile(np.arange(len(tets)), 4)
    fs = np.sort(f, axis=1)
    return fs, owner


def face_structure(tets):
    """Interior face pairs (tet a, tet b) and boundary faces of the mesh."""
    fs, owner = _faces(tets)
    n = int(tets.max()) + 1
    key = (fs[:, 0].astype(np.int64) * n + fs[:, 1]) * n + fs[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    interior = np.stack([owner[order[same]], owner[order[same + 1]]], axis=1)
    counts = np.bincount(np.unique(ks, return_inverse=True)[1])
    uniq_first = np.unique(ks, return_index=True)[1]
    bmask = counts == 1
    boundary = fs[order[uniq_first[bmask]]]
    return interior, boundary


def p1_stiffness(X, tets, weight):
    """Weighted P1 stiffness matrix L_ij = sum_e w_e vol_e grad(phi_i).grad(phi_j)
    (positive semi-definite) and the lumped volume mass."""
    n = X.shape[0]
    vol, Dinv = _rest(X, tets)
    grads = np.concatenate([-Dinv.sum(axis=1, keepdims=True), Dinv], axis=1)  # [t,4,3]
    Ke = (weight * vol)[:, None, None] * np.einsum("tac,tbc->tab", grads, grads)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    L = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    M = _vertex_volume(n, tets, vol)
    return L, M


def _biharmonic(X, sub_tets, weight, dir_idx, dir_val):
    """Solve L^T M^{-1} L u = 0 on the sub-mesh with Dirichlet values; returns
    u on the sub-mesh vertices (global indices of sub_tets' vertices)."""
    verts, local = np.unique(sub_tets, return_inverse=True)
    lt = local.reshape(-1, 4)
    return verts, _biharmonic_local(X[verts], lt, weight, verts, dir_idx, dir_val)


def _biharmonic_job(args):
    return _biharmonic_local(*args)


def _biharmonic_local(Xl, lt, weight, verts, dir_idx, dir_val):
    L, M = p1_stiffness(Xl, lt, weight)
    K = (L.T @ sp.diags(1.0 / M) @ L).tocsr()
    nl = len(verts)
    gl = {int(g): i for i, g in enumerate(verts)}
    d_local = np.array([gl[int(g)] for g in dir_idx if int(g) in gl], dtype=np.int64)
    d_vals = np.array([v for g, v in zip(dir_idx, dir_val) if int(g) in gl], dtype=np.float64)
    u = np.zeros(nl)
    if len(d_local):
        d_local, first = np.unique(d_local, return_index=True)
        d_vals = d_vals[first]
        u[d_local] = d_vals
    free = np.setdiff1d(np.arange(nl), d_local)
    if len(free):
        Kff = K[free][:, free]
        rhs = -(K[free][:, d_local] @ u[d_local]) if len(d_local) else np.zeros(len(free))
        reg = 1e-12 * abs(Kff.diagonal()).max()
        lu = spla.splu((Kff + reg * sp.eye(len(free))).tocsc(), permc_spec="MMD_AT_PLUS_A",
                       diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
        u[free] = lu.solve(rhs)
    return u


def _run_jobs(jobs, workers):
    """Run the subdomain solves, in a spawned process pool when ``workers`` > 1
    (spawn, so that it is safe in a process that already uses CUDA)."""
    if workers is None:
        import os
        workers = min(16, os.cpu_count() or 1) if len(jobs) >= 16 else 1
    if workers <= 1:
        return [_biharmonic_job(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_biharmonic_job, jobs, chunksize=max(1, len(jobs) // (4 * workers)))


def build_sms_basis(X, tets, E, m_target, dirichlet=None, seed=0, workers=None, distance="graph"):
    """Build the SMS basis.  Returns a dict with ``origins`` [m,3], per-vertex
    CSR ``vrow``/``handle``/``phi``, the vertex ``labels`` and tet
    ``partition`` used, and ``u_dbc`` (per-vertex Dirichlet weight, zeros
    without Dirichlet vertices).  ``distance`` selects the K-means distance
    ("graph" or "heat", see ``kmeans_partition``)."""
    X = np.asarray(X, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    n = X.shape[0]
    pinned = np.zeros(n, bool) if dirichlet is None else np.asarray(dirichlet).astype(bool)
    vlabels, _ = kmeans_partition(X, tets, E, m_target, seed=seed, distance=distance)
    part = tet_partition(tets, vlabels)
    used = np.unique(part)
    remap = -np.ones(part.max() + 1, dtype=np.int64)
    remap[used] = np.arange(len(used))
    part = remap[part]
    m = len(used)
    vol, _ = _rest(X, tets)
    w, _ = stiffness_weights(tets, E)
    # handle vertex per partition: vertex of the partition nearest its centroid
    centroid_tet = X[tets].mean(axis=1)
    hv = np.zeros(m, dtype=np.int64)
    for i in range(m):
        sel = np.nonzero(part == i)[0]
        g = (vol[sel, None] * centroid_tet[sel]).sum(0) / vol[sel].sum()
        cand = np.unique(tets[sel])
        hv[i] = cand[np.argmin(((X[cand] - g) ** 2).sum(1))]
    origins = X[hv].copy()
    # partition adjacency through shared faces
    interior, boundary = face_structure(tets)
    pa, pb = part[interior[:, 0]], part[interior[:, 1]]
    cross = pa != pb
    nb_sets = [set() for _ in range(m)]
    for a, b in zip(pa[cross], pb[cross]):
        nb_sets[a].add(int(b))
        nb_sets[b].add(int(a))
    bnd_key = set(map(tuple, np.sort(boundary, axis=1).tolist()))
    fs_all, owner_all = _faces(tets)
    # per-handle clipped weights (subdomain problems are independent)
    jobs = []
    for i in range(m):
        sub_parts = [i] + sorted(nb_sets[i])
        sub_mask = np.isin(part, sub_parts)
        sub = np.nonzero(sub_mask)[0]
        sub_tets = tets[sub]
        # internal boundary of T_i: faces of T_i seen once inside T_i but not on the mesh boundary
        fsel = sub_mask[owner_all]
        fs = fs_all[fsel]
        keys, cnt = np.unique(fs, axis=0, return_counts=True)
        ib = [f for f, c in zip(keys.tolist(), cnt) if c == 1 and tuple(f) not in bnd_key]
        ib_verts = np.unique(np.array(ib, dtype=np.int64)) if ib else np.zeros(0, np.int64)
        dir_idx = [hv[i]] + [hv[j] for j in nb_sets[i]]
        dir_val = [1.0] + [0.0] * len(nb_sets[i])
        extra = np.setdiff1d(ib_verts, np.array(dir_idx))
        extra = np.concatenate([extra, np.nonzero(pinned)[0]])
        extra = np.setdiff1d(extra, np.array([hv[i]]))
        dir_idx = dir_idx + extra.tolist()
        dir_val = dir_val + [0.0] * len(extra)
        verts, local = np.unique(sub_tets, return_inverse=True)
        jobs.append((X[verts], local.reshape(-1, 4), w[sub], verts, dir_idx, dir_val))
    results = _run_jobs(jobs, workers)
    upos = []  # (verts, values)
    for job, u in zip(jobs, results):
        u = np.maximum(u, 0.0)
        keep = u > 0
        upos.append((job[3][keep], u[keep]))
    # Dirichlet basis
    u_dbc = np.zeros(n)
    if pinned.any():
        dparts = sorted(set(part[np.isin(tets, np.nonzero(pinned)[0]).any(axis=1)].tolist()))
        region = set(dparts)
        for i in dparts:
            region |= nb_sets[i]
        sub_mask = np.isin(part, sorted(region))
        sub_tets = tets[sub_mask]
        fsel = sub_mask[owner_all]
        keys, cnt = np.unique(fs_all[fsel], axis=0, return_counts=True)
        ib = [f for f, c in zip(keys.tolist(), cnt) if c == 1 and tuple(f) not in bnd_key]
        ib_verts = np.unique(np.array(ib, dtype=np.int64)) if ib else np.zeros(0, np.int64)
        pin_idx = np.nonzero(pinned)[0]
        zero_idx = np.setdiff1d(np.concatenate([hv[dparts], ib_verts]), pin_idx)
        verts, u = _biharmonic(X, sub_tets, w[sub_mask], pin_idx.tolist() + zero_idx.tolist(),
                               [1.0] * len(pin_idx) + [0.0] * len(zero_idx))
        u_dbc[verts] = np.maximum(u, 0.0)
        u_dbc[pin_idx] = 1.0
    # partition of unity
    denom = u_dbc.copy()
    for verts, vals in upos:
        np.add.at(denom, verts, vals)
    rows, cols, vals = [], [], []
    for i, (verts, u) in enumerate(upos):
        ok = denom[verts] > 0
        rows.append(verts[ok])
        cols.append(np.full(ok.sum(), i))
        vals.append(u[ok] / denom[verts[ok]])
    zero = np.nonzero(denom <= 0)[0]
    if len(zero):
        rows.append(zero)
        cols.append(vlabels_to_part(zero, tets, part))
        vals.append(np.ones(len(zero)))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    vrow = np.zeros(n + 1, dtype=np.int32)
    np.add.at(vrow, rows + 1, 1)
    vrow = np.cumsum(vrow).astype(np.int32)
    phi_dbc = np.where(denom > 0, u_dbc / np.where(denom > 0, denom, 1.0), 0.0)
    supports = [verts for verts, _ in upos]
    return {"origins": origins, "vrow": vrow, "handle": cols.astype(np.int32), "phi": vals,
            "labels": vlabels, "partition": part, "handle_vertex": hv, "u_dbc": u_dbc,
            "phi_dbc": phi_dbc, "neighbours": [sorted(s) for s in nb_sets], "supports": supports}


def refinement_cg_iterations(tets, partition, handle_vertex):
    """The refinement's CG count (Sec. 3.7.2): for each partition, the largest
    number of mesh-edge hops from its handle vertex (the vertex nearest its
    centroid) to a vertex of the partition, the path running through the
    partition's own tets; the mean over partitions; and the fixed count of
    full-space CG iterations, 20 or 40, whichever is nearer that mean.
    Vertices that the partition's tets do not connect to the handle vertex
    are left out.  Returns (mean hops, per-partition hops, 20 or 40)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    tets = np.asarray(tets, dtype=np.int64)
    partition = np.asarray(partition, dtype=np.int64)
    hops = []
    for i, hv in enumerate(np.asarray(handle_vertex, dtype=np.int64)):
        sub = tets[partition == i]
        if len(sub) == 0:
            continue
        verts, local = np.unique(sub, return_inverse=True)
        lt = local.reshape(-1, 4)
        a = np.concatenate([lt[:, p] for p in range(4) for q in range(4) if p != q])
        b = np.concatenate([lt[:, q] for p in range(4) for q in range(4) if p != q])
        G = sp.coo_matrix((np.ones(len(a)), (a, b)), shape=(len(verts), len(verts))).tocsr()
        src = np.searchsorted(verts, hv)
        if src >= len(verts) or verts[src] != hv:
            continue
        d = shortest_path(G, unweighted=True, indices=src)
        hops.append(int(np.max(d[np.isfinite(d)])))
    mean = float(np.mean(hops)) if hops else 0.0
    return mean, hops, (20 if abs(mean - 20) <= abs(mean - 40) else 40)


def vlabels_to_part(verts, tets, part):
    """Partition of some tet containing each vertex (first such tet)."""
    n = int(tets.max()) + 1
    first = np.full(n, -1, dtype=np.int64)
    for e in range(len(tets) - 1, -1, -1):
        first[tets[e]] = e
    return part[first[verts]]


def affine_basis(X, dirichlet=None):
    """Per-object affine handle at the centre of mass with phi = 1 (Sec. 3.4);
    with Dirichlet vertices the weight is zero there (those DOFs are fixed)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    pinned = np.zeros(n, bool) if dirichlet is None else np.asarray(dirichlet).astype(bool)
    origins = X.mean(axis=0, keepdims=True)
    phi = np.where(pinned, 0.0, 1.0)
    return {"origins": origins, "vrow": np.arange(n + 1, dtype=np.int32),
            "handle": np.zeros(n, dtype=np.int32), "phi": phi}
