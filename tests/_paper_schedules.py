"""Emulations of the paper's Hierarchy-Scan schedules (test helpers).

Each routine runs one of the paper's per-joint parallel algorithms on the
CPU, with every "for all jointID in parallel" step done as a phase that reads
the values of the previous phase (double buffering) and every barrier
counted.  They compose general 4x4 matrices with numpy and count the
products each joint's thread performs, so the oracle's sequential traversal
can be checked against schedules written from a different description of
the same product (Eq. 1), and the paper's operation counts can be checked.

Readings of the garbled listings (Sec. 2 Alg. 1; Sec. 3.1 Alg. 2 and Eq. 2;
Sec. 3.2.1 Alg. 3; Sec. 3.2.2 Alg. 4):
  * Alg. 1 advances to the parent of the current ancestor and multiplies the
    ancestors' LOCAL matrices into a separate result.
  * Alg. 2 round d multiplies by the 2^(d-1)-th ancestor's running product.
  * MaxParentOutBlock(i) is the nearest ancestor of i outside i's 64-node
    block; the out-of-block loop walks it repeatedly, multiplying that
    ancestor's in-block partial product.
  * Alg. 4 takes a node plus up to 7 ancestors serially, then up to 7 jumps
    of stride 8 (the 8th in-block ancestor), then the out-of-block walk.
"""
import numpy as np


def _h(A):
    """3x4 -> 4x4 homogeneous."""
    H = np.zeros(A.shape[:-2] + (4, 4))
    H[..., :3, :] = A
    H[..., 3, 3] = 1
    return H


def depths(parents):
    d = np.zeros(len(parents), int)
    for i, p in enumerate(parents):
        d[i] = 1 if p < 0 else d[p] + 1
    return d


def alg1_gateau(parents, L):
    """One thread per joint walks to the root multiplying local matrices."""
    Lh = _h(L)
    n = len(parents)
    out = np.empty_like(Lh)
    prods = np.zeros(n, int)
    for j in range(n):
        m = Lh[j].copy()
        a = parents[j]
        while a >= 0:
            m = Lh[a] @ m
            prods[j] += 1
            a = parents[a]
        out[j] = m
    return out[:, :3, :], prods


def alg2_jump(parents, L):
    """Pointer jumping: round d multiplies by the 2^(d-1)-th ancestor."""
    n = len(parents)
    M = _h(L)
    anc = np.array(parents, int)
    rounds = 0
    prods = np.zeros(n, int)
    D = depths(parents).max() if n else 0
    R = int(np.ceil(np.log2(D))) if D > 1 else 0
    for _ in range(R):
        M2, anc2 = M.copy(), anc.copy()
        for j in range(n):
            a = anc[j]
            if a >= 0:
                M2[j] = M[a] @ M[j]
                anc2[j] = anc[a]
                prods[j] += 1
        M, anc = M2, anc2
        rounds += 1
    return M[:, :3, :], prods, rounds


def _blocks(parents, B):
    n = len(parents)
    blk = np.arange(n) // B
    inb_par = np.array([p if (p >= 0 and blk[p] == blk[i]) else -1 for i, p in enumerate(parents)])
    # nearest ancestor outside the block = parent of the block-local root
    out_par = np.full(n, -1)
    for i in range(n):
        r = i
        while inb_par[r] >= 0:
            r = inb_par[r]
        out_par[i] = parents[r]
    return inb_par, out_par


def _out_walk(M_in, out_par, prods):
    n = len(out_par)
    M = M_in.copy()
    for j in range(n):
        a = out_par[j]
        while a >= 0:
            M[j] = M_in[a] @ M[j]
            prods[j] += 1
            a = out_par[a]
    return M


def alg3_blocks(parents, L, B=64):
    """6 in-block jump rounds (log2 64), a barrier after each, then the
    out-of-block walk over block-exit ancestors."""
    n = len(parents)
    inb_par, out_par = _blocks(parents, B)
    M = _h(L)
    anc = inb_par.copy()
    prods = np.zeros(n, int)
    barriers = 0
    for _ in range(int(np.log2(B))):
        M2, anc2 = M.copy(), anc.copy()
        for j in range(n):
            a = anc[j]
            if a >= 0:
                M2[j] = M[a] @ M[j]
                anc2[j] = anc[a]
                prods[j] += 1
        M, anc = M2, anc2
        barriers += 1
    M = _out_walk(M, out_par, prods)
    return M[:, :3, :], prods, barriers


def alg4_compress(parents, L, B=64, S=8):
    """State compression: each thread multiplies up to S-1 in-block
    ancestors serially, barrier, up to S-1 jumps of stride S over the
    in-block partial products, barrier, then the out-of-block walk."""
    n = len(parents)
    inb_par, out_par = _blocks(parents, B)
    Lh = _h(L)
    prods = np.zeros(n, int)
    M1 = Lh.copy()
    far = np.empty(n, int)  # S-th in-block ancestor
    for j in range(n):
        a = inb_par[j]
        k = 0
        while a >= 0 and k < S - 1:
            M1[j] = Lh[a] @ M1[j]
            prods[j] += 1
            a = inb_par[a]
            k += 1
        far[j] = a  # in-block ancestor S levels up (or -1)
    barriers = 1
    M2 = M1.copy()
    for j in range(n):
        a = far[j]
        k = 0
        while a >= 0 and k < S - 1:
            M2[j] = M1[a] @ M2[j]
            prods[j] += 1
            a = far[a]
            k += 1
    barriers += 1
    M = _out_walk(M2, out_par, prods)
    return M[:, :3, :], prods, barriers
