"""Quadtree over the inclusion grid, near lists and proxy circles (paper
Sec. 3: each Gamma_j is a leaf cell; Sec. 4: the near field of a cell is its
edge-adjacent neighbours; Sec. 4.4: cells indexed along the Morton Z-order).

Choices where the paper is silent:
  * inclusion j sits in grid cell (ix, iy) = round((c_j - origin) / spacing),
    origin = the smallest centre coordinates; the grid is padded to
    2^L x 2^L, L = ceil(log2(max(nx, ny))); empty boxes are dropped;
  * a level-l box has centre origin + spacing (b 2^(L-l) + (2^(L-l) - 1)/2);
  * spacing 0 (an arbitrary arrangement, Sec. 4.4's general layouts): the
    quadtree of the centres' bounding square, deep enough for one centre per
    cell (auto_cells); a leaf's centre is its inclusion's centre, a parent's
    the centre of its cell;
  * r_cell = largest distance from the box centre to any node of the box's
    inclusions; the proxy circle has radius R_p = f r_cell (f = 1.5) and p
    equispaced points, p = opts["proxy_points"] if positive, otherwise
    p = max(32, 8 ceil((2 k0 R_p + c)/8)), c = ceil(ln(1/tol)/ln f); with
    opts["proxy_scale"] = s != 1 the count is max(16, 8 ceil(s p / 8)) (the
    rule's count stays in box["p_rule"]);
  * near(b) = edge-adjacent boxes of the same level, plus every box that has a
    node closer than R_p to b's centre (so all far nodes lie outside the
    proxy circle), in Morton order;
  * levels L, L-1, ..., 1 are compressed; level 0 is the top dense system.

Pinned by tests/test_oracle_tree.py (Morton order, near lists of a regular
grid against hand-counted neighbours, proxy validity).
"""
import math

import numpy as np


def morton(bx, by):
    code = 0
    for b in range(32):
        code |= ((bx >> b) & 1) << (2 * b)
        code |= ((by >> b) & 1) << (2 * b + 1)
    return code


def auto_cells(cent):
    """Cells of an arbitrary arrangement (spacing 0): the bounding square of the
    centres (side E, the larger extent, widened by a factor 1 + 2^-30) in
    2^L x 2^L cells, L the smallest depth (up to 20) at which no two centres
    share a cell; cell indices floor((c - origin) / (E / 2^L))."""
    origin = cent.min(0)
    ext = float(np.max(cent.max(0) - origin))
    if len(cent) == 1 or ext == 0.0:
        return origin, 1.0, 0, np.zeros((len(cent), 2), dtype=np.int64)
    side = ext * (1.0 + 2.0 ** -30)
    for L in range(1, 21):
        cell = side / (1 << L)
        ij = np.floor((cent - origin) / cell).astype(np.int64)
        if len({(int(a), int(b)) for a, b in ij}) == len(ij):
            return origin, cell, L, ij
    raise ValueError("inclusion centres too close to separate")


def build(prob, nds, opts):
    cent = np.array([[inc["cx"], inc["cy"]] for inc in prob["inclusions"]])
    s = float(prob["spacing"])
    general = s == 0.0      # arbitrary arrangement: quadtree over the centres' bounding square
    if general:
        origin, s, L, ij = auto_cells(cent)
    else:
        origin = cent.min(0)
        ij = np.rint((cent - origin) / s).astype(np.int64)
        if len({(int(a), int(b)) for a, b in ij}) != len(ij):
            raise ValueError("two inclusions share a grid cell")
        side = int(ij.max()) + 1
        L = 0 if side <= 1 else int(math.ceil(math.log2(side)))
    factor = float(opts.get("proxy_factor", 1.5))
    tol = float(opts["tol"])
    k0 = float(opts.get("k_rule", prob["k_out"]))   # the largest wavenumber the proxies must resolve
    levels = {}
    # leaves
    keys = [(int(a), int(b)) for a, b in ij]
    order = sorted(range(len(keys)), key=lambda j: morton(*keys[j]))
    levels[L] = [{"key": keys[j], "leaves": [j], "children": []} for j in order]
    for lev in range(L - 1, -1, -1):
        parents = {}
        for ci, ch in enumerate(levels[lev + 1]):
            pk = (ch["key"][0] >> 1, ch["key"][1] >> 1)
            parents.setdefault(pk, []).append(ci)
        boxes = []
        for pk in sorted(parents, key=lambda k: morton(*k)):
            kids = parents[pk]
            leaves = [j for c in kids for j in levels[lev + 1][c]["leaves"]]
            boxes.append({"key": pk, "leaves": leaves, "children": kids})
        levels[lev] = boxes
    ctol = math.ceil(math.log(1.0 / tol) / math.log(factor))
    for lev, boxes in levels.items():
        scale = 2 ** (L - lev)
        for b in boxes:
            if not general:
                c = origin + s * (np.array(b["key"], dtype=np.float64) * scale + (scale - 1) / 2.0)
            elif lev == L:
                c = cent[b["leaves"][0]].copy()     # a leaf's proxy circle around its inclusion
            else:
                c = origin + s * (np.array(b["key"], dtype=np.float64) * scale + scale / 2.0)
            pts = np.concatenate([nds[j]["x"] for j in b["leaves"]])
            b["center"] = c
            b["r_cell"] = float(np.max(np.hypot(*(pts - c).T)))
            b["R_p"] = factor * b["r_cell"]
            pp = int(opts.get("proxy_points", 0) or 0)
            if pp <= 0:
                pp = max(32, 8 * math.ceil((2 * k0 * b["R_p"] + ctol) / 8))
                b["p_rule"] = pp
                pscale = float(opts.get("proxy_scale", 1.0) or 1.0)
                if pscale != 1.0:
                    pp = max(16, 8 * math.ceil(pscale * pp / 8))
            else:
                b["p_rule"] = pp
            b["p"] = pp
        for bi, b in enumerate(boxes):
            near = []
            for bj, o in enumerate(boxes):
                if bj == bi:
                    continue
                dk = abs(o["key"][0] - b["key"][0]) + abs(o["key"][1] - b["key"][1])
                if dk == 1:
                    near.append(bj)
                    continue
                if np.hypot(*(o["center"] - b["center"])) - o["r_cell"] >= b["R_p"]:
                    continue
                pts = np.concatenate([nds[j]["x"] for j in o["leaves"]])
                if np.min(np.hypot(*(pts - b["center"]).T)) < b["R_p"]:
                    near.append(bj)
            b["near"] = near
    return {"L": L, "levels": levels, "origin": origin}


def heldout_points(box):
    """The held-out ring of the proxy adequacy check: as many points as the
    proxy circle on the same circle, turned by half their spacing (the
    midpoints between proxy points)."""
    p = box["p"]
    th = 2 * math.pi * (np.arange(p) + 0.5) / p
    nrm = np.stack([np.cos(th), np.sin(th)], -1)
    x = box["center"] + box["R_p"] * nrm
    w = np.full(p, 2 * math.pi * box["R_p"] / p)
    return x, nrm, w


def proxy_points(box):
    p = box["p"]
    th = 2 * math.pi * np.arange(p) / p
    nrm = np.stack([np.cos(th), np.sin(th)], -1)
    x = box["center"] + box["R_p"] * nrm
    w = np.full(p, 2 * math.pi * box["R_p"] / p)
    return x, nrm, w
