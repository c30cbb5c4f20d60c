"""Octree, near lists and interaction lists (paper Sec. 2 and Sec. 3).

Readings (the paper delegates the details to its NESA reference):
* sources are the quadrature points of the triangles (7 per triangle), so every
  source lies in exactly one leaf;
* the root cube has side leaf_size * 2**(n_levels-1) and is centred on the centre of
  the mesh's vertex bounding box; level l boxes have side w_l = root / 2**l;
  leaf index of a point = floor((x - origin)/w_L) clamped to [0, 2**L - 1] per axis;
  n_levels = 0 takes the fewest levels whose root spans the largest side of the box;
* with points_per_leaf = P > 0 instead (Sec. 3: a group is subdivided while it holds
  at least P sources on average), the root cube is the bounding cube (side = the
  largest side of the box, same centre) and the leaf level L is the deepest level
  l <= 19 whose occupied boxes hold on average at least P points;
* two boxes of one level touch when their integer coordinates differ by at most one
  in every axis (a box touches itself);
* near field (Eq. 9): at the leaf level, every pair of touching leaves;
* coarsest far level l0 (Sec. 2 and Sec. 3): the coarsest level with at least 4
  occupied boxes along the longest dimension of the mesh's bounding box (L if none);
* interaction list (Sec. 3): at l0 every non-touching box of l0; at l > l0 the children
  of the boxes touching the parent that do not touch the box itself.
"""
import numpy as np

from .quadrature import triangle_points


MAX_DEPTH = 19


def depth_for_points_per_leaf(points, origin, root, P):
    """Deepest level l <= MAX_DEPTH whose occupied boxes hold at least P points on average."""
    best = 0
    for l in range(MAX_DEPTH + 1):
        w = root / 2.0 ** l
        ijk = np.clip(np.floor((points - origin) / w).astype(np.int64), 0, 2 ** l - 1)
        nbox = len(np.unique(ijk, axis=0))
        if len(points) >= P * nbox:
            best = l
        else:
            break
    return best


def point_leaf_coords(points, origin, leaf_width, levels):
    """Integer leaf coordinates of points: floor((x - origin) / w_L) clamped to
    [0, 2**L - 1] per axis (L = levels - 1)."""
    nb = 2 ** (levels - 1)
    ijk = np.floor((np.asarray(points) - origin) / leaf_width).astype(np.int64)
    return np.clip(ijk, 0, nb - 1)


def leaf_geometry(vertices, leaf_size, n_levels):
    """(origin, leaf width) of the tree with a given leaf size and number of levels."""
    lo, hi = vertices.min(0), vertices.max(0)
    root = leaf_size * 2.0 ** (n_levels - 1)
    return 0.5 * (lo + hi) - 0.5 * root, root / 2.0 ** (n_levels - 1)


class Tree:
    def __init__(self, vertices, triangles, leaf_size, n_levels, points_per_leaf=0):
        lo, hi = vertices.min(0), vertices.max(0)
        self.center = 0.5 * (lo + hi)
        self.extent = hi - lo
        self.points = triangle_points(vertices, triangles).reshape(-1, 3)  # point id = 7 t + p
        if points_per_leaf > 0:
            self.root = float(self.extent.max())
            self.origin = self.center - 0.5 * self.root
            self.L = depth_for_points_per_leaf(self.points, self.origin, self.root, points_per_leaf)
        else:
            if n_levels < 0:
                raise ValueError("n_levels >= 0")
            if n_levels > 0:
                self.L = n_levels - 1
            else:
                self.L = 0
                while self.L < MAX_DEPTH and leaf_size * 2.0 ** self.L < self.extent.max():
                    self.L += 1
            self.root = leaf_size * 2.0 ** self.L
            self.origin = self.center - 0.5 * self.root
        self.point_leaf_ijk = point_leaf_coords(self.points, self.origin, self.width(self.L), self.L + 1)
        # boxes per level: sorted list of integer coordinate triples
        self.boxes = {}
        for l in range(self.L + 1):
            c = self.point_leaf_ijk >> (self.L - l)
            self.boxes[l] = sorted(set(map(tuple, c.tolist())))
        # points per leaf (ascending point id)
        self.leaf_points = {}
        for pid, c in enumerate(map(tuple, self.point_leaf_ijk.tolist())):
            self.leaf_points.setdefault(c, []).append(pid)
        axis = int(np.argmax(self.extent))
        self.l0 = self.L
        for l in range(self.L + 1):
            if len({b[axis] for b in self.boxes[l]}) >= 4:
                self.l0 = l
                break

    def width(self, level):
        return self.root / 2.0 ** level

    def box_center(self, level, ijk):
        return self.origin + (np.asarray(ijk, dtype=np.float64) + 0.5) * self.width(level)

    @staticmethod
    def touch(a, b):
        return max(abs(a[0] - b[0]), abs(a[1] - b[1]), abs(a[2] - b[2])) <= 1

    @staticmethod
    def parent(b):
        return (b[0] >> 1, b[1] >> 1, b[2] >> 1)

    def near_list(self, leaf):
        """Touching leaves (including the leaf itself)."""
        return [b for b in self.boxes[self.L] if self.touch(leaf, b)]

    def interaction_list(self, level, box):
        if level < self.l0:
            return []
        if level == self.l0:
            return [b for b in self.boxes[level] if not self.touch(box, b)]
        p = self.parent(box)
        out = []
        for b in self.boxes[level]:
            if self.touch(p, self.parent(b)) and not self.touch(box, b):
                out.append(b)
        return out

    def children(self, level, box):
        """Occupied children (at level+1) of a box."""
        return [b for b in self.boxes[level + 1] if self.parent(b) == tuple(box)]
