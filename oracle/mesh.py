"""Uniform box meshes for the oracle (Section 2: the partition Omega_h, skeleton E_h).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Elements are numbered lexicographically with x fastest.  Global faces are numbered with all
x-normal faces first (index i + (nx+1)*(j + ny*k)), then all y-normal faces
(i + nx*(j + (ny+1)*k)), then all z-normal faces (i + nx*(j + ny*k)).  Each global face of
axis a has a "left" element (on its -a side; it sees the face as its local face 2a+1) and
a "right" element (on its +a side; local face 2a).  -1 marks a missing side (boundary).
Boundary faces are numbered in global face order.
"""
import numpy as np


class BoxMesh:
    def __init__(self, d, n, lo=None, hi=None):
        self.d = d
        self.n = tuple(int(v) for v in n)[:d]
        self.lo = np.zeros(d) if lo is None else np.asarray(lo, dtype=np.float64)[:d]
        self.hi = np.ones(d) if hi is None else np.asarray(hi, dtype=np.float64)[:d]
        self.h = (self.hi - self.lo) / np.array(self.n, dtype=np.float64)
        self.nel = int(np.prod(self.n))
        self._build()

    def elem_index(self, idx):
        """idx: tuple of integer arrays (i, j[, k]) -> lexicographic element numbers."""
        e = np.zeros_like(idx[0])
        stride = 1
        for a in range(self.d):
            e = e + idx[a] * stride
            stride *= self.n[a]
        return e

    def elem_coords(self):
        """Integer coordinates (nel, d) of every element."""
        grids = np.meshgrid(*[np.arange(m) for m in self.n], indexing="ij")
        return np.stack([g.transpose(tuple(range(self.d))[::-1]).ravel() for g in grids], axis=1)

    def _build(self):
        d = self.d
        ec = self.elem_coords()
        self.elem_lo = self.lo[None, :] + ec * self.h[None, :]
        # neighbour across each local face, -1 at the boundary
        self.nbr = np.full((self.nel, 2 * d), -1, dtype=np.int64)
        for a in range(d):
            for side, step in ((0, -1), (1, 1)):
                c = ec.copy()
                c[:, a] += step
                ok = (c[:, a] >= 0) & (c[:, a] < self.n[a])
                e = self.elem_index(tuple(c[:, b] for b in range(d)))
                self.nbr[ok, 2 * a + side] = e[ok]
        # global faces per axis
        self.faces = []   # list of (axis, left, right) arrays, in global order
        self.elem_face = np.zeros((self.nel, 2 * d), dtype=np.int64)  # global face id of local face
        offset = 0
        for a in range(d):
            shape = list(self.n)
            shape[a] += 1
            grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
            fc = np.stack([g.transpose(tuple(range(d))[::-1]).ravel() for g in grids], axis=1)
            nf = fc.shape[0]
            left = np.full(nf, -1, dtype=np.int64)
            right = np.full(nf, -1, dtype=np.int64)
            cl = fc.copy()
            cl[:, a] -= 1
            okl = cl[:, a] >= 0
            left[okl] = self.elem_index(tuple(cl[okl, b] for b in range(d)))
            okr = fc[:, a] < self.n[a]
            right[okr] = self.elem_index(tuple(fc[okr, b] for b in range(d)))
            ids = offset + np.arange(nf)
            self.elem_face[left[okl], 2 * a + 1] = ids[okl]
            self.elem_face[right[okr], 2 * a] = ids[okr]
            self.faces.append((a, left, right, fc))
            offset += nf
        self.nface = offset
        self.face_axis = np.concatenate([np.full(len(f[1]), f[0]) for f in self.faces])
        self.face_left = np.concatenate([f[1] for f in self.faces])
        self.face_right = np.concatenate([f[2] for f in self.faces])
        self.is_boundary = (self.face_left < 0) | (self.face_right < 0)
        self.bface_ids = np.nonzero(self.is_boundary)[0]
        self.nbface = len(self.bface_ids)
        self.bface_index = np.full(self.nface, -1, dtype=np.int64)
        self.bface_index[self.bface_ids] = np.arange(self.nbface)
        # physical lower corner of every face (its tangential extent is h along other axes)
        self.face_lo = np.concatenate([self.lo[None, :] + f[3] * self.h[None, :] for f in self.faces])
