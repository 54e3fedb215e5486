"""A literal FP64 transcription of one step of the coupled metaball/LBM method,
for grids of at most 8^3 nodes.

TEST INFRASTRUCTURE ONLY.  It is written from the paper's equations and the
readings the oracle states (node classification §2.3.1 Eq. (26), the
metaball function Eq. (4), refilling §2.3.3 Eq. (30), the D3Q19 BGK step with
Guo forcing §2.2 Eqs. (14)-(18), VIBB §2.3.1 Eqs. (19)-(25) with the q of
Eq. (27), halfway bounce-back §2.3.5 item 1, the Galilean-invariant momentum
exchange §2.3.2 Eqs. (28)-(29) and the missing force points §2.3.5 item 2,
Eqs. (31)-(32)), and it shares no code with oracle/lbm_oracle.c.  Where the
oracle visits search boxes, lists links while it sweeps and accumulates
per-thread partial sums, this transcription works by brute force: the
metaball value of every particle at every node, every link of every node,
one loop per rule.  The tests compare the two to 1e-14.

Conventions: node (x, y, z) sits at position (x, y, z); non-periodic faces are
halfway walls at -1/2 and n - 1/2; populations are f[i][z][y][x] in this
module's own direction order (`E`), post-collision values of the time level
they belong to.  For a link from a fluid node x_f toward a solid node
x_s = x_f + d, d is the lattice vector pointing into the solid and the unknown
population travels along -d.
"""
from __future__ import annotations

import itertools

import numpy as np

# D3Q19: the rest vector, the six axis vectors and the twelve face diagonals,
# weights 1/3, 1/18, 1/36 (fourth-order isotropic with c_s^2 = 1/3).
E = np.array([v for v in itertools.product((-1, 0, 1), repeat=3) if sum(abs(c) for c in v) <= 2], dtype=np.int64)
W = np.array([{0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[int(np.abs(v).sum())] for v in E])
OPP = np.array([int(np.flatnonzero((E == -v).all(axis=1))[0]) for v in E])


def equilibrium(i: int, rho: float, u: np.ndarray) -> float:
    """Eq. (16) with C = 1."""
    eu = float(E[i] @ u)
    return W[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * float(u @ u))


def rotation(q) -> np.ndarray:
    """Rotation matrix of the unit quaternion q = (w, x, y, z), body -> world."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


class Step:
    """State of one small lattice: populations, node owners and particles."""

    def __init__(self, shape_xyz, periodic, tau, force=(0.0, 0.0, 0.0), rho0=1.0, c0=1.0):
        self.n = tuple(int(v) for v in shape_xyz)          # (nx, ny, nz)
        assert max(self.n) <= 8, "brute force is meant for grids of at most 8^3"
        self.per = tuple(bool(p) for p in periodic)
        self.tau, self.rho0, self.c0 = float(tau), float(rho0), float(c0)
        self.F = np.asarray(force, dtype=np.float64)
        nx, ny, nz = self.n
        self.f = np.zeros((19, nz, ny, nx))
        self.own = -np.ones((nz, ny, nx), dtype=np.int64)   # owner of the previous step (-1 fluid)
        self.parts = []
        self.Fh = np.zeros((0, 3))
        self.Th = np.zeros((0, 3))
        self.nlinks = 0
        self.nrefill = 0
        self.nhalfway = 0   # particle links that fell back to halfway bounce-back
        self.nmissing = 0   # missing force points
        self.ndouble = 0    # nodes inside two or more particles

    # geometry ------------------------------------------------------------
    def set_particles(self, parts):
        """parts: dicts with cp (body frame), K, x, q, v, w (world)."""
        self.parts = []
        for p in parts:
            q = np.asarray(p["q"], dtype=np.float64)
            q = q / np.sqrt(q @ q)
            R = rotation(q)
            cpw = np.asarray(p["x"], dtype=np.float64) + np.asarray(p["cp"], dtype=np.float64) @ R.T
            self.parts.append(dict(cpw=cpw, K=np.asarray(p["K"], dtype=np.float64),
                                   x=np.asarray(p["x"], dtype=np.float64), v=np.asarray(p["v"], dtype=np.float64),
                                   w=np.asarray(p["w"], dtype=np.float64)))

    def image(self, d: np.ndarray) -> np.ndarray:
        """Minimum-image displacement on the periodic axes."""
        d = np.array(d, dtype=np.float64)
        for a in range(3):
            if self.per[a]:
                L = float(self.n[a])
                d[a] -= L * np.floor(d[a] / L + 0.5)
        return d

    def M(self, j: int, pos) -> float:
        """Eq. (4): sum_k K_k / |x - x_k|^2 (minimum image)."""
        p = self.parts[j]
        total = 0.0
        for c, K in zip(p["cpw"], p["K"]):
            r = self.image(np.asarray(pos, dtype=np.float64) - c)
            total += K / float(r @ r)
        return total

    def surface_velocity(self, j: int, pos):
        """u = v_p + w_p x (pos - x_p) and the arm pos - x_p (§2.3.1)."""
        p = self.parts[j]
        arm = self.image(np.asarray(pos, dtype=np.float64) - p["x"])
        return p["v"] + np.cross(p["w"], arm), arm

    def inside(self, c):
        """The node at integer position c, wrapped on periodic axes; None beyond a wall."""
        out = []
        for a in range(3):
            v = int(c[a])
            if v < 0 or v >= self.n[a]:
                if not self.per[a]:
                    return None
                v %= self.n[a]
            out.append(v)
        return tuple(out)

    def classify(self):
        """Owner of every node: solid of particle j when M_j >= c0 (Eq. (26)
        with the surface value c0), the largest M_j where several cover it,
        ties to the lower index; -1 for fluid.  Every node, every particle."""
        nx, ny, nz = self.n
        own = -np.ones((nz, ny, nx), dtype=np.int64)
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            vals = [self.M(j, (x, y, z)) for j in range(len(self.parts))]
            best = -1
            for j, m in enumerate(vals):
                if m >= self.c0 and (best < 0 or m > vals[best]):
                    best = j
            own[z, y, x] = best
            self.ndouble += sum(m >= self.c0 for m in vals) > 1
        return own

    # the step --------------------------------------------------------------
    def step(self):
        nx, ny, nz = self.n
        f = self.f
        old = self.own
        self.ndouble = self.nhalfway = self.nmissing = 0
        new = self.classify()
        F = self.F
        tau = self.tau

        # refilling of uncovered nodes, Eq. (30): a population whose opposite
        # streams in from a node that was fluid is bounced back with the
        # surface velocity there; the others take f^eq(rho0, u_new)
        nref = 0
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            if not (old[z, y, x] >= 0 and new[z, y, x] < 0):
                continue
            nref += 1
            u_new, _ = self.surface_velocity(int(old[z, y, x]), (x, y, z))
            vals = np.zeros(19)
            for i in range(19):
                nb = self.inside((x + E[i][0], y + E[i][1], z + E[i][2]))
                if nb is not None and old[nb[2], nb[1], nb[0]] < 0:
                    vals[i] = f[OPP[i], nb[2], nb[1], nb[0]] + 6.0 * W[OPP[i]] * self.rho0 * float(E[i] @ u_new)
                else:
                    vals[i] = equilibrium(i, self.rho0, u_new)
            f[:, z, y, x] = vals

        def moments_of_stored(node):
            """rho and the velocity of the collision that produced the stored
            post-collision populations: (sum f e - F/2)/rho."""
            fz = f[:, node[2], node[1], node[0]]
            rho = float(fz.sum())
            return rho, (fz @ E - 0.5 * F) / rho

        np_ = len(self.parts)
        Fh = np.zeros((np_, 3))
        Th = np.zeros((np_, 3))
        out = f.copy()
        links = 0
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            if new[z, y, x] >= 0:
                continue
            fin = np.zeros(19)
            xf = np.array([x, y, z], dtype=np.float64)
            for i in range(19):
                io = OPP[i]
                src = self.inside((x - E[i][0], y - E[i][1], z - E[i][2]))
                if src is None:                       # box wall: halfway, at rest
                    fin[i] = f[io, z, y, x]
                    continue
                j = int(new[src[2], src[1], src[0]])
                if j < 0:                             # plain streaming
                    fin[i] = f[i, src[2], src[1], src[0]]
                    continue
                # particle link: d = -e_i points into the solid x_s = x_f + d
                d = -E[i].astype(np.float64)
                Mf, Ms = self.M(j, xf), self.M(j, xf + d)
                q = (self.c0 - Mf) / (Ms - Mf)        # Eq. (27)
                xw = xf + q * d
                uw, arm = self.surface_velocity(j, xw)
                rho_f, u_f = moments_of_stored((x, y, z))
                eu_w = float(E[i] @ uw)
                ff = self.inside((x + E[i][0], y + E[i][1], z + E[i][2]))   # x_ff = x_f - d
                if ff is None or new[ff[2], ff[1], ff[0]] >= 0:
                    # not enough fluid nodes for VIBB: halfway bounce-back
                    val = f[io, z, y, x] + 6.0 * W[io] * rho_f * eu_w
                    self.nhalfway += 1
                else:
                    rho_ff, u_ff = moments_of_stored(ff)
                    f_f, f_ff = f[io, z, y, x], f[io, ff[2], ff[1], ff[0]]
                    neq_d = 2 * q * (f_f - equilibrium(io, rho_f, u_f)) + \
                        (1 - 2 * q) * (f_ff - equilibrium(io, rho_ff, u_ff))        # Eq. (21)
                    if q <= 0.5:
                        rho_d = 2 * q * rho_f + (1 - 2 * q) * rho_ff                 # Eq. (22)
                        u_star = 2 * q * u_f + (1 - 2 * q) * u_ff                   # Eq. (23)
                    else:
                        rho_d = rho_f
                        u_star = (1 - q) / q * u_f + (2 * q - 1) / q * uw
                    u_2star = (1 - q) / (1 + q) * u_ff + 2 * q / (1 + q) * uw        # Eq. (24)
                    u_d = u_star / 3 + 2 * u_2star / 3                              # Eq. (25)
                    val = equilibrium(io, rho_d, u_d) + neq_d + 6.0 * W[io] * rho_f * eu_w   # Eqs. (19)-(20)
                fin[i] = val
                links += 1
                # Eq. (28)-(29): outgoing f+ along d at t, incoming along -d at t+1
                dP = (d - uw) * f[io, z, y, x] - (-d - uw) * val
                Fh[j] += dP
                Th[j] += np.cross(arm, dP)
            rho = float(fin.sum())
            u = (fin @ E + 0.5 * F) / rho
            for i in range(19):
                eu = float(E[i] @ u)
                S = (1.0 - 0.5 / tau) * W[i] * float((3.0 * (E[i] - u) + 9.0 * eu * E[i]) @ F)
                out[i, z, y, x] = fin[i] + (equilibrium(i, rho, u) - fin[i]) / tau + S

        # missing force points, Eqs. (31)-(32): every link y -> x_s = y + d
        # that crosses particle j's surface (M_j(y) < c0 <= M_j(x_s)) and that
        # Eq. (28) did not see (y not a fluid node, or x_s owned by another
        # particle) takes the equilibrium exchange with rho0 and u_w
        for j in range(np_):
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                xs = np.array([x, y, z], dtype=np.float64)
                Ms = self.M(j, xs)
                if Ms < self.c0:
                    continue
                for i in range(19):
                    if not E[i].any():
                        continue
                    d = E[i].astype(np.float64)
                    yp = xs - d
                    My = self.M(j, yp)
                    if My >= self.c0:
                        continue
                    ynode = self.inside(yp.astype(np.int64))
                    seen = ynode is not None and new[ynode[2], ynode[1], ynode[0]] < 0 and new[z, y, x] == j
                    if seen:
                        continue
                    self.nmissing += 1
                    q = (self.c0 - My) / (Ms - My)
                    uw, arm = self.surface_velocity(j, yp + q * d)
                    dP = (d - uw) * equilibrium(i, self.rho0, uw) - (-d - uw) * equilibrium(OPP[i], self.rho0, uw)
                    Fh[j] += dP
                    Th[j] += np.cross(arm, dP)

        self.f = out
        self.own = new
        self.Fh, self.Th = Fh, Th
        self.nlinks, self.nrefill = links, nref
