"""Block-structured AMR of the reacting-flow step, as a plain CPU oracle.

Test infrastructure: imported only by the tests, the smoke check and the
benchmark's CPU baseline, never by the product path.

Follows Sec. 3 (the multi-layer block structure, Sec. 3.1, and the main loop
and solver of Algorithms 2 and 3) on top of the single-grid oracle
(oracle.py) for the flux, Newton and chemistry arithmetic of Sec. 4. The
structure, in the paper's terms:

* Layer B_0 is the whole base grid (nx0 x ny0 cells, physical boundaries).
* Layer B_i (i >= 1) holds blocks of B x B cells at twice the resolution of
  layer i-1 (the "one to four" refinement). Block positions are fixed: block
  (bx, by) of layer i covers the layer-i cells [bx B, bx B + B) x
  [by B, by B + B), i.e. the layer-(i-1) subregion [bx B/2, (bx+1) B/2) x
  [by B/2, (by+1) B/2), which is one quarter of layer-(i-1) block
  (bx // 2, by // 2) (Sec. 3.1.1; 2 x 2 subregions per parent block).
* info of a block (Sec. 3.1.3): its position (bx, by) (the glob_index), its
  parent block, and the neighbour blocks to the north, south, west and east
  in the same layer (EXTERNAL where there is none inside the domain,
  PHYSICAL where the side lies on a wall or zero-gradient boundary).
* get_refinement_grid_mask: layer-(i-1) cells with |grad T| > threshold, by
  central differences over the layer, one-sided where the neighbouring cell
  is outside the domain or outside the layer's valid blocks;
  buffer grids: the mask dilated by n_buffer cells (Chebyshev distance).
  get_refinement_block_mask: a subregion is refined when it holds a masked or
  buffer cell and its parent block is valid (Sec. 3.1.2).
* get_ghost_block: 3 ghost cells per side from the same-layer neighbours
  (across a periodic boundary too); on a side that lies on the domain's
  physical boundary, the physical ghosts of that boundary built from the
  block itself (wall mirror or zero-gradient copy, as on layer 0); on any
  other side without a neighbour (an external boundary, Sec. 3.1.3) NaN
  (the paper's NAN block).
* update_external_boundary: the cells within n_boundary = 3 of an external
  side take the layer-(i-1) values of the cell that contains them ("one to
  four" copy), after every Runge-Kutta stage (Algorithm 3 and the remark
  after it). These are exactly the cells whose update reads a ghost of that
  side, so no NaN survives.
* advance_source_term: the point-implicit chemistry over the layer's dt on
  every cell of every block.
* Crossover advance (Fig. 2a): layer i takes two steps of dt_i / 2 on layer
  i + 1 before each of its own steps of dt_i, deepest layer first
  (Algorithm 2); then interpolate_fine_to_coarse ("four to one" arithmetic
  mean, layers ..., 2, 1 in turn) once per base step, onto the parent cells
  whose children are all outside the external band (the band holds copies
  of the parent, so averaging it back would freeze that region).
* Synchronous advance (Fig. 2b): every layer takes one step of the deepest
  layer's dt, deepest layer first, then the four-to-one means; a step then
  advances dt_base / 2^levels.
* The blocks are regenerated every regrid_every base steps (before the
  solve, as in Algorithm 2); a block that exists before and after keeps its
  data (find_and_update_unaltered_block), a new block is refined from its
  parent layer.

Readings where the paper is silent: block size B = 16 cells (8 x 8 parent
cells); the LF speeds of Eq. 4.11 for a refined layer are the maxima over all
of its blocks' cells at each stage input; T of a cell filled by the
one-to-four copy is the parent's T; after the four-to-one mean a parent cell's
T comes from Newton warm-started from its previous T; the base-layer dt comes
from the CFL of the base layer at the start of the base step, and layer i uses
dt / 2^i; the blocks of a layer are ordered by (by, bx).
"""
from __future__ import annotations

import numpy as np

import oracle as orc

NG = 3  # ghost cells per side (WENO5 stencil half-width), n_ghost = n_boundary


EXTERNAL = -1   # no neighbour inside the domain: the external boundary of Sec. 3.1.3
PHYSICAL = -2   # the side lies on the domain's wall or zero-gradient boundary
BC_WALL, BC_ZEROGRAD, BC_PERIODIC = 0, 1, 2


class Layer:
    """Layer B_i, i >= 1: blocks in (by, bx) order, data [nblk, nv, B, B] and T [nblk, B, B].
    nbx, nby: blocks of the layer's index space along x and y; bc: the domain's boundaries."""

    def __init__(self, level, pos, U, T, nbx, nby, bc):
        self.level = level
        self.pos = list(pos)                                # glob_index (bx, by) per block
        self.index = {p: k for k, p in enumerate(self.pos)}
        self.U = U
        self.T = T
        self.nbx, self.nby, self.bc = nbx, nby, list(bc)

    def neighbours(self, k):
        """(north, south, west, east): block number in this layer, EXTERNAL or PHYSICAL."""
        bx, by = self.pos[k]
        out = []
        for (qx, qy), side in (((bx, by + 1), 3), ((bx, by - 1), 2), ((bx - 1, by), 0), ((bx + 1, by), 1)):
            inside = 0 <= qx < self.nbx and 0 <= qy < self.nby
            if not inside:
                if self.bc[side] != BC_PERIODIC:
                    out.append(PHYSICAL)
                    continue
                qx, qy = qx % self.nbx, qy % self.nby
            out.append(self.index.get((qx, qy), EXTERNAL))
        return tuple(out)


class AMROracle:
    def __init__(self, mech, grid, U0, T0, levels=2, threshold=1e6, n_buffer=2, B=16, regrid_every=10,
                 chem=True, force_blocks=None, synchronous=False):
        assert B % 2 == 0 and grid["nx"] % (B // 2) == 0 and grid["ny"] % (B // 2) == 0
        self.m = mech
        self.g0 = dict(grid)
        self.nv = orc.nvar(mech)
        self.B = B
        self.levels = levels
        self.threshold = threshold
        self.n_buffer = n_buffer
        self.regrid_every = regrid_every
        self.chem = chem
        self.force_blocks = force_blocks      # optional {level: set of (bx, by)} overriding the criterion
        self.synchronous = synchronous
        self.U0 = np.array(U0, dtype=np.float64)
        self.T0 = np.array(T0, dtype=np.float64)
        self.layers = [None] + [self._layer(i, [], np.zeros((0, self.nv, B, B)), np.zeros((0, B, B)))
                                for i in range(1, levels + 1)]
        self.nstep = 0
        self.t = 0.0
        self.trace = []                        # (layer, dt) of every solve, in order

    def _layer(self, i, pos, U, T):
        nx, ny = self.ncols(i)
        return Layer(i, pos, U, T, nx // self.B, ny // self.B, self.g0["bc"])

    # ---- geometry -------------------------------------------------------------------------
    def h(self, i):
        return self.g0["dx"] / 2 ** i, self.g0["dy"] / 2 ** i

    def ncols(self, i):
        """Cells of layer i's index space along x and y."""
        return self.g0["nx"] * 2 ** i, self.g0["ny"] * 2 ** i

    def layer_values(self, i, gx, gy):
        """U [nv, ...], T [...] of layer i at global cells (gx, gy) (arrays); layer 0 or valid blocks."""
        if i == 0:
            return self.U0[:, gy, gx], self.T0[gy, gx]
        L, B = self.layers[i], self.B
        k = np.array([L.index[(int(a), int(b))] for a, b in zip((gx // B).ravel(), (gy // B).ravel())])
        k = k.reshape(np.shape(gx))
        return L.U[k, :, gy % B, gx % B].transpose(-1, *range(np.ndim(gx))), L.T[k, gy % B, gx % B]

    def parent_copy(self, i, bx, by):
        """One-to-four copy of the parent layer onto block (bx, by) of layer i: U [nv, B, B], T [B, B]."""
        B = self.B
        gy, gx = np.meshgrid(by * B + np.arange(B), bx * B + np.arange(B), indexing="ij")
        return self.layer_values(i - 1, gx // 2, gy // 2)

    # ---- refinement (Sec. 3.1.2) ----------------------------------------------------------------
    @staticmethod
    def grad_T(T, dx, dy, valid=None):
        """|grad T| by central differences; one-sided where the neighbour is
        outside the array or not valid; 0 on invalid cells."""
        ny, nx = T.shape
        if valid is None:
            valid = np.ones(T.shape, dtype=bool)
        g = np.zeros_like(T)
        for j in range(ny):
            for i in range(nx):
                if not valid[j, i]:
                    continue
                ip = i + 1 if i + 1 < nx and valid[j, i + 1] else i
                im = i - 1 if i > 0 and valid[j, i - 1] else i
                jp = j + 1 if j + 1 < ny and valid[j + 1, i] else j
                jm = j - 1 if j > 0 and valid[j - 1, i] else j
                gx = (T[j, ip] - T[j, im]) / ((ip - im) * dx) if ip != im else 0.0
                gy = (T[jp, i] - T[jm, i]) / ((jp - jm) * dy) if jp != jm else 0.0
                g[j, i] = np.sqrt(gx * gx + gy * gy)
        return g

    def layer_T(self, i):
        """T of layer i over its whole index space and the mask of valid cells."""
        if i == 0:
            return self.T0, np.ones(self.T0.shape, dtype=bool)
        nx, ny = self.ncols(i)
        T = np.zeros((ny, nx))
        valid = np.zeros((ny, nx), dtype=bool)
        L, B = self.layers[i], self.B
        for k, (bx, by) in enumerate(L.pos):
            T[by * B:(by + 1) * B, bx * B:(bx + 1) * B] = L.T[k]
            valid[by * B:(by + 1) * B, bx * B:(bx + 1) * B] = True
        return T, valid

    def refinement_grid_mask(self, i):
        """get_refinement_grid_mask on layer i-1, in layer-(i-1) global cells."""
        dx, dy = self.h(i - 1)
        T, valid = self.layer_T(i - 1)
        return self.grad_T(T, dx, dy, valid) > self.threshold

    def refinement_block_mask(self, i):
        """get_refinement_block_mask: the set of (bx, by) of layer i to refine."""
        if self.force_blocks is not None:
            return sorted(self.force_blocks.get(i, set()), key=lambda p: (p[1], p[0]))
        mask = self.refinement_grid_mask(i)
        ny, nx = mask.shape
        nb = self.n_buffer
        dil = np.zeros_like(mask)
        for sy in range(-nb, nb + 1):            # buffer grids: dilation by n_buffer
            for sx in range(-nb, nb + 1):
                ys, yd = slice(max(sy, 0), ny + min(sy, 0)), slice(max(-sy, 0), ny + min(-sy, 0))
                xs, xd = slice(max(sx, 0), nx + min(sx, 0)), slice(max(-sx, 0), nx + min(-sx, 0))
                dil[yd, xd] |= mask[ys, xs]
        h = self.B // 2
        nbx, nby = self.ncols(i)[0] // self.B, self.ncols(i)[1] // self.B
        out = []
        for by in range(nby):
            for bx in range(nbx):
                if i >= 2 and (bx // 2, by // 2) not in self.layers[i - 1].index:
                    continue
                if dil[by * h:(by + 1) * h, bx * h:(bx + 1) * h].any():
                    out.append((bx, by))
        return out

    def regrid(self):
        """Regenerate layers 1..levels (Algorithm 2, initialize/update)."""
        for i in range(1, self.levels + 1):
            pos = self.refinement_block_mask(i)
            old = self.layers[i]
            U = np.zeros((len(pos), self.nv, self.B, self.B))
            T = np.zeros((len(pos), self.B, self.B))
            for k, (bx, by) in enumerate(pos):
                if (bx, by) in old.index:                       # unaltered block keeps its data
                    U[k], T[k] = old.U[old.index[(bx, by)]], old.T[old.index[(bx, by)]]
                else:                                            # new block: one-to-four refinement
                    U[k], T[k] = self.parent_copy(i, bx, by)
            self.layers[i] = self._layer(i, pos, U, T)

    # ---- solver of a refined layer (Algorithm 3) ---------------------------------------------
    def ghost_block(self, L, U, T, k):
        """get_ghost_block: block k with 3 ghost cells per side (NaN on external sides)."""
        B, nv = self.B, self.nv
        P = np.full((nv, B + 2 * NG, B + 2 * NG), np.nan)
        PT = np.full((B + 2 * NG, B + 2 * NG), np.nan)
        P[:, NG:NG + B, NG:NG + B], PT[NG:NG + B, NG:NG + B] = U[k], T[k]
        n, s, w, e = L.neighbours(k)
        bc = self.g0["bc"]
        g = np.arange(NG)
        if n >= 0:
            P[:, NG + B:, NG:NG + B], PT[NG + B:, NG:NG + B] = U[n][:, :NG, :], T[n][:NG, :]
        elif n == PHYSICAL:                      # ghost NG+B+g mirrors cell B-1-g, or copies B-1
            src = B - 1 - g if bc[3] == BC_WALL else np.full(NG, B - 1)
            P[:, NG + B:, NG:NG + B], PT[NG + B:, NG:NG + B] = U[k][:, src, :], T[k][src, :]
            if bc[3] == BC_WALL:
                P[2, NG + B:, NG:NG + B] *= -1.0
        if s >= 0:
            P[:, :NG, NG:NG + B], PT[:NG, NG:NG + B] = U[s][:, B - NG:, :], T[s][B - NG:, :]
        elif s == PHYSICAL:                      # ghost NG-1-g mirrors cell g, or copies 0
            src = (NG - 1 - g) if bc[2] == BC_WALL else np.zeros(NG, dtype=int)
            P[:, :NG, NG:NG + B], PT[:NG, NG:NG + B] = U[k][:, src, :], T[k][src, :]
            if bc[2] == BC_WALL:
                P[2, :NG, NG:NG + B] *= -1.0
        if w >= 0:
            P[:, NG:NG + B, :NG], PT[NG:NG + B, :NG] = U[w][:, :, B - NG:], T[w][:, B - NG:]
        elif w == PHYSICAL:
            src = (NG - 1 - g) if bc[0] == BC_WALL else np.zeros(NG, dtype=int)
            P[:, NG:NG + B, :NG], PT[NG:NG + B, :NG] = U[k][:, :, src], T[k][:, src]
            if bc[0] == BC_WALL:
                P[1, NG:NG + B, :NG] *= -1.0
        if e >= 0:
            P[:, NG:NG + B, NG + B:], PT[NG:NG + B, NG + B:] = U[e][:, :, :NG], T[e][:, :NG]
        elif e == PHYSICAL:
            src = B - 1 - g if bc[1] == BC_WALL else np.full(NG, B - 1)
            P[:, NG:NG + B, NG + B:], PT[NG:NG + B, NG + B:] = U[k][:, :, src], T[k][:, src]
            if bc[1] == BC_WALL:
                P[1, NG:NG + B, NG + B:] *= -1.0
        return P, PT

    def external_band(self, L, k):
        """Cells of block k within n_boundary of an external side."""
        B = self.B
        n, s, w, e = L.neighbours(k)
        band = np.zeros((B, B), dtype=bool)
        if n == EXTERNAL:
            band[B - NG:, :] = True
        if s == EXTERNAL:
            band[:NG, :] = True
        if w == EXTERNAL:
            band[:, :NG] = True
        if e == EXTERNAL:
            band[:, B - NG:] = True
        return band

    def solve_layer(self, i, dt):
        """One step of layer i: RK3 of the flux terms with ghost blocks and the external-boundary
        update after every stage, then the source term (Algorithm 3)."""
        self.trace.append((i, dt))
        if i == 0:
            self.U0, self.T0, st, _, _ = orc.step(self.m, self.g0, self.U0, self.T0, 1, dt=dt, chem=self.chem)
            assert st == 0, st
            return
        L = self.layers[i]
        if not L.pos:
            return
        dx, dy = self.h(i)
        eps = self.g0.get("weno_eps", 1e-6)
        gi = dict(self.g0, nx=self.B, ny=self.B, dx=dx, dy=dy)
        bands = [self.external_band(L, k) for k in range(len(L.pos))]
        parents = [self.parent_copy(i, bx, by) for (bx, by) in L.pos]

        def rhs_all(U, T):
            alpha = orc.lf_alpha(self.m, U.transpose(1, 0, 2, 3), T)
            out = np.empty_like(U)
            for k in range(len(L.pos)):
                P, PT = self.ghost_block(L, U, T, k)
                out[k] = orc.rhs_ghosted(self.m, self.B, self.B, dx, dy, P, PT, alpha, eps)
            return out

        def finish(Unew, Twarm):
            """update_external_boundary, then Newton T of the other cells (warm start)."""
            Tnew = np.empty_like(Twarm)
            for k in range(len(L.pos)):
                band = bands[k]
                pU, pT = parents[k]
                Unew[k][:, band] = pU[:, band]
                Tk, st = orc.newton(self.m, gi, Unew[k], Twarm[k])
                assert st == 0, st
                Tk[band] = pT[band]
                Tnew[k] = Tk
            return Unew, Tnew

        Un, Tn = L.U, L.T
        U1, T1 = finish(Un + dt * rhs_all(Un, Tn), Tn)
        U2, T2 = finish(0.75 * Un + 0.25 * (U1 + dt * rhs_all(U1, T1)), T1)
        Us, Ts = finish((1.0 / 3.0) * Un + (2.0 / 3.0) * (U2 + dt * rhs_all(U2, T2)), T2)
        if self.chem:                                             # advance_source_term
            for k in range(len(L.pos)):
                Uc, st = orc.point_implicit(self.m, Us[k], Ts[k], dt)
                assert st == 0, st
                Tc, st = orc.newton(self.m, gi, Uc, Ts[k])
                assert st == 0, st
                Us[k], Ts[k] = Uc, Tc
        L.U, L.T = Us, Ts

    def advance(self, i, dt):
        """Crossover advance (Fig. 2a): two steps of layer i+1 at dt/2, then one of layer i."""
        if i < self.levels and self.layers[i + 1].pos:
            self.advance(i + 1, 0.5 * dt)
            self.advance(i + 1, 0.5 * dt)
        self.solve_layer(i, dt)

    def fine_to_coarse(self):
        """interpolate_fine_to_coarse: four-to-one arithmetic mean, layers ..., 2, 1,
        onto the parent cells none of whose four children lies in the block's
        external band (those children are copies of the parent, not values
        the fine solver computed; the parent keeps its own value there)."""
        h = self.B // 2
        for i in range(self.levels, 0, -1):
            L = self.layers[i]
            for k, (bx, by) in enumerate(L.pos):
                f = L.U[k]
                band = self.external_band(L, k)
                keep = band[0::2, 0::2] | band[0::2, 1::2] | band[1::2, 0::2] | band[1::2, 1::2]
                mean = 0.25 * ((f[:, 0::2, 0::2] + f[:, 0::2, 1::2]) + (f[:, 1::2, 0::2] + f[:, 1::2, 1::2]))
                if i - 1 == 0:
                    ys, xs = slice(by * h, (by + 1) * h), slice(bx * h, (bx + 1) * h)
                    Tw = self.T0[ys, xs]
                    Tn, st = orc.newton(self.m, dict(self.g0, nx=h, ny=h), mean, Tw)
                    assert st == 0, st
                    mean[:, keep], Tn[keep] = self.U0[:, ys, xs][:, keep], Tw[keep]
                    self.U0[:, ys, xs], self.T0[ys, xs] = mean, Tn
                else:
                    P = self.layers[i - 1]
                    kp = P.index[(bx // 2, by // 2)]
                    ys = slice((by % 2) * h, (by % 2 + 1) * h)
                    xs = slice((bx % 2) * h, (bx % 2 + 1) * h)
                    Tw = P.T[kp][ys, xs]
                    Tn, st = orc.newton(self.m, dict(self.g0, nx=h, ny=h), mean, Tw)
                    assert st == 0, st
                    mean[:, keep], Tn[keep] = P.U[kp][:, ys, xs][:, keep], Tw[keep]
                    P.U[kp][:, ys, xs], P.T[kp][ys, xs] = mean, Tn

    def step(self, dt=0.0, cfl=0.0):
        """One step (Algorithm 2). Crossover: a base step of dt (the CFL dt of
        layer 0 when dt <= 0). Synchronous: every layer advances dt (the
        CFL dt of layer 0 divided by 2^levels when dt <= 0). Returns the dt
        advanced."""
        if self.nstep % self.regrid_every == 0:
            self.regrid()
        if dt <= 0.0:
            dt = orc.cfl_dt(self.m, self.g0, self.U0, self.T0, cfl)
            if self.synchronous:
                dt /= 2 ** self.levels
        if self.synchronous:
            for i in range(self.levels, -1, -1):
                if i == 0 or self.layers[i].pos:
                    self.solve_layer(i, dt)
        else:
            self.advance(0, dt)
        self.fine_to_coarse()
        self.nstep += 1
        self.t += dt
        return dt

    def cell_updates_per_step(self):
        """Cell updates of one step: base cells plus the cells of layer i, times
        2^i (crossover) or once (synchronous)."""
        n = self.g0["nx"] * self.g0["ny"]
        for i in range(1, self.levels + 1):
            n += len(self.layers[i].pos) * self.B * self.B * (1 if self.synchronous else 2 ** i)
        return n
