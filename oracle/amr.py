"""Berger-Oliger AMR driver of the oracle: levels, patches, ghost cells, subcycling,
coarsening, mass reflux and regridding, built on the C primitives of the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
* Sec. 2, Eqs. (1)-(2): dx^{l+1} = dx^l / r^l; time ratio r_t^l = max(r_x, r_y) = r^l
  (the fixed choice), or with dynamic_rt the ratio GeoClaw chooses per step (Sec. 2): the
  fewest steps of level l per step of its parent that keep its Courant number at cfl,
  r_t = ceil(dt_parent * rate_l / cfl) within [1, r^l], rate_l the level's largest
  speed / cell size from the previous step (or from the initial speeds); the first step
  after a regrid takes r^l (those speeds were measured on the old patches).
* Sec. 2.1 refinement (Eqs. (4), (5), (10), bottom-up layer loop) for new fine cells
  and for fine ghost cells (after linear interpolation of the coarse state in time).
* Sec. 2.2, Eq. (11): coarse cells under fine patches take the mean of their fine cells,
  every component.
Not in the paper (this project's reading, standard Berger-Oliger/Colella practice): the
conservative correction of the layer masses at coarse/fine edges (reflux), the nesting
margin of two coarse cells, top-down regridding, and the time step from the largest wave
speeds of the previous coarse step.

Storage mirrors the problem, not the GPU: every level is a dense numpy array over the
domain; each patch is stepped as its own array with a filled ghost ring.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O
from oracle import cluster as C

NG = 2


class Level:
    def __init__(self, nx, ny, dx, dy, F):
        self.nx, self.ny, self.dx, self.dy = nx, ny, dx, dy
        self.q = np.zeros((F, ny, nx))
        self.q_old = None
        self.B = None
        self.patches = []
        self.fx = None  # interface mass flux of this level as a coarse level [M][ny][nx+1]
        self.fy = None
        self.acc_x = None  # accumulated dt * boundary mass flux as a fine level
        self.acc_y = None

    def in_patch_mask(self):
        m = np.zeros((self.ny, self.nx), dtype=bool)
        for (i0, j0, i1, j1) in self.patches:
            m[j0:j1, i0:i1] = True
        return m


class OracleAMR:
    def __init__(self, P, domain, nx0, ny0, max_levels, ratios, B_finest, flag_tol=1e-3, n_buf=2,
                 cluster_eff=0.7, min_side=16, max_side=64, cfl=0.9, n_nest=2, dynamic_rt=False, cfl_max=1.0):
        self.P = P
        self.dynamic_rt = dynamic_rt
        self.M = P.M
        self.F = 3 * P.M
        self.x0, self.y0, self.x1, self.y1 = domain
        self.L = max_levels
        self.r = list(ratios)
        self.flag_tol, self.n_buf, self.eff = flag_tol, n_buf, cluster_eff
        self.min_side, self.max_side, self.cfl, self.n_nest = min_side, max_side, cfl, n_nest
        self.cfl_max = cfl_max
        self.lev = []
        nx, ny = nx0, ny0
        for l in range(max_levels):
            self.lev.append(Level(nx, ny, (self.x1 - self.x0) / nx, (self.y1 - self.y0) / ny, self.F))
            if l + 1 < max_levels:
                nx *= self.r[l]
                ny *= self.r[l]
        self.lev[0].patches = [(0, 0, nx0, ny0)]
        # Bathymetry per level: recursive r x r means of the finest samples (operator of Eq. (11)).
        B = np.ascontiguousarray(B_finest, dtype=float)
        self.lev[-1].B = B
        for l in range(max_levels - 2, -1, -1):
            B = O.bathy_average(B, self.r[l])
            self.lev[l].B = B
        self.t = 0.0
        self.dt = None
        self.smax = [np.zeros(2) for _ in range(max_levels)]
        self.rates = [0.0] * max_levels   # largest speed / cell size per level, for the next step
        self.fresh = False                # this coarse step follows a regrid: fixed ratios
        self.level_steps = [0] * max_levels
        self.level_dt = [0.0] * max_levels  # step of each level in the last coarse step
        self.rejected = 0                     # coarse-step attempts rejected (Courant > cfl_max)
        self.rejected_smax = None             # wave speeds measured by the last rejected attempt
        self.history = []                     # (Courant number, kept) of every automatic attempt
        self.cfl_failed = False               # a member gave up after the retry budget

    # ------------------------------------------------------------------ helpers
    def set_state(self, level, q):
        self.lev[level].q = np.array(q, dtype=float, copy=True)

    def set_patches(self, level, boxes):
        self.lev[level].patches = [tuple(int(v) for v in b) for b in boxes]

    def _padded_level(self, l, q):
        """Dense level array with a wall-mirror ghost ring of 2 (domain boundary)."""
        qp, Bp = O.pad(q, self.lev[l].B)
        O.fill_walls(self.M, qp, Bp)
        return qp, Bp

    def interp_box(self, l, qc, box_c):
        """Refinement (Sec. 2.1) of the coarse cells box_c of level l into level l+1 values."""
        r = self.r[l]
        qp, Bp = self._padded_level(l, qc)
        ci0, cj0, ci1, cj1 = box_c
        Bf = self.lev[l + 1].B[cj0 * r:cj1 * r, ci0 * r:ci1 * r]
        return O.interp_fine(self.P, r, qp, Bp, box_c, Bf)

    def interp_into(self, l, qc, fine_mask):
        """Fills the fine cells of level l+1 marked in fine_mask by refinement of qc."""
        r = self.r[l]
        Fl = self.lev[l + 1]
        js, is_ = np.nonzero(fine_mask)
        if len(js) == 0:
            return
        box = (is_.min() // r, js.min() // r, is_.max() // r + 1, js.max() // r + 1)
        vals = self.interp_box(l, qc, box)
        sub = Fl.q[:, box[1] * r:box[3] * r, box[0] * r:box[2] * r]
        m = fine_mask[box[1] * r:box[3] * r, box[0] * r:box[2] * r]
        sub[:, m] = vals[:, m]

    def coarse_state_at(self, l, alpha):
        """State of level l at fraction alpha in [0, 1] of its last step: linear in time
        between the states before (q_old) and after (q) that step, the coarse values the
        ghost cells of the finer level refine from at each of its substeps."""
        V = self.lev[l]
        return (1.0 - alpha) * V.q_old + alpha * V.q

    def patch_array(self, l, box, alpha):
        """Patch array [F][h+4][w+4] of level l with its ghost ring: patch and sibling cells
        from the level, other in-domain cells by refinement of the coarse state interpolated
        in time at alpha, out-of-domain cells by wall mirroring of those."""
        V = self.lev[l]
        i0, j0, i1, j1 = box
        gi0, gj0, gi1, gj1 = i0 - NG, j0 - NG, i1 + NG, j1 + NG
        # in-domain source region of the ring (mirrors fold into [0, n))
        si0, sj0 = max(gi0, 0), max(gj0, 0)
        si1, sj1 = min(gi1, V.nx), min(gj1, V.ny)
        region = V.q[:, sj0:sj1, si0:si1].copy()
        if l > 0:
            inside = V.in_patch_mask()[sj0:sj1, si0:si1]
            if not inside.all():
                qc = self.coarse_state_at(l - 1, alpha)
                r = self.r[l - 1]
                box_c = (si0 // r, sj0 // r, -(-si1 // r), -(-sj1 // r))
                vals = self.interp_box(l - 1, qc, box_c)
                ox, oy = si0 - box_c[0] * r, sj0 - box_c[1] * r
                vals = vals[:, oy:oy + (sj1 - sj0), ox:ox + (si1 - si0)]
                region[:, ~inside] = vals[:, ~inside]
        out = np.zeros((self.F, j1 - j0 + 2 * NG, i1 - i0 + 2 * NG))
        Bout = np.zeros((j1 - j0 + 2 * NG, i1 - i0 + 2 * NG))
        for jj in range(gj0, gj1):
            sj, fy = jj, 1.0
            if sj < 0:
                sj, fy = -1 - sj, -1.0
            elif sj >= V.ny:
                sj, fy = 2 * V.ny - 1 - sj, -1.0
            for ii in range(gi0, gi1):
                si, fx = ii, 1.0
                if si < 0:
                    si, fx = -1 - si, -1.0
                elif si >= V.nx:
                    si, fx = 2 * V.nx - 1 - si, -1.0
                v = region[:, sj - sj0, si - si0].copy()
                for m in range(self.M):
                    v[3 * m + 1] *= fx
                    v[3 * m + 2] *= fy
                out[:, jj - gj0, ii - gi0] = v
                Bout[jj - gj0, ii - gi0] = V.B[sj, si]
        return np.ascontiguousarray(out), np.ascontiguousarray(Bout)

    # ------------------------------------------------------------------ stepping
    def step_level(self, l, dt, alpha=0.0, record=True):
        """One step of every patch of level l (ghosts at time fraction alpha of the parent step).
        Records coarse interface fluxes and accumulates fine boundary fluxes for the reflux."""
        V = self.lev[l]
        V.q_old = V.q.copy()
        new = V.q.copy()
        smax = np.zeros(2)
        in_patch = V.in_patch_mask()
        for box in V.patches:
            qp, Bp = self.patch_array(l, box, alpha)
            s, _, fx, fy = O.step_patch(self.P, qp, Bp, V.dx, V.dy, dt, want_flux=True)
            smax = np.maximum(smax, s)
            i0, j0, i1, j1 = box
            new[:, j0:j1, i0:i1] = qp[:, NG:-NG, NG:-NG]
            if record and l + 1 < self.L and self.lev[l + 1].patches:
                V.fx[:, j0:j1, i0:i1 + 1] = fx
                V.fy[:, j0:j1 + 1, i0:i1] = fy
            if record and l > 0:
                # boundary edges of this patch whose outer cell is in no patch of the level
                for e, ii in ((0, i0), (i1 - i0, i1)):
                    for j in range(j0, j1):
                        if 0 < ii < V.nx:
                            other = ii - 1 if e == 0 else ii
                            if not in_patch[j, other]:
                                V.acc_x[:, j, ii] += dt * fx[:, j - j0, e]
                for e, jj in ((0, j0), (j1 - j0, j1)):
                    for i in range(i0, i1):
                        if 0 < jj < V.ny:
                            other = jj - 1 if e == 0 else jj
                            if not in_patch[other, i]:
                                V.acc_y[:, jj, i] += dt * fy[:, e, i - i0]
        V.q = new
        self.smax[l] = np.maximum(self.smax[l], smax)
        return smax

    def covered_mask(self, l):
        """Cells of level l covered by level l+1 patches."""
        V = self.lev[l]
        m = np.zeros((V.ny, V.nx), dtype=bool)
        if l + 1 < self.L:
            r = self.r[l]
            for (i0, j0, i1, j1) in self.lev[l + 1].patches:
                m[j0 // r:j1 // r, i0 // r:i1 // r] = True
        return m

    def average_down(self, l):
        """Sec. 2.2, Eq. (11): level-l cells under level l+1 patches := mean of fine cells."""
        r = self.r[l]
        V, Fl = self.lev[l], self.lev[l + 1]
        for (i0, j0, i1, j1) in Fl.patches:
            avg = O.average_coarse(Fl.q[:, j0:j1, i0:i1], r)
            V.q[:, j0 // r:j1 // r, i0 // r:i1 // r] = avg

    def reflux(self, l, dt):
        """Mass reflux at the coarse/fine edges of level l: the coarse mass flux through an
        edge next to an uncovered coarse cell is replaced by the time and space mean of the
        fine mass fluxes through the same edge."""
        r = self.r[l]
        V, Fl = self.lev[l], self.lev[l + 1]
        cov = self.covered_mask(l)
        inp = V.in_patch_mask() if l > 0 else np.ones_like(cov)
        for m in range(self.M):
            for j in range(V.ny):
                for i in range(1, V.nx):
                    a, b = cov[j, i - 1], cov[j, i]
                    if a == b:
                        continue
                    fine = sum(Fl.acc_x[m, j * r + k, i * r] for k in range(r))
                    corr = (dt * V.fx[m, j, i] - fine / r) / V.dx
                    if not a and inp[j, i - 1]:
                        V.q[3 * m, j, i - 1] += corr
                    if not b and inp[j, i]:
                        V.q[3 * m, j, i] -= corr
            for j in range(1, V.ny):
                for i in range(V.nx):
                    a, b = cov[j - 1, i], cov[j, i]
                    if a == b:
                        continue
                    fine = sum(Fl.acc_y[m, j * r, i * r + k] for k in range(r))
                    corr = (dt * V.fy[m, j, i] - fine / r) / V.dy
                    if not a and inp[j - 1, i]:
                        V.q[3 * m, j - 1, i] += corr
                    if not b and inp[j, i]:
                        V.q[3 * m, j, i] -= corr
        Fl.acc_x[:] = 0.0
        Fl.acc_y[:] = 0.0

    def _alloc_flux(self):
        for l, V in enumerate(self.lev):
            if V.fx is None:
                V.fx = np.zeros((self.M, V.ny, V.nx + 1))
                V.fy = np.zeros((self.M, V.ny + 1, V.nx))
                V.acc_x = np.zeros((self.M, V.ny, V.nx + 1))
                V.acc_y = np.zeros((self.M, V.ny + 1, V.nx))

    def time_ratio(self, l, dt_parent):
        """Steps of level l per step of its parent (l >= 1)."""
        r = self.r[l - 1]
        if not self.dynamic_rt or self.fresh or self.rates[l] <= 0.0:
            return r
        need = math.ceil((dt_parent * self.rates[l]) / self.cfl)
        return min(r, max(1, need))

    def substep_fraction(self, l, s, rt):
        """Time of the start of substep s of level l as a fraction of its parent's step,
        when the parent step is taken in rt equal substeps (Sec. 2, time refinement)."""
        return s / rt

    def advance_level(self, l, dt, alpha):
        self.step_level(l, dt, alpha)
        self.level_steps[l] += 1
        self.level_dt[l] = dt
        if l + 1 < self.L and self.lev[l + 1].patches:
            rt = self.time_ratio(l + 1, dt)
            for s in range(rt):
                self.advance_level(l + 1, dt / rt, self.substep_fraction(l + 1, s, rt))
            self.average_down(l)
            self.reflux(l, dt)

    def initial_dt(self):
        g = self.P.g
        best = np.inf
        fac = 1.0
        for l, V in enumerate(self.lev):
            if l > 0:
                fac *= self.r[l - 1]
            if not V.patches:
                continue
            m = V.in_patch_mask() if l > 0 else np.ones((V.ny, V.nx), bool)
            # largest layer speed plus the one-layer gravity wave speed of the whole column
            htot = sum(V.q[3 * k] for k in range(self.M))
            umax = np.zeros_like(htot)
            for k in range(self.M):
                h = V.q[3 * k]
                wet = h > self.P.dry_tol
                hs = np.where(wet, h, 1.0)
                u = np.where(wet, np.abs(V.q[3 * k + 1]) / hs, 0.0)
                v = np.where(wet, np.abs(V.q[3 * k + 2]) / hs, 0.0)
                umax = np.maximum(umax, np.maximum(u, v))
            s = umax + np.sqrt(g * np.maximum(htot, 0.0))
            smax = s[m].max()
            self.rates[l] = smax / min(V.dx, V.dy)
            if smax > 0:
                best = min(best, fac * min(V.dx, V.dy) / smax)
        return self.cfl * best

    def next_dt(self):
        best = np.inf
        fac = 1.0
        for l, V in enumerate(self.lev):
            if l > 0:
                fac *= self.r[l - 1]
            if not V.patches:
                continue
            rate = max(self.smax[l][0] / V.dx, self.smax[l][1] / V.dy)
            self.rates[l] = rate
            if rate > 0:
                best = min(best, fac / rate)
        return self.cfl * best

    def courant(self):
        """Courant number of the last coarse step: the largest over the levels of the level's
        step times its largest wave speed per cell size, max(sx * (1/dx), sy * (1/dy))."""
        c = 0.0
        for l, V in enumerate(self.lev):
            c = max(c, self.level_dt[l] * max(self.smax[l][0] * (1.0 / V.dx), self.smax[l][1] * (1.0 / V.dy)))
        return c

    def advance(self, n_coarse_steps, regrid_interval=0, dt=None):
        """n accepted coarse steps. With automatic time steps (dt None) an attempt whose
        Courant number exceeds cfl_max is rejected: every level returns to its state before
        the attempt and the step is retaken in the next round with the time step the usual
        rule gives from the wave speeds that attempt measured (dt * cfl / Courant number for
        the level that bounds it). Regrids happen at the start of rounds k < n with
        k % regrid_interval == 0; the rounds after the first n (retakes only) never regrid.
        After n + 8 extra rounds the run gives up (cfl_failed)."""
        self._alloc_flux()
        done, k = 0, 0
        while done < n_coarse_steps:
            if k >= 2 * n_coarse_steps + 8:
                self.cfl_failed = True
                return
            if k < n_coarse_steps and regrid_interval and k % regrid_interval == 0 and self.L > 1:
                self.regrid(0)
                self.fresh = True  # the last speeds were measured on the old patches
            step_dt = dt if dt is not None else (self.initial_dt() if self.dt is None else self.next_dt())
            self.smax = [np.zeros(2) for _ in range(self.L)]
            self.level_dt = [0.0] * self.L
            saved = [V.q.copy() for V in self.lev] if dt is None else None
            self.advance_level(0, step_dt, 0.0)
            self.fresh = False
            self.dt = step_dt
            k += 1
            if dt is None:
                c = self.courant()
                kept = not (c > self.cfl_max)
                self.history.append((c, kept))
                if not kept:
                    for V, q in zip(self.lev, saved):
                        V.q = q
                    self.rejected += 1
                    self.rejected_smax = [s.copy() for s in self.smax]
                    continue
            self.t += step_dt
            done += 1

    # ------------------------------------------------------------------ regrid
    def flags(self, l):
        V = self.lev[l]
        avail = V.in_patch_mask().astype(np.uint8) if l > 0 else np.ones((V.ny, V.nx), np.uint8)
        return O.flags(self.M, V.q, V.B, avail, self.P.dry_tol, V.dx, V.dy, self.flag_tol)

    def regrid(self, base=0):
        """Top-down: new level l+1 boxes from level-l flags, newly covered fine cells by
        refinement of level l; cells already in an old fine patch keep their values."""
        for l in range(base, self.L - 1):
            V, Fl = self.lev[l], self.lev[l + 1]
            if l > 0 and not V.patches:
                Fl.patches = []
                continue
            fl = self.flags(l)
            boxes = C.cluster(fl, l, V.patches, self.r[l], self.n_buf, self.eff, self.min_side, self.max_side,
                              self.n_nest)
            old = Fl.in_patch_mask()
            Fl.patches = boxes
            new = Fl.in_patch_mask()
            self.interp_into(l, V.q, new & ~old)

    def mass(self):
        """Composite mass per layer: uncovered cells of every level times their area."""
        out = np.zeros(self.M)
        for l, V in enumerate(self.lev):
            if not V.patches:
                continue
            m = V.in_patch_mask() if l > 0 else np.ones((V.ny, V.nx), bool)
            m = m & ~self.covered_mask(l)
            for k in range(self.M):
                out[k] += V.q[3 * k][m].sum() * V.dx * V.dy
        return out
