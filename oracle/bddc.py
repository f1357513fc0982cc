"""BDDC preconditioner and PCG for the statically condensed VEM Stokes system.

Test infrastructure only (see ``oracle/__init__.py``).

Paper, Sec. 4-6:
* Subdomain split of the DOFs into interior (I) and interface (Gamma);
  pressure Q = Q_I (+) Q_0 with Q_0 the subdomain constants (Eq. discVQ).
* Interface problem S^ u^ = g^ (Eq. globInt) obtained by static
  condensation with subdomain Dirichlet solves (Eq. uipi).
* Partially assembled space V~ = V^_Pi (+) prod V_Delta; change of basis
  so that each primal constraint is an explicit DOF (Sec. 4.3).
* Preconditioner M^{-1} = R~_D^T S~^{-1} R~_D (Eq. BDDCprec), evaluated as a
  coarse saddle problem plus independent constrained local problems.
* Primal set (Sec. 5.1): all subdomain vertices, per macro edge the three
  component means, per macro face the three component integrals and the
  normal flux (Eq. primalfacen); linearly dependent functionals removed
  by an SVD.  Edge-flux functionals (Eq. primaledgen) vanish identically
  in this DOF set (a mesh-face flux is a face DOF), so they add nothing.
* Deluxe scaling on macro faces, D_F^(k) = (S_F^(i) + S_F^(j))^{-1} S_F^(k)
  with S_F the principal minor of the subdomain Schur complement on the
  dual face coordinates (Sec. 6); counting scaling 1/card on macro edges
  (Eq. pseudoinv), or, as an option, the deluxe formula on edges too.
* Adaptive primal enrichment (Sec. 6): generalized eigenproblems
  (S~_i : S~_j) psi = nu (S_i : S_j) psi per face, A:B = (A^-1 + B^-1)^-1;
  eigenvectors with nu < 1/nu_tol give extra primal rows (S_i : S_j) psi.
* CG stop: ||r||_2 <= rtol ||r_0||_2 on the interface residual (u_Gamma,
  p_0) (Sec. 7); Lanczos estimate of the extreme eigenvalues of M^{-1} S^.

Readings: the interior pressure space Q_I^(i) is the zero-mean subspace
(enforced by a bordering row); the coarse saddle matrix is bordered by
sum_i |Omega_i| p_0,i = 0 (the global constant pressure is its null space).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .poly import dim2


class _UF:
    def __init__(self):
        self.p = {}

    def find(self, a):
        self.p.setdefault(a, a)
        while self.p[a] != a:
            self.p[a] = self.p[self.p[a]]
            a = self.p[a]
        return a

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            self.p[max(ra, rb)] = min(ra, rb)


class _BorderedSolver:
    """Exact solves with [K  [0;w]; [0 w^T]  0] (w acts on the trailing
    pressure block): sparse LU plus two steps of iterative refinement, so
    that the local problems are solved to working accuracy also when the
    viscosity jumps by orders of magnitude (pivoted LU alone loses digits)."""

    def __init__(self, K, w):
        n = K.shape[0]
        col = np.zeros(n)
        col[n - len(w):] = w
        self.Kb = sp.bmat([[K, sp.csr_matrix(col[:, None])], [sp.csr_matrix(col[None, :]), None]],
                          format="csc")
        self.lu = spla.splu(self.Kb)

    def solve(self, b):
        x = self.lu.solve(b)
        for _ in range(2):
            x = x + self.lu.solve(b - self.Kb @ x)
        return x


def _bordered_lu(K, w):
    return _BorderedSolver(K, w)


def _bsolve(lu, rhs):
    pad = np.zeros((1,) + rhs.shape[1:])
    x = lu.solve(np.concatenate([rhs, pad], axis=0))
    return x[:-1]


class BDDC:
    """Oracle BDDC over a ``vem.System`` and an element -> subdomain map.

    constraints: tuple from {'vertex','edge','face','flux'} or 'all'
    (every interface DOF primal).  scaling: 'deluxe' (faces; edges by
    counting), 'deluxe_edges' (faces and edges deluxe) or 'multiplicity'.
    adaptive: None or nu_tol.
    """

    def __init__(self, S, part, constraints=("vertex", "edge", "face", "flux"),
                 scaling="deluxe", adaptive=None, svd_tol=1e-10):
        self.S = S
        topo, dm = S.topo, S.dm
        self.part = np.asarray(part)
        self.N = int(self.part.max()) + 1
        if scaling not in ("deluxe", "deluxe_edges", "multiplicity"):
            raise ValueError("scaling must be 'deluxe', 'deluxe_edges' or 'multiplicity'")
        self.scaling = scaling
        self.nvf = len(dm.free)
        self.npr = dm.npress
        self.K = S.free_matrix().tocsr()
        npk = dm.c["press"]
        # ---- entity of each velocity DOF and sharing sets
        ent_of = np.empty(dm.nvel, dtype=object)
        for v in range(topo.nV):
            for c in range(3):
                ent_of[3 * v + c] = ("v", v)
        ce, cf = dm.c["edge"], dm.c["face"]
        for ed in range(topo.nEd):
            for j in range(ce):
                ent_of[dm.off_e + ed * ce + j] = ("e", ed)
        for f in range(topo.nF):
            for j in range(cf):
                ent_of[dm.off_f + f * cf + j] = ("f", f)
        for e in range(topo.nE):
            for j in range(dm.n_elem_int):
                ent_of[dm.off_k + e * dm.n_elem_int + j] = ("k", e)
        share = {}
        for e in range(topo.nE):
            s = int(self.part[e])
            for v in topo.elem_vertices[e]:
                share.setdefault(("v", v), set()).add(s)
            for ed in topo.elem_edges[e]:
                share.setdefault(("e", ed), set()).add(s)
            for f, _ in topo.elem_faces[e]:
                share.setdefault(("f", f), set()).add(s)
        # ---- subdomain local DOFs (global free-velocity indices)
        self.vel = []
        self.prs = []
        for i in range(self.N):
            els = np.nonzero(self.part == i)[0]
            d = set()
            for e in els:
                for g in dm.element_dofs(topo, e):
                    if not dm.fixed[g]:
                        d.add(int(dm.free_index[g]))
            self.vel.append(np.array(sorted(d), dtype=np.int64))
            self.prs.append(np.concatenate([np.arange(e * npk, (e + 1) * npk) for e in els]))
        mult = np.zeros(self.nvf, dtype=int)
        for i in range(self.N):
            mult[self.vel[i]] += 1
        self.mult = mult
        gfree = dm.free
        iface = np.nonzero(mult >= 2)[0]
        # ---- macro entities: components of interface mesh entities with equal sharing set
        ents = {}
        for g in iface:
            ent = ent_of[gfree[g]]
            ents.setdefault(ent, []).append(int(g))
        uf = _UF()
        key = {ent: tuple(sorted(share[ent])) for ent in ents}
        for ent in ents:
            uf.find(ent)
            if ent[0] == "e":
                a, b = topo.edges[ent[1]]
                for v in (("v", a), ("v", b)):
                    if v in ents and key[v] == key[ent]:
                        uf.union(ent, v)
            if ent[0] == "f":
                for ed in topo.face_edges[ent[1]]:
                    if ("e", ed) in ents and key[("e", ed)] == key[ent]:
                        uf.union(ent, ("e", ed))
                for v in topo.face_loops[ent[1]]:
                    if ("v", v) in ents and key[("v", v)] == key[ent]:
                        uf.union(ent, ("v", v))
        comps = {}
        for ent in sorted(ents):
            comps.setdefault(uf.find(ent), []).append(ent)
        self.macro = []
        for root in sorted(comps):
            members = comps[root]
            sset = key[members[0]]
            dofs = sorted(g for ent in members for g in ents[ent])
            if len(members) == 1 and members[0][0] == "v":
                kind = "vertex"
            elif len(sset) == 2:
                kind = "face"
            else:
                kind = "edge"
            self.macro.append(dict(kind=kind, share=sset, ents=members, dofs=np.array(dofs)))
        # ---- constraint rows and change of basis per macro entity
        nint = dim2(dm.k - 2)
        for G in self.macro:
            G["C"] = self._constraints(G, constraints, topo, dm, gfree, ent_of, nint)
        self.adaptive = adaptive
        self._setup(svd_tol)
        if adaptive is not None and scaling in ("deluxe", "deluxe_edges"):
            self._adapt(adaptive, svd_tol)

    # ------------------------------------------------------------- constraints
    def _constraints(self, G, constraints, topo, dm, gfree, ent_of, nint):
        n = len(G["dofs"])
        pos = {g: a for a, g in enumerate(G["dofs"])}
        rows = []
        if constraints == "all":
            return np.eye(n)
        if G["kind"] == "vertex":
            return np.eye(n) if "vertex" in constraints else np.zeros((0, n))
        if G["kind"] == "edge":
            if "edge" in constraints:
                for c in range(3):
                    r = np.zeros(n)
                    for g in G["dofs"]:
                        gg = gfree[g]
                        ent = ent_of[gg]
                        if ent[0] == "v":
                            comp = gg % 3
                        else:
                            comp = (gg - dm.off_e) % 3
                        if comp == c:
                            r[pos[g]] = 1.0
                    rows.append(r / r.sum())
            return np.array(rows).reshape(-1, n)
        # face
        i0 = G["share"][0]
        if "face" in constraints or "flux" in constraints:
            comp_rows = [np.zeros(n) for _ in range(3)]
            flux = np.zeros(n)
            for ent in G["ents"]:
                if ent[0] != "f":
                    continue
                f = ent[1]
                F = _face_geom(topo.xyz, topo.face_loops[f])
                base = dm.off_f + f * dm.c["face"]        # beta = 0 block: (n, t1, t2)
                gn, g1, g2 = (dm.free_index[base + t] for t in range(3))
                for c in range(3):
                    comp_rows[c][pos[gn]] += F["area"] * F["n"][c]
                    comp_rows[c][pos[g1]] += F["area"] * F["t1"][c]
                    comp_rows[c][pos[g2]] += F["area"] * F["t2"][c]
                # outward orientation from the first subdomain sharing the face
                sgn = self._face_sign(f, i0)
                flux[pos[gn]] += sgn * F["area"]
            if "face" in constraints:
                rows += comp_rows
            if "flux" in constraints:
                rows.append(flux)
        return np.array(rows).reshape(-1, n)

    def _face_sign(self, f, sub):
        if not hasattr(self, "_face_elems"):
            fe = {}
            for e in range(self.S.topo.nE):
                for ff, s in self.S.topo.elem_faces[e]:
                    fe.setdefault(ff, []).append((e, s))
            self._face_elems = fe
        for e, s in self._face_elems[f]:
            if self.part[e] == sub:
                return s
        raise ValueError("face not on subdomain")

    # ------------------------------------------------------------- setup
    def _setup(self, svd_tol):
        # change of basis: T_G = [dual | primal], orthonormal, from an SVD of C_G
        self.ncoarse_vel = 0
        for G in self.macro:
            C = G["C"]
            n = len(G["dofs"])
            if C.shape[0] == 0:
                G["T"] = np.eye(n)
                G["ndual"] = n
            else:
                U, s, Vt = np.linalg.svd(C)
                r = int(np.sum(s > svd_tol * s[0]))
                G["T"] = np.hstack([Vt[r:].T, Vt[:r].T])
                G["ndual"] = n - r
            G["nprim"] = n - G["ndual"]
            G["coarse"] = np.arange(self.ncoarse_vel, self.ncoarse_vel + G["nprim"])
            self.ncoarse_vel += G["nprim"]
        self.ncoarse = self.ncoarse_vel + self.N         # + p_0 per subdomain
        self.NPi = self.ncoarse
        self.subs = []
        for i in range(self.N):
            self.subs.append(self._local(i))
        self._coarse()
        self._deluxe()

    def _local(self, i):
        S = self.S
        vel, prs = self.vel[i], self.prs[i]
        nv, npl = len(vel), len(prs)
        lpos = {int(g): a for a, g in enumerate(vel)}
        idx = np.concatenate([vel, self.nvf + prs])
        K = S.local_matrix(np.nonzero(self.part == i)[0])[idx][:, idx]
        # local T (velocity part), primal/dual bookkeeping
        is_iface = self.mult[vel] >= 2
        interior = np.nonzero(~is_iface)[0]
        prim_cols, prim_global = [], []
        dual_index = {}
        cols_T = []
        for gi, G in enumerate(self.macro):
            if i not in G["share"]:
                continue
            loc = np.array([lpos[int(g)] for g in G["dofs"]])
            Tg = G["T"]
            dual_index[gi] = []
            for c in range(Tg.shape[1]):
                cols_T.append((loc, Tg[:, c]))
                if c < G["ndual"]:
                    dual_index[gi].append(len(cols_T) - 1)
                else:
                    prim_global.append(G["coarse"][c - G["ndual"]])
                    prim_cols.append(len(cols_T) - 1)
        # assemble T: local velocity coordinates = [interior..., entity columns...]
        ncols = len(interior) + len(cols_T)
        assert ncols == nv
        Tm = np.zeros((nv, nv))
        for a, ia in enumerate(interior):
            Tm[ia, a] = 1.0
        for c, (loc, v) in enumerate(cols_T):
            Tm[loc, len(interior) + c] = v
        Tsp = sp.csr_matrix(Tm)
        nI = len(interior)
        dual = [nI + c for gi in dual_index for c in dual_index[gi]]
        prim = [nI + c for c in prim_cols]
        Kv = K[:nv, :nv]
        Bl = K[nv:, :nv]
        At = (Tsp.T @ Kv @ Tsp).tocsr()
        Bt = (Bl @ Tsp).tocsr()
        w = S.wmean[prs]
        ones_p = np.zeros(npl)
        # 1_{Omega_i} in element-monomial coefficients: the constant coefficient of every element
        npk = S.dm.c["press"]
        ones_p[0::npk] = 1.0
        # Dirichlet: interior velocity + zero-mean pressure
        KII = sp.bmat([[At[interior_idx(nI)][:, interior_idx(nI)], Bt[:, :nI].T],
                       [Bt[:, :nI], None]], format="csc")
        luD = _bordered_lu(KII, w)
        # Neumann: r = interior + dual
        r = np.array(list(range(nI)) + dual, dtype=np.int64)
        Krr = sp.bmat([[At[r][:, r], Bt[:, r].T], [Bt[:, r], None]], format="csc")
        luN = _bordered_lu(Krr, w)
        # primal columns: velocity primal coords, then p_0 (column 1_Omega_i)
        KrP_v = sp.vstack([At[r][:, prim], Bt[:, prim]]).toarray()
        p0_col = np.concatenate([Bt[:, r].T @ ones_p, np.zeros(npl)])
        KrP = np.hstack([KrP_v, p0_col[:, None]])
        KPP = np.zeros((len(prim) + 1, len(prim) + 1))
        KPP[:len(prim), :len(prim)] = At[prim][:, prim].toarray()
        bp = Bt[:, prim].T @ ones_p
        KPP[:len(prim), -1] = bp
        KPP[-1, :len(prim)] = bp
        Phi_r = -_bsolve(luN, KrP)
        SPi = KPP + KrP.T @ Phi_r
        glob = np.concatenate([np.array(prim_global, dtype=np.int64), [self.ncoarse_vel + i]])
        return dict(vel=vel, prs=prs, nv=nv, npl=npl, T=Tsp, nI=nI, interior=interior,
                    dual=np.array(dual, dtype=np.int64), prim=np.array(prim, dtype=np.int64),
                    dual_index=dual_index, r=r, At=At, Bt=Bt, w=w, ones_p=ones_p,
                    luD=luD, luN=luN, Phi_r=Phi_r, SPi=SPi, glob=glob, lpos=lpos)

    def _coarse(self):
        Kc = np.zeros((self.ncoarse, self.ncoarse))
        for sub in self.subs:
            g = sub["glob"]
            Kc[np.ix_(g, g)] += sub["SPi"]
        vol = np.array([self.S.wmean[self.prs[i]][0::self.S.dm.c["press"]].sum() for i in range(self.N)])
        self.omega_vol = vol
        bord = np.zeros(self.ncoarse)
        bord[self.ncoarse_vel:] = vol
        Kb = np.zeros((self.ncoarse + 1, self.ncoarse + 1))
        Kb[:-1, :-1] = Kc
        Kb[:-1, -1] = bord
        Kb[-1, :-1] = bord
        self.Kc = Kc
        self.Kc_lu = sla.lu_factor(Kb)

    # ---- Dirichlet solve with interface data (local velocity coords in T basis)
    def _dirichlet(self, sub, rhs_I, rhs_p):
        x = _bsolve(sub["luD"], np.concatenate([rhs_I, rhs_p]))
        return x[:sub["nI"]], x[sub["nI"]:]

    def _schur_cols(self, sub, cols):
        """S_Gamma^(i) applied to unit vectors of local T-basis interface
        coordinates ``cols`` (indices into the local velocity coordinates);
        returns the full local-velocity result block [nv, len(cols)]."""
        nv, nI = sub["nv"], sub["nI"]
        At, Bt = sub["At"], sub["Bt"]
        E = np.zeros((nv, len(cols)))
        E[cols, np.arange(len(cols))] = 1.0
        rhs_I = -(At[:nI] @ E)
        rhs_p = -(Bt @ E)
        X = _bsolve(sub["luD"], np.vstack([rhs_I, rhs_p]))
        W = E.copy()
        W[:nI] = X[:nI]
        P = X[nI:]
        return At @ W + Bt.T @ P

    def _deluxe(self):
        """Deluxe blocks D_G^(k) = (sum_{j in N_G} S_G^(j))^{-1} S_G^(k), with
        S_G^(k) the principal minor of the subdomain Schur complement on the
        dual coordinates of the macro entity G: on every macro face (Sec. 6,
        N_F = {i, j}), and with scaling 'deluxe_edges' also on every macro
        edge, over the card(N_E) >= 3 subdomains sharing it (the same
        formula; the paper's edges use 1/card, Eq. pseudoinv)."""
        self.SF = {}
        self.DF = {}
        kinds = {"deluxe": ("face",), "deluxe_edges": ("face", "edge")}.get(self.scaling, ())
        for gi, G in enumerate(self.macro):
            if G["kind"] not in kinds or G["ndual"] == 0:
                continue
            blocks = {}
            for i in G["share"]:
                sub = self.subs[i]
                cols = self._dual_cols(sub, gi)
                R = self._schur_cols(sub, cols)
                blocks[i] = R[cols]
                blocks[i] = 0.5 * (blocks[i] + blocks[i].T)
            Ssum = sum(blocks[s] for s in G["share"])
            self.SF[gi] = blocks
            self.DF[gi] = {s: np.linalg.solve(Ssum, blocks[s]) for s in G["share"]}

    def _dual_cols(self, sub, gi):
        # local coordinate indices of the dual columns of macro entity gi
        return np.array([sub["nI"] + c for c in sub["dual_index"][gi]], dtype=np.int64)

    # ------------------------------------------------------------- adaptive
    def _adapt(self, nu_tol, svd_tol):
        """Adds eigenvector-based primal rows per macro face (Sec. 6); the
        eigenvalues of every face are kept in self.adapt_eigs."""
        added = 0
        self.adapt_eigs = {}
        for gi, G in enumerate(self.macro):
            if gi not in self.SF or G["kind"] != "face":
                continue
            i, j = G["share"]
            St = {}
            for s in (i, j):
                sub = self.subs[s]
                cols = self._dual_cols(sub, gi)
                # S~ = Schur complement of the Neumann matrix onto F_Delta:
                # (E^T K_rr^{-1} E)^{-1} with E the unit columns of F_Delta
                nr = len(sub["r"]) + sub["npl"]
                rpos = {int(c): a for a, c in enumerate(sub["r"])}
                E = np.zeros((nr, len(cols)))
                for a, c in enumerate(cols):
                    E[rpos[int(c)], a] = 1.0
                X = _bsolve(sub["luN"], E)
                St[s] = np.linalg.inv(E.T @ X)
                St[s] = 0.5 * (St[s] + St[s].T)
            Si, Sj = self.SF[gi][i], self.SF[gi][j]
            par = lambda A, B: A @ np.linalg.solve(A + B, B)
            A = par(St[i], St[j])
            Bm = par(Si, Sj)
            A = 0.5 * (A + A.T)
            Bm = 0.5 * (Bm + Bm.T)
            lam, V = sla.eigh(A, Bm)
            self.adapt_eigs[gi] = lam
            sel = lam < 1.0 / nu_tol
            if not sel.any():
                continue
            rows_dual = (Bm @ V[:, sel]).T                 # in dual T-coordinates
            Qd = G["T"][:, :G["ndual"]]
            extra = rows_dual @ Qd.T                        # back to original face DOFs
            G["C"] = np.vstack([G["C"], extra])
            added += int(sel.sum())
        self.n_adaptive = added
        if added:
            self._setup(svd_tol)

    # ------------------------------------------------------------- apply
    def interface_parts(self, r):
        """(r_Gamma over free velocity interface DOFs, r_0 per subdomain)."""
        npk = self.S.dm.c["press"]
        r0 = np.array([r[self.nvf + self.prs[i]][0::npk].sum() for i in range(self.N)])
        return r[:self.nvf] * (self.mult >= 2), r0

    def apply(self, r):
        """z = M^{-1} r with the harmonic (Dirichlet) extension; r, z over the
        free velocity DOFs followed by all pressures."""
        npk = self.S.dm.c["press"]
        rG, r0 = self.interface_parts(r)
        # (1) restriction R~_D: primal coordinates (global) and scaled dual parts
        rC = np.zeros(self.ncoarse)
        rC[self.ncoarse_vel:] = r0
        for G in self.macro:
            rt = G["T"].T @ rG[G["dofs"]]
            rC[G["coarse"]] = rt[G["ndual"]:]
        g_dual = []
        for i, sub in enumerate(self.subs):
            gd = np.zeros(len(sub["r"]))
            for gi in sub["dual_index"]:
                G = self.macro[gi]
                rt = (G["T"].T @ rG[G["dofs"]])[:G["ndual"]]
                cols = self._dual_cols(sub, gi)
                rpos = np.searchsorted(sub["r"], cols)
                gd[rpos] = self._scale_T(gi, i, rt)
            g_dual.append(gd)
        # (2) coarse + local solves
        rhsC = rC.copy()
        for i, sub in enumerate(self.subs):
            rr = np.concatenate([g_dual[i], np.zeros(sub["npl"])])
            rhsC[sub["glob"]] += sub["Phi_r"].T @ rr
        uC = sla.lu_solve(self.Kc_lu, np.concatenate([rhsC, [0.0]]))[:-1]
        self.last_uC = uC
        wloc = []
        for i, sub in enumerate(self.subs):
            rr = np.concatenate([g_dual[i], np.zeros(sub["npl"])])
            zr = _bsolve(sub["luN"], rr)
            wr = zr + sub["Phi_r"] @ uC[sub["glob"]]
            wloc.append(wr)
        # (3) R~_D^T: scaled sum of dual parts, primal from uC; back to original basis
        zG = np.zeros(self.nvf)
        for gi, G in enumerate(self.macro):
            zt = np.zeros(len(G["dofs"]))
            zt[G["ndual"]:] = uC[G["coarse"]]
            for i in G["share"]:
                sub = self.subs[i]
                cols = self._dual_cols(sub, gi)
                rpos = np.searchsorted(sub["r"], cols)
                zt[:G["ndual"]] += self._scale(gi, i, wloc[i][rpos])
            zG[G["dofs"]] = G["T"] @ zt
        # (4) harmonic extension into every subdomain, pressure = zero-mean part + p_0
        z = np.zeros(self.nvf + self.npr)
        z[:self.nvf] = zG
        for i, sub in enumerate(self.subs):
            nI = sub["nI"]
            vloc = sub["T"].T @ zG[sub["vel"]]             # local T-basis coordinates
            vloc[:nI] = 0.0
            rhs_I = -(sub["At"][:nI] @ vloc)
            rhs_p = -(sub["Bt"] @ vloc)
            zI, zp = self._dirichlet(sub, rhs_I, rhs_p)
            z[sub["vel"][sub["interior"]]] = zI
            z[self.nvf + sub["prs"]] = zp + uC[self.ncoarse_vel + i] * sub["ones_p"]
        return z

    def _scale(self, gi, i, w):
        G = self.macro[gi]
        if gi in self.DF:
            return self.DF[gi][i] @ w
        return w / len(G["share"])

    def _scale_T(self, gi, i, r):
        G = self.macro[gi]
        if gi in self.DF:
            return self.DF[gi][i].T @ r
        return r / len(G["share"])

    # ------------------------------------------------------------- solve
    def initial_guess(self, F):
        """Interior Dirichlet solves with zero interface data (r_I = 0)."""
        x = np.zeros(self.nvf + self.npr)
        for sub in self.subs:
            nI = sub["nI"]
            fI = (sub["T"].T @ F[sub["vel"]])[:nI]
            zI, zp = self._dirichlet(sub, fI, np.zeros(sub["npl"]))
            x[sub["vel"][sub["interior"]]] = zI
            x[self.nvf + sub["prs"]] = zp
        return x

    def iface_norm(self, r):
        rG, r0 = self.interface_parts(r)
        return np.sqrt(rG @ rG + r0 @ r0)

    def pcg(self, F, rtol=1e-8, maxit=500, x0=None):
        """PCG on the full system with harmonic iterates (equivalent to CG on
        S^ u^ = g^).  Returns dict(x, iters, lam_min, lam_max, kappa, hist)."""
        K = self.K
        x = self.initial_guess(F) if x0 is None else x0.copy()
        r = F - K @ x
        n0 = self.iface_norm(r)
        hist = [n0]
        alphas, betas = [], []
        if n0 <= 1e-14 * np.linalg.norm(F):
            # no interface (one subdomain): the Dirichlet solve is the solution
            return dict(x=x, iters=0, lam_min=1.0, lam_max=1.0, kappa=1.0, hist=hist)
        z = self.apply(r)
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit:
            Ap = K @ p
            pAp = p @ Ap
            alpha = rz / pAp
            x += alpha * p
            r -= alpha * Ap
            it += 1
            alphas.append(alpha)
            nr = self.iface_norm(r)
            hist.append(nr)
            if nr <= rtol * n0:
                break
            z = self.apply(r)
            rz_new = r @ z
            beta = rz_new / rz
            betas.append(beta)
            rz = rz_new
            p = z + beta * p
        lmin, lmax = lanczos_extremes(alphas, betas)
        return dict(x=x, iters=it, lam_min=lmin, lam_max=lmax, kappa=lmax / lmin, hist=hist)


def interior_idx(n):
    return np.arange(n)


def lanczos_extremes(alphas, betas):
    """Extreme eigenvalues of the CG Lanczos matrix: diagonal
    1/a_j + b_{j-1}/a_{j-1}, off-diagonal sqrt(b_j)/a_j."""
    m = len(alphas)
    if m == 0:
        return 1.0, 1.0
    d = np.zeros(m)
    e = np.zeros(max(m - 1, 0))
    for j in range(m):
        d[j] = 1.0 / alphas[j]
        if j > 0:
            d[j] += betas[j - 1] / alphas[j - 1]
        if j < m - 1:
            e[j] = np.sqrt(betas[j]) / alphas[j]
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[0]), float(ev[-1])


def _face_geom(xyz, loop):
    P = xyz[list(loop)]
    n = np.zeros(3)
    for i in range(len(P)):
        n += np.cross(P[i], P[(i + 1) % len(P)])
    area = 0.5 * np.linalg.norm(n)
    nrm = n / np.linalg.norm(n)
    t1 = P[1] - P[0]
    t1 = t1 - nrm * (t1 @ nrm)
    t1 /= np.linalg.norm(t1)
    return dict(n=nrm, t1=t1, t2=np.cross(nrm, t1), area=area)
