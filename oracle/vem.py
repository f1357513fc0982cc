"""Divergence-free VEM of degree k for 3D Stokes: DOFs, projectors, local
and global matrices, and the bordered direct solve.

Test infrastructure only (see ``oracle/__init__.py``).

Paper: Sec. 3 (virtual element discretization).
* Pressure: Q_h^K = P_{k-1}(K), per element, discontinuous (Eq. globdiscpre).
* Face space with enhancement (Eq. faceSpace), element space (Eq. vemSpace)
  and its enhanced version (Eq. velSpace).
* DOFs D1 (vertex values), D2 (k-1 edge points), D3 (face normal and
  tangential moments against P_{k-2}(f)), D4 (moments against
  x ^ [P_{k-3}]^3), D5 (moments of div v against P_{k-1} without constants).
* a_h^K = consistency + stabilization (Eq. discreteA); load (Eq. discreteF).

Readings where the paper is silent (all also listed in the design notes):
* x in "x ^ p" is xi = (x - x_K)/h_K with x_K the vertex average, h_K the
  element diameter.
* Scaled monomials; D3 uses the face vertex average, diameter, the global
  face normal n_f, t1 = unit first edge, t2 = n_f x t1, and the moments
  are averages (1/|f|) int; D4 and D5 are averages (1/|K|) int.
* D2 points: interior Gauss-Lobatto nodes, ordered from the lower-index
  vertex.
* For k = 4 the one dependent D4 generator (xi ^ (xi_3 e_3), since
  xi ^ xi = 0) is dropped by greedy selection in (monomial, component)
  order.
* a_h^K is nu_K times the printed form; Pi^0_{k-1} eps is the symmetric part
  of Pi^0_{k-1} grad.  Stabilization (the paper defers the D-recipe to its
  reference): S = diag(max((A_c)_ii, h_K)) on the DOF vector.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .poly import (exps2, exps3, dim2, dim3, mono2, mono3, dmono2, dmono3,
                   op_lap2, op_lap3, op_mul3, helmholtz_split, quad_tri, quad_tet,
                   gauss01, gauss_lobatto_interior, cross_xi, index3)


# ------------------------------------------------------------------ topology

class Topology:
    """Vertices, edges and faces of a polyhedral mesh, with boundary flags."""

    def __init__(self, mesh):
        self.xyz = np.asarray(mesh["xyz"], dtype=np.float64)
        fp, fv = mesh["face_ptr"], mesh["face_vtx"]
        ep, ef = mesh["elem_ptr"], mesh["elem_face"]
        self.nV = len(self.xyz)
        self.nF = len(fp) - 1
        self.nE = len(ep) - 1
        self.face_loops = [tuple(int(v) for v in fv[fp[f]:fp[f + 1]]) for f in range(self.nF)]
        self.elem_faces = [[(abs(int(s)) - 1, 1 if s > 0 else -1) for s in ef[ep[e]:ep[e + 1]]]
                           for e in range(self.nE)]
        edges = {}
        self.face_edges = []
        for f, loop in enumerate(self.face_loops):
            fe = []
            for i in range(len(loop)):
                a, b = loop[i], loop[(i + 1) % len(loop)]
                key = (min(a, b), max(a, b))
                if key not in edges:
                    edges[key] = len(edges)
                fe.append(edges[key])
            self.face_edges.append(fe)
        self.edges = sorted(edges, key=lambda k: edges[k])
        self.nEd = len(self.edges)
        self.edge_id = edges
        count = np.zeros(self.nF, dtype=int)
        for e in range(self.nE):
            for f, _ in self.elem_faces[e]:
                count[f] += 1
        self.bnd_face = count == 1
        self.bnd_vertex = np.zeros(self.nV, dtype=bool)
        self.bnd_edge = np.zeros(self.nEd, dtype=bool)
        for f in np.nonzero(self.bnd_face)[0]:
            self.bnd_vertex[list(self.face_loops[f])] = True
            self.bnd_edge[self.face_edges[f]] = True
        self.elem_vertices = []
        self.elem_edges = []
        for e in range(self.nE):
            vs, es = set(), set()
            for f, _ in self.elem_faces[e]:
                vs.update(self.face_loops[f])
                es.update(self.face_edges[f])
            self.elem_vertices.append(sorted(vs))
            self.elem_edges.append(sorted(es))


# ------------------------------------------------------------------ DOFs

def counts(k):
    """Per-entity DOF counts (velocity components included) and pressure dim."""
    nd4 = 3 * dim3(k - 3) - dim3(k - 4)
    return dict(vertex=3, edge=3 * (k - 1), face=3 * dim2(k - 2),
                d4=nd4, d5=dim3(k - 1) - 1, press=dim3(k - 1))


def total_dofs(nV, nEd, nF, nE, k):
    """Total DOF count, all entities and the pressure included (Sec. 3)."""
    c = counts(k)
    return (nV * c["vertex"] + nEd * c["edge"] + nF * c["face"]
            + nE * (c["d4"] + c["d5"] + c["press"]))


class DofMap:
    """Global velocity numbering (all entities) and the free/Dirichlet split.

    Order: vertex DOFs (3 per vertex), edge DOFs (per edge, per point, per
    component), face DOFs (per face, per P_{k-2} monomial, (n, t1, t2)),
    then per element D4 and D5.  Pressure: per element, dim P_{k-1}
    coefficients of the scaled monomials.

    reduced: the reduced scheme (Remark after the convergence theorem, Sec.
    3): the velocity is restricted to fields whose element divergence
    moments of degree >= 1 vanish (every D5 DOF is fixed to zero, like a
    Dirichlet DOF) and the pressure to one constant per element.  The
    velocity of the full scheme is divergence-free, so it lies in that
    subspace and the two schemes give the same velocity.
    """

    def __init__(self, topo, k, reduced=False):
        self.k = k
        self.reduced = reduced
        c = dict(counts(k))
        self.press_full = c["press"]
        if reduced:
            c["press"] = 1
        self.c = c
        self.off_v = 0
        self.off_e = topo.nV * 3
        self.off_f = self.off_e + topo.nEd * c["edge"]
        self.off_k = self.off_f + topo.nF * c["face"]
        self.n_elem_int = c["d4"] + c["d5"]
        self.nvel = self.off_k + topo.nE * self.n_elem_int
        fixed = np.zeros(self.nvel, dtype=bool)
        for v in np.nonzero(topo.bnd_vertex)[0]:
            fixed[3 * v:3 * v + 3] = True
        for ed in np.nonzero(topo.bnd_edge)[0]:
            fixed[self.off_e + ed * c["edge"]: self.off_e + (ed + 1) * c["edge"]] = True
        for f in np.nonzero(topo.bnd_face)[0]:
            fixed[self.off_f + f * c["face"]: self.off_f + (f + 1) * c["face"]] = True
        if reduced:
            for e in range(topo.nE):
                b = self.off_k + e * self.n_elem_int + c["d4"]
                fixed[b:b + c["d5"]] = True
        self.fixed = fixed
        self.free = np.nonzero(~fixed)[0]
        self.free_index = -np.ones(self.nvel, dtype=np.int64)
        self.free_index[self.free] = np.arange(len(self.free))
        self.npress = topo.nE * c["press"]

    def element_dofs(self, topo, e):
        """Global velocity DOF ids of element e in element-local order:
        vertices (sorted), edges (sorted by id), faces (element order), D4, D5."""
        k, c = self.k, self.c
        ids = []
        for v in topo.elem_vertices[e]:
            ids += [3 * v, 3 * v + 1, 3 * v + 2]
        for ed in topo.elem_edges[e]:
            ids += list(range(self.off_e + ed * c["edge"], self.off_e + (ed + 1) * c["edge"]))
        for f, _ in topo.elem_faces[e]:
            ids += list(range(self.off_f + f * c["face"], self.off_f + (f + 1) * c["face"]))
        ids += list(range(self.off_k + e * self.n_elem_int, self.off_k + (e + 1) * self.n_elem_int))
        return np.array(ids, dtype=np.int64)


# ------------------------------------------------------------------ geometry

def face_frame(xyz, loop):
    P = xyz[list(loop)]
    n = np.zeros(3)
    for i in range(len(P)):
        a, b = P[i], P[(i + 1) % len(P)]
        n += np.cross(a, b)              # Newell normal (2 x area vector)
    area_vec = 0.5 * n
    nrm = n / np.linalg.norm(n)
    t1 = P[1] - P[0]
    t1 = t1 - nrm * (t1 @ nrm)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nrm, t1)
    xc = P.mean(axis=0)
    hf = max(np.linalg.norm(P[i] - P[j]) for i in range(len(P)) for j in range(i + 1, len(P)))
    return dict(P=P, n=nrm, t1=t1, t2=t2, xc=xc, h=hf, area=np.linalg.norm(area_vec),
                W=face_whitening(P, xc, t1, t2))


def face_whitening(P, xc, t1, t2):
    """Face-local coordinates of the scaled monomials: (s, t) = W (xi1, xi2)
    with xi = ((x - xc).t1, (x - xc).t2) and W = Sigma^{-1/2} / sqrt(24),
    Sigma = (1/|f|) int_f xi xi^T dA (second moments about xc, exact on the
    fan triangles from vertex 0).  The paper leaves the polynomial basis of
    the face moments open; P_n(f) and its homogeneous parts about xc are
    invariant under this linear map, so only the basis changes, and it stays
    well conditioned on thin faces.  For a square W = I / diam, the plain
    diameter scaling."""
    q = np.stack([(P - xc) @ t1, (P - xc) @ t2], axis=1)
    S = np.zeros((2, 2))
    area = 0.0
    for i in range(1, len(q) - 1):
        a, b, c = q[0], q[i], q[i + 1]
        ar = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        sm = a + b + c
        S += ar / 12.0 * (np.outer(a, a) + np.outer(b, b) + np.outer(c, c) + np.outer(sm, sm))
        area += ar
    S /= area
    # inverse square root of a 2x2 SPD matrix in closed form:
    # sqrt(S) = (S + d I) / tau, d = sqrt(det S), tau = sqrt(tr S + 2 d)
    d = np.sqrt(S[0, 0] * S[1, 1] - S[0, 1] ** 2)
    tau = np.sqrt(S[0, 0] + S[1, 1] + 2.0 * d)
    adj = np.array([[S[1, 1] + d, -S[0, 1]], [-S[0, 1], S[0, 0] + d]])
    return adj / (d * tau * np.sqrt(24.0))


def face_quadrature(F, deg):
    """Points [Q,3] and weights on a planar polygon (fan from vertex 0)."""
    ref, w = quad_tri(deg)
    pts, wts = [], []
    P = F["P"]
    for i in range(1, len(P) - 1):
        a, b, c = P[0], P[i], P[i + 1]
        J = np.linalg.norm(np.cross(b - a, c - a))
        pts.append(a + np.outer(ref[:, 0], b - a) + np.outer(ref[:, 1], c - a))
        wts.append(w * J)
    return np.vstack(pts), np.concatenate(wts)


def face_local(F, x):
    d = x - F["xc"]
    return np.stack([d @ F["t1"], d @ F["t2"]], axis=1) @ F["W"].T


# ------------------------------------------------------------------ face projectors

def face_projectors(xyz, loop, k):
    """Per scalar component: Pi^nabla_{k,f} and Pi^0_{k+1,f} (Eq. faceSpace).

    Face-local scalar DOF vector s = [vertex values (m, loop order),
    edge interior values (m*(k-1), loop-traversal order), averaged
    moments (1/|f|) int v m_b for m_b in P_{k-2}(f)].
    Returns (F, PiN [dim2(k), len s], Pi0 [dim2(k+1), len s]).
    """
    F = face_frame(xyz, loop)
    m = len(loop)
    nb = m * k
    nint = dim2(k - 2)
    ns = nb + nint
    Wf = F["W"]
    qp, qw = face_quadrature(F, 2 * k + 4)
    st = face_local(F, qp)
    Nk = dim2(k)
    # stiffness and boundary rows of the Pi^nabla system; the gradient in
    # the (t1, t2) frame is W^T grad_st
    Gx = [Wf[0, j] * dmono2(k, st, 0) + Wf[1, j] * dmono2(k, st, 1) for j in range(2)]
    G = sum((g * qw[:, None]).T @ g for g in Gx)
    Bv = np.zeros((Nk, ns))
    # -int Lap m_b v  via internal moments: Lap m_b = tr(W W^T Hess_st m_b) in P_{k-2}
    if k >= 2:
        L = op_lap2(k, Wf @ Wf.T)[:nint, :]        # [nint, Nk]
        Bv[:, nb:] -= F["area"] * L.T
    # boundary terms
    gl = gauss_lobatto_interior(k)
    nodes = np.concatenate([[0.0], gl, [1.0]])
    gq, gw = gauss01(k + 2)
    # Lagrange basis on the k+1 nodes, evaluated at the Gauss points
    lag = np.ones((len(gq), k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            if a != b:
                lag[:, a] *= (gq - nodes[b]) / (nodes[a] - nodes[b])
    bnd_row = np.zeros(ns)            # int_{df} v as a functional of s
    bnd_mono = np.zeros(Nk)           # int_{df} m_g
    for i in range(m):
        va, vb = loop[i], loop[(i + 1) % m]
        A, B = xyz[va], xyz[vb]
        le = np.linalg.norm(B - A)
        d = (B - A) / le
        ne = np.cross(d, F["n"])
        x = A[None, :] + np.outer(gq, B - A)
        stq = face_local(F, x)
        nw = Wf @ np.array([F["t1"] @ ne, F["t2"] @ ne])
        dn = dmono2(k, stq, 0) * nw[0] + dmono2(k, stq, 1) * nw[1]
        # map of the k+1 nodal values (traversal order) to s indices
        idx = [i] + [m + i * (k - 1) + j for j in range(k - 1)] + [(i + 1) % m]
        W = gw * le
        contrib = (dn * W[:, None]).T @ lag          # [Nk, k+1]
        for a, s_i in enumerate(idx):
            Bv[:, s_i] += contrib[:, a]
            bnd_row[s_i] += (W @ lag[:, a])
        bnd_mono += W @ mono2(k, stq)
    G[0, :] = bnd_mono
    Bv[0, :] = bnd_row
    PiN = np.linalg.solve(G, Bv)
    # Pi^0_{k+1}: moments up to k-2 from DOFs, k-1..k+1 from Pi^nabla (enhancement)
    N1 = dim2(k + 1)
    M = mono2(k + 1, st)
    Mass = (M * qw[:, None]).T @ M
    R = np.zeros((N1, ns))
    R[:nint, nb:] = F["area"] * np.eye(nint)
    R[nint:, :] = Mass[nint:, :Nk] @ PiN
    Pi0 = np.linalg.solve(Mass, R)
    return F, PiN, Pi0


# ------------------------------------------------------------------ element

def _d4_basis(k):
    """Greedy independent subset of {xi ^ (m_b e_c) : m_b in P_{k-3}} and the
    expansion of every generator in it.  Generators as [P_{k-2}]^3 coefficient
    vectors.  Returns (kept list of (b, c), coef [ngen, nkept])."""
    if k < 3:
        return [], np.zeros((0, 0))
    n = k - 3
    C = cross_xi(n)                      # [3 N_{n+1}, 3 N_n]
    N0 = dim3(n)
    gens = []
    for b in range(N0):
        for c in range(3):
            r = np.zeros(3 * N0)
            r[c * N0 + b] = 1.0
            gens.append(((b, c), C @ r))
    kept, mats = [], []
    for key, g in gens:
        trial = np.array(mats + [g])
        if np.linalg.matrix_rank(trial, tol=1e-10) == len(trial):
            kept.append(key)
            mats.append(g)
    Km = np.array(mats).T
    coef = np.array([np.linalg.lstsq(Km, g, rcond=None)[0] for _, g in gens])
    return kept, coef


class Element:
    """All projector matrices and local matrices of one element."""

    def __init__(self, topo, dm, e, nu=1.0, load_deg=None):
        self.e = e
        k = dm.k
        self.k = k
        xyz = topo.xyz
        c = dm.c
        self.verts = topo.elem_vertices[e]
        self.edges = topo.elem_edges[e]
        self.faces = topo.elem_faces[e]
        nvx, ned, nfc = len(self.verts), len(self.edges), len(self.faces)
        self.off_e = 3 * nvx
        self.off_f = self.off_e + ned * c["edge"]
        self.off_4 = self.off_f + nfc * c["face"]
        self.off_5 = self.off_4 + c["d4"]
        self.nK = self.off_5 + c["d5"]
        nK = self.nK
        self.dofs = dm.element_dofs(topo, e)
        assert len(self.dofs) == nK
        vpos = {v: i for i, v in enumerate(self.verts)}
        epos = {ed: i for i, ed in enumerate(self.edges)}
        # geometry
        P = xyz[self.verts]
        self.xK = P.mean(axis=0)
        self.hK = max(np.linalg.norm(P[i] - P[j]) for i in range(len(P)) for j in range(i + 1, len(P)))
        # volume quadrature: tets (x_K, face fan triangle), signed volumes
        deg = 2 * k + 2
        self.vq_pts, self.vq_w = self._vol_quad(topo, deg)
        self.vol = self.vq_w.sum()
        xi = (self.vq_pts - self.xK) / self.hK
        self.xi = xi
        # face data
        self.fdata = []
        nint = dim2(k - 2)
        for fi, (f, sgn) in enumerate(self.faces):
            loop = topo.face_loops[f]
            F, PiN, Pi0 = face_projectors(xyz, loop, k)
            m = len(loop)
            ns = m * k + nint
            sel = np.zeros((3, ns, nK))
            for comp in range(3):
                for i, v in enumerate(loop):
                    sel[comp, i, 3 * vpos[v] + comp] = 1.0
                for i in range(m):
                    va, vb = loop[i], loop[(i + 1) % m]
                    ed = topo.edge_id[(min(va, vb), max(va, vb))]
                    base = self.off_e + epos[ed] * c["edge"]
                    for j in range(k - 1):
                        jj = j if va < vb else k - 2 - j
                        sel[comp, m + i * (k - 1) + j, base + 3 * jj + comp] = 1.0
                fbase = self.off_f + fi * c["face"]
                for b in range(nint):
                    for t, vec in enumerate((F["n"], F["t1"], F["t2"])):
                        sel[comp, m * k + b, fbase + 3 * b + t] = vec[comp]
            qp, qw = face_quadrature(F, 2 * k + 4)
            self.fdata.append(dict(f=f, sgn=sgn, F=F, PiN=PiN, Pi0=Pi0, sel=sel,
                                   qp=qp, qw=qw, st=face_local(F, qp)))
        self._build(nu)
        self.load_deg = load_deg

    def _vol_quad(self, topo, deg):
        ref, w = quad_tet(deg)
        pts, wts = [], []
        for f, sgn in self.faces:
            loop = list(topo.face_loops[f])
            if sgn < 0:
                loop = loop[::-1]
            P = topo.xyz[loop]
            for i in range(1, len(P) - 1):
                a, b, cc = P[0], P[i], P[i + 1]
                J = np.linalg.det(np.stack([a - self.xK, b - self.xK, cc - self.xK], 1))
                pts.append(self.xK + np.outer(ref[:, 0], a - self.xK) + np.outer(ref[:, 1], b - self.xK)
                           + np.outer(ref[:, 2], cc - self.xK))
                wts.append(w * J)
        return np.vstack(pts), np.concatenate(wts)

    # -- boundary functional: int_{dK} v_comp * q  with q given at face quad points
    def _bnd(self, comp, qvals_per_face, normal_dir=None):
        row = np.zeros(self.nK)
        k = self.k
        for fd, qv in zip(self.fdata, qvals_per_face):
            w = fd["qw"] * qv
            if normal_dir is not None:
                w = w * fd["sgn"] * fd["F"]["n"][normal_dir]
            M = mono2(k + 1, fd["st"])
            row += (w @ M) @ fd["Pi0"] @ fd["sel"][comp]
        return row

    def _grad_moment(self, qfun_vol, qfun_face):
        """Row r with r . dofs = int_K v . grad q  (q in P_{k+1}, given as callables
        of physical points) = -int div v q + sum_f int_f (v.n_K) q."""
        qv = qfun_vol(self.vq_pts)
        Mv = mono3(self.k - 1, self.xi)
        row = -((self.vq_w * qv) @ Mv) @ self.DIV
        for fd in self.fdata:
            qf = qfun_face(fd["qp"])
            for comp in range(3):
                w = fd["qw"] * qf * fd["sgn"] * fd["F"]["n"][comp]
                row += (w @ mono2(self.k + 1, fd["st"])) @ fd["Pi0"] @ fd["sel"][comp]
        return row

    def _poly_fun(self, coef, n):
        """Callable evaluating the scalar polynomial sum coef_a m_a(xi(x))."""
        xK, hK = self.xK, self.hK
        return lambda x: mono3(n, (x - xK) / hK) @ coef

    def _vec_moments(self, n, use_enh):
        """Rows for int_K v . (m_a e_c) for all a in P_n, c (component-major)."""
        k = self.k
        Qc, Rc = helmholtz_split(n)
        Nn = dim3(n)
        out = np.zeros((3 * Nn, self.nK))
        Nr = dim3(n - 1) if n >= 1 else 0
        for col in range(3 * Nn):
            Q = Qc[:, col]
            row = np.zeros(self.nK)
            if np.any(Q != 0):
                qf = self._poly_fun(Q, n + 1)
                row += self.hK * self._grad_moment(qf, qf)
            if Nr > 0:
                R = Rc[:, col]
                row += self._xi_cross_moment(R, n - 1, use_enh)
            out[col] = row
        return out

    def _xi_cross_moment(self, R, nr, use_enh):
        """Row for int_K v . (xi ^ R), R in [P_nr]^3 (component-major coefs)."""
        k = self.k
        Nr = dim3(nr)
        row = np.zeros(self.nK)
        ex = exps3(nr)
        low = np.array([sum(e) <= k - 3 for e in ex])
        # D4 part (degree <= k-3)
        if k >= 3 and low.any():
            N4 = dim3(k - 3)
            for c in range(3):
                for a in range(Nr):
                    if low[a] and R[c * Nr + a] != 0:
                        g = a * 3 + c            # generator index (b major, c minor)
                        row[self.off_4:self.off_5] += R[c * Nr + a] * self.vol * self.d4coef[g]
        hi = ~low
        if hi.any() and np.any(R.reshape(3, Nr)[:, hi] != 0):
            assert use_enh, "enhancement needed before Pi^nabla is known"
            Rh = R.reshape(3, Nr).copy()
            Rh[:, low] = 0.0
            C = cross_xi(nr)
            W = C @ Rh.ravel()                     # xi ^ R_hi in [P_{nr+1}]^3
            N1 = dim3(nr + 1)
            Mw = mono3(nr + 1, self.xi)
            Mk = mono3(k, self.xi)
            Nk = dim3(k)
            for comp in range(3):
                wv = Mw @ W[comp * N1:(comp + 1) * N1]
                row += ((self.vq_w * wv) @ Mk) @ self.PiN[comp * Nk:(comp + 1) * Nk]
        return row

    def _build(self, nu):
        k, nK = self.k, self.nK
        hK = self.hK
        nint = dim2(k - 2)
        self.d4kept, self.d4coef = _d4_basis(k)
        # (1) divergence in P_{k-1}
        Nd = dim3(k - 1)
        mom = np.zeros((Nd, nK))
        for fi, fd in enumerate(self.fdata):
            mom[0, self.off_f + fi * 3 * nint + 0] += fd["sgn"] * fd["F"]["area"]
        for a in range(1, Nd):
            mom[a, self.off_5 + a - 1] = self.vol
        Mv = mono3(k - 1, self.xi)
        self.Mkm1 = (Mv * self.vq_w[:, None]).T @ Mv
        self.DIV = np.linalg.solve(self.Mkm1, mom)
        self.Bmom = mom                               # int_K div v m_a (B_K rows)
        # (2) Pi^nabla_k (vector, component-major coefficients)
        Nk = dim3(k)
        Gm = [dmono3(k, self.xi, j) / hK for j in range(3)]
        G = sum((g * self.vq_w[:, None]).T @ g for g in Gm)
        bnd_mono = np.zeros(Nk)
        for fd in self.fdata:
            bnd_mono += fd["qw"] @ mono3(k, (fd["qp"] - self.xK) / hK)
        G[0, :] = bnd_mono
        lap = op_lap3(k) / hK ** 2                    # [N_{k-2}, Nk]
        if k >= 2:
            VM = self._vec_moments(k - 2, use_enh=False)   # [3 N_{k-2}, nK]
        Nl = dim3(max(k - 2, 0))
        PiN = np.zeros((3 * Nk, nK))
        for comp in range(3):
            rhs = np.zeros((Nk, nK))
            for a in range(1, Nk):
                r = -lap[:, a] @ VM[comp * Nl:(comp + 1) * Nl] if k >= 2 else 0.0
                # boundary: int_dK v_c (grad m_a . n_K)
                qs = []
                for fd in self.fdata:
                    xi_f = (fd["qp"] - self.xK) / hK
                    g = sum(dmono3(k, xi_f, j)[:, a] / hK * fd["F"]["n"][j] for j in range(3)) * fd["sgn"]
                    qs.append(g)
                r = r + self._bnd(comp, qs)
                rhs[a] = r
            rhs[0] = self._bnd(comp, [np.ones(len(fd["qw"])) for fd in self.fdata])
            PiN[comp * Nk:(comp + 1) * Nk] = np.linalg.solve(G, rhs)
        self.PiN = PiN
        # (3) Pi^0_{k-1} grad v : tensor entries (i, j) -> [N_{k-1}, nK]
        Nm = dim3(k - 1)
        VMm = VM if k >= 2 else None
        Gt = {}
        for i in range(3):
            for j in range(3):
                rhs = np.zeros((Nm, nK))
                for a in range(Nm):
                    # -int v_i d_j m_a : d_j m_a = (1/h) dxi_j m_a in P_{k-2}
                    ea = exps3(k - 1)[a]
                    r = np.zeros(nK)
                    if ea[j] > 0 and k >= 2:
                        ee = list(ea)
                        ee[j] -= 1
                        b = index3(k - 2)[tuple(ee)]
                        r -= (ea[j] / hK) * VMm[i * Nl + b]
                    qs = [mono3(k - 1, (fd["qp"] - self.xK) / hK)[:, a] for fd in self.fdata]
                    r += self._bnd(i, qs, normal_dir=j)
                    rhs[a] = r
                Gt[(i, j)] = np.linalg.solve(self.Mkm1, rhs)
        self.Gt = Gt
        Ac = np.zeros((nK, nK))
        for i in range(3):
            for j in range(3):
                E = 0.5 * (Gt[(i, j)] + Gt[(j, i)])
                Ac += E.T @ self.Mkm1 @ E
        self.Ac = Ac
        # (4) DOFs of the [P_k]^3 basis and the stabilization
        self.D = self.poly_dofs()
        s = np.maximum(np.diag(Ac), hK)
        IP = np.eye(nK) - self.D @ PiN
        self.Stab = IP.T @ (s[:, None] * IP)
        self.A = nu * (Ac + self.Stab)
        # (5) Pi^0_k v
        VMk = self._vec_moments(k, use_enh=True)       # [3 Nk, nK]
        Mk = mono3(k, self.xi)
        self.Mk = (Mk * self.vq_w[:, None]).T @ Mk
        self.Pi0 = np.vstack([np.linalg.solve(self.Mk, VMk[c * Nk:(c + 1) * Nk]) for c in range(3)])
        self.B = self.Bmom

    # DOFs of polynomial fields (used for the stabilization and the tests)
    def poly_dofs(self, fun=None, div=None):
        """DOF vector of a vector field.  Default: the DOFs of every function of
        the [P_k]^3 scaled-monomial basis (component-major), as [nK, 3 N_k].
        Otherwise ``fun(x)`` -> [P,3] values and ``div(x)`` -> [P] its
        divergence (needed for D5)."""
        k = self.k
        if fun is None:
            Nk = dim3(k)
            cols = []
            for c in range(3):
                for a in range(Nk):
                    def ev(x, c=c, a=a):
                        out = np.zeros((len(x), 3))
                        out[:, c] = mono3(k, (x - self.xK) / self.hK)[:, a]
                        return out

                    def dv(x, c=c, a=a):
                        return dmono3(k, (x - self.xK) / self.hK, c)[:, a] / self.hK
                    cols.append(self._dofs_of(ev, dv))
            return np.stack(cols, axis=1)
        return self._dofs_of(fun, div)

    def _dofs_of(self, fun, div):
        k = self.k
        xyz = self._topo_xyz
        out = np.zeros(self.nK)
        for i, v in enumerate(self.verts):
            out[3 * i:3 * i + 3] = fun(xyz[v][None, :])[0]
        gl = gauss_lobatto_interior(k)
        for ie, (a, b) in enumerate(self._edge_pairs):
            for j, t in enumerate(gl):
                x = xyz[a] + t * (xyz[b] - xyz[a])
                base = self.off_e + ie * 3 * (k - 1) + 3 * j
                out[base:base + 3] = fun(x[None, :])[0]
        nint = dim2(k - 2)
        for fi, fd in enumerate(self.fdata):
            vals = fun(fd["qp"])
            F = fd["F"]
            M = mono2(k - 2, fd["st"])
            for b in range(nint):
                for t, vec in enumerate((F["n"], F["t1"], F["t2"])):
                    out[self.off_f + fi * 3 * nint + 3 * b + t] = (fd["qw"] * (vals @ vec)) @ M[:, b] / F["area"]
        vals = fun(self.vq_pts)
        if k >= 3:
            M4 = mono3(k - 3, self.xi)
            for j, (b, c) in enumerate(self.d4kept):
                e_c = np.zeros(3)
                e_c[c] = 1.0
                g = M4[:, b][:, None] * np.cross(self.xi, e_c)
                out[self.off_4 + j] = (self.vq_w * np.sum(vals * g, axis=1)).sum() / self.vol
        if self.nK > self.off_5:
            dv = div(self.vq_pts)
            M5 = mono3(k - 1, self.xi)
            for a in range(1, dim3(k - 1)):
                out[self.off_5 + a - 1] = (self.vq_w * dv * M5[:, a]).sum() / self.vol
        return out

    def load(self, f):
        """Local load vector F_K = Pi0_k^T [int f_c m_a] (Eq. discreteF)."""
        k = self.k
        deg = self.load_deg if self.load_deg is not None else k + 9
        pts, w = self._vol_quad(self._topo, deg)
        fv = f(pts)
        M = mono3(k, (pts - self.xK) / self.hK)
        mom = np.concatenate([(w * fv[:, c]) @ M for c in range(3)])
        return self.Pi0.T @ mom


def build_element(topo, dm, e, nu=1.0, load_deg=None):
    el = Element.__new__(Element)
    el._topo = topo
    el._topo_xyz = topo.xyz
    el._edge_pairs = [topo.edges[ed] for ed in topo.elem_edges[e]]
    Element.__init__(el, topo, dm, e, nu, load_deg)
    return el


# ------------------------------------------------------------------ assembly

class System:
    """Global saddle system (Eq. MatrixForm) over all velocity DOFs and the
    element pressures; Dirichlet velocity DOFs are eliminated on solve."""

    def __init__(self, mesh, k, nu, f=None, load_deg=None, elements=None, reduced=False, prebuilt=None):
        """``prebuilt``: optional {e: (Element, F_K or None)} made elsewhere by
        ``build_element`` and ``Element.load`` with these same arguments (the
        test suite builds elements in worker processes); the assembly below
        is the same either way."""
        self.topo = Topology(mesh)
        self.dm = DofMap(self.topo, k, reduced)
        self.k = k
        topo, dm = self.topo, self.dm
        ne = topo.nE
        npk = dm.c["press"]
        rows, cols, vals = [], [], []
        brow, bcol, bval = [], [], []
        F = np.zeros(dm.nvel)
        self.wmean = np.zeros(dm.npress)
        self.elements = {}
        els = range(ne) if elements is None else elements
        for e in els:
            if prebuilt is not None:
                el, fk = prebuilt[e]
                el._topo = topo
                el._topo_xyz = topo.xyz
            else:
                el = build_element(topo, dm, e, nu[e], load_deg)
                fk = el.load(f) if f is not None else None
            d = el.dofs
            rows.append(np.repeat(d, len(d)))
            cols.append(np.tile(d, len(d)))
            vals.append(el.A.ravel())
            pr = np.arange(e * npk, (e + 1) * npk)
            brow.append(np.repeat(pr, len(d)))
            bcol.append(np.tile(d, npk))
            bval.append(el.B[:npk].ravel())
            if fk is not None:
                F[d] += fk
            self.wmean[pr] = (el.vq_w @ mono3(k - 1, el.xi))[:npk]     # int_K m_a
            self.elements[e] = el
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(dm.nvel, dm.nvel))
        self.B = sp.csr_matrix((np.concatenate(bval), (np.concatenate(brow), np.concatenate(bcol))),
                               shape=(dm.npress, dm.nvel))
        self.F = F

    def local_matrix(self, elements):
        """Sum of the element matrices of ``elements`` (a subdomain's Neumann
        matrix), in the global free-velocity + pressure numbering."""
        dm = self.dm
        nvf = len(dm.free)
        rows, cols, vals = [], [], []
        npk = dm.c["press"]
        for e in elements:
            el = self.elements[e]
            d = dm.free_index[el.dofs]
            keep = d >= 0
            dk = d[keep]
            Ak = el.A[np.ix_(keep, keep)]
            rows.append(np.repeat(dk, len(dk)))
            cols.append(np.tile(dk, len(dk)))
            vals.append(Ak.ravel())
            pr = nvf + np.arange(e * npk, (e + 1) * npk)
            Bk = el.B[:npk, keep]
            rows.append(np.repeat(pr, len(dk)))
            cols.append(np.tile(dk, len(pr)))
            vals.append(Bk.ravel())
            rows.append(np.repeat(dk, len(pr)))
            cols.append(np.tile(pr, len(dk)))
            vals.append(Bk.T.ravel())
        n = nvf + dm.npress
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))

    def free_matrix(self):
        """K = [A_ff B_f^T; B_f 0] over free velocity and all pressures."""
        fr = self.dm.free
        Aff = self.A[fr][:, fr]
        Bf = self.B[:, fr]
        return sp.bmat([[Aff, Bf.T], [Bf, None]], format="csr")

    def solve_direct(self, u_bnd=None, F=None):
        """Bordered direct solve with int_Omega p = 0 (zero-mean pressure).

        ``u_bnd``: values of all velocity DOFs used on the Dirichlet ones.
        Returns (u over all velocity DOFs, p)."""
        dm = self.dm
        fr, fx = dm.free, np.nonzero(dm.fixed)[0]
        F = self.F if F is None else F
        ud = np.zeros(len(fx)) if u_bnd is None else u_bnd[fx]
        Aff = self.A[fr][:, fr]
        Afd = self.A[fr][:, fx]
        Bf = self.B[:, fr]
        Bd = self.B[:, fx]
        w = self.wmean[:, None]
        Kb = sp.bmat([[Aff, Bf.T, None], [Bf, None, sp.csr_matrix(w)],
                      [None, sp.csr_matrix(w.T), None]], format="csc")
        rhs = np.concatenate([F[fr] - Afd @ ud, -Bd @ ud, [0.0]])
        x = spla.splu(Kb).solve(rhs)
        u = np.zeros(dm.nvel)
        u[fr] = x[:len(fr)]
        u[fx] = ud
        p = x[len(fr):len(fr) + dm.npress]
        return u, p

    def full_pressure(self, u, p0, F=None):
        """Reduced scheme: the P_{k-1} pressure coefficients of every element
        from the velocity u (all DOFs) and the element constants p0.  The
        higher coefficients p^ follow from the element's D5 velocity rows,
        A_5 u + B_0,5^T p0 + B^_5^T p^ = F_5 (B^_5 = |K| I on the D5 DOFs)."""
        dm = self.dm
        assert dm.reduced
        F = self.F if F is None else F
        npf = dm.press_full
        Au = self.A @ u
        p = np.zeros(self.topo.nE * npf)
        for e, el in self.elements.items():
            j = np.arange(el.off_5, el.nK)
            g = el.dofs[j]
            rhs = F[g] - Au[g] - el.B[0, j] * p0[e]
            p[e * npf] = p0[e]
            if len(j):
                p[e * npf + 1:(e + 1) * npf] = np.linalg.solve(el.B[1:, j].T, rhs)
        return p
