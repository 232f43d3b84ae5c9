"""Python front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference arm may
import this module. It builds and loads ``oracle/liblhe_oracle.so`` (plain C, gcc,
``-O2 -ffp-contract=off``) and shares nothing with the CUDA library: its own velocity
table, weights, initialisation, stepping, boundary schemes and adjoint, all written
from arXiv:2410.13165 (see the citations in lhe_oracle.c).

Layout: populations are numpy float64 arrays of shape (Q, S), S = prod(n), site index
i_1 + n_1*(i_2 + ...) (x_1 fastest); the state is the PRE-collision population.

Dirichlet data given as jets (Model.step_jets, Sec. 3.2) and their cotangent (Model.jet_grad, the
transpose of the same formulas) are written in numpy here; jet_grad is pinned by central differences
of step_jets (tests/test_oracle_jets.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lhe_oracle.c")
_LIBPATH = os.path.join(_HERE, "liblhe_oracle.so")
_lock = threading.Lock()
_lib = None

MAXD, MAXQ, MAXMODES = 5, 51, 16
BC = {"periodic": 0, "fullway": 1, "halfway": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over sites; FMA contraction off)."""
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lhe_oracle.h"))
    ):
        tmp = _LIBPATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class OrcModel(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("Q", ctypes.c_int),
        ("n", ctypes.c_int64 * MAXD), ("x0", ctypes.c_double * MAXD),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("u", ctypes.c_double * MAXD), ("s", ctypes.c_double), ("R", ctypes.c_double),
        ("e", ctypes.c_int * (MAXQ * MAXD)), ("omega", ctypes.c_double * MAXQ),
        ("bc", ctypes.c_int), ("bc_order", ctypes.c_int),
    ]


class OrcWave(ctypes.Structure):
    _fields_ = [
        ("nmodes", ctypes.c_int), ("b", ctypes.c_double), ("g", ctypes.c_double * MAXD),
        ("a", ctypes.c_double * MAXMODES), ("kappa", ctypes.c_double * (MAXMODES * MAXD)),
        ("theta", ctypes.c_double * MAXMODES),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def load(path: str) -> ctypes.CDLL:
    """Load an oracle library built from lhe_oracle.c (the default build, or a copy with a planted
    mistake that a test compiles to show that a pin catches it) and declare its signatures."""
    L = ctypes.CDLL(path)
    L.orc_velocities.argtypes = [ctypes.c_int, _I]
    L.orc_moment_matrix.argtypes = [ctypes.c_int, _I, _D]
    L.orc_eps.argtypes = [ctypes.c_int, _D, _D, _D]
    L.orc_m4_rule.argtypes = [ctypes.c_int, _D, ctypes.c_double]
    L.orc_m4_rule.restype = ctypes.c_double
    L.orc_weights_closed.argtypes = [ctypes.c_int, _D, _D, _D]
    L.orc_solve.argtypes = [ctypes.c_int, _D, _D]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    P = ctypes.POINTER(OrcModel)
    W = ctypes.POINTER(OrcWave)
    L.orc_init.argtypes = [P, ctypes.c_int, _D, _D, _D]
    L.orc_fd_grad.argtypes = [P, _D, _D]
    L.orc_step.argtypes = [P, W, ctypes.c_int64, _D, _D, _D, _D]
    L.orc_phi.argtypes = [P, _D, _D]
    L.orc_exact.argtypes = [P, W, _D, ctypes.c_double]
    L.orc_exact.restype = ctypes.c_double
    L.orc_dir_deriv.argtypes = [P, W, _D, ctypes.c_double, _D, ctypes.c_int, ctypes.c_int]
    L.orc_dir_deriv.restype = ctypes.c_double
    L.orc_node_coord.argtypes = [P, ctypes.c_int64, _D]
    L.orc_exact_field.argtypes = [P, W, ctypes.c_double, _D]
    L.orc_exact_grad_field.argtypes = [P, W, ctypes.c_double, _D]
    L.orc_entropy.argtypes = [P, _D]
    L.orc_entropy.restype = ctypes.c_double
    L.orc_adjoint_step.argtypes = [P, _D, _D, _D]
    L.orc_adjoint_init.argtypes = [P, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    return L


def build_variant(source: str, out_path: str) -> str:
    """Compile C source text (lhe_oracle.c with a planted mistake) with the oracle's own flags."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source)
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           "-std=c11", "-I", _HERE, "-o", out_path, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(_LIBPATH)
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(_D)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ------------------------------------------------------------------ lattice / equilibrium

def velocities(d: int) -> np.ndarray:
    e = (ctypes.c_int * (MAXQ * MAXD))()
    Q = lib().orc_velocities(d, e)
    if Q < 0:
        raise ValueError("d must be 1..5")
    return np.array(e[: Q * d], dtype=np.int64).reshape(Q, d)


def moment_matrix(d: int) -> np.ndarray:
    e = velocities(d)
    Q = e.shape[0]
    ei = (ctypes.c_int * (Q * d))(*[int(v) for v in e.ravel()])
    M = np.zeros(Q * Q)
    lib().orc_moment_matrix(d, ei, _p(M))
    return M.reshape(Q, Q)


def _pairs(d, m4):
    npairs = d * (d - 1) // 2
    if np.isscalar(m4):
        return np.full(max(npairs, 1), float(m4))
    a = np.asarray(m4, dtype=np.float64).ravel()
    assert a.size == npairs
    return np.ascontiguousarray(a if npairs else np.zeros(1))


def eps(d: int, sigma, m4) -> np.ndarray:
    sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    out = np.zeros(2 * d * d + 1)
    lib().orc_eps(d, _p(sig), _p(_pairs(d, m4)), _p(out))
    return out


def m4_rule(d: int, sigma, g: float = 0.5) -> float:
    sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    return lib().orc_m4_rule(d, _p(sig), float(g))


def weights_closed(d: int, sigma, m4) -> np.ndarray:
    sig = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    out = np.zeros(2 * d * d + 1)
    if lib().orc_weights_closed(d, _p(sig), _p(_pairs(d, m4)), _p(out)) < 0:
        raise ValueError("bad d")
    return out


def weights_solve(d: int, sigma, m4) -> np.ndarray:
    """omega = M^{-1} eps by the oracle's own Gaussian elimination (Eq. below (epsilon))."""
    M = np.ascontiguousarray(moment_matrix(d))
    b = eps(d, sigma, m4)
    if lib().orc_solve(M.shape[0], _p(M), _p(b)) != 0:
        raise ValueError("singular moment matrix")
    return b


# ------------------------------------------------------------------ model

class Model:
    """A DdQ(2d^2+1) problem on a box. Grids (paper's RMSE grids, Eq. (rmse)):
    periodic  : n nodes at lo + i dx, dx = L/n;
    full-way  : n nodes at lo + i dx, dx = L/(n-1) (nodes on both faces);
    half-way  : n nodes at lo + (i + 1/2) dx, dx = L/n (walls at mid-link)."""

    def __init__(self, d, n, lo, hi, u, tau=0.5, R=0.0, g=0.5, m4=None, bc="periodic", bc_order=4, c=1.0):
        n = [int(v) for v in (n if np.ndim(n) else [n] * d)]
        lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,)).copy()
        hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,)).copy()
        L = hi - lo
        kind = BC[bc]
        span = [(n[i] - 1) if kind == 1 else n[i] for i in range(d)]
        dxs = L / np.asarray(span, dtype=np.float64)
        if np.max(np.abs(dxs - dxs[0])) > 1e-12 * abs(dxs[0]):
            raise ValueError("the lattice must be square (equal dx in every dimension)")
        self.d, self.n, self.bc, self.bc_order = d, n, bc, bc_order
        self.dx = float(dxs[0])
        self.c = float(c)
        self.dt = self.dx / self.c
        self.u = np.asarray(u, dtype=np.float64).reshape(d)
        self.sigma = self.u / self.c
        self.tau, self.s, self.R = float(tau), 1.0 / float(tau), float(R)
        self.m4 = m4_rule(d, self.sigma, g) if m4 is None else m4
        self.omega = weights_closed(d, self.sigma, self.m4)
        self.e = velocities(d)
        self.Q = self.e.shape[0]
        self.S = int(np.prod(n))
        self.x0 = lo + (0.5 * self.dx if kind == 2 else 0.0)
        m = OrcModel()
        m.d, m.Q = d, self.Q
        for i in range(d):
            m.n[i] = n[i]
            m.x0[i] = self.x0[i]
            m.u[i] = self.u[i]
        m.dx, m.dt, m.s, m.R = self.dx, self.dt, self.s, self.R
        for k in range(self.Q):
            m.omega[k] = self.omega[k]
            for i in range(d):
                m.e[k * d + i] = int(self.e[k, i])
        m.bc, m.bc_order = kind, int(bc_order)
        self._m = m

    # geometry
    def coords(self) -> np.ndarray:
        """(d, S) node coordinates, x_1 fastest."""
        axes = [self.x0[i] + self.dx * np.arange(self.n[i]) for i in range(self.d)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        return np.stack([g.ravel() for g in grids])

    def wave(self, a=(), kappa=(), theta=(), b=0.0, g=None) -> OrcWave:
        w = OrcWave()
        a = list(a)
        assert len(a) <= MAXMODES
        w.nmodes, w.b = len(a), float(b)
        for i in range(self.d):
            w.g[i] = 0.0 if g is None else float(g[i])
        for mo in range(len(a)):
            w.a[mo] = float(a[mo])
            w.theta[mo] = float(theta[mo]) if len(theta) else 0.0
            for i in range(self.d):
                w.kappa[mo * MAXD + i] = float(kappa[mo][i])
        return w

    def exact(self, w: OrcWave, t: float) -> np.ndarray:
        out = np.empty(self.S)
        lib().orc_exact_field(ctypes.byref(self._m), ctypes.byref(w), float(t), _p(out))
        return out

    def exact_grad(self, w: OrcWave, t: float) -> np.ndarray:
        out = np.empty((self.d, self.S))
        lib().orc_exact_grad_field(ctypes.byref(self._m), ctypes.byref(w), float(t), _p(out))
        return out

    # scheme
    def init(self, phi0, grad=None, order=3) -> np.ndarray:
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(self.S)
        if order == 3 and grad is None:
            grad = self.fd_grad(phi0)
        g = None if grad is None else np.ascontiguousarray(grad, dtype=np.float64).reshape(self.d, self.S)
        f = np.empty((self.Q, self.S))
        lib().orc_init(ctypes.byref(self._m), int(order), _p(phi0), _p(g), _p(f))
        return f

    def fd_grad(self, phi) -> np.ndarray:
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.S)
        out = np.empty((self.d, self.S))
        lib().orc_fd_grad(ctypes.byref(self._m), _p(phi), _p(out))
        return out

    def step(self, f, n0=0, nsteps=1, wave: OrcWave | None = None, Rfield=None) -> np.ndarray:
        """Advance the pre-collision state f from step n0 by nsteps steps."""
        if self.bc != "periodic" and wave is None:
            raise ValueError("Dirichlet boundaries need boundary data (wave)")
        w = wave if wave is not None else OrcWave()
        cur = np.ascontiguousarray(f, dtype=np.float64).copy()
        star = np.empty_like(cur)
        nxt = np.empty_like(cur)
        Rf = None if Rfield is None else np.ascontiguousarray(Rfield, dtype=np.float64).reshape(self.S)
        L = lib()
        for n in range(n0, n0 + nsteps):
            L.orc_step(ctypes.byref(self._m), ctypes.byref(w), n, _p(Rf), _p(cur), _p(star), _p(nxt))
            cur, nxt = nxt, cur
        return cur

    def _jet_links(self) -> dict:
        """The unknown populations of a Dirichlet box (Sec. 3.2): every (site, link k) whose pull source
        site - e_k lies outside the box, site-major, links in the order of k; with c_k, the opposite link,
        the weights, and the position of each derivative tuple in a jet (orders 0..3 in (t, x_1..x_d),
        tuples non-decreasing, by length then lexicographic)."""
        import itertools

        d, S, Q = self.d, self.S, self.Q
        pos, j = {}, 0
        for q in range(4):
            for tup in itertools.combinations_with_replacement(range(d + 1), q):
                pos[tup] = j
                j += 1
        idx = np.stack(np.unravel_index(np.arange(S), self.n[::-1])[::-1])  # (d, S), x_1 fastest
        sites, links = [], []
        for site in range(S):
            for k in range(Q):
                src = idx[:, site] - self.e[k]
                if np.any(src < 0) or np.any(src >= np.asarray(self.n)):
                    sites.append(site)
                    links.append(k)
        sites, links = np.asarray(sites, dtype=np.int64), np.asarray(links, dtype=np.int64)
        kb = np.array([int(np.nonzero(np.all(self.e == -self.e[k], axis=1))[0][0]) for k in links], dtype=np.int64)
        return {"pos": pos, "jlen": j, "sites": sites, "links": links, "ck": self.c * self.e[links].astype(np.float64),
                "kb": kb, "wk": self.omega[links], "wkb": self.omega[kb]}

    def _dir_deriv(self, jl, J, p, q):
        """d_t^q (c_k . grad)^p phi from the jets J (U, jlen) of the unknown populations, summed over
        ordered spatial tuples."""
        import itertools

        ck, pos = jl["ck"], jl["pos"]
        out = np.zeros(len(jl["links"]))
        for sp in itertools.product(range(1, self.d + 1), repeat=p):
            w = np.ones(len(jl["links"]))
            for i in sp:
                w = w * ck[:, i - 1]
            out += w * J[:, pos[tuple(sorted((0,) * q + sp))]]
        return out

    def _dir_deriv_T(self, jl, g, p, q):
        """Transpose of _dir_deriv: the (U, jlen) cotangent of the jets for the cotangent g (U,) of
        d_t^q (c_k . grad)^p phi."""
        import itertools

        ck, pos = jl["ck"], jl["pos"]
        G = np.zeros((len(jl["links"]), jl["jlen"]))
        for sp in itertools.product(range(1, self.d + 1), repeat=p):
            w = np.ones(len(jl["links"]))
            for i in sp:
                w = w * ck[:, i - 1]
            G[:, pos[tuple(sorted((0,) * q + sp))]] += w * g
        return G

    def jet_grad(self, lam):
        """Cotangent of the Dirichlet jets of one step (the transpose of the map from jets to unknown
        populations in step_jets, Eq. (bun1) / Eq. (bun2)). lam = dL/df (Q, S) of the pre-collision
        state that the step produced, so the cotangent of each unknown population's value is
        lam_k(site). The R terms and -f*_kbar do not depend on the jets. Returns (points (P, d),
        grad (P, jlen)): full-way one point per boundary node (ascending site), the sum over its
        unknown links; half-way one point per unknown population, at x - c_k dt/2, in the order of
        _jet_links."""
        jl = self._jet_links()
        sites, links, wk, wkb = jl["sites"], jl["links"], jl["wk"], jl["wkb"]
        dt = self.dt
        g = np.asarray(lam, dtype=np.float64).reshape(self.Q, self.S)[links, sites]
        T = lambda coef, p, q: self._dir_deriv_T(jl, coef * g, p, q)  # noqa: E731
        X = self.coords()
        if self.bc == "fullway":
            G = T(wk, 0, 0)
            if self.bc_order >= 3:
                G = G - T(0.5 * dt * wk, 1, 0) - T(0.5 * dt * wk, 0, 1)
            if self.bc_order >= 4:
                G = G + T(dt ** 3 / 8.0 * wk, 1, 2) + T(dt ** 3 / 8.0 * wk, 2, 1) \
                    + T(dt ** 3 / 24.0 * wk, 0, 3) + T(dt ** 3 / 24.0 * wk, 3, 0)
            nodes, inv = np.unique(sites, return_inverse=True)
            out = np.zeros((len(nodes), jl["jlen"]))
            np.add.at(out, inv, G)
            return X[:, nodes].T.copy(), out
        wsum, wdif = wk + wkb, wk - wkb
        G = T(wsum, 0, 0)
        if self.bc_order >= 2:
            G = G + T(0.5 * dt * wsum, 0, 1)
        if self.bc_order >= 3:
            G = G - T(dt * dt / 8.0 * wsum, 2, 0) - T(dt * dt / 4.0 * wdif, 1, 1)
        if self.bc_order >= 4:
            G = G - T(dt ** 3 / 8.0 * wdif, 1, 2) - T(dt ** 3 / 16.0 * wsum, 2, 1) - T(dt ** 3 / 24.0 * wsum, 0, 3)
        return (X[:, sites].T - 0.5 * dt * jl["ck"]).copy(), G

    def step_jets(self, f, n0, nsteps, jet_fn, Rfield_fn=None) -> np.ndarray:
        """Dirichlet steps with the boundary data given as jets of phi: jet_fn(points (P, d), t)
        returns (P, J) arrays of every derivative of order 0..3 in (t, x_1..x_d), ordered by length
        and then lexicographically over non-decreasing variable tuples (0: t, i: x_i). The unknown
        populations follow Eq. (bun1) (at the node, t + dt) and Eq. (bun2) (at x - c_k dt/2, t) with
        the directional derivatives d_t^q (c . grad)^p phi formed from the jets, term by term as in
        boundary_value of lhe_oracle.c. Rfield_fn(n) (optional) gives the per-site source R(x, t_n) of
        the collision at t_n; the schemes' R terms take it at the boundary node at the time of their
        data: full-way t_{n+1} (Rfield_fn(n + 1)), half-way t_n (Rfield_fn(n))."""
        if self.bc == "periodic":
            raise ValueError("jets are Dirichlet data")
        S = self.S
        jl = self._jet_links()
        sites, links, ck, kb, wk, wkb = jl["sites"], jl["links"], jl["ck"], jl["kb"], jl["wk"], jl["wkb"]
        X = self.coords()
        dt = self.dt

        def dir_deriv(J, p, q):
            return self._dir_deriv(jl, J, p, q)

        w = OrcWave()  # no wave data: the unknown populations are replaced below
        cur = np.ascontiguousarray(f, dtype=np.float64).copy()
        star = np.empty_like(cur)
        nxt = np.empty_like(cur)
        L = lib()
        for n in range(n0, n0 + nsteps):
            Rf = None if Rfield_fn is None else np.ascontiguousarray(Rfield_fn(n), dtype=np.float64).reshape(S)
            L.orc_step(ctypes.byref(self._m), ctypes.byref(w), n, _p(Rf), _p(cur), _p(star), _p(nxt))
            Rn = np.full(len(sites), self.R) if Rf is None else Rf[sites]  # source at the boundary node
            if self.bc == "fullway" and Rfield_fn is not None:
                Rn = np.ascontiguousarray(Rfield_fn(n + 1), dtype=np.float64).reshape(S)[sites]
            if self.bc == "fullway":
                t1 = (n + 1) * dt
                J = np.asarray(jet_fn(X[:, sites].T.copy(), t1), dtype=np.float64)
                feq = wk * dir_deriv(J, 0, 0)
                if self.bc_order == 1:
                    val = feq
                else:
                    val = feq - 0.5 * dt * wk * dir_deriv(J, 1, 0) - 0.5 * dt * wk * dir_deriv(J, 0, 1) + 0.5 * dt * wk * Rn
                    if self.bc_order >= 4:
                        val = val + dt ** 3 / 8.0 * wk * dir_deriv(J, 1, 2) + dt ** 3 / 8.0 * wk * dir_deriv(J, 2, 1) \
                            + dt ** 3 / 24.0 * wk * dir_deriv(J, 0, 3) + dt ** 3 / 24.0 * wk * dir_deriv(J, 3, 0)
            else:
                t0 = n * dt
                J = np.asarray(jet_fn((X[:, sites].T - 0.5 * dt * ck).copy(), t0), dtype=np.float64)
                wsum, wdif = wk + wkb, wk - wkb
                B = wsum * dir_deriv(J, 0, 0)
                if self.bc_order >= 2:
                    B = B + 0.5 * dt * wsum * dir_deriv(J, 0, 1) + 0.5 * dt * (wk * Rn + wkb * Rn)
                if self.bc_order >= 3:
                    B = B - dt * dt / 8.0 * wsum * dir_deriv(J, 2, 0) - dt * dt / 4.0 * wdif * dir_deriv(J, 1, 1)
                if self.bc_order >= 4:
                    B = B - dt ** 3 / 8.0 * wdif * dir_deriv(J, 1, 2) - dt ** 3 / 16.0 * wsum * dir_deriv(J, 2, 1) \
                        - dt ** 3 / 24.0 * wsum * dir_deriv(J, 0, 3)
                val = -star[kb, sites] + B
            nxt[links, sites] = val
            cur, nxt = nxt, cur
        return cur

    def phi(self, f) -> np.ndarray:
        out = np.empty(self.S)
        lib().orc_phi(ctypes.byref(self._m), _p(np.ascontiguousarray(f)), _p(out))
        return out

    def entropy(self, f) -> float:
        return lib().orc_entropy(ctypes.byref(self._m), _p(np.ascontiguousarray(f)))

    # adjoint (periodic and Dirichlet boxes)
    def adjoint_step(self, lam_next, gR=None) -> np.ndarray:
        lam = np.empty_like(lam_next)
        lib().orc_adjoint_step(ctypes.byref(self._m), _p(np.ascontiguousarray(lam_next)), _p(lam), _p(gR))
        return lam

    def adjoint_init(self, lam0, order=3, grad_is_fd=True):
        gphi = np.empty(self.S)
        ggrad = np.zeros((self.d, self.S))
        lib().orc_adjoint_init(ctypes.byref(self._m), int(order), int(bool(grad_is_fd)),
                               _p(np.ascontiguousarray(lam0)), _p(gphi), _p(ggrad))
        return gphi, ggrad

    def gradient(self, phi0, Rfield, target, T, order=3, grad=None, wave=None):
        """Loss L = 1/2 sum_x (phi(T) - target)^2 and its exact discrete gradients w.r.t. phi0,
        the source field R(x) and (when grad is given) grad phi0. Dirichlet boxes take their
        boundary data (wave) and an explicit grad phi0; the R gradient is then that of the
        collision source only. Stores every state (tiny grids)."""
        grad_is_fd = grad is None
        if self.bc != "periodic" and grad_is_fd:
            raise ValueError("Dirichlet boxes need an explicit grad phi0")
        f = self.init(phi0, grad, order)
        states = [f]
        for n in range(T):
            f = self.step(f, n0=n, nsteps=1, wave=wave, Rfield=Rfield)
            states.append(f)
        phiT = self.phi(f)
        r = phiT - np.asarray(target).reshape(self.S)
        loss = 0.5 * float(np.dot(r, r))
        lam = np.ascontiguousarray(np.broadcast_to(r, (self.Q, self.S)).copy())
        gR = np.zeros(self.S)
        for n in range(T - 1, -1, -1):
            lam = self.adjoint_step(lam, gR)
        gphi0, ggrad = self.adjoint_init(lam, order, grad_is_fd)
        return loss, gphi0, gR, ggrad


def rmse(phi, phi_exact) -> float:
    """Eq. (rmse): root-mean-square error over all lattice points."""
    d = np.asarray(phi) - np.asarray(phi_exact)
    return float(np.sqrt(np.mean(d * d)))


# ---------------------------------------------------------------------- stability maps (Sec. 4)

def amplification_matrix(d: int, sigma, xi, s: float = 2.0, g: float = 0.5) -> np.ndarray:
    """Eq. (G) in moment space: G(xi) = M T(xi) M^{-1} ((1 - s) I + s eps e_1^T), T = diag(exp(-i c_k . xi))
    (the i of the Fourier variable restored), eps the EDF moment vector with the m4 rule."""
    sigma = np.asarray(sigma, dtype=np.float64)
    M = moment_matrix(d)
    e = velocities(d)
    ep = eps(d, sigma, m4_rule(d, sigma, g)) if d > 1 else eps(d, sigma, 0.0)
    Q = M.shape[0]
    T = np.diag(np.exp(-1j * (e @ np.asarray(xi, dtype=np.float64))))
    E1 = np.zeros(Q)
    E1[0] = 1.0
    C = (1.0 - s) * np.eye(Q) + s * np.outer(ep, E1)
    return M @ T @ np.linalg.solve(M, C)


def stability_map(d: int, sigmas, nxi: int, tau: float = 0.5, g: float = 0.5):
    """For each velocity sigma (rows of sigmas): min_k omega_k (Prop. 1: the microscopic entropy
    conditions are omega_k > 0) and the largest spectral radius of G(xi) over the grid
    xi_i = -pi + 2 pi j / nxi, j = 0..nxi-1 (von Neumann L2 stability, Sec. 4.2)."""
    sigmas = np.atleast_2d(np.asarray(sigmas, dtype=np.float64))
    grid = -np.pi + 2.0 * np.pi * np.arange(nxi) / nxi
    xis = np.stack(np.meshgrid(*([grid] * d), indexing="ij"), axis=-1).reshape(-1, d)
    omin, rho = np.empty(len(sigmas)), np.empty(len(sigmas))
    for p, sig in enumerate(sigmas):
        m4 = m4_rule(d, sig, g) if d > 1 else 0.0
        omin[p] = np.min(weights_closed(d, sig, m4))
        rho[p] = max(np.max(np.abs(np.linalg.eigvals(amplification_matrix(d, sig, xi, 1.0 / tau, g)))) for xi in xis)
    return rho, omin
