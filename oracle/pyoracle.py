"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Arrays are numpy float64 / int32 in the library's interface layouts:
weights ``W[var][coef][cell]``, point values ``u[var][q][cell]``,
coordinates ``xyz[axis][q][cell]``, neighbour table ``nbr[side][cell]``.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None

LIM_NONE, LIM_COMPONENT, LIM_CHARACTERISTIC = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE = 0, 1

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_I32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, _I, _D, _D, _I, C.c_int, _I, C.c_int, C.c_double,
                                 C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                 C.c_double, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_last_error.restype = C.c_char_p
        for name in ("orc_n_cells",):
            getattr(L, name).restype = C.c_int64
            getattr(L, name).argtypes = [C.c_void_p]
        for name in ("orc_n_nodes", "orc_n_basis", "orc_n_vars", "orc_n_qpoints",
                     "orc_n_l1points"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_void_p]
        L.orc_cell_levels.argtypes = [C.c_void_p, _I32]
        L.orc_cell_dx.argtypes = [C.c_void_p, _D]
        L.orc_neighbor_table.argtypes = [C.c_void_p, _I32]
        L.orc_node_children.argtypes = [C.c_void_p, _I32]
        L.orc_quad_points.argtypes = [C.c_void_p, _D]
        L.orc_l1_points.argtypes = [C.c_void_p, _D]
        L.orc_project.argtypes = [C.c_void_p, _D, _D]
        L.orc_rhs.argtypes = [C.c_void_p, _D, _D]
        L.orc_compute_dt.restype = C.c_double
        L.orc_compute_dt.argtypes = [C.c_void_p, _D]
        L.orc_set_accel.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_rk_step.restype = C.c_double
        L.orc_rk_step.argtypes = [C.c_void_p, _D, C.c_double]
        L.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
        for name in ("orc_slope_limit", "orc_positivity_limit", "orc_limit"):
            getattr(L, name).argtypes = [C.c_void_p, _D]
        L.orc_totals.argtypes = [C.c_void_p, _D, _D]
        L.orc_l1_density.restype = C.c_double
        L.orc_l1_density.argtypes = [C.c_void_p, _D, _D]
        L.orc_node_weights.argtypes = [C.c_void_p, _D, _D]
        L.orc_n_base.restype = C.c_int
        L.orc_n_base.argtypes = [C.c_void_p]
        L.orc_adapt_flags.argtypes = [C.c_void_p, _D, C.c_double, C.c_double, _I]
        L.orc_adapt_project.argtypes = [C.c_void_p, C.c_void_p, _D, _D]
        L.orc_rhs_cells.argtypes = [C.c_void_p, _D, _I32, C.c_int, _D]
        L.orc_limit_cells.argtypes = [C.c_void_p, _D, _I32, C.c_int, _D]
        L.orc_rk_step_jvp.argtypes = [C.c_void_p, _D, _D, C.c_double, _D, _D]
        L.orc_gauss_legendre.argtypes = [C.c_int, _D, _D]
        L.orc_gauss_lobatto.argtypes = [C.c_int, _D, _D]
        L.orc_legendre.argtypes = [C.c_int, C.c_double, _D, _D]
        L.orc_basis_exponents.argtypes = [C.c_int, C.c_int, _I]
        L.orc_basis_exponents_tensor.argtypes = [C.c_int, C.c_int, _I]
        L.orc_basis_phi_tensor.restype = C.c_double
        L.orc_basis_phi_tensor.argtypes = [C.c_int, C.c_int, C.c_int, _D]
        L.orc_basis_phi.restype = C.c_double
        L.orc_basis_phi.argtypes = [C.c_int, C.c_int, C.c_int, _D]
        L.orc_basis_dphi.restype = C.c_double
        L.orc_basis_dphi.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D]
        L.orc_refinement_matrix.argtypes = [C.c_int, C.c_int, C.c_int, _D]
        L.orc_eigen_matrices.argtypes = [C.c_int, C.c_double, _D, C.c_int, _D, _D]
        L.orc_flux.argtypes = [C.c_int, C.c_double, _D, C.c_int, _D]
        L.orc_flux_jacobian.argtypes = [C.c_int, C.c_double, _D, C.c_int, _D]
        L.orc_hllc.argtypes = [C.c_int, C.c_double, _D, _D, C.c_int, _D]
        L.orc_rk_tableau.restype = C.c_int
        L.orc_rk_tableau.argtypes = [C.c_int, _D, _D, _D]
        L.orc_rk_ode.restype = C.c_double
        L.orc_rk_ode.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int]
        L.orc_minmod_b.restype = C.c_double
        L.orc_minmod_b.argtypes = [C.c_double] * 5
        L.orc_solve_tau.restype = C.c_double
        L.orc_solve_tau.argtypes = [C.c_int, C.c_double, C.c_double, _D, _D]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One DG problem on the CPU oracle."""

    def __init__(self, dim, n, lo, hi, k, gamma=1.4, bc=None, refine_boxes=(), rk_order=2,
                 cfl=0.2, limiter=LIM_NONE, beta=1.0, Mtilde=0.5, positivity=False, eps=1e-10,
                 basis="total"):
        """basis: "total" (total degree <= k, the paper's) or "tensor" (Q_k)"""
        L = lib()
        self.dim, self.k, self.gamma = dim, k, gamma
        n3 = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
        lo3 = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
        hi3 = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
        bc = bc if bc is not None else [BC_PERIODIC] * dim
        bc3 = (C.c_int * 3)(*(list(bc) + [0] * (3 - len(bc))))
        boxes = np.ascontiguousarray(np.array(refine_boxes, dtype=np.int32).reshape(-1))
        nb = len(refine_boxes)
        bptr = boxes.ctypes.data_as(_I) if nb else None
        if basis not in ("total", "tensor"):
            raise ValueError("basis: 'total' or 'tensor'")
        self._h = L.orc_create(dim, n3, lo3, hi3, bc3, nb, bptr, k, gamma, rk_order, cfl,
                               limiter, beta, Mtilde, int(bool(positivity)), eps,
                               int(basis == "tensor"))
        if not self._h:
            raise ValueError(L.orc_last_error().decode())
        self.n_cells = L.orc_n_cells(self._h)
        self.n_nodes = L.orc_n_nodes(self._h)
        self.N = L.orc_n_basis(self._h)
        self.nv = L.orc_n_vars(self._h)
        self.nq = L.orc_n_qpoints(self._h)
        self.nq_l1 = L.orc_n_l1points(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.nv, self.N, self.n_cells)

    def levels(self):
        out = np.zeros(self.n_cells, np.int32)
        lib().orc_cell_levels(self._h, out.ctypes.data_as(_I32))
        return out

    def cell_dx(self):
        out = np.zeros(self.n_cells)
        lib().orc_cell_dx(self._h, _d(out))
        return out

    def neighbor_table(self):
        out = np.zeros((2 * self.dim, self.n_cells), np.int32)
        lib().orc_neighbor_table(self._h, out.ctypes.data_as(_I32))
        return out

    def node_children(self):
        out = np.zeros((self.n_nodes, 2 ** self.dim), np.int32)
        lib().orc_node_children(self._h, out.ctypes.data_as(_I32))
        return out

    def quad_points(self):
        out = np.zeros((self.dim, self.nq, self.n_cells))
        lib().orc_quad_points(self._h, _d(out))
        return out

    def l1_points(self):
        out = np.zeros((self.dim, self.nq_l1, self.n_cells))
        lib().orc_l1_points(self._h, _d(out))
        return out

    def project(self, u_q):
        u_q = _f64(u_q)
        assert u_q.shape == (self.nv, self.nq, self.n_cells)
        W = np.zeros(self.shape)
        lib().orc_project(self._h, _d(u_q), _d(W))
        return W

    def rhs(self, W):
        W = _f64(W)
        out = np.zeros(self.shape)
        lib().orc_rhs(self._h, _d(W), _d(out))
        return out

    def set_accel(self, accel):
        """external acceleration [dim][Q][cells] at quad_points() (None removes it)"""
        if accel is None:
            lib().orc_set_accel(self._h, None)
            self._accel = None
            return
        self._accel = _f64(accel)
        assert self._accel.shape == (self.dim, self.nq, self.n_cells)
        lib().orc_set_accel(self._h, self._accel.ctypes.data_as(C.c_void_p))

    def compute_dt(self, W):
        W = _f64(W)
        return lib().orc_compute_dt(self._h, _d(W))

    def set_threads(self, n):
        """OpenMP threads of rk_step's right-hand side (gather form when n > 1)."""
        lib().orc_set_threads(self._h, int(n))

    def rk_step(self, W, dt=0.0):
        """Advance a copy of W by one step; returns (W_new, dt_used)."""
        W = _f64(W).copy()
        dt = lib().orc_rk_step(self._h, _d(W), dt)
        return W, dt

    def slope_limit(self, W):
        W = _f64(W).copy()
        lib().orc_slope_limit(self._h, _d(W))
        return W

    def positivity_limit(self, W):
        W = _f64(W).copy()
        lib().orc_positivity_limit(self._h, _d(W))
        return W

    def limit(self, W):
        W = _f64(W).copy()
        lib().orc_limit(self._h, _d(W))
        return W

    def totals(self, W):
        W = _f64(W)
        out = np.zeros(self.nv)
        lib().orc_totals(self._h, _d(W), _d(out))
        return out

    def l1_density(self, W, rho_exact):
        W, rho_exact = _f64(W), _f64(rho_exact)
        assert rho_exact.shape == (self.nq_l1, self.n_cells)
        return lib().orc_l1_density(self._h, _d(W), _d(rho_exact))

    def rhs_cells(self, W, cells):
        """dW/dt of the listed cells only, [nv][N][len(cells)]."""
        W = _f64(W)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((len(cells), self.nv, self.N))
        lib().orc_rhs_cells(self._h, _d(W), cells.ctypes.data_as(_I32), len(cells), _d(out))
        return np.moveaxis(out, 0, 2)

    def limit_cells(self, W, cells):
        """Limited weights (slope then positivity) of the listed cells, [nv][N][len(cells)]."""
        W = _f64(W)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((len(cells), self.nv, self.N))
        lib().orc_limit_cells(self._h, _d(W), cells.ctypes.data_as(_I32), len(cells), _d(out))
        return np.moveaxis(out, 0, 2)

    def node_weights(self, W):
        W = _f64(W)
        out = np.zeros((self.nv, self.N, self.n_nodes))
        lib().orc_node_weights(self._h, _d(W), _d(out))
        return out

    def adapt_flags(self, W, w_t=0.01, alpha=1.1):
        """new refinement flag of every base cell (lexicographic, x fastest)"""
        W = _f64(W)
        out = np.zeros(lib().orc_n_base(self._h), dtype=np.int32)
        lib().orc_adapt_flags(self._h, _d(W), w_t, alpha, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out

    def adapt_project(self, old, W_old):
        """this mesh's state from W_old on `old` (same base grid)"""
        W_old = _f64(W_old)
        out = np.zeros(self.shape)
        lib().orc_adapt_project(self._h, old._h, _d(W_old), _d(out))
        return out

    def rk_step_jvp(self, W, V, dt):
        W, V = _f64(W), _f64(V)
        Wo, JV = np.zeros(self.shape), np.zeros(self.shape)
        lib().orc_rk_step_jvp(self._h, _d(W), _d(V), dt, _d(Wo), _d(JV))
        return Wo, JV


# ---- building blocks -------------------------------------------------------

def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(n, _d(x), _d(w))
    return x, w


def gauss_lobatto(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_lobatto(n, _d(x), _d(w))
    return x, w


def legendre(n, x):
    P, dP = np.zeros(n + 2), np.zeros(n + 2)
    lib().orc_legendre(n, float(x), _d(P), _d(dP))
    return P[: n + 1], dP[: n + 1]


def basis_exponents(dim, k):
    N = (k + 1) * (k + 2) // 2 if dim == 2 else (k + 1) * (k + 2) * (k + 3) // 6
    e = np.zeros((N, 3), np.int32)
    lib().orc_basis_exponents(dim, k, e.ctypes.data_as(_I))
    return e


def basis_exponents_tensor(dim, k):
    e = np.zeros(((k + 1) ** dim, 3), np.int32)
    lib().orc_basis_exponents_tensor(dim, k, e.ctypes.data_as(_I))
    return e


def basis_phi_tensor(dim, k, l, xi):
    x = _f64(list(xi) + [0.0] * (3 - len(xi)))
    return lib().orc_basis_phi_tensor(dim, k, l, _d(x))


def basis_phi(dim, k, l, xi):
    x = _f64(list(xi) + [0.0] * (3 - len(xi)))
    return lib().orc_basis_phi(dim, k, l, _d(x))


def basis_dphi(dim, k, l, a, xi):
    x = _f64(list(xi) + [0.0] * (3 - len(xi)))
    return lib().orc_basis_dphi(dim, k, l, a, _d(x))


def refinement_matrix(dim, k, child):
    N = len(basis_exponents(dim, k))
    P = np.zeros((N, N))
    lib().orc_refinement_matrix(dim, k, child, _d(P))
    return P


def eigen_matrices(dim, gamma, u, a):
    nv = dim + 2
    L, R = np.zeros((nv, nv)), np.zeros((nv, nv))
    lib().orc_eigen_matrices(dim, gamma, _d(_f64(u)), a, _d(L), _d(R))
    return L, R


def flux(dim, gamma, u, a):
    f = np.zeros(dim + 2)
    lib().orc_flux(dim, gamma, _d(_f64(u)), a, _d(f))
    return f


def flux_jacobian(dim, gamma, u, a):
    J = np.zeros((dim + 2, dim + 2))
    lib().orc_flux_jacobian(dim, gamma, _d(_f64(u)), a, _d(J))
    return J


def hllc(dim, gamma, uL, uR, a):
    F = np.zeros(dim + 2)
    lib().orc_hllc(dim, gamma, _d(_f64(uL)), _d(_f64(uR)), a, _d(F))
    return F


def rk_tableau(order):
    A, b, c = np.zeros(25), np.zeros(5), np.zeros(5)
    s = lib().orc_rk_tableau(order, _d(A), _d(b), _d(c))
    return A[: s * s].reshape(s, s), b[:s], c[:s]


def rk_ode(order, problem, y0, t_end, nsteps):
    return lib().orc_rk_ode(order, problem, y0, t_end, nsteps)


def minmod_b(a, b, c, Mtilde, dx):
    return lib().orc_minmod_b(a, b, c, Mtilde, dx)


def solve_tau(dim, gamma, eps, ubar, u):
    return lib().orc_solve_tau(dim, gamma, eps, _d(_f64(ubar)), _d(_f64(u)))
