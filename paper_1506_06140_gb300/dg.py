"""Thin Python binding of libdg (ctypes).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step of the computation runs in libdg's kernels.  There is
no CPU path: if ``libdg.so`` is missing this module raises on first use.
"""
import ctypes as C
import json
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdg.so")

DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_OOM, DG_ERR_NONPHYSICAL, DG_ERR_TIMEOUT, \
    DG_ERR_UNSUPPORTED = range(7)
DG_BC_PERIODIC, DG_BC_TRANSMISSIVE = 0, 1
LIMITERS = {"none": 0, "component": 1, "characteristic": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_tc": 2, "mixed": 3, "mixed_tc": 4}
BASES = {"total": 0, "tensor": 1}

EXPORTS = ["dg_default_options", "dg_create", "dg_destroy", "dg_last_error", "dg_sizes",
           "dg_quad_points", "dg_l1_points", "dg_project", "dg_rhs", "dg_compute_dt",
           "dg_rk_step", "dg_advance", "dg_rk_step_adjoint", "dg_limit", "dg_totals",
           "dg_l1_density", "dg_node_weights", "dg_neighbor_table", "dg_cell_levels",
           "dg_status", "dg_profile_begin", "dg_profile_end", "dg_totals_noalloc",
           "dg_create_batch", "dg_batch_advance", "dg_n_problems", "dg_tiles",
           "dg_limiter_counts", "dg_set_tiles", "dg_adapt_mark", "dg_adapt_set", "dg_regrid",
           "dg_set_gravity", "dg_test_force_timeout", "dg_set_advance_mode", "dg_advance_mode",
           "dg_advance_dt", "dg_set_overlap", "dg_overlap", "dg_test_flux_math",
           "dg_test_mesh_tables", "dg_test_stage_program"]
DG_TEST_OP_DOUBLES = 27
KERNEL_KINDS = ["face", "cell", "limit", "dt", "other", "adjoint"]
ADVANCE_MODES = {"graph": 0, "persistent": 1}


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("bc", C.c_int * 3), ("n_refine_boxes", C.c_int),
                ("refine_boxes", C.POINTER(C.c_int32))]


class Options(C.Structure):
    _fields_ = [("rk_order", C.c_int), ("cfl", C.c_double), ("slope_limiter", C.c_int),
                ("beta", C.c_double), ("Mtilde", C.c_double), ("positivity", C.c_int),
                ("eps", C.c_double), ("precision", C.c_int), ("autotune", C.c_int),
                ("basis", C.c_int)]


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libdg error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load libdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdg.so not found at %s: build it with "
                           "paper_1506_06140_gb300.build.build()" % path)
    L = C.CDLL(path)
    vp, i32p, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)
    L.dg_default_options.argtypes = [C.POINTER(Options)]
    L.dg_create.argtypes = [C.POINTER(MeshDesc), C.c_int, C.c_double, C.POINTER(Options),
                            C.POINTER(vp)]
    L.dg_destroy.argtypes = [vp]
    L.dg_last_error.restype = C.c_char_p
    L.dg_last_error.argtypes = [vp]
    L.dg_sizes.argtypes = [vp, C.POINTER(C.c_int64)] + [C.POINTER(C.c_int)] * 5
    for name in ("dg_quad_points", "dg_l1_points"):
        getattr(L, name).argtypes = [vp, vp, vp]
    L.dg_project.argtypes = [vp, vp, vp, vp]
    L.dg_rhs.argtypes = [vp, vp, vp, vp]
    L.dg_compute_dt.argtypes = [vp, vp, vp, vp]
    L.dg_rk_step.argtypes = [vp, vp, C.c_double, vp, vp]
    L.dg_advance.argtypes = [vp, vp, C.c_int, vp, vp]
    L.dg_advance_dt.argtypes = [vp, vp, C.c_int, C.c_double, vp]
    L.dg_set_overlap.argtypes = [vp, C.c_int]
    L.dg_test_flux_math.argtypes = [C.c_int, vp, vp, C.c_int64, vp]
    L.dg_overlap.argtypes = [vp, C.POINTER(C.c_int)]
    L.dg_rk_step_adjoint.argtypes = [vp, vp, C.c_double, vp, vp, vp]
    L.dg_limit.argtypes = [vp, vp, vp]
    L.dg_totals.argtypes = [vp, vp, vp, vp]
    L.dg_l1_density.argtypes = [vp, vp, vp, vp, vp]
    L.dg_node_weights.argtypes = [vp, vp, vp, vp]
    L.dg_neighbor_table.argtypes = [vp, i32p]
    L.dg_cell_levels.argtypes = [vp, i32p]
    L.dg_status.argtypes = [vp, C.POINTER(C.c_int)]
    L.dg_create_batch.argtypes = [C.POINTER(MeshDesc), C.POINTER(C.c_double), C.c_int, C.c_int,
                                  C.POINTER(Options), C.POINTER(vp)]
    L.dg_batch_advance.argtypes = [vp, vp, C.c_int, vp, vp]
    L.dg_n_problems.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64)]
    L.dg_totals_noalloc.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_double, vp, vp,
                                     vp, vp]
    i64p = C.POINTER(C.c_int64)
    L.dg_adapt_mark.argtypes = [vp, vp, C.c_double, C.c_double, i32p, i64p, i64p, vp]
    L.dg_adapt_set.argtypes = [vp, i32p, i64p, i64p, vp]
    L.dg_regrid.argtypes = [vp, vp, vp, vp]
    L.dg_set_gravity.argtypes = [vp, vp, vp]
    L.dg_test_force_timeout.argtypes = [vp]
    L.dg_test_mesh_tables.argtypes = [C.POINTER(MeshDesc), C.c_int, i64p, i32p, i32p, i32p, i32p, i32p]
    L.dg_test_stage_program.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int,
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.dg_set_advance_mode.argtypes = [vp, C.c_int]
    L.dg_advance_mode.argtypes = [vp, C.POINTER(C.c_int)]
    L.dg_profile_begin.argtypes = [vp]
    L.dg_profile_end.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int]
    for name in EXPORTS:
        getattr(L, name).restype = C.c_int if name != "dg_last_error" else C.c_char_p
    _lib = L
    return L


CHECKPOINT_VERSION = 1


def _plain_mesh(m):
    """A mesh dict with plain JSON values (for checkpoints)."""
    d = int(m["dim"])
    return dict(dim=d, n=[int(x) for x in m["n"][:d]], lo=[float(x) for x in m["lo"][:d]],
                hi=[float(x) for x in m["hi"][:d]],
                bc=[int(x) for x in (m.get("bc") or [DG_BC_PERIODIC] * d)[:d]],
                refine_boxes=[[int(x) for x in b] for b in (m.get("refine_boxes") or [])])


def _fill_desc(md, m):
    """Fills the MeshDesc md from a mesh dict; returns the refinement-box
    array md points into (keep it alive while md is used)."""
    md.dim = m["dim"]
    for a in range(3):
        md.n[a] = int(m["n"][a]) if a < md.dim else 1
        md.lo[a] = float(m["lo"][a]) if a < md.dim else 0.0
        md.hi[a] = float(m["hi"][a]) if a < md.dim else 1.0
        bc = m.get("bc") or [DG_BC_PERIODIC] * md.dim
        md.bc[a] = int(bc[a]) if a < md.dim else 0
    boxes = m.get("refine_boxes") or []
    arr = np.ascontiguousarray(np.array(boxes, dtype=np.int32).reshape(-1))
    md.n_refine_boxes = len(boxes)
    md.refine_boxes = arr.ctypes.data_as(C.POINTER(C.c_int32)) if len(boxes) else None
    return arr


def mesh_tables(mesh):
    """Test hook, host only: the mesh tables the library builds for a mesh
    dict, or a list of them for an ensemble (dg_test_mesh_tables), as numpy
    arrays: nbr [2 dim][cells], levels [cells], faces [3][faces] (minus cell,
    plus cell, packed info), sface [2 dim][cells] and prob [cells], plus the
    node count."""
    L = load()
    meshes = list(mesh) if isinstance(mesh, (list, tuple)) else [mesh]
    descs = (MeshDesc * len(meshes))()
    keep = [_fill_desc(md, m) for md, m in zip(descs, meshes)]
    counts = (C.c_int64 * 3)()
    r = L.dg_test_mesh_tables(descs, len(meshes), counts, None, None, None, None, None)
    if r != DG_OK:
        raise DGError(r, "dg_test_mesh_tables")
    nc, nf, nn = counts[0], counts[1], counts[2]
    d = meshes[0]["dim"]
    nbr = np.empty((2 * d, nc), np.int32)
    lev = np.empty(nc, np.int32)
    faces = np.empty((3, nf), np.int32)
    sface = np.empty((2 * d, nc), np.int32)
    prob = np.empty(nc, np.int32)
    p32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    r = L.dg_test_mesh_tables(descs, len(meshes), counts, p32(nbr), p32(lev), p32(faces), p32(sface),
                              p32(prob))
    del keep
    if r != DG_OK:
        raise DGError(r, "dg_test_mesh_tables")
    return dict(nbr=nbr, levels=lev, faces=faces, sface=sface, prob=prob, n_nodes=nn)


def stage_program(rk_order, limited):
    """Test hook, host only: the stage program of one RK step
    (dg_test_stage_program) as a list of dicts (in_reg, ins, outs, C, ck,
    lim_src, lim_dst) and the number of scratch registers."""
    L = load()
    n_ops, n_regs = C.c_int(), C.c_int()
    r = L.dg_test_stage_program(int(rk_order), int(limited), None, 0, C.byref(n_ops), C.byref(n_regs))
    if r != DG_OK:
        raise DGError(r, "dg_test_stage_program")
    buf = np.zeros((n_ops.value, DG_TEST_OP_DOUBLES))
    r = L.dg_test_stage_program(int(rk_order), int(limited), buf.ctypes.data_as(C.POINTER(C.c_double)),
                                n_ops.value, C.byref(n_ops), C.byref(n_regs))
    if r != DG_OK:
        raise DGError(r, "dg_test_stage_program")
    ops = []
    for rec in buf:
        n_in, n_out = int(rec[1]), int(rec[2])
        ops.append(dict(in_reg=int(rec[0]), ins=[int(x) for x in rec[5:5 + n_in]],
                        outs=[int(x) for x in rec[9:9 + n_out]],
                        C=rec[12:24].reshape(3, 4)[:n_out, :n_in].copy(), ck=rec[24:24 + n_out].copy(),
                        lim_src=int(rec[3]), lim_dst=int(rec[4])))
    return ops, n_regs.value


def flux_math_check(op, x):
    """Test hook: the flux formulas' reciprocal ("recip", FP64; "recip32", FP32)
    or square root ("sqrt", "sqrt32") of every entry of the float64 CUDA
    tensor x (dg_test_flux_math; the FP32 ones of float(x), widened)."""
    L = load()
    assert x.is_cuda and x.dtype == torch.float64
    x = x.contiguous()
    out = torch.empty_like(x)
    r = L.dg_test_flux_math({"recip": 0, "sqrt": 1, "recip32": 2, "sqrt32": 3}[op], _ptr(x), _ptr(out),
                             x.numel(), _stream())
    if r != DG_OK:
        raise DGError(r, "dg_test_flux_math")
    return out


def totals_noalloc(W, dim, dx0, levels=None, out=None):
    """Conserved totals of a state without a handle and without any device
    allocation inside the library (see dg_totals_noalloc in include/dg.h).
    W: [dim+2][N][cells] float64/float32 CUDA tensor; levels: optional int32
    CUDA tensor of per-cell refinement levels; out: float64 CUDA tensor [dim+2]."""
    L = load()
    assert W.is_cuda and W.is_contiguous() and W.dim() == 3 and W.shape[0] == dim + 2
    prec = PRECISIONS["fp64"] if W.dtype == torch.float64 else PRECISIONS["fp32"]
    if levels is not None:
        assert levels.device == W.device and levels.dtype == torch.int32
        assert levels.numel() == W.shape[2]
    if out is None:
        out = torch.empty(dim + 2, dtype=torch.float64, device=W.device)
    assert out.device == W.device and out.dtype == torch.float64 and out.numel() >= dim + 2
    # the library runs on the current device and looks up its scratch there:
    # make W's device current and launch on that device's current stream
    with torch.cuda.device(W.device):
        r = L.dg_totals_noalloc(dim, W.shape[1], W.shape[2], prec, float(dx0),
                                _ptr(levels) if levels is not None else None, _ptr(W), _ptr(out),
                                torch.cuda.current_stream(W.device).cuda_stream)
    if r != DG_OK:
        raise DGError(r, "dg_totals_noalloc failed")
    return out


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """One DG problem on the current CUDA device (see include/dg.h)."""

    def __init__(self, mesh, k, gamma=1.4, rk_order=3, cfl=0.2, limiter="none", beta=1.0,
                 Mtilde=0.5, positivity=False, eps=1e-10, precision="fp64", autotune=False,
                 basis="total"):
        """mesh: one mesh dict, or a list of them for an ensemble of
        independent problems advanced together (dg_create_batch).
        basis: "total" (the paper's total-degree space) or "tensor" (Q_k,
        (k+1)^2 coefficients per variable; 2D, fp64/fp32, no limiter)."""
        L = load()
        self._L = L
        meshes = list(mesh) if isinstance(mesh, (list, tuple)) else [mesh]
        self.batch = isinstance(mesh, (list, tuple))
        # the arguments save_checkpoint records to rebuild the handle
        self._args = dict(meshes=[dict(m) for m in meshes], k=k, gamma=gamma, rk_order=rk_order, cfl=cfl, limiter=limiter,
                          beta=beta, Mtilde=Mtilde, positivity=positivity, eps=eps, precision=precision,
                          basis=basis)
        self.mesh = dict(meshes[0])
        self.dim, self.k, self.gamma = meshes[0]["dim"], k, gamma
        descs = (MeshDesc * len(meshes))()
        self._boxes = [_fill_desc(md, m) for md, m in zip(descs, meshes)]
        opt = Options()
        L.dg_default_options(C.byref(opt))
        opt.rk_order, opt.cfl = rk_order, cfl
        opt.slope_limiter = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
        opt.beta, opt.Mtilde = beta, Mtilde
        opt.positivity, opt.eps = int(bool(positivity)), eps
        opt.precision = PRECISIONS[precision]
        opt.autotune = int(bool(autotune))
        opt.basis = BASES[basis]
        self.precision = precision
        self.basis = basis
        self.dtype = torch.float64 if precision in ("fp64", "mixed", "mixed_tc") else torch.float32
        torch.cuda.init()
        h = C.c_void_p()
        if self.batch:
            gam = (C.c_double * len(meshes))(*([gamma] * len(meshes)))
            r = L.dg_create_batch(descs, gam, len(meshes), k, C.byref(opt), C.byref(h))
        else:
            r = L.dg_create(descs, k, gamma, C.byref(opt), C.byref(h))
        if r != DG_OK:
            raise DGError(r, L.dg_last_error(None).decode())
        self._h = h
        self._next_cells = None
        self._sizes()
        self.n_base = int(np.prod([int(self.mesh["n"][a]) for a in range(self.dim)]))
        self.device = torch.device("cuda", torch.cuda.current_device())
        npb = C.c_int()
        self._check(L.dg_n_problems(h, C.byref(npb), None))
        self.n_problems = npb.value
        offs = (C.c_int64 * (self.n_problems + 1))()
        self._check(L.dg_n_problems(h, C.byref(npb), offs))
        self.cell_offsets = np.array(offs[:], dtype=np.int64)

    def _sizes(self):
        nc, N, nv, nq, nq1, nn = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(self._L.dg_sizes(self._h, C.byref(nc), C.byref(N), C.byref(nv), C.byref(nq),
                                     C.byref(nq1), C.byref(nn)))
        self.n_cells, self.N, self.nv = nc.value, N.value, nv.value
        self.nq, self.nq1, self.n_nodes = nq.value, nq1.value, nn.value
        if hasattr(self, "cell_offsets"):
            self.cell_offsets = np.array([0, self.n_cells], dtype=np.int64)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.dg_destroy(h)
            self._h = None

    def _check(self, r):
        if r != DG_OK:
            raise DGError(r, self._L.dg_last_error(self._h if hasattr(self, "_h") else None).decode())

    def _state(self, W):
        assert W.is_cuda and W.dtype == self.dtype and W.is_contiguous(), "bad state tensor"
        assert tuple(W.shape) == (self.nv, self.N, self.n_cells), "bad state shape"
        return _ptr(W)

    # -- allocation helpers (torch owns the memory) --
    def empty_state(self):
        return torch.empty((self.nv, self.N, self.n_cells), dtype=self.dtype, device=self.device)

    def dt_buffer(self, n_steps=1):
        """device buffer for timesteps: one per problem and step"""
        return torch.zeros(n_steps * self.n_problems, dtype=torch.float64, device=self.device)

    def scalar(self, n=1):
        return torch.zeros(n, dtype=torch.float64, device=self.device)

    # -- C-ABI calls --
    def quad_points(self):
        out = torch.empty((self.dim, self.nq, self.n_cells), dtype=torch.float64, device=self.device)
        self._check(self._L.dg_quad_points(self._h, _ptr(out), _stream()))
        return out

    def l1_points(self):
        out = torch.empty((self.dim, self.nq1, self.n_cells), dtype=torch.float64, device=self.device)
        self._check(self._L.dg_l1_points(self._h, _ptr(out), _stream()))
        return out

    def project(self, u, out=None):
        u = u.to(device=self.device, dtype=torch.float64).contiguous()
        assert tuple(u.shape) == (self.nv, self.nq, self.n_cells)
        W = self.empty_state() if out is None else out
        self._check(self._L.dg_project(self._h, _ptr(u), self._state(W), _stream()))
        return W

    def rhs(self, W, out=None):
        out = self.empty_state() if out is None else out
        self._check(self._L.dg_rhs(self._h, self._state(W), self._state(out), _stream()))
        return out

    def compute_dt(self, W, out=None):
        out = self.scalar(self.n_problems) if out is None else out
        self._check(self._L.dg_compute_dt(self._h, self._state(W), _ptr(out), _stream()))
        return out

    def rk_step(self, W, dt=0.0, dt_out=None):
        """One RK step in place; dt <= 0 uses the CFL timestep."""
        p = _ptr(dt_out) if dt_out is not None else None
        self._check(self._L.dg_rk_step(self._h, self._state(W), float(dt), p, _stream()))
        return W

    def advance(self, W, n_steps, dt_hist=None, dt=None):
        """n_steps steps in place through a cached CUDA graph: CFL steps, or
        steps of the fixed timestep dt (dg_advance_dt; no dt_hist then)."""
        if dt is not None:
            assert dt_hist is None
            self._check(self._L.dg_advance_dt(self._h, self._state(W), int(n_steps), float(dt), _stream()))
            return W
        p = _ptr(dt_hist) if dt_hist is not None else None
        self._check(self._L.dg_advance(self._h, self._state(W), int(n_steps), p, _stream()))
        return W

    def rk_step_adjoint(self, W_n, dt, lam_np1, out=None):
        out = self.empty_state() if out is None else out
        self._check(self._L.dg_rk_step_adjoint(self._h, self._state(W_n), float(dt),
                                               self._state(lam_np1), self._state(out), _stream()))
        return out

    def limit(self, W):
        self._check(self._L.dg_limit(self._h, self._state(W), _stream()))
        return W

    def totals(self, W, out=None):
        out = self.scalar(self.nv) if out is None else out
        self._check(self._L.dg_totals(self._h, self._state(W), _ptr(out), _stream()))
        return out

    def l1_density(self, W, rho_ref, out=None):
        rho_ref = rho_ref.to(device=self.device, dtype=torch.float64).contiguous()
        assert tuple(rho_ref.shape) == (self.nq1, self.n_cells)
        out = self.scalar() if out is None else out
        self._check(self._L.dg_l1_density(self._h, self._state(W), _ptr(rho_ref), _ptr(out),
                                          _stream()))
        return out

    def node_weights(self, W):
        out = torch.empty((self.nv, self.N, max(self.n_nodes, 1)), dtype=self.dtype,
                          device=self.device)
        self._check(self._L.dg_node_weights(self._h, self._state(W), _ptr(out), _stream()))
        return out[:, :, : self.n_nodes]

    def neighbor_table(self):
        out = np.zeros((2 * self.dim, self.n_cells), np.int32)
        self._check(self._L.dg_neighbor_table(self._h, out.ctypes.data_as(C.POINTER(C.c_int32))))
        return out

    def levels(self):
        out = np.zeros(self.n_cells, np.int32)
        self._check(self._L.dg_cell_levels(self._h, out.ctypes.data_as(C.POINTER(C.c_int32))))
        return out

    def set_gravity(self, accel):
        """external acceleration [dim][nq][cells] at quad_points() (None removes it)"""
        if accel is None:
            self._check(self._L.dg_set_gravity(self._h, None, _stream()))
            return
        a = torch.as_tensor(accel).to(device=self.device, dtype=torch.float64).contiguous()
        assert tuple(a.shape) == (self.dim, self.nq, self.n_cells)
        self._check(self._L.dg_set_gravity(self._h, _ptr(a), _stream()))

    # -- mesh adaptation (single problems) --
    def adapt_mark(self, W, w_t=0.01, alpha=1.1, flags=False):
        """Decide the next refinement from W (dg_adapt_mark): returns
        (cells of the next mesh, base cells that change[, int32 flags per base cell])."""
        nc, ch = C.c_int64(), C.c_int64()
        fl = np.zeros(self.n_base, np.int32) if flags else None
        fp = fl.ctypes.data_as(C.POINTER(C.c_int32)) if flags else None
        self._check(self._L.dg_adapt_mark(self._h, self._state(W), float(w_t), float(alpha), fp,
                                          C.byref(nc), C.byref(ch), _stream()))
        self._next_cells = nc.value
        return (nc.value, ch.value, fl) if flags else (nc.value, ch.value)

    def set_refinement(self, flags):
        """Mark the next refinement explicitly (nonzero = refined base cell)."""
        fl = np.ascontiguousarray(np.asarray(flags, dtype=np.int32).reshape(-1))
        assert fl.size == self.n_base
        nc, ch = C.c_int64(), C.c_int64()
        self._check(self._L.dg_adapt_set(self._h, fl.ctypes.data_as(C.POINTER(C.c_int32)),
                                         C.byref(nc), C.byref(ch), _stream()))
        self._next_cells = nc.value
        return nc.value, ch.value

    def regrid(self, W_old, out=None):
        """Move to the marked mesh; returns the state projected onto it."""
        assert self._next_cells is not None, "no refinement marked"
        shape = (self.nv, self.N, self._next_cells)
        W_new = torch.empty(shape, dtype=self.dtype, device=self.device) if out is None else out
        assert W_new.is_cuda and W_new.is_contiguous() and W_new.dtype == self.dtype
        assert tuple(W_new.shape) == shape
        self._check(self._L.dg_regrid(self._h, self._state(W_old), _ptr(W_new), _stream()))
        self._next_cells = None
        self._sizes()
        return W_new

    def adapt(self, W, w_t=0.01, alpha=1.1):
        """One adaptation after a step (Sec. 4): returns (state on the adapted
        mesh, base cells changed); W itself is returned when nothing changes."""
        nc, changed = self.adapt_mark(W, w_t, alpha)
        if changed == 0:
            return W, 0
        return self.regrid(W), changed

    def refinement(self):
        """int32 flag per base cell of the current mesh (1 refined)"""
        lv = self.levels()
        out = np.zeros(self.n_base, np.int32)
        c, nch = 0, 1 << self.dim
        for b in range(self.n_base):
            out[b] = lv[c]
            c += nch if lv[c] else 1
        return out

    # -- checkpoint / resume --
    def save_checkpoint(self, path, W, **meta):
        """Writes what resuming needs to one .npz file: the state W (copied to
        the host), the constructor's arguments, the current refinement of the
        base cells (a single problem's mesh after adaptation) and meta (JSON
        values, e.g. t= and step=).  Not recorded: the tiles (from_checkpoint
        can autotune again), the advance mode and a gravity field (set it
        again after resuming)."""
        assert tuple(W.shape) == (self.nv, self.N, self.n_cells), "bad state shape"
        a = self._args
        limiter = a["limiter"] if isinstance(a["limiter"], str) else int(a["limiter"])
        config = dict(meshes=[_plain_mesh(m) for m in a["meshes"]], batch=self.batch, k=int(a["k"]),
                      gamma=float(a["gamma"]), rk_order=int(a["rk_order"]), cfl=float(a["cfl"]),
                      limiter=limiter, beta=float(a["beta"]), Mtilde=float(a["Mtilde"]),
                      positivity=bool(a["positivity"]), eps=float(a["eps"]), precision=a["precision"],
                      basis=a["basis"])
        ref = np.zeros(0, np.int32) if self.batch else self.refinement()
        with open(path, "wb") as f:
            np.savez(f, version=np.int64(CHECKPOINT_VERSION), config=np.array(json.dumps(config)),
                     refinement=ref, W=W.detach().cpu().numpy(), meta=np.array(json.dumps(meta)))

    @classmethod
    def from_checkpoint(cls, path, autotune=False):
        """(solver, W, meta) from a save_checkpoint file: the handle is built
        from the recorded arguments, moved to the recorded refinement, and W
        is the recorded state on this device."""
        with np.load(path, allow_pickle=False) as d:
            version = int(d["version"])
            if version != CHECKPOINT_VERSION:
                raise ValueError("checkpoint version %d, expected %d" % (version, CHECKPOINT_VERSION))
            cfg = json.loads(str(d["config"]))
            ref = np.array(d["refinement"], dtype=np.int32)
            Wh = np.array(d["W"])
            meta = json.loads(str(d["meta"]))
        meshes, batch = cfg.pop("meshes"), cfg.pop("batch")
        s = cls(meshes if batch else meshes[0], autotune=autotune, **cfg)
        if not batch and not np.array_equal(s.refinement(), ref):
            s.set_refinement(ref)
            s.regrid(s.empty_state().zero_())  # the projected values are replaced by W below
        W = torch.as_tensor(Wh).to(device=s.device, dtype=s.dtype).contiguous()
        if tuple(W.shape) != (s.nv, s.N, s.n_cells):
            raise ValueError("checkpoint state %s does not fit the rebuilt mesh %s"
                             % (tuple(W.shape), (s.nv, s.N, s.n_cells)))
        return s, W, meta

    def profile_begin(self):
        self._check(self._L.dg_profile_begin(self._h))

    def profile_end(self):
        """{kind: (launches, total_ms)} of the launches since profile_begin."""
        n = len(KERNEL_KINDS)
        cnt, ms = (C.c_int * n)(), (C.c_double * n)()
        self._check(self._L.dg_profile_end(self._h, cnt, ms, n))
        return {k: (cnt[i], ms[i]) for i, k in enumerate(KERNEL_KINDS)}

    def limiter_counts(self, reset=False, out=None):
        """device int64[3]: cell passes changed by the slope / positivity limiter,
        and cell passes examined by the FP64 positivity pass"""
        out = torch.zeros(3, dtype=torch.int64, device=self.device) if out is None else out
        self._check(self._L.dg_limiter_counts(self._h, _ptr(out), int(bool(reset)), _stream()))
        return out

    def set_tiles(self, cell_tile, face_tile):
        """cell_tile 16/32/64 (or 1: one thread per cell, FP32 2D; 2: two variables
        per thread as packed FP32 pairs, FP32 2D), face_tile 16/32/64 (or 0: the
        fused face + cell kernel, single 2D uniform meshes)"""
        self._check(self._L.dg_set_tiles(self._h, int(cell_tile), int(face_tile)))

    def tiles(self):
        """(cells per block of the cell kernel, faces per block of the face kernel)"""
        ct, ft = C.c_int(), C.c_int()
        self._check(self._L.dg_tiles(self._h, C.byref(ct), C.byref(ft)))
        return ct.value, ft.value

    def set_advance_mode(self, mode):
        """"graph" or "persistent": how advance() runs its steps (see dg_set_advance_mode)"""
        self._check(self._L.dg_set_advance_mode(self._h, ADVANCE_MODES[mode]))

    def set_overlap(self, on):
        """launch the step's kernels as programmatic dependents (dg_set_overlap)"""
        self._check(self._L.dg_set_overlap(self._h, int(bool(on))))

    def overlap(self):
        v = C.c_int()
        self._check(self._L.dg_overlap(self._h, C.byref(v)))
        return bool(v.value)

    def advance_mode(self):
        m = C.c_int()
        self._check(self._L.dg_advance_mode(self._h, C.byref(m)))
        return {v: k for k, v in ADVANCE_MODES.items()}[m.value]

    def force_timeout(self):
        """Test hook: the next tensor-core cell launch outside a graph gives up
        a bounded wait in its first CTA (see dg_test_force_timeout)."""
        self._check(self._L.dg_test_force_timeout(self._h))

    def status(self):
        s = C.c_int()
        self._check(self._L.dg_status(self._h, C.byref(s)))
        return s.value
