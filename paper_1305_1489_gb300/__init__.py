"""GB300-native HDG hot path (Fu, Gatica, Sayas, arXiv 1305.1489) -- Python binding.

Thin marshalling layer over the C ABI of libhdg (include/hdg.h): the functions below carry
the C names and only convert torch tensors / numpy arrays into pointers.  Every step of the
computation runs in the CUDA kernels of libhdg; there is no CPU path.  PyTorch provides
device memory and the CUDA stream.

    mesh = HDGMesh(coords, elements, dirichlet, neumann, k)   # hdg_mesh_create
    X, Y, Z = mesh.volume_nodes()                             # hdg_quadrature_nodes
    mesh.set_coefficients(kappa, c, f)                        # hdg_set_coefficients
    mesh.set_boundary_data(uD, gN)                            # hdg_set_boundary_data
    mesh.assemble_condense()                                  # hdg_assemble_condense
    uhat, iters, relres = mesh.solve_trace(1e-10)             # hdg_solve_trace
    q, u = mesh.recover(uhat)                                 # hdg_recover
    ustar = mesh.postprocess(q, u)                            # hdg_postprocess
"""

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (HDG_DF32, HDG_FP64, HDG_METHOD_BDM, HDG_METHOD_HDG, HDG_MIXED_BF16, HDG_MIXED_FP32,  # noqa: F401
                   HDG_RULE_CONICAL, HDG_RULE_SYMMETRIC, HDGError)

__all__ = ["HDGMesh", "HDGError", "HDG_FP64", "HDG_MIXED_FP32", "HDG_DF32", "HDG_MIXED_BF16", "HDG_METHOD_HDG", "HDG_METHOD_BDM",
           "HDG_RULE_CONICAL", "HDG_RULE_SYMMETRIC",
           "build", "load_library"]


def build(**kw):
    from .buildlib import build as _b
    return _b(**kw)


def load_library():
    return _lib.load()


def _ptr(t):
    """Device/host pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to libhdg must be contiguous"
    return t.data_ptr()


def _dev_f64(t, shape, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


# ---------------------------------------------------------------- C-named thin wrappers
def hdg_mesh_create(coords, elems, dirichlet, neumann, k, stream=0):
    lib = _lib.load()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    dirichlet = np.ascontiguousarray(np.asarray(dirichlet).reshape(-1, 3), dtype=np.int32)
    neumann = np.ascontiguousarray(np.asarray(neumann).reshape(-1, 3), dtype=np.int32)
    h = C.c_void_p()
    _lib.check(lib.hdg_mesh_create(
        _ptr(coords), coords.shape[0], _ptr(elems), elems.shape[0],
        _ptr(dirichlet) if len(dirichlet) else None, len(dirichlet),
        _ptr(neumann) if len(neumann) else None, len(neumann), int(k), C.c_void_p(stream), C.byref(h)))
    return h


def hdg_mesh_destroy(h):
    return _lib.check(_lib.load().hdg_mesh_destroy(h))


def hdg_mesh_get_info(h):
    info = _lib.MeshInfo()
    _lib.check(_lib.load().hdg_mesh_get_info(h, C.byref(info)))
    return {f: getattr(info, f) for f, _ in _lib.MeshInfo._fields_}


def hdg_mesh_get_faces(h, nelt, nfc):
    faces = np.zeros((nfc, 4), np.int32)
    fbe = np.zeros((nelt, 4), np.int32)
    perm = np.zeros((nelt, 4), np.int32)
    _lib.check(_lib.load().hdg_mesh_get_faces(h, _ptr(faces), _ptr(fbe), _ptr(perm)))
    return faces, fbe, perm


def hdg_quadrature_nodes(h, X, Y, Z, FX, FY, FZ):
    return _lib.check(_lib.load().hdg_quadrature_nodes(h, _ptr(X), _ptr(Y), _ptr(Z), _ptr(FX), _ptr(FY), _ptr(FZ)))


def hdg_set_coefficients(h, kappa, c, beta, f, tau):
    return _lib.check(_lib.load().hdg_set_coefficients(h, _ptr(kappa), _ptr(c), _ptr(beta), _ptr(f), _ptr(tau)))


def hdg_element_face_nodes(h, X, Y, Z):
    return _lib.check(_lib.load().hdg_element_face_nodes(h, _ptr(X), _ptr(Y), _ptr(Z)))


def hdg_set_face_convection(h, beta_f):
    return _lib.check(_lib.load().hdg_set_face_convection(h, _ptr(beta_f)))


def hdg_set_boundary_data(h, uD, gN):
    return _lib.check(_lib.load().hdg_set_boundary_data(h, _ptr(uD), _ptr(gN)))


def hdg_assemble_condense(h, precision=HDG_FP64):
    return _lib.check(_lib.load().hdg_assemble_condense(h, precision))


def hdg_get_condensed(h, Cm, Cf):
    return _lib.check(_lib.load().hdg_get_condensed(h, _ptr(Cm), _ptr(Cf)))


def hdg_solve_trace(h, precision, rtol, maxit, x0, uhat):
    it = C.c_int(0)
    rr = C.c_double(0.0)
    code = _lib.load().hdg_solve_trace(h, precision, float(rtol), int(maxit), _ptr(x0), _ptr(uhat),
                                       C.byref(it), C.byref(rr))
    return code, it.value, rr.value


def hdg_set_inner_tolerance(h, rtol):
    return _lib.check(_lib.load().hdg_set_inner_tolerance(h, float(rtol)))


def hdg_trace_residual(h, x, r):
    rn = C.c_double(0.0)
    bn = C.c_double(0.0)
    _lib.check(_lib.load().hdg_trace_residual(h, _ptr(x), _ptr(r), C.byref(rn), C.byref(bn)))
    return rn.value, bn.value


def hdg_recover(h, uhat, q, u):
    return _lib.check(_lib.load().hdg_recover(h, _ptr(uhat), _ptr(q), _ptr(u)))


def hdg_postprocess(h, q, u, ustar):
    return _lib.check(_lib.load().hdg_postprocess(h, _ptr(q), _ptr(u), _ptr(ustar)))


def hdg_projection(h, q_vol, u_vol, q_face, u_face, Pq, Pu):
    return _lib.check(_lib.load().hdg_projection(h, _ptr(q_vol), _ptr(u_vol), _ptr(q_face), _ptr(u_face),
                                                 _ptr(Pq), _ptr(Pu)))


def hdg_face_projection(h, vals, Pu):
    return _lib.check(_lib.load().hdg_face_projection(h, _ptr(vals), _ptr(Pu)))


def hdg_volume_norm2(h, degree, coef, vals):
    out = (C.c_double * 2)()
    _lib.check(_lib.load().hdg_volume_norm2(h, int(degree), _ptr(coef) if coef is not None else None,
                                            _ptr(vals) if vals is not None else None, out))
    return out[0], out[1]


def hdg_face_norm2(h, coef, vals):
    out = (C.c_double * 2)()
    _lib.check(_lib.load().hdg_face_norm2(h, _ptr(coef) if coef is not None else None,
                                          _ptr(vals) if vals is not None else None, out))
    return out[0], out[1]


def hdg_launch_count(h):
    return int(_lib.load().hdg_launch_count(h))


# ---------------------------------------------------------------- convenience handle
class HDGMesh:
    """Owns one hdg_mesh handle; tensors passed in are kept alive while the library borrows them."""

    def __init__(self, coords, elements, dirichlet, neumann, k, stream=None, _handle=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("HDGMesh needs a CUDA device: libhdg has no CPU path")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._owned = _handle is None
        self._h = _handle if _handle is not None else hdg_mesh_create(coords, elements, dirichlet, neumann, k,
                                                                     self.stream.cuda_stream)
        self.info = hdg_mesh_get_info(self._h)
        for key in ("nelt", "nfc", "k", "n", "d2", "m", "n1", "nq", "nf"):
            setattr(self, key, self.info[key])
        self._keep = {}

    def set_volume_rule(self, rule):
        """hdg_set_volume_rule: HDG_RULE_CONICAL or HDG_RULE_SYMMETRIC (call before setting the
        coefficients; self.nq follows)."""
        _lib.check(_lib.load().hdg_set_volume_rule(self._h, int(rule)))
        self.info = hdg_mesh_get_info(self._h)
        self.nq = self.info["nq"]
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None) is not None:
            if getattr(self, "_owned", True):
                hdg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def faces(self):
        """(faces [nfc,4], facebyele [nelt,4], perm [nelt,4]) as numpy int32."""
        return hdg_mesh_get_faces(self._h, self.nelt, self.nfc)

    def volume_nodes(self):
        X, Y, Z = (self._empty(self.nelt, self.nq) for _ in range(3))
        hdg_quadrature_nodes(self._h, X, Y, Z, None, None, None)
        return X, Y, Z

    def face_nodes(self):
        X, Y, Z = (self._empty(self.nfc, self.nf) for _ in range(3))
        hdg_quadrature_nodes(self._h, None, None, None, X, Y, Z)
        return X, Y, Z

    def element_face_nodes(self):
        """F_K(q_hat_r^l): X, Y, Z [nelt, 4, nf] (where beta enters the face integrals)."""
        X, Y, Z = (self._empty(self.nelt, 4, self.nf) for _ in range(3))
        hdg_element_face_nodes(self._h, X, Y, Z)
        return X, Y, Z

    def set_coefficients(self, kappa, c, f, tau=None, beta=None, beta_faces=None):
        """kappa, c, f [nelt, nq]; tau [nelt, 4]; beta [3, nelt, nq] and beta_faces
        [3, nelt, 4, nf] (convection, both or neither)."""
        kappa = _dev_f64(kappa, (self.nelt, self.nq), "kappa")
        c = _dev_f64(c, (self.nelt, self.nq), "c")
        f = _dev_f64(f, (self.nelt, self.nq), "f")
        if tau is not None:
            tau = _dev_f64(tau, (self.nelt, 4), "tau")
        if (beta is None) != (beta_faces is None):
            raise ValueError("beta and beta_faces go together")
        if beta is not None:
            beta = _dev_f64(beta, (3, self.nelt, self.nq), "beta")
            beta_faces = _dev_f64(beta_faces, (3, self.nelt, 4, self.nf), "beta_faces")
        self._keep.update(kappa=kappa, c=c, f=f, tau=tau, beta=beta, beta_faces=beta_faces)
        hdg_set_coefficients(self._h, kappa, c, beta, f, tau)
        if beta is not None:
            hdg_set_face_convection(self._h, beta_faces)

    def set_boundary_data(self, uD=None, gN=None):
        if uD is not None:
            uD = _dev_f64(uD, (self.nfc, self.nf), "uD")
        if gN is not None:
            gN = _dev_f64(gN, (3, self.nfc, self.nf), "gN")
        self._keep.update(uD=uD, gN=gN)
        hdg_set_boundary_data(self._h, uD, gN)

    def assemble_condense(self, precision=HDG_FP64):
        hdg_assemble_condense(self._h, precision)

    def condensed(self):
        Cm = self._empty(self.nelt, self.m, self.m)
        Cf = self._empty(self.nelt, self.m)
        hdg_get_condensed(self._h, Cm, Cf)
        return Cm, Cf

    def solve_trace(self, rtol=1e-10, maxit=20000, x0=None, precision=HDG_FP64, raise_on_fail=True):
        uhat = self._empty(self.nfc, self.d2)
        if x0 is not None:
            x0 = _dev_f64(x0, (self.nfc, self.d2), "x0")
        code, it, rr = hdg_solve_trace(self._h, precision, rtol, maxit, x0, uhat)
        if code != 0 and raise_on_fail:
            raise HDGError(code, _lib.last_error())
        return uhat, it, rr

    def set_coarse_space(self, sizes, nodes, weights):
        """Two-level preconditioner from nested P1 levels (hdg_set_coarse_space); sizes=None
        removes it."""
        lib = _lib.load()
        if sizes is None:
            _lib.check(lib.hdg_set_coarse_space(self._h, 0, None, None, None))
            return
        sz = np.ascontiguousarray(sizes, dtype=np.int64)
        nd = np.ascontiguousarray(nodes, dtype=np.int32)
        wt = np.ascontiguousarray(weights, dtype=np.float64)
        if nd.shape != wt.shape or nd.ndim != 2 or nd.shape[1] != 4:
            raise ValueError("nodes and weights must both be [R, 4]")
        _lib.check(lib.hdg_set_coarse_space(self._h, len(sz), _ptr(sz), _ptr(nd), _ptr(wt)))

    def autotune(self):
        """Pick the persistent grids and the operator form (element pass + face sum, or one
        face-major pass) of the trace-solve kernels (FP64 and FP32) and the launch shape of the
        double-float assembly by timing (hdg_autotune); returns a dict of the choices and the
        best times."""
        t = _lib.Tuning()
        _lib.check(_lib.load().hdg_autotune(self._h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in _lib.Tuning._fields_}

    def apply(self, x):
        """y = H x on the free faces (hdg_trace_apply; Dirichlet rows 0)."""
        y = self._empty(self.nfc, self.d2)
        _lib.check(_lib.load().hdg_trace_apply(self._h, _dev_f64(x, (self.nfc, self.d2), "x").data_ptr(),
                                               y.data_ptr()))
        return y

    def precond_apply(self, r):
        z = self._empty(self.nfc, self.d2)
        _lib.check(_lib.load().hdg_coarse_precond_apply(self._h, _dev_f64(r, (self.nfc, self.d2), "r").data_ptr(),
                                                        z.data_ptr()))
        return z

    def set_inner_tolerance(self, rtol):
        hdg_set_inner_tolerance(self._h, rtol)

    def residual(self, x):
        r = self._empty(self.nfc, self.d2)
        rn, bn = hdg_trace_residual(self._h, _dev_f64(x, (self.nfc, self.d2), "x"), r)
        return r, rn, bn

    def recover(self, uhat):
        q = self._empty(self.nelt, 3, self.n)
        u = self._empty(self.nelt, self.n)
        hdg_recover(self._h, _dev_f64(uhat, (self.nfc, self.d2), "uhat"), q, u)
        return q, u

    def postprocess(self, q, u):
        ustar = self._empty(self.nelt, self.n1)
        hdg_postprocess(self._h, _dev_f64(q, (self.nelt, 3, self.n), "q"),
                        _dev_f64(u, (self.nelt, self.n), "u"), ustar)
        return ustar

    def set_method(self, method):
        """HDG_METHOD_HDG (default) or HDG_METHOD_BDM (hybridised BDM: tau = 0, u_h in
        P_{k-1}) for the next assembly."""
        _lib.check(_lib.load().hdg_set_method(self._h, int(method)))

    def projection(self, q_vol, u_vol, q_face, u_face):
        """HDG projection of eq. 9.13: q_vol [3, nelt, nq], u_vol [nelt, nq] at the volume
        nodes; q_face [3, nelt, 4, nf], u_face [nelt, 4, nf] at the element face nodes.
        Returns (Pi q [nelt, 3, n], Pi u [nelt, n])."""
        Pq = self._empty(self.nelt, 3, self.n)
        Pu = self._empty(self.nelt, self.n)
        hdg_projection(self._h, _dev_f64(q_vol, (3, self.nelt, self.nq), "q_vol"),
                       _dev_f64(u_vol, (self.nelt, self.nq), "u_vol"),
                       _dev_f64(q_face, (3, self.nelt, 4, self.nf), "q_face"),
                       _dev_f64(u_face, (self.nelt, 4, self.nf), "u_face"), Pq, Pu)
        return Pq, Pu

    def face_projection(self, vals):
        """eq. 9.12 on every face from the values [nfc, nf] at the face nodes: [nfc, d2]."""
        Pu = self._empty(self.nfc, self.d2)
        hdg_face_projection(self._h, _dev_f64(vals, (self.nfc, self.nf), "vals"), Pu)
        return Pu

    def volume_norm2(self, coef=None, vals=None, degree=None):
        """(sum_K |K| sum_q omega_q (vals - coef . P)^2, sum ... vals^2); coef in the degree-k
        (default) or degree-(k+1) basis."""
        degree = self.k if degree is None else degree
        dim = self.n if degree == self.k else self.n1
        c = None if coef is None else _dev_f64(coef, (self.nelt, dim), "coef")
        v = None if vals is None else _dev_f64(vals, (self.nelt, self.nq), "vals")
        return hdg_volume_norm2(self._h, degree, c, v)

    def face_norm2(self, coef=None, vals=None):
        """(||vals - coef . D||_h^2, ||vals||_h^2) of eq. 10.2."""
        c = None if coef is None else _dev_f64(coef, (self.nfc, self.d2), "coef")
        v = None if vals is None else _dev_f64(vals, (self.nfc, self.nf), "vals")
        return hdg_face_norm2(self._h, c, v)

    def mass_contraction(self, g, mode=0):
        """hdg_mass_contraction: sum_q |K| omega_q g P_i P_j for the n(n+1)/2 pairs (i <= j),
        [nelt, n(n+1)/2] FP32; mode 0 tensor cores (BF16 operands), 1 CUDA cores on the same
        BF16 operands, 2 CUDA cores in FP32."""
        import torch
        g = _dev_f64(g, (self.nelt, self.nq), "g")
        out = torch.empty((self.nelt, self.n * (self.n + 1) // 2), dtype=torch.float32, device=g.device)
        _lib.check(_lib.load().hdg_mass_contraction(self._h, g.data_ptr(), int(mode), out.data_ptr()))
        return out

    def assemble_condense_host(self, host, precision=HDG_DF32, chunks=16):
        """hdg_assemble_condense_host: the assembly from host arrays (numpy arrays or CPU
        tensors, pinned for overlap) given in `host` by name (kappa, c, f required; beta,
        beta_f, tau, uD, gN optional), copied chunk by chunk beside the condensation.  The host
        arrays must stay alive until the call returns."""
        def hp(name, shape):
            a = host.get(name)
            if a is None:
                return None
            if hasattr(a, "is_cuda"):
                if a.is_cuda or a.dtype != __import__("torch").float64 or not a.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous float64 CPU tensor")
                if tuple(a.shape) != shape:
                    raise ValueError(f"{name} must have shape {shape}")
                return a.data_ptr()
            a = np.asarray(a)
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.shape != shape:
                raise ValueError(f"{name} must be a C-contiguous float64 array of shape {shape}")
            return a.ctypes.data
        nf = self.nf
        hi = _lib.HostInputs(hp("kappa", (self.nelt, self.nq)), hp("c", (self.nelt, self.nq)), hp("f", (self.nelt, self.nq)),
                        hp("beta", (3, self.nelt, self.nq)), hp("beta_f", (3, self.nelt, 4, nf)),
                        hp("tau", (self.nelt, 4)), hp("uD", (self.nfc, nf)), hp("gN", (3, self.nfc, nf)))
        self._host_keep = host  # the mesh now reads library copies; nothing else to keep alive
        _lib.check(_lib.load().hdg_assemble_condense_host(self._h, int(precision), C.byref(hi), int(chunks)))

    def recover_host(self, uhat, q_host, u_host, chunks=16):
        """hdg_recover_host: q [nelt, 3, n] and u [nelt, n] written into host arrays (CPU
        float64 tensors or numpy arrays, pinned for overlap), chunk by chunk."""
        uhat = _dev_f64(uhat, (self.nfc, self.d2), "uhat")

        def hp(a, shape, name):
            if hasattr(a, "is_cuda"):
                if a.is_cuda or tuple(a.shape) != shape or not a.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous CPU tensor of shape {shape}")
                return a.data_ptr()
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.shape != shape:
                raise ValueError(f"{name} must be a C-contiguous float64 array of shape {shape}")
            return a.ctypes.data
        _lib.check(_lib.load().hdg_recover_host(self._h, uhat.data_ptr(), hp(q_host, (self.nelt, 3, self.n), "q"),
                                                hp(u_host, (self.nelt, self.n), "u"), int(chunks)))

    def mixed_masses(self):
        """hdg_mixed_masses: the FP32 masses of the HDG_MIXED_BF16 assembly for the current
        coefficients, [nelt, stride] = [M_{kappa^-1} pairs | M_c pairs | f^K | padding]."""
        import torch
        st = C.c_int(0)
        lib = _lib.load()
        _lib.check(lib.hdg_mixed_masses(self._h, None, C.byref(st)))
        out = torch.empty((self.nelt, st.value), dtype=torch.float32, device="cuda")
        _lib.check(lib.hdg_mixed_masses(self._h, out.data_ptr(), C.byref(st)))
        return out

    @property
    def launches(self):
        return hdg_launch_count(self._h)


# ---------------------------------------------------------------- batched problems
class HDGBatch:
    """Many independent problems solved together (hdg_batch_*): problems of equal degree form
    one union mesh per group; one CUDA graph launch runs the whole batch."""

    def __init__(self, meshes, stream=None):
        """meshes: list of (coords, elements, dirichlet, neumann, k)."""
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nprob = len(meshes)
        arrs = []
        for (c, e, d, n, k) in meshes:
            arrs.append((np.ascontiguousarray(c, np.float64), np.ascontiguousarray(e, np.int32),
                         np.ascontiguousarray(np.asarray(d).reshape(-1, 3), np.int32),
                         np.ascontiguousarray(np.asarray(n).reshape(-1, 3), np.int32), int(k)))
        self._arrs = arrs
        N = self.nprob
        P = C.c_void_p
        cp = (P * N)(*[a[0].ctypes.data for a in arrs])
        ep = (P * N)(*[a[1].ctypes.data for a in arrs])
        dp = (P * N)(*[a[2].ctypes.data if len(a[2]) else None for a in arrs])
        npp = (P * N)(*[a[3].ctypes.data if len(a[3]) else None for a in arrs])
        nv = (C.c_int64 * N)(*[len(a[0]) for a in arrs])
        ne = (C.c_int64 * N)(*[len(a[1]) for a in arrs])
        nd = (C.c_int64 * N)(*[len(a[2]) for a in arrs])
        nn = (C.c_int64 * N)(*[len(a[3]) for a in arrs])
        kk = (C.c_int * N)(*[a[4] for a in arrs])
        h = C.c_void_p()
        lib = _lib.load()
        _lib.check(lib.hdg_batch_create(N, cp, nv, ep, ne, dp, nd, npp, nn, kk, C.c_void_p(self.stream.cuda_stream),
                                        C.byref(h)))
        self._h = h
        ng = C.c_int(0)
        _lib.check(lib.hdg_batch_num_groups(h, C.byref(ng)))
        self.groups = []
        for g in range(ng.value):
            mh = C.c_void_p()
            k = C.c_int(0)
            npg = C.c_int(0)
            _lib.check(lib.hdg_batch_group(h, g, C.byref(mh), C.byref(k), C.byref(npg), None, None, None))
            ids = np.zeros(npg.value, np.int32)
            eo = np.zeros(npg.value + 1, np.int64)
            fo = np.zeros(npg.value + 1, np.int64)
            _lib.check(lib.hdg_batch_group(h, g, None, None, None, ids.ctypes.data, eo.ctypes.data, fo.ctypes.data))
            mesh = HDGMesh(None, None, None, None, k.value, stream=self.stream, _handle=mh)
            self.groups.append(dict(mesh=mesh, k=k.value, probs=ids, elem_off=eo, face_off=fo))

    def set_coarse_spaces(self, hierarchies):
        """Two-level preconditioner for every group: hierarchies[p] = (sizes, nodes, weights) of
        problem p in its own numbering (as for HDGMesh.set_coarse_space).  Per group the levels
        of its problems are joined block-diagonally (node and vertex numbers offset in union
        order); a problem with fewer levels repeats its coarsest level (identity rows) so that
        all have the group's depth.  hierarchies=None removes the coarse spaces."""
        for G in self.groups:
            M = G["mesh"]
            if hierarchies is None:
                M.set_coarse_space(None, None, None)
                continue
            hs = [hierarchies[p] for p in G["probs"]]
            depth = max(2, max(len(h[0]) for h in hs))
            sizes = np.zeros(depth, np.int64)
            per = []  # per problem: list of per-level row blocks (nodes, weights) and level sizes
            for (sz, nd, wt), p in zip(hs, G["probs"]):
                nver = len(self._arrs[p][0])
                szp = list(sz) + [sz[-1]] * (depth - len(sz))
                blocks = [(nd[:nver], wt[:nver])]
                off = nver
                for l in range(depth - 1):
                    if l < len(sz) - 1:
                        blocks.append((nd[off:off + sz[l]], wt[off:off + sz[l]]))
                        off += sz[l]
                    else:  # repeat the coarsest level
                        n_ = szp[l]
                        ident = np.full((n_, 4), -1, np.int32)
                        ident[:, 0] = np.arange(n_)
                        w_ = np.zeros((n_, 4))
                        w_[:, 0] = 1.0
                        blocks.append((ident, w_))
                per.append((szp, blocks))
                sizes += np.asarray(szp, np.int64)
            rows_n, rows_w = [], []
            for b in range(depth):  # block b: mesh vertices (b = 0) or level b-1 nodes
                tgt_off = 0
                for szp, blocks in per:
                    nd, wt = blocks[b]
                    nd = np.asarray(nd, np.int64)
                    rows_n.append(np.where(nd >= 0, nd + tgt_off, -1))
                    rows_w.append(np.asarray(wt, np.float64))
                    tgt_off += szp[b]
            M.set_coarse_space(sizes, np.concatenate(rows_n).astype(np.int32), np.concatenate(rows_w))

    def autotune(self, precision=HDG_DF32):
        """hdg_autotune on every group mesh (assembles each group once first); the batch graph
        is rebuilt with the tuned shapes at the next run.  Returns the choices per group."""
        out = []
        for G in self.groups:
            G["mesh"].assemble_condense(precision)
            out.append(G["mesh"].autotune())
        return out

    def set_solve_precision(self, precision):
        """HDG_FP64 (default) or HDG_MIXED_FP32 for the batch's trace solves."""
        _lib.check(_lib.load().hdg_batch_set_solve_precision(self._h, int(precision)))

    def set_inner_tolerance(self, rtol):
        for G in self.groups:
            G["mesh"].set_inner_tolerance(rtol)

    def run(self, precision=HDG_FP64, rtol=1e-10, maxit=20000, raise_on_fail=True):
        relres = np.zeros(self.nprob)
        iters = np.zeros(len(self.groups), np.int32)
        code = _lib.load().hdg_batch_run(self._h, precision, float(rtol), int(maxit), relres.ctypes.data,
                                         iters.ctypes.data)
        if code != 0 and raise_on_fail:
            raise HDGError(code, _lib.last_error())
        return relres, iters

    def solution(self, g):
        """(u_hat, q, u) of group g in union numbering, copied into new CUDA tensors."""
        G = self.groups[g]
        M = G["mesh"]
        uh, q, u = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _lib.check(_lib.load().hdg_batch_solution(self._h, g, C.byref(uh), C.byref(q), C.byref(u)))
        out = []
        for ptr, shape in ((uh, (M.nfc, M.d2)), (q, (M.nelt, 3, M.n)), (u, (M.nelt, M.n))):
            out.append(_device_view(ptr.value, int(np.prod(shape))).view(shape).clone())
        return tuple(out)

    def set_volume_rule(self, rule):
        """hdg_set_volume_rule: HDG_RULE_CONICAL or HDG_RULE_SYMMETRIC (call before setting the
        coefficients; self.nq follows)."""
        _lib.check(_lib.load().hdg_set_volume_rule(self._h, int(rule)))
        self.info = hdg_mesh_get_info(self._h)
        self.nq = self.info["nq"]
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None) is not None:
            for G in self.groups:
                G["mesh"]._h = None
            _lib.load().hdg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr, numel):
    """A float64 CUDA tensor aliasing library-owned device memory (no copy)."""
    import torch

    class _Arr:
        __cuda_array_interface__ = {"shape": (numel,), "typestr": "<f8", "data": (ptr, False), "version": 3,
                                    "strides": None}
    return torch.as_tensor(_Arr(), device="cuda")
