"""Learned initial guess for the trace solve (argument marshalling over libhdg's kernels).

A small network phi_theta maps a coefficient field kappa = exp(g) (here g a Gaussian random
field with parameters xi), seen through g at the coarse nodes, to the coefficients c of a
continuous piecewise-linear coarse field.  Its training targets are the coarse Galerkin solutions
c* = (Pi^T H Pi)^-1 Pi^T b of the trace system (hdg_coarse_solve), i.e. the trace in range(Pi)
closest to the solution in the energy norm.  At solve time x0 = alpha Pi phi_theta(xi) with the
energy-optimal alpha (hdg_coarse_guess), and PCG runs from x0 to the same residual tolerance as
from zero, so the method's answer and stopping test do not depend on the network.

Every arithmetic step runs in libhdg: GEMM, bias, tanh forward/backward, mean-squared loss,
Adam (hdg_nn_*), prolongation, coarse solve and the trace solve.  PyTorch holds the buffers.
"""

import ctypes as C

import numpy as np

from . import _lib

__all__ = ["MLP", "CoarseSpace"]


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class CoarseSpace:
    """Per-vertex interpolation (nodes int32 [nver,4], weights f64 [nver,4]) of nc coarse values."""

    def __init__(self, nodes, weights, nc):
        import torch
        self.nodes = torch.from_numpy(np.ascontiguousarray(nodes, np.int32)).cuda()
        self.weights = torch.from_numpy(np.ascontiguousarray(weights, np.float64)).cuda()
        self.nc = int(nc)

    def prolong(self, mesh, c):
        import torch
        out = torch.empty((mesh.nfc, mesh.d2), dtype=torch.float64, device="cuda")
        _lib.check(_lib.load().hdg_prolong(mesh._h, _p(self.nodes), _p(self.weights), _p(c), _p(out)))
        return out

    def restrict(self, mesh, y):
        import torch
        out = torch.empty(self.nc, dtype=torch.float64, device="cuda")
        _lib.check(_lib.load().hdg_restrict(mesh._h, _p(self.nodes), _p(self.weights), self.nc, _p(y), _p(out)))
        return out

    def coarse_solve(self, mesh, rtol=1e-10, maxit=5000):
        import torch
        c = torch.empty(self.nc, dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        rr = C.c_double(0.0)
        _lib.check(_lib.load().hdg_coarse_solve(mesh._h, _p(self.nodes), _p(self.weights), self.nc, _p(c),
                                                float(rtol), int(maxit), C.byref(it), C.byref(rr)))
        return c, it.value, rr.value

    def guess(self, mesh, c):
        import torch
        x0 = torch.empty((mesh.nfc, mesh.d2), dtype=torch.float64, device="cuda")
        a = C.c_double(0.0)
        _lib.check(_lib.load().hdg_coarse_guess(mesh._h, _p(self.nodes), _p(self.weights), _p(c), _p(x0),
                                                C.byref(a)))
        return x0, a.value


class MLP:
    """x -> tanh(x W1^T + b1) -> ... -> x W_L^T + b_L (last layer linear), FP32 on the GPU."""

    def __init__(self, sizes, seed=7, params=None):
        import torch
        self.sizes = list(sizes)
        rng = np.random.default_rng(seed)
        self.params = []
        for i in range(len(sizes) - 1):
            if params is not None:
                W, b = params[2 * i], params[2 * i + 1]
            else:
                W = rng.normal(0.0, 1.0 / np.sqrt(sizes[i]), size=(sizes[i + 1], sizes[i]))
                b = np.zeros(sizes[i + 1])
            self.params += [torch.from_numpy(np.ascontiguousarray(W, np.float32)).cuda(),
                            torch.from_numpy(np.ascontiguousarray(b, np.float32)).cuda()]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self.stream = torch.cuda.current_stream().cuda_stream

    def forward(self, x):
        """x: float32 CUDA [B, in].  Returns (y, activations)."""
        import torch
        lib = _lib.load()
        acts = [x.contiguous()]
        h = acts[0]
        nl = len(self.params) // 2
        for i in range(nl):
            W, b = self.params[2 * i], self.params[2 * i + 1]
            B, nin = h.shape
            nout = W.shape[0]
            out = torch.empty((B, nout), dtype=torch.float32, device="cuda")
            _lib.check(lib.hdg_nn_gemm(B, nout, nin, _p(h), nin, 1, _p(W), 1, nin, _p(out), nout, 0.0, _p(b),
                                       1 if i < nl - 1 else 0, C.c_void_p(self.stream)))
            acts.append(out)
            h = out
        return h, acts

    def backward(self, acts, dy):
        """Gradients of the parameters for the output gradient dy (float32 CUDA [B, out])."""
        import torch
        lib = _lib.load()
        nl = len(self.params) // 2
        grads = [None] * len(self.params)
        dz = dy.contiguous().clone()
        for i in reversed(range(nl)):
            W = self.params[2 * i]
            h_in = acts[i]
            B, nin = h_in.shape
            nout = W.shape[0]
            dW = torch.empty_like(W)
            db = torch.empty(nout, dtype=torch.float32, device="cuda")
            _lib.check(lib.hdg_nn_gemm(nout, nin, B, _p(dz), 1, nout, _p(h_in), nin, 1, _p(dW), nin, 0.0, None, 0,
                                       C.c_void_p(self.stream)))
            _lib.check(lib.hdg_nn_colsum(B, nout, _p(dz), _p(db), C.c_void_p(self.stream)))
            grads[2 * i], grads[2 * i + 1] = dW, db
            if i > 0:
                dh = torch.empty((B, nin), dtype=torch.float32, device="cuda")
                _lib.check(lib.hdg_nn_gemm(B, nin, nout, _p(dz), nout, 1, _p(W), nin, 1, _p(dh), nin, 0.0, None, 0,
                                           C.c_void_p(self.stream)))
                _lib.check(lib.hdg_nn_tanh_bwd(dh.numel(), _p(acts[i]), _p(dh), C.c_void_p(self.stream)))
                dz = dh
        return grads

    def loss_grad(self, y, t):
        import torch
        g = torch.empty_like(y)
        part = torch.zeros(64, dtype=torch.float32, device="cuda")
        _lib.check(_lib.load().hdg_nn_mse(y.numel(), _p(y), _p(t.contiguous()), _p(g), _p(part),
                                          C.c_void_p(self.stream)))
        return part, g

    def train_step(self, x, t, lr=1e-3):
        y, acts = self.forward(x)
        part, g = self.loss_grad(y, t)
        grads = self.backward(acts, g)
        self.step_count += 1
        lib = _lib.load()
        for p, gr, m, v in zip(self.params, grads, self.m, self.v):
            _lib.check(lib.hdg_nn_adam(p.numel(), _p(p), _p(gr), _p(m), _p(v), lr, 0.9, 0.999, 1e-8,
                                       self.step_count, C.c_void_p(self.stream)))
        return part

    def host_params(self):
        return [p.double().cpu().numpy() for p in self.params]


def fourier_field(X, Y, Z, omega, amps, sigma, exponentiate=True, out=None):
    """exp(g) (or g) of the random Fourier field at device points X, Y, Z (hdg_fourier_field)."""
    import torch
    if out is None:
        out = torch.empty_like(X)
    omega = omega if isinstance(omega, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(omega, np.float64))
    amps = amps if isinstance(amps, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(amps, np.float64))
    omega, amps = omega.cuda().contiguous(), amps.cuda().contiguous()
    _lib.check(_lib.load().hdg_fourier_field(X.numel(), _p(X), _p(Y), _p(Z), omega.shape[0], _p(omega), _p(amps),
                                             float(sigma), 1 if exponentiate else 0, _p(out),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


class LearnedGuess:
    """Network-predicted coarse correction x0 = alpha Pi phi(xi) for a family of fields
    kappa = exp(g_xi) on one mesh (c, f, tau and the boundary data fixed).

    mesh:   an HDGMesh whose coefficients are set with the arrays this object owns
    coarse: CoarseSpace on a coarser nested grid
    omega:  [M, 3] frequencies of the field, sigma its standard deviation
    feature_points: [nfeat, 3] points where g is sampled as the network's input (the coarse
            nodes)
    """

    def __init__(self, mesh, coarse, omega, sigma, c, f, feature_points, hidden=(256, 256), seed=7,
                 assemble_precision=None):
        import torch
        from . import HDG_DF32
        self.mesh, self.coarse, self.sigma = mesh, coarse, float(sigma)
        self.omega = torch.from_numpy(np.ascontiguousarray(omega, np.float64)).cuda()
        self.nmodes = self.omega.shape[0]
        self.X, self.Y, self.Z = mesh.volume_nodes()
        self.kappa = torch.empty_like(self.X)
        self.c, self.f = c, f
        self.asm = HDG_DF32 if assemble_precision is None else assemble_precision
        P = torch.from_numpy(np.ascontiguousarray(feature_points, np.float64)).cuda()
        self.FX, self.FY, self.FZ = (P[:, i].contiguous() for i in range(3))
        self.sizes = [P.shape[0], *hidden, coarse.nc]
        self.net = MLP(self.sizes, seed=seed)
        self.mean = self.std = None
        self.history = []

    def features(self, amps):
        """Network input of the field xi: g at the feature points (FP32 device [nfeat])."""
        import torch
        g = fourier_field(self.FX, self.FY, self.FZ, self.omega, amps, self.sigma, False)
        out = torch.empty(g.numel(), dtype=torch.float32, device="cuda")
        _lib.check(_lib.load().hdg_nn_to_f32(g.numel(), _p(g), _p(out),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return out

    # -- one field on the mesh
    def set_field(self, amps):
        fourier_field(self.X, self.Y, self.Z, self.omega, amps, self.sigma, True, out=self.kappa)
        self.mesh.set_coefficients(self.kappa, self.c, self.f)
        self.mesh.assemble_condense(self.asm)

    def target(self, amps, rtol=1e-8, maxit=5000):
        """Coarse Galerkin solution c* = (Pi^T H Pi)^-1 Pi^T b of the field xi: the energy
        projection onto range(Pi) of the trace the method solves for (H u_hat = b)."""
        self.set_field(amps)
        c, it, rr = self.coarse.coarse_solve(self.mesh, rtol, maxit)
        return c, it, rr

    def generate(self, amps_list, rtol=1e-8):
        """Training pairs: inputs [N, nfeat] (host, float32) and targets [N, nc] (host, float64)."""
        T = np.empty((len(amps_list), self.coarse.nc))
        A = np.empty((len(amps_list), self.sizes[0]), np.float32)
        its = []
        for i, a in enumerate(amps_list):
            c, it, _ = self.target(a, rtol)
            T[i] = c.cpu().numpy()
            A[i] = self.features(a).cpu().numpy()
            its.append(it)
        return A, T, its

    # -- training (all arithmetic in the hdg_nn_* kernels)
    def fit(self, A, T, epochs=200, batch=64, lr=1e-3, seed=0):
        import torch
        lib = _lib.load()
        st = C.c_void_p(self.net.stream)
        M, N = T.shape
        Td64 = torch.from_numpy(np.ascontiguousarray(T, np.float64)).cuda()
        self.mean = torch.empty(N, dtype=torch.float64, device="cuda")
        self.std = torch.empty(N, dtype=torch.float64, device="cuda")
        _lib.check(lib.hdg_nn_colstats(M, N, _p(Td64), _p(self.mean), _p(self.std), st))
        Tn32 = torch.empty((M, N), dtype=torch.float32, device="cuda")
        _lib.check(lib.hdg_nn_standardize(M, N, _p(Td64), _p(self.mean), _p(self.std), _p(Tn32), st))
        Tn = Tn32.cpu().numpy()
        rng = np.random.default_rng(seed)
        n = len(A)
        nb = max(1, n // batch)
        for ep in range(epochs):
            perm = rng.permutation(n)
            Ad = torch.from_numpy(np.ascontiguousarray(A[perm], np.float32)).cuda()
            Td = torch.from_numpy(np.ascontiguousarray(Tn[perm], np.float32)).cuda()
            parts = []
            for b in range(nb):
                sl = slice(b * batch, (b + 1) * batch)
                parts.append(self.net.train_step(Ad[sl], Td[sl], lr))
            if ep == epochs - 1 or ep % 10 == 0:
                self.history.append((ep, float(np.mean([p.cpu().numpy().sum() for p in parts]))))
        return self.history

    def predict(self, amps):
        """c = phi(xi) as FP64 device [nc] (the target normalisation folded into the last
        layer by fold_normalisation)."""
        import torch
        x = self.features(amps)[None, :]
        y, _ = self.net.forward(x)
        yd = torch.empty(self.coarse.nc, dtype=torch.float64, device="cuda")
        _lib.check(_lib.load().hdg_nn_to_f64(yd.numel(), _p(y), _p(yd), C.c_void_p(self.net.stream)))
        return yd

    def fold_normalisation(self):
        """Fold the target normalisation into the last layer (hdg_nn_fold_affine) so phi(xi)
        is c itself."""
        import torch
        W, b = self.net.params[-2], self.net.params[-1]
        _lib.check(_lib.load().hdg_nn_fold_affine(W.shape[0], W.shape[1], _p(W), _p(b), _p(self.mean), _p(self.std),
                                                  C.c_void_p(self.net.stream)))
        self.mean = torch.zeros_like(self.mean)
        self.std = torch.ones_like(self.std)

    def guess(self, amps):
        """x0 = alpha Pi phi(xi) (after set_field).  Returns (x0, alpha)."""
        return self.coarse.guess(self.mesh, self.predict(amps))

    def solve(self, amps, rtol=1e-10, maxit=20000, precision=None, use_guess=True, assemble=True):
        """Trace solve of the field xi to the relative residual rtol, started from the learned
        x0.  The energy-optimal alpha makes x0 no worse than zero in the energy norm; a guess
        that is not finite or has alpha <= 0, or a solve from x0 that fails, falls back to the
        zero start.  assemble=False: the field is already set and assembled.  Returns
        (uhat, iters, relres, used_guess)."""
        from . import HDG_FP64
        prec = HDG_FP64 if precision is None else precision
        if assemble:
            self.set_field(amps)
        if use_guess:
            x0, alpha = self.guess(amps)
            if np.isfinite(alpha) and alpha > 0.0:
                uhat, it, rr = self.mesh.solve_trace(rtol, maxit, x0=x0, precision=prec, raise_on_fail=False)
                if rr <= rtol:
                    return uhat, it, rr, True
        uhat, it, rr = self.mesh.solve_trace(rtol, maxit, precision=prec)
        return uhat, it, rr, False
