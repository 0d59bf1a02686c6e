"""Python binding of libbie.so (include/bie.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
arguments to the C structs and pointers of the ABI.  Host arrays are numpy
float64 arrays; device arrays are torch CUDA float64 tensors (passed by data
pointer with on_device = 1).  If the library has not been built the first
call raises -- there is no fallback implementation.

The functions carry the C names:
    bie_default_opts, bie_init, bie_destroy, bie_size, bie_nodes, bie_apply,
    bie_rhs, bie_solve, bie_velocities, bie_step, bie_get_state,
    bie_set_state, bie_set_stream, bie_close_info, bie_near_shape, bie_profile, bie_profile_read,
    bie_apply_static, bie_init_batch, bie_cells, bie_features, bie_set_warm_net,
    bie_get_history, bie_set_history,
    bie_net_init, bie_net_destroy, bie_net_last_error, bie_net_size,
    bie_net_set_stream, bie_net_set_params, bie_net_get_params,
    bie_net_forward, bie_net_loss_grad, bie_net_adam_step
and `Context` wraps them for a workload dict, or a list of them for a batch
of independent cells (see workloads.py); `Net` wraps the warm-start network.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbie.so")

BIE_OK, BIE_EINVAL, BIE_ENOCONV, BIE_ECOLLIDE, BIE_ENUMERIC, BIE_ECUDA, BIE_ENOMEM = 0, -1, -2, -3, -4, -5, -6
BIE_FP64, BIE_MIXED, BIE_DF64 = 0, 1, 2
BIE_NET_FEATURES, BIE_NET_HIDDEN = 13, 64
BIE_NEAR32_SHAPES = 5
# (packed, targets per thread, CTAs per SM) of each single-precision near-sum tile shape
NEAR32_SHAPES = [(1, 2, 5), (1, 1, 8), (1, 3, 4), (0, 3, 4), (0, 2, 5)]
_NAMES = {0: "BIE_OK", -1: "BIE_EINVAL", -2: "BIE_ENOCONV", -3: "BIE_ECOLLIDE", -4: "BIE_ENUMERIC",
          -5: "BIE_ECUDA", -6: "BIE_ENOMEM"}

c_double, c_int32, c_void_p = ctypes.c_double, ctypes.c_int32, ctypes.c_void_p
P_DOUBLE = ctypes.POINTER(ctypes.c_double)


class Lattice(ctypes.Structure):
    _fields_ = [("e1", c_double * 2), ("e2", c_double * 2), ("center", c_double * 2)]


class Body(ctypes.Structure):
    _fields_ = [("n_nodes", c_int32), ("shape", c_int32), ("p", c_double * 4), ("xc", c_double * 2),
                ("theta", c_double)]


class Cell(ctypes.Structure):
    _fields_ = [("lattice", Lattice), ("mu", c_double), ("gamma", c_double), ("n_bodies", c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("n_proxy", c_int32), ("proxy_radius", c_double), ("n_coll", c_int32),
                ("lam_rel", c_double), ("gmres_tol", c_double), ("gmres_max", c_int32), ("inner_tol", c_double),
                ("max_refine", c_int32), ("warm_start", c_int32), ("min_gap", c_double), ("device", c_int32),
                ("close_factor", c_double), ("close_capacity", c_int32), ("residual", c_int32),
                ("autotune", c_int32), ("graph", c_int32), ("precond", c_int32), ("n_images", c_int32),
                ("close_rule", c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("refinements", c_int32), ("applies64", c_int32),
                ("applies32", c_int32), ("rel_residual", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProfileInfo(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("near32_launches", c_int32), ("near32_ms", c_double),
                ("near64_launches", c_int32), ("near64_ms", c_double),
                ("neardf_launches", c_int32), ("neardf_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library():
    """Load libbie.so (raises if it is missing: build it with
    paper_1912_04501_gb300._build.build() or __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build the CUDA library first")
    L = ctypes.CDLL(LIB_PATH)
    vp = c_void_p
    sig = {
        "bie_default_opts": (None, [ctypes.POINTER(Opts)]),
        "bie_init": (c_int32, [ctypes.POINTER(vp), ctypes.POINTER(Lattice), c_double, c_double, c_int32,
                               ctypes.POINTER(Body), ctypes.POINTER(Opts)]),
        "bie_init_batch": (c_int32, [ctypes.POINTER(vp), c_int32, ctypes.POINTER(Cell), ctypes.POINTER(Body),
                                     ctypes.POINTER(Opts)]),
        "bie_cells": (c_int32, [vp, ctypes.POINTER(c_int32), vp, vp, ctypes.POINTER(SolveInfo)]),
        "bie_destroy": (None, [vp]),
        "bie_last_error": (ctypes.c_char_p, [vp]),
        "bie_size": (c_int32, [vp, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
        "bie_set_stream": (c_int32, [vp, vp]),
        "bie_nodes": (c_int32, [vp, vp, vp, vp, vp, c_int32]),
        "bie_apply": (c_int32, [vp, vp, vp, c_int32, c_int32]),
        "bie_rhs": (c_int32, [vp, vp, c_int32]),
        "bie_solve": (c_int32, [vp, vp, vp, c_int32, c_int32, ctypes.POINTER(SolveInfo)]),
        "bie_velocities": (c_int32, [vp, vp, vp, vp, vp, c_int32]),
        "bie_step": (c_int32, [vp, c_double, c_int32, vp, ctypes.POINTER(SolveInfo)]),
        "bie_get_state": (c_int32, [vp, vp, vp, vp, vp, vp]),
        "bie_set_state": (c_int32, [vp, c_double, vp, vp, vp, vp]),
        "bie_close_info": (c_int32, [vp, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
        "bie_near_shape": (c_int32, [vp, ctypes.POINTER(c_int32), vp]),
        "bie_apply_static": (c_int32, [vp, vp, vp]),
        "bie_device_sms": (c_int32, [vp, ctypes.POINTER(c_int32)]),
        "bie_mu_eff_contour": (c_int32, [vp, vp, vp, c_int32]),
        "bie_set_partition": (c_int32, [vp, c_int32, c_int32, vp, vp]),
        "bie_alu_peak": (c_int32, [c_int32, vp, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double)]),
        "bie_profile": (c_int32, [vp, c_int32]),
        "bie_profile_read": (c_int32, [vp, ctypes.POINTER(ProfileInfo)]),
        "bie_features": (c_int32, [vp, vp, c_int32]),
        "bie_get_history": (c_int32, [vp, vp, vp, ctypes.POINTER(c_double), ctypes.POINTER(c_int32)]),
        "bie_set_history": (c_int32, [vp, vp, vp, c_double]),
        "bie_set_warm_net": (c_int32, [vp, vp]),
        "bie_net_init": (c_int32, [ctypes.POINTER(vp), c_int32, c_int32]),
        "bie_net_destroy": (None, [vp]),
        "bie_net_last_error": (ctypes.c_char_p, [vp]),
        "bie_net_size": (c_int32, [vp, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
        "bie_net_set_stream": (c_int32, [vp, vp]),
        "bie_net_set_params": (c_int32, [vp, vp]),
        "bie_net_get_params": (c_int32, [vp, vp]),
        "bie_net_forward": (c_int32, [vp, vp, c_int32, vp]),
        "bie_net_loss_grad": (c_int32, [vp, vp, vp, vp, c_int32, vp, ctypes.POINTER(c_double)]),
        "bie_net_adam_step": (c_int32, [vp, c_double, c_double, c_double, c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/bie.h that the loaded library exports."""
    L = library()
    return [n for n in ("bie_default_opts", "bie_init", "bie_destroy", "bie_last_error", "bie_size",
                        "bie_set_stream", "bie_nodes", "bie_apply", "bie_rhs", "bie_solve", "bie_velocities",
                        "bie_step", "bie_get_state", "bie_set_state", "bie_close_info", "bie_profile",
                        "bie_profile_read", "bie_apply_static", "bie_init_batch", "bie_cells", "bie_features",
                        "bie_set_warm_net", "bie_net_init", "bie_net_destroy", "bie_net_last_error",
                        "bie_net_size", "bie_net_set_stream", "bie_net_set_params", "bie_net_get_params",
                        "bie_net_forward", "bie_net_loss_grad", "bie_net_adam_step", "bie_get_history",
                        "bie_set_history", "bie_near_shape", "bie_device_sms", "bie_alu_peak", "bie_mu_eff_contour", "bie_set_partition")
            if hasattr(L, n)]


def _ptr(a):
    """(pointer, on_device) of a numpy float64 array or a torch float64 tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):  # torch tensor
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float64")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def bie_default_opts():
    o = Opts()
    library().bie_default_opts(ctypes.byref(o))
    return o


def _lattice(cell):
    return Lattice((c_double * 2)(*cell["e1"]), (c_double * 2)(*cell["e2"]), (c_double * 2)(*cell["centre"]))


class Context:
    """One unit cell (a workload dict: bie_init) or a batch of independent
    cells (a list of them: bie_init_batch) on the GPU."""

    def __init__(self, cell, precision=BIE_MIXED, **opts):
        L = library()
        o = bie_default_opts()
        cells = list(cell) if isinstance(cell, (list, tuple)) else [cell]
        self.batch = isinstance(cell, (list, tuple))
        sv = cells[0].get("solver", {})
        o.precision = precision
        for k in ("n_proxy", "proxy_radius", "n_coll"):
            if k in sv:
                setattr(o, k, sv[k])
        if "gmres_tol" in sv:
            o.gmres_tol = sv["gmres_tol"]
        known = {name for name, _ in Opts._fields_}
        for k, v in opts.items():
            if k not in known:
                raise TypeError(f"unknown option {k!r} (bie_opts has {sorted(known)})")
            setattr(o, k, v)
        all_bodies = [bd for c in cells for bd in c["bodies"]]
        bodies = (Body * len(all_bodies))()
        for b, bd in zip(bodies, all_bodies):
            b.n_nodes = int(bd["n"])
            if bd.get("shape", "ellipse") == "star":
                b.shape = 1
                b.p = (c_double * 4)(bd["r0"], bd["eps"], float(bd["k"]), 0.0)
            else:
                b.shape = 0
                b.p = (c_double * 4)(bd["a"], bd["b"], 0.0, 0.0)
            b.xc = (c_double * 2)(*bd["xc"])
            b.theta = bd["theta"]
        h = c_void_p()
        if self.batch:
            cs = (Cell * len(cells))()
            for ct, c in zip(cs, cells):
                ct.lattice = _lattice(c)
                ct.mu, ct.gamma, ct.n_bodies = c["mu"], c["gamma"], len(c["bodies"])
            rc = L.bie_init_batch(ctypes.byref(h), len(cells), cs, bodies, ctypes.byref(o))
        else:
            lat = _lattice(cell)
            rc = L.bie_init(ctypes.byref(h), ctypes.byref(lat), cell["mu"], cell["gamma"], len(cell["bodies"]),
                            bodies, ctypes.byref(o))
        if rc != 0:
            raise BieError(rc, "bie_init failed (invalid input or CUDA error)")
        self.h = h
        self.opts = o
        n, nb = c_int32(), c_int32()
        L.bie_size(h, ctypes.byref(n), ctypes.byref(nb))
        self.N, self.n_bodies = n.value, nb.value
        self.n_cells = len(cells)
        no = np.zeros(self.n_cells + 1, dtype=np.int32)
        bo = np.zeros(self.n_cells + 1, dtype=np.int32)
        self._check(L.bie_cells(h, None, no.ctypes.data, bo.ctypes.data, None))
        self.node_offsets, self.body_offsets = no, bo

    def _check(self, rc):
        if rc != 0:
            raise BieError(rc, library().bie_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            library().bie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        self._check(library().bie_set_stream(self.h, c_void_p(stream_handle)))

    def nodes(self):
        x, n = np.zeros(2 * self.N), np.zeros(2 * self.N)
        w, k = np.zeros(self.N), np.zeros(self.N)
        self._check(library().bie_nodes(self.h, x.ctypes.data, n.ctypes.data, w.ctypes.data, k.ctypes.data, 0))
        return x.reshape(-1, 2), n.reshape(-1, 2), w, k

    def apply(self, sigma, out=None, precision=BIE_FP64):
        if out is None:
            out = np.zeros(2 * self.N)
        ps, ds = _ptr(sigma)
        po, do = _ptr(out)
        if ds != do:
            raise ValueError("sigma and out must both be host or both device")
        self._check(library().bie_apply(self.h, ps, po, precision, ds))
        return out

    def rhs(self):
        b = np.zeros(2 * self.N)
        self._check(library().bie_rhs(self.h, b.ctypes.data, 0))
        return b

    def solve(self, rhs=None, guess=None, allow_noconv=False):
        sigma = np.zeros(2 * self.N) if guess is None else np.array(guess, dtype=np.float64).ravel()
        info = SolveInfo()
        pr, _ = _ptr(None if rhs is None else np.ascontiguousarray(rhs, dtype=np.float64).ravel())
        rc = library().bie_solve(self.h, pr, sigma.ctypes.data, 0 if guess is None else 1, 0, ctypes.byref(info))
        if rc != 0 and not (allow_noconv and rc == BIE_ENOCONV):
            self._check(rc)
        return sigma, info.as_dict()

    def cell_info(self):
        """Per-cell statistics of the last solve (list of dicts)."""
        infos = (SolveInfo * self.n_cells)()
        self._check(library().bie_cells(self.h, None, None, None, infos))
        return [i.as_dict() for i in infos]

    def velocities(self, sigma):
        """(v (n_bodies x 2), omega, mu_eff): mu_eff a float for one cell, an
        array of one value per cell for a batch."""
        v, om, mu = np.zeros(2 * self.n_bodies), np.zeros(self.n_bodies), np.zeros(self.n_cells)
        s = np.ascontiguousarray(sigma, dtype=np.float64).ravel()
        self._check(library().bie_velocities(self.h, s.ctypes.data, v.ctypes.data, om.ctypes.data,
                                             mu.ctypes.data, 0))
        return v.reshape(-1, 2), om, (mu if self.batch else float(mu[0]))

    def set_partition(self, body_begin, body_end, exchange):
        """bie_set_partition: own the targets of bodies [body_begin, body_end);
        exchange is a ctypes callback (shard.EXCHANGE) or None to switch off."""
        fn = ctypes.cast(exchange, c_void_p) if exchange is not None else None
        self._exchange = exchange
        self._check(library().bie_set_partition(self.h, int(body_begin), int(body_end), fn, None))

    def mu_eff_contour(self, sigma):
        """mu_eff by the contour-deformation formula (n_images 4 contexts):
        a float for one cell, one value per cell for a batch."""
        mu = np.zeros(self.n_cells)
        s = np.ascontiguousarray(sigma, dtype=np.float64).ravel()
        self._check(library().bie_mu_eff_contour(self.h, s.ctypes.data, mu.ctypes.data, 0))
        return mu if self.batch else float(mu[0])

    def step(self, dt, n_steps=1):
        """mu_eff per step (n_steps) for one cell, (n_steps x n_cells) for a batch."""
        mu = np.zeros(max(1, n_steps) * self.n_cells)
        info = SolveInfo()
        self._check(library().bie_step(self.h, dt, n_steps, mu.ctypes.data, ctypes.byref(info)))
        mu = mu[:n_steps * self.n_cells]
        return (mu.reshape(n_steps, self.n_cells) if self.batch else mu), info.as_dict()

    def get_state(self):
        t = np.zeros(1)
        e2 = np.zeros(2 * self.n_cells)
        xc = np.zeros(2 * self.n_bodies)
        th = np.zeros(self.n_bodies)
        sg = np.zeros(2 * self.N)
        self._check(library().bie_get_state(self.h, t.ctypes.data, e2.ctypes.data, xc.ctypes.data,
                                            th.ctypes.data, sg.ctypes.data))
        s2, d2 = np.zeros(2 * self.N), np.zeros(2 * self.N)
        dtp, have = c_double(), c_int32()
        self._check(library().bie_get_history(self.h, s2.ctypes.data, d2.ctypes.data, ctypes.byref(dtp),
                                              ctypes.byref(have)))
        return dict(t=float(t[0]), e2=(e2.reshape(-1, 2) if self.batch else e2), xc=xc.reshape(-1, 2), theta=th,
                    sigma=sg, sigma_prev2=(s2 if have.value & 1 else None), d2=(d2 if have.value & 2 else None),
                    dt_prev=dtp.value)

    def apply_static(self, sigma, out):
        """bie_apply_static on device tensors (no device allocation inside the
        library; asynchronous on the context's stream)."""
        ps, ds = _ptr(sigma)
        po, do = _ptr(out)
        if not (ds and do):
            raise ValueError("bie_apply_static takes device tensors")
        n = 2 * self.N
        if sigma.numel() != n or out.numel() != n:
            raise ValueError(f"sigma and out must hold 2N = {n} doubles each")
        dev = self.opts.device
        if sigma.device.index != dev or out.device.index != dev:
            raise ValueError(f"sigma and out must be on the context's device cuda:{dev}")
        a0, a1 = ps, ps + 8 * n
        b0, b1 = po, po + 8 * n
        if a0 < b1 and b0 < a1:
            raise ValueError("sigma and out must not overlap")
        self._check(library().bie_apply_static(self.h, ps, po))
        return out

    def features(self, out=None):
        """Node features (N x BIE_NET_FEATURES float32) of the current geometry
        and stored densities; into a device tensor `out` if given."""
        if out is None:
            X = np.zeros((self.N, BIE_NET_FEATURES), dtype=np.float32)
            self._check(library().bie_features(self.h, X.ctypes.data, 0))
            return X
        self._check(library().bie_features(self.h, out.data_ptr(), 1))
        return out

    def set_warm_net(self, net):
        """Attach a Net for warm_start = 2 (None detaches)."""
        self._warm_net = net
        self._check(library().bie_set_warm_net(self.h, None if net is None else net.h))

    def near_shape(self):
        """(index of the single-precision near-sum tile shape in use, median
        launch time in ms of each shape as opts.autotune measured it)."""
        sh = c_int32()
        ms = (ctypes.c_float * BIE_NEAR32_SHAPES)()
        self._check(library().bie_near_shape(self.h, ctypes.byref(sh), ms))
        return sh.value, list(ms)

    def device_sms(self):
        """Streaming multiprocessors of the context's device (queried at init)."""
        n = c_int32()
        self._check(library().bie_device_sms(self.h, ctypes.byref(n)))
        return n.value

    def close_info(self):
        n, u = c_int32(), c_int32()
        self._check(library().bie_close_info(self.h, ctypes.byref(n), ctypes.byref(u)))
        return n.value, u.value

    def profile(self, enable=True):
        self._check(library().bie_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        info = ProfileInfo()
        self._check(library().bie_profile_read(self.h, ctypes.byref(info)))
        return info.as_dict()

    def set_state(self, t, e2, xc, theta, sigma=None, sigma_prev2=None, dt_prev=0.0, d2=None):
        e2 = np.ascontiguousarray(e2, dtype=np.float64).ravel()
        if e2.size != 2 * self.n_cells:
            raise ValueError("e2 needs two entries per cell")
        xc = np.ascontiguousarray(xc, dtype=np.float64).ravel()
        th = np.ascontiguousarray(theta, dtype=np.float64)
        sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64).ravel()
        self._check(library().bie_set_state(self.h, float(t), e2.ctypes.data, xc.ctypes.data, th.ctypes.data,
                                            None if sg is None else sg.ctypes.data))
        s2 = None if sigma_prev2 is None else np.ascontiguousarray(sigma_prev2, dtype=np.float64).ravel()
        dd = None if d2 is None else np.ascontiguousarray(d2, dtype=np.float64).ravel()
        self._check(library().bie_set_history(self.h, None if s2 is None else s2.ctypes.data,
                                              None if dd is None else dd.ctypes.data, float(dt_prev)))


def alu_peak(device=0, stream_handle=None):
    """Measured FMA throughput of a device in TFLOP/s (bie_alu_peak):
    dict(ffma=..., ffma2=..., dfma=...)."""
    a, b, d = c_double(), c_double(), c_double()
    rc = library().bie_alu_peak(device, c_void_p(stream_handle), ctypes.byref(a), ctypes.byref(b), ctypes.byref(d))
    if rc != 0:
        raise BieError(rc, "bie_alu_peak failed")
    return dict(ffma=a.value, ffma2=b.value, dfma=d.value)


class Net:
    """The warm-start network (bie_net_*): forward, loss gradient and Adam on
    device tensors (torch float32, contiguous)."""

    def __init__(self, n_in=BIE_NET_FEATURES, device=0):
        L = library()
        h = c_void_p()
        rc = L.bie_net_init(ctypes.byref(h), n_in, device)
        if rc != 0:
            raise BieError(rc, "bie_net_init failed")
        self.h = h
        ni, hid, npar = c_int32(), c_int32(), c_int32()
        L.bie_net_size(h, ctypes.byref(ni), ctypes.byref(hid), ctypes.byref(npar))
        self.n_in, self.hidden, self.n_params = ni.value, hid.value, npar.value

    def _check(self, rc):
        if rc != 0:
            raise BieError(rc, library().bie_net_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            library().bie_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        self._check(library().bie_net_set_stream(self.h, c_void_p(stream_handle)))

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self._check(library().bie_net_set_params(self.h, p.ctypes.data))

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        self._check(library().bie_net_get_params(self.h, p.ctypes.data))
        return p

    @staticmethod
    def _dev(t, cols):
        if not (hasattr(t, "is_cuda") and t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if cols and (t.dim() != 2 or t.shape[1] != cols):
            raise ValueError(f"expected shape (N, {cols})")
        return t.data_ptr()

    def forward(self, X, Y):
        self._check(library().bie_net_forward(self.h, self._dev(X, self.n_in), X.shape[0], self._dev(Y, 2)))
        return Y

    def loss_grad(self, X, T, W, with_grad=True):
        g = np.zeros(self.n_params, dtype=np.float32) if with_grad else None
        loss = c_double()
        self._check(library().bie_net_loss_grad(self.h, self._dev(X, self.n_in), self._dev(T, 2), self._dev(W, 0),
                                                X.shape[0], None if g is None else g.ctypes.data,
                                                ctypes.byref(loss)))
        return loss.value, g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(library().bie_net_adam_step(self.h, lr, beta1, beta2, eps))
