"""Thin PyTorch binding of libfst.so.

Every function here only checks and marshals arguments: tensors in, device
pointers plus the current CUDA stream out to the C ABI, output tensors
allocated with torch when the caller passes none. All arithmetic runs in the
library's kernels.

Layout: FP32 CUDA tensors in structure-of-arrays form, environment index
last and contiguous: q (nq, B), qd/qdd/tau (nv, B), poses (n_b, 12, B),
J (n_links, 6, nv, B), M (nv, nv, B). `soa(x)` / `aos(x)` convert from/to
the (B, ...) layout most training code uses.
"""
from __future__ import annotations

import ctypes
import hashlib

import numpy as np
import torch

from . import _ffi
from ._ffi import check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def soa(x: torch.Tensor) -> torch.Tensor:
    """(B, ...) -> (..., B) contiguous."""
    return x.movedim(0, -1).contiguous()


def aos(x: torch.Tensor) -> torch.Tensor:
    """(..., B) -> (B, ...) view."""
    return x.movedim(-1, 0)


class Model:
    """A kinematic tree uploaded to the current CUDA device.

    `tree` is any object with the body-table fields parent, jtype, axis,
    T_joint, T_link, mass, com, I_com and gravity (see workloads.Tree)."""

    def __init__(self, tree, device=None, specialize=False):
        L = _ffi.lib()
        n = len(tree.parent)
        arr = (_ffi.BodyDesc * n)()
        for i in range(n):
            d = arr[i]
            d.parent = int(tree.parent[i])
            d.type = int(tree.jtype[i])
            for k in range(3):
                d.axis[k] = float(tree.axis[i][k])
                d.com[k] = float(tree.com[i][k])
            for k in range(12):
                d.T_joint[k] = float(tree.T_joint[i][k])
                d.T_link[k] = float(tree.T_link[i][k])
            d.mass = float(tree.mass[i])
            for k in range(6):
                d.I_com[k] = float(tree.I_com[i][k])
        g = (ctypes.c_double * 3)(*[float(x) for x in tree.gravity])
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.fst_model_create(arr, n, g, ctypes.byref(handle)))
        self._h = handle
        nq, nv, nb, depth = (ctypes.c_int32() for _ in range(4))
        check(L.fst_model_info(self._h, ctypes.byref(nq), ctypes.byref(nv), ctypes.byref(nb), ctypes.byref(depth)))
        self.nq, self.nv, self.n_bodies, self.depth = nq.value, nv.value, nb.value, depth.value
        self.name = getattr(tree, "name", "tree")
        self.ee = tuple(getattr(tree, "ee", ()))
        h = hashlib.sha1()
        for f in ("parent", "jtype", "axis", "T_joint", "T_link", "mass", "com", "I_com", "gravity"):
            h.update(np.ascontiguousarray(np.asarray(getattr(tree, f), dtype=np.float64)).tobytes())
        self.fingerprint = h.hexdigest()[:16]
        if specialize:
            self.specialize(None if specialize is True else specialize)

    def specialize(self, kinds=None):
        """Compile kernels specialised for this tree (fst_model_specialize);
        `kinds` is an iterable of names from _ffi.SPEC_KINDS, None = all."""
        mask = 0 if kinds is None else sum(1 << _ffi.SPEC_KINDS.index(k) for k in kinds)
        with torch.cuda.device(self.device):
            check(_ffi.lib().fst_model_specialize(self._h, mask))
        return self.specialized()

    def theta(self):
        """The model's own inertial parameters (n_b, 10), float32, on its device."""
        buf = (ctypes.c_float * (self.n_bodies * 10))()
        check(_ffi.lib().fst_model_theta(self._h, buf))
        return torch.tensor(list(buf), dtype=torch.float32).view(self.n_bodies, 10).to(self.device)

    def set_launch(self, kinds=None, block=0, variant="auto"):
        """Launch configuration (fst_model_set_launch) of the given kernel
        kinds (names from _ffi.SPEC_KINDS, None = all): threads per block
        (0 = built-in heuristic) and variant ("auto", "generic",
        "specialized", "level", "mixed" (eval only))."""
        mask = 0 if kinds is None else sum(1 << _ffi.SPEC_KINDS.index(k) for k in kinds)
        check(_ffi.lib().fst_model_set_launch(self._h, mask, int(block), _ffi.VARIANTS[variant]))

    ROLES = {"none": -1, "aba": 0, "crba": 1, "rnea": 2, "kin": 3}

    def set_sm_roles(self, roles):
        """Role of every SM id for the "pinned" variant (fst_model_set_sm_roles):
        a sequence of role names ("aba", "crba", "rnea", "kin", "none") or
        codes, indexed by SM id."""
        codes = [self.ROLES[r] if isinstance(r, str) else int(r) for r in roles]
        arr = (ctypes.c_int32 * len(codes))(*codes)
        with torch.cuda.device(self.device):
            check(_ffi.lib().fst_model_set_sm_roles(self._h, arr, len(codes)))

    def specialized(self):
        """Names of the kernel kinds that run specialised for this model."""
        m = ctypes.c_uint32()
        check(_ffi.lib().fst_model_specialized(self._h, ctypes.byref(m)))
        return tuple(k for i, k in enumerate(_ffi.SPEC_KINDS) if (m.value >> i) & 1)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _ffi.lib().fst_model_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        return f"Model({self.name}: n_b={self.n_bodies}, nq={self.nq}, nv={self.nv}, depth={self.depth})"


def set_smem_carveout(percent: int):
    """fst_set_smem_carveout: -1 = per kernel, else one percentage for all."""
    check(_ffi.lib().fst_set_smem_carveout(int(percent)))


def _check_in(x, rows, name, model):
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if x.dtype != torch.float32 or x.device != model.device:
        raise ValueError(f"{name} must be float32 on {model.device}, got {x.dtype} on {x.device}")
    if x.dim() != 2 or x.shape[0] != rows or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous ({rows}, B) tensor, got {tuple(x.shape)}")
    return x.shape[1]


def _check_shape(x, shape, name, model):
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if (tuple(x.shape) != tuple(shape) or x.dtype != torch.float32 or x.device != model.device
            or not x.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 {tuple(shape)} tensor on {model.device}")


def _host_out_ok(t):
    """A pinned host tensor the device can write with its own pointer
    (fst_device_can_access)."""
    if t.device.type != "cpu" or not t.is_pinned():
        return False
    ok = ctypes.c_int32()
    with torch.cuda.device(torch.cuda.current_device()):
        check(_ffi.lib().fst_device_can_access(ctypes.c_void_p(t.data_ptr()), ctypes.byref(ok)))
    return bool(ok.value)


def _out(out, shape, model):
    """An output tensor: on the model's device, or pinned host memory the
    device addresses directly (the kernels then write to the host)."""
    if out is None:
        return torch.empty(shape, dtype=torch.float32, device=model.device)
    if out.shape != torch.Size(shape) or out.dtype != torch.float32 or not out.is_contiguous() or \
            (out.device != model.device and not _host_out_ok(out)):
        raise ValueError(f"out must be a contiguous float32 {shape} tensor on {model.device} "
                         "(or in pinned host memory the device can address)")
    return out


def _theta(theta, model):
    if theta is None:
        return None
    if theta.dtype != torch.float32 or theta.device != model.device or theta.shape != (model.n_bodies, 10) \
            or not theta.is_contiguous():
        raise ValueError(f"theta must be a contiguous float32 ({model.n_bodies}, 10) tensor on {model.device}")
    return theta


def fk(model: Model, q, out=None):
    """World poses (n_b, 12, B): R row-major then p, for every body."""
    B = _check_in(q, model.nq, "q", model)
    out = _out(out, (model.n_bodies, 12, B), model)
    check(_ffi.lib().fst_fk(model.handle, B, _ptr(q), _ptr(out), _stream()))
    return out


def jacobian(model: Model, q, links, out=None):
    """World-frame Jacobians (n_links, 6, nv, B), rows [v; w]."""
    B = _check_in(q, model.nq, "q", model)
    links = [int(l) for l in links]
    arr = (ctypes.c_int32 * len(links))(*links)
    out = _out(out, (len(links), 6, model.nv, B), model)
    check(_ffi.lib().fst_jacobian(model.handle, B, _ptr(q), arr, len(links), _ptr(out), _stream()))
    return out


def rnea(model: Model, q, qd, qdd, theta=None, out=None):
    """Inverse dynamics tau (nv, B)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd")):
        if _check_in(x, model.nv, nm, model) != B:
            raise ValueError(f"{nm} batch size differs from q")
    out = _out(out, (model.nv, B), model)
    check(_ffi.lib().fst_rnea(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                              _ptr(out), _stream()))
    return out


def crba(model: Model, q, theta=None, out=None):
    """Mass matrix (nv, nv, B)."""
    B = _check_in(q, model.nq, "q", model)
    out = _out(out, (model.nv, model.nv, B), model)
    check(_ffi.lib().fst_crba(model.handle, B, _ptr(q), _ptr(_theta(theta, model)), _ptr(out), _stream()))
    return out


def aba(model: Model, q, qd, tau, theta=None, out=None):
    """Forward dynamics qdd (nv, B)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (tau, "tau")):
        if _check_in(x, model.nv, nm, model) != B:
            raise ValueError(f"{nm} batch size differs from q")
    out = _out(out, (model.nv, B), model)
    check(_ffi.lib().fst_aba(model.handle, B, _ptr(q), _ptr(qd), _ptr(tau), _ptr(_theta(theta, model)),
                             _ptr(out), _stream()))
    return out


def eval(model: Model, q, qd=None, qdd=None, tau=None, *, fk=False, links=None, rnea=False, crba=False,
         aba=False, theta=None, out=None, tau_bar=None, q_bar=False, qd_bar=False, qdd_bar=False,
         one_sweep=False, packed=False):
    """Every requested operator in one fused launch (fst_eval).

    fk=True requests poses; links=[...] the Jacobians of those bodies;
    rnea=True tau (needs qd, qdd); crba=True M; aba=True qdd (needs qd, tau).
    q_bar/qd_bar/qdd_bar=True request the RNEA adjoint for the cotangent
    tau_bar (nv, B) in the same pass; tau_bar="tau" uses the computed tau
    (with rnea=True). one_sweep=True computes poses and Jacobians from the
    RNEA sweep's own joint transforms. packed=True writes M as its upper
    triangle (nv (nv + 1) / 2, B) and J as the support-path columns of each
    link (packed_layout(), (j_rows, B)). Returns a dict with the requested
    outputs ("poses", "J", "tau", "M", "qdd", "q_bar", "qd_bar", "qdd_bar");
    `out` may supply preallocated tensors under the same keys."""
    B = _check_in(q, model.nq, "q", model)
    out = dict(out or {})
    io = _ffi.EvalIO()
    io.q = q.data_ptr()
    vjp = q_bar or qd_bar or qdd_bar
    if vjp and tau_bar is None:
        raise ValueError("the RNEA adjoint needs tau_bar (a (nv, B) tensor, or 'tau' with rnea=True)")
    if isinstance(tau_bar, str) and (tau_bar != "tau" or not rnea):
        raise ValueError("tau_bar='tau' needs rnea=True")
    if rnea or aba or vjp:
        _check_in(qd, model.nv, "qd", model)
        io.qd = qd.data_ptr()
    if rnea or vjp:
        _check_in(qdd, model.nv, "qdd", model)
        io.qdd = qdd.data_ptr()
    if aba:
        _check_in(tau, model.nv, "tau", model)
        io.tau = tau.data_ptr()
    res = {}
    if fk:
        res["poses"] = _out(out.get("poses"), (model.n_bodies, 12, B), model)
        io.poses = res["poses"].data_ptr()
    link_arr = None
    if links:
        links = [int(l) for l in links]
        link_arr = (ctypes.c_int32 * len(links))(*links)
        jshape = (packed_layout(model, links)[1], B) if packed else (len(links), 6, model.nv, B)
        res["J"] = _out(out.get("J"), jshape, model)
        io.J = res["J"].data_ptr()
        io.links = link_arr
        io.n_links = len(links)
    if rnea:
        res["tau"] = _out(out.get("tau"), (model.nv, B), model)
        io.tau_out = res["tau"].data_ptr()
    if crba:
        mshape = (model.nv * (model.nv + 1) // 2, B) if packed else (model.nv, model.nv, B)
        res["M"] = _out(out.get("M"), mshape, model)
        io.M = res["M"].data_ptr()
    if aba:
        res["qdd"] = _out(out.get("qdd"), (model.nv, B), model)
        io.qdd_out = res["qdd"].data_ptr()
    if vjp:
        if isinstance(tau_bar, str):
            io.tau_bar = io.tau_out
        else:
            _check_in(tau_bar, model.nv, "tau_bar", model)
            io.tau_bar = tau_bar.data_ptr()
        for key, want, rows in (("q_bar", q_bar, model.nq), ("qd_bar", qd_bar, model.nv),
                                ("qdd_bar", qdd_bar, model.nv)):
            if want:
                res[key] = _out(out.get(key), (rows, B), model)
                setattr(io, key, res[key].data_ptr())
    io.flags = (_ffi.EVAL_ONE_SWEEP if one_sweep else 0) | (_ffi.EVAL_PACKED if packed else 0)
    check(_ffi.lib().fst_eval(model.handle, B, ctypes.byref(io), _ptr(_theta(theta, model)), _stream()))
    return res


def packed_layout(model: Model, links):
    """The packed Jacobian layout of eval(packed=True) (fst_packed_layout):
    (support-path columns per link, rows of the packed J, rows of the packed
    M)."""
    links = [int(l) for l in links]
    arr = (ctypes.c_int32 * max(len(links), 1))(*links)
    cols = (ctypes.c_int32 * max(len(links), 1))()
    jr, mr = ctypes.c_int32(), ctypes.c_int32()
    check(_ffi.lib().fst_packed_layout(model.handle, arr, len(links), cols, ctypes.byref(jr), ctypes.byref(mr)))
    return [cols[k] for k in range(len(links))], jr.value, mr.value


# ---------------------------------------------------------------------------
# adjoints
# ---------------------------------------------------------------------------

def adjoint_scratch(model: Model, B: int) -> torch.Tensor:
    """Device scratch for the thetabar partial sums of B environments."""
    n = ctypes.c_size_t()
    check(_ffi.lib().fst_adjoint_scratch_bytes(model.handle, int(B), ctypes.byref(n)))
    return torch.empty(max(int(n.value), 4), dtype=torch.uint8, device=model.device)


def _scratch(model, B, scratch):
    if scratch is None:
        scratch = adjoint_scratch(model, B)
    return _ptr(scratch), scratch.numel() * scratch.element_size()


def fk_vjp(model: Model, q, poses_bar, out=None):
    """q_bar (nq, B) for the cotangent poses_bar (n_b, 12, B) of fk()."""
    B = _check_in(q, model.nq, "q", model)
    if poses_bar.shape != (model.n_bodies, 12, B) or not poses_bar.is_contiguous() or poses_bar.dtype != torch.float32:
        raise ValueError(f"poses_bar must be a contiguous float32 ({model.n_bodies}, 12, {B}) tensor")
    out = _out(out, (model.nq, B), model)
    check(_ffi.lib().fst_fk_vjp(model.handle, B, _ptr(q), _ptr(poses_bar), _ptr(out), _stream()))
    return out


def rnea_vjp(model: Model, q, qd, qdd, tau_bar, theta=None, *, q_bar=True, qd_bar=True, qdd_bar=True,
             theta_bar=True, scratch=None):
    """Cotangents of rnea() for tau_bar (nv, B). Returns a dict with the
    requested keys among "q", "qd", "qdd" ((nq|nv, B)) and "theta" (n_b, 10,
    summed over environments)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd"), (tau_bar, "tau_bar")):
        _check_in(x, model.nv, nm, model)
    res = {}
    if q_bar:
        res["q"] = _out(None, (model.nq, B), model)
    if qd_bar:
        res["qd"] = _out(None, (model.nv, B), model)
    if qdd_bar:
        res["qdd"] = _out(None, (model.nv, B), model)
    if theta_bar:
        res["theta"] = _out(None, (model.n_bodies, 10), model)
    sp, sb = _scratch(model, B, scratch) if theta_bar else (None, 0)
    check(_ffi.lib().fst_rnea_vjp(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                                  _ptr(tau_bar), _ptr(res.get("q")), _ptr(res.get("qd")), _ptr(res.get("qdd")),
                                  _ptr(res.get("theta")), sp, sb, _stream()))
    return res


def rnea_tape(model: Model, B: int):
    """Device buffer for the store variant's forward tape ([n_b][30][B])."""
    n = ctypes.c_size_t()
    check(_ffi.lib().fst_rnea_tape_bytes(model.handle, B, ctypes.byref(n)))
    import torch
    return torch.empty(max(n.value // 4, 1), dtype=torch.float32, device=model.device)


def rnea_store(model: Model, q, qd, qdd, theta=None, tape=None, out=None, tau=True):
    """RNEA that also writes the forward tape for rnea_vjp_stored.
    Returns (tau or None, tape)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd")):
        if _check_in(x, model.nv, nm, model) != B:
            raise ValueError(f"{nm} batch size differs from q")
    tape = rnea_tape(model, B) if tape is None else tape
    out = _out(out, (model.nv, B), model) if tau else None
    check(_ffi.lib().fst_rnea_store(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                                    _ptr(out), _ptr(tape), tape.numel() * 4, _stream()))
    return out, tape


def rnea_vjp_stored(model: Model, q, qd, tape, tau_bar, theta=None, *, q_bar=True, qd_bar=True, qdd_bar=True,
                    theta_bar=True, scratch=None):
    """rnea_vjp() from a tape written by rnea_store() (no forward sweep)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (tau_bar, "tau_bar")):
        _check_in(x, model.nv, nm, model)
    res = {}
    if q_bar:
        res["q"] = _out(None, (model.nq, B), model)
    if qd_bar:
        res["qd"] = _out(None, (model.nv, B), model)
    if qdd_bar:
        res["qdd"] = _out(None, (model.nv, B), model)
    if theta_bar:
        res["theta"] = _out(None, (model.n_bodies, 10), model)
    sp, sb = _scratch(model, B, scratch) if theta_bar else (None, 0)
    check(_ffi.lib().fst_rnea_vjp_stored(model.handle, B, _ptr(q), _ptr(qd), _ptr(_theta(theta, model)), _ptr(tape),
                                         tape.numel() * 4, _ptr(tau_bar), _ptr(res.get("q")), _ptr(res.get("qd")),
                                         _ptr(res.get("qdd")), _ptr(res.get("theta")), sp, sb, _stream()))
    return res


def jacobian_vjp(model: Model, q, links, J_bar):
    """q_bar (nq, B) for the cotangent J_bar (n_links, 6, nv, B) of jacobian()."""
    B = _check_in(q, model.nq, "q", model)
    links = [int(l) for l in links]
    _check_shape(J_bar, (len(links), 6, model.nv, B), "J_bar", model)
    arr = (ctypes.c_int32 * len(links))(*links)
    q_bar = _out(None, (model.nq, B), model)
    check(_ffi.lib().fst_jacobian_vjp(model.handle, B, _ptr(q), arr, len(links), _ptr(J_bar), _ptr(q_bar), _stream()))
    return q_bar


def crba_vjp(model: Model, q, M_bar, theta=None, *, q_bar=True, theta_bar=True, scratch=None):
    """Cotangents of crba() for M_bar (nv, nv, B): a dict with keys among
    "q" (nq, B) and "theta" (n_b, 10, summed over environments)."""
    B = _check_in(q, model.nq, "q", model)
    _check_shape(M_bar, (model.nv, model.nv, B), "M_bar", model)
    res = {}
    if q_bar:
        res["q"] = _out(None, (model.nq, B), model)
    if theta_bar:
        res["theta"] = _out(None, (model.n_bodies, 10), model)
    sp, sb = _scratch(model, B, scratch) if theta_bar else (None, 0)
    check(_ffi.lib().fst_crba_vjp(model.handle, B, _ptr(q), _ptr(_theta(theta, model)), _ptr(M_bar),
                                  _ptr(res.get("q")), _ptr(res.get("theta")), sp, sb, _stream()))
    return res


def rnea_derivatives(model: Model, q, qd, qdd, theta=None, *, dq=True, dqd=True):
    """Dense d tau / d q (tangent directions) and d tau / d qd, (nv, nv, B)
    each (row = tau component, column = direction). Returns a dict with the
    requested keys "q", "qd"."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd")):
        if _check_in(x, model.nv, nm, model) != B:
            raise ValueError(f"{nm} batch size differs from q")
    res = {}
    if dq:
        res["q"] = _out(None, (model.nv, model.nv, B), model)
    if dqd:
        res["qd"] = _out(None, (model.nv, model.nv, B), model)
    check(_ffi.lib().fst_rnea_derivatives(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                                          _ptr(res.get("q")), _ptr(res.get("qd")), _stream()))
    return res


def aba_derivatives(model: Model, q, qd, tau, theta=None, *, dq=True, dqd=True, qdd=False):
    """Dense d qdd / d q (tangent directions), d qdd / d qd and
    d qdd / d tau = M^-1, (nv, nv, B) each, at qdd = ABA(q, qd, tau).
    Returns a dict with keys "q", "qd" (as requested), "tau" (M^-1) and,
    with qdd=True, "qdd" (nv, B)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (tau, "tau")):
        if _check_in(x, model.nv, nm, model) != B:
            raise ValueError(f"{nm} batch size differs from q")
    res = {"tau": _out(None, (model.nv, model.nv, B), model)}
    if dq:
        res["q"] = _out(None, (model.nv, model.nv, B), model)
    if dqd:
        res["qd"] = _out(None, (model.nv, model.nv, B), model)
    if qdd:
        res["qdd"] = _out(None, (model.nv, B), model)
    check(_ffi.lib().fst_aba_derivatives(model.handle, B, _ptr(q), _ptr(qd), _ptr(tau), _ptr(_theta(theta, model)),
                                         _ptr(res.get("qdd")), _ptr(res.get("q")), _ptr(res.get("qd")),
                                         _ptr(res["tau"]), _stream()))
    return res


def aba_vjp(model: Model, q, qd, qdd, qdd_bar, theta=None, *, q_bar=True, qd_bar=True, tau_bar=True,
            theta_bar=True, scratch=None):
    """Cotangents of aba() for qdd_bar (nv, B); qdd is aba()'s result.
    Returns a dict with keys among "q", "qd", "tau", "theta"."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd"), (qdd_bar, "qdd_bar")):
        _check_in(x, model.nv, nm, model)
    res = {}
    if q_bar:
        res["q"] = _out(None, (model.nq, B), model)
    if qd_bar:
        res["qd"] = _out(None, (model.nv, B), model)
    if tau_bar:
        res["tau"] = _out(None, (model.nv, B), model)
    if theta_bar:
        res["theta"] = _out(None, (model.n_bodies, 10), model)
    sp, sb = _scratch(model, B, scratch) if theta_bar else (None, 0)
    check(_ffi.lib().fst_aba_vjp(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                                 _ptr(qdd_bar), _ptr(res.get("q")), _ptr(res.get("qd")), _ptr(res.get("tau")),
                                 _ptr(res.get("theta")), sp, sb, _stream()))
    return res


def rnea_loss_grad(model: Model, q, qd, qdd, tau_meas, theta=None, *, q_bar=False, qd_bar=False, scratch=None,
                   out=None):
    """L = sum (rnea(q, qd, qdd; theta) - tau_meas)^2 and dL/dtheta in one
    pass. Returns (L as a 0-d tensor, theta_bar (n_b, 10), q_bar, qd_bar)."""
    B = _check_in(q, model.nq, "q", model)
    for x, nm in ((qd, "qd"), (qdd, "qdd"), (tau_meas, "tau_meas")):
        _check_in(x, model.nv, nm, model)
    buf = _out(out, (model.n_bodies * 10 + 1,), model)
    qb = _out(None, (model.nq, B), model) if q_bar else None
    qdb = _out(None, (model.nv, B), model) if qd_bar else None
    sp, sb = _scratch(model, B, scratch)
    check(_ffi.lib().fst_rnea_loss_grad(model.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(_theta(theta, model)),
                                        _ptr(tau_meas), _ptr(buf), _ptr(qb), _ptr(qdb), sp, sb, _stream()))
    return buf[-1], buf[:-1].view(model.n_bodies, 10), qb, qdb


# ---------------------------------------------------------------------------
# mixed batches of several trees
# ---------------------------------------------------------------------------

class MultiBatch:
    """Several models evaluated in one persistent launch (fst_multi_eval)."""

    def __init__(self, models):
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        h = ctypes.c_void_p()
        check(_ffi.lib().fst_multi_create(arr, len(self.models), ctypes.byref(h)))
        self._h = h

    def set_launch(self, block=64, variant="generic"):
        """Launch form of eval() (fst_multi_set_launch): "generic" (one
        environment per thread) or "level" (level-parallel, 32 environments
        per item), with `block` threads per block."""
        check(_ffi.lib().fst_multi_set_launch(self._h, int(block), _ffi.VARIANTS[variant]))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _ffi.lib().fst_multi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, items):
        """items[k] for models[k]: dict with "q" and, as needed, "qd", "qdd",
        "tau", plus flags fk/rnea/crba/aba and optional preallocated outputs
        under "out". Returns one dict of outputs per model."""
        if len(items) != len(self.models):
            raise ValueError("one item per model")
        ios = (_ffi.MultiIO * len(items))()
        results = []
        for k, (m, it) in enumerate(zip(self.models, items)):
            q = it["q"]
            B = _check_in(q, m.nq, "q", m)
            io = ios[k]
            io.B = B
            io.q = q.data_ptr()
            for name in ("qd", "qdd", "tau"):
                if it.get(name) is not None:
                    _check_in(it[name], m.nv, name, m)
                    setattr(io, name, it[name].data_ptr())
            out = dict(it.get("out") or {})
            res = {}
            if it.get("fk"):
                res["poses"] = _out(out.get("poses"), (m.n_bodies, 12, B), m)
                io.poses = res["poses"].data_ptr()
            if it.get("rnea"):
                res["tau"] = _out(out.get("tau"), (m.nv, B), m)
                io.tau_out = res["tau"].data_ptr()
            if it.get("crba"):
                res["M"] = _out(out.get("M"), (m.nv, m.nv, B), m)
                io.M = res["M"].data_ptr()
            if it.get("aba"):
                res["qdd"] = _out(out.get("qdd"), (m.nv, B), m)
                io.qdd_out = res["qdd"].data_ptr()
            results.append(res)
        check(_ffi.lib().fst_multi_eval(self._h, ios, _stream()))
        return results


def fp32_probe(blocks_per_sm: int = 4, iters: int = 1 << 16, out=None):
    """Launches the FP32 FMA throughput probe (fst_fp32_probe) on the current
    stream. Returns (flops of the launch, the output buffer); time the call
    with CUDA events around it."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n = sms * blocks_per_sm * 256
    if out is None or out.numel() < n:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = ctypes.c_double()
    check(_ffi.lib().fst_fp32_probe(int(blocks_per_sm), int(iters), _ptr(out), out.numel() * 4, ctypes.byref(fl),
                                    _stream()))
    return fl.value, out


_SM_IDS = {}


def sm_ids(device=None):
    """The hardware ids of the device's SMs (fst_sm_ids), sorted; probed once
    per device."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    if dev not in _SM_IDS:
        buf = (ctypes.c_int32 * 1024)()
        n = ctypes.c_int32()
        with torch.cuda.device(dev):
            check(_ffi.lib().fst_sm_ids(buf, 1024, ctypes.byref(n)))
        _SM_IDS[dev] = [buf[k] for k in range(min(n.value, 1024))]
    return _SM_IDS[dev]


class SmPartition:
    """Disjoint SM sets of one device, each with a stream whose kernels run
    only on its SMs (fst_sm_partition_create: CUDA green contexts), also
    inside a CUDA graph captured from another stream that forks into them.
    `streams[k]` is a torch stream of partition k, `sm_counts[k]` its SMs
    (each request rounded up to groups of 8). Keep the object alive while
    any launch or graph that uses its streams can still run."""

    def __init__(self, sm_counts, device=None):
        dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
        counts = [int(c) for c in sm_counts]
        arr = (ctypes.c_int32 * len(counts))(*counts)
        h = ctypes.c_void_p()
        check(_ffi.lib().fst_sm_partition_create(int(dev), arr, len(counts), ctypes.byref(h)))
        self._h = h
        self.device = dev
        self.streams, self.sm_counts = [], []
        for k in range(len(counts)):
            s, c = ctypes.c_void_p(), ctypes.c_int32()
            check(_ffi.lib().fst_sm_partition_info(h, k, ctypes.byref(s), ctypes.byref(c)))
            self.streams.append(torch.cuda.ExternalStream(s.value, device=torch.device("cuda", dev)))
            self.sm_counts.append(c.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            _ffi.lib().fst_sm_partition_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_PARTITIONS = {}


def sm_partition(sm_counts, device=None):
    """A shared SmPartition per (device, SM counts): step plans that use the
    same split reuse one set of green contexts for the life of the process."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    key = (dev, tuple(int(c) for c in sm_counts))
    if key not in _PARTITIONS:
        _PARTITIONS[key] = SmPartition(key[1], dev)
    return _PARTITIONS[key]
