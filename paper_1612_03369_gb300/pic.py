"""Thin ctypes binding of libpic.so (include/pic.h).

Every function has the name of its C entry point and only marshals
arguments: torch tensors supply device memory (data_ptr) and the current
CUDA stream; every step of the particle path runs in the library's kernels.
There is no CPU fallback: if libpic.so is missing or cannot be loaded, the
import of this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CAPACITY, PIC_ERR_CUDA, PIC_ERR_NOT_CONVERGED, PIC_ERR_TIMEOUT, \
    PIC_ERR_STATE = range(8)
PIC_EULER, PIC_RK2, PIC_RK4 = 1, 2, 4
PIC_FP64, PIC_FP32_BASIS, PIC_FP32_BASIS_STAGE_DF = 0, 1, 2
PIC_AVG_ARITHMETIC, PIC_AVG_GEOMETRIC, PIC_AVG_HARMONIC = 0, 1, 2
PIC_TAPE_STAGES, PIC_TAPE_CHECKPOINTS = 0, 1
PIC_STATUS_NEWTON_NONCONV, PIC_STATUS_CAPACITY, PIC_STATUS_GLOBAL_SEARCH, PIC_STATUS_BOUNDS = 1, 2, 4, 8
LOST = 0xFFFFFFFF

# name -> (restype, argtypes)
_P, _I, _U32, _U64, _SZ, _F64 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_size_t, C.c_double
SIGNATURES = {
    "pic_create_mesh": (_I, [_I, _P, _P, _I, _P, _P]),
    "pic_destroy_mesh": (_I, [_P]),
    "pic_set_velocity_dofs": (_I, [_P, _P, _P, _P]),
    "pic_seed_particles": (_I, [_P, _P, _U32, _U64, _U64, _I, _SZ, _P, _P]),
    "pic_destroy_particles": (_I, [_P]),
    "pic_set_properties": (_I, [_P, _I, _P, _P]),
    "pic_advect": (_I, [_P, _P, _F64, _I, _I, _I, _P]),
    "pic_stage_velocity_dofs": (_I, [_P, _P, _P]),
    "pic_commit_velocity_dofs": (_I, [_P, _P]),
    "pic_cell_weights": (_I, [_P, _P, _P, _P]),
    "pic_draw_cell_counts": (_I, [_U32, _P, _U64, _U64, _P, _P]),
    "pic_seed_particles_mh": (_I, [_P, _P, _P, _U32, _U64, _U64, _I, _SZ, _P, _P]),
    "pic_import_particles": (_I, [_P, _SZ, _P, _U64, _I, _SZ, _P, _P, _P]),
    "pic_advect_properties": (_I, [_P, _P, _F64, _I, _I, _P, _P]),
    "pic_locate": (_I, [_P, _P, _P]),
    "pic_advect_record": (_I, [_P, _P, _F64, _I, _I, _P, _P]),
    "pic_advect_record_tape": (_I, [_P, _P, _F64, _I, _I, _I, _P, _P]),
    "pic_tape_adjoint": (_I, [_P, _P, _P, _P, _P]),
    "pic_destroy_tape": (_I, [_P]),
    "pic_rebin": (_I, [_P, _P]),
    "pic_locate_points": (_I, [_P, _SZ, _P, _P, _P, _P, _P]),
    "pic_sort_by_cell": (_I, [_SZ, _P, _P, _U32, _P, _P, _P]),
    "pic_sort_by_cell_noalloc": (_I, [_SZ, _P, _P, _U32, _P, _P, _P]),
    "pic_interpolate_to_cells": (_I, [_P, _P, _I, _I, _P, _P, _F64, _P]),
    "pic_interpolate_to_vertices": (_I, [_P, _P, _I, _P, _P, _F64, _P]),
    "pic_project_linear": (_I, [_P, _P, _I, _P, _P, _F64, _P]),
    "pic_get_state": (_I, [_P, _P, _P, _P]),
    "pic_get_stats": (_I, [_P, _P, _P, _P, _P]),
    "pic_get_counters": (_I, [_P, _P, _I]),
    "pic_export": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pic_cell_offsets": (_I, [_P, _P, _P]),
    "pic_export_range": (_I, [_P, _SZ, _SZ, C.c_longlong, _P, _P, _P, _P, _P, _P]),
    "pic_merge_particles": (_I, [_P, _U32, _U32, _SZ, _P, _P, _P, _P, C.c_longlong, _P, _P]),
    "pic_timing_enable": (_I, [_P, _I]),
    "pic_set_advect_staging": (_I, [_P, _I]),
    "pic_timing_read": (_I, [_P, _P, _P, _P]),
    "pic_kernel_launches": (_U64, []),
    "pic_ensemble_create": (_I, [_I, _P, _P, _P, _P, _I, _P, _P]),
    "pic_ensemble_destroy": (_I, [_P]),
    "pic_ensemble_set_dt": (_I, [_P, _P, _P]),
    "pic_ensemble_run": (_I, [_P, _I, _I, _I, _I, _P]),
    "pic_ensemble_tune": (_I, [_P, _I, _P, _P, _P, _P]),
    "pic_ensemble_state": (_I, [_P, _P, _P, _P]),
    "pic_ensemble_export": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "pic_barrier_selftest": (_I, [_F64, _P]),
    "pic_last_error": (C.c_char_p, []),
    "pic_version": (C.c_char_p, []),
}


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libpic.so not built at %s (run __graft_entry__.build())" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


class PicError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.pic_last_error().decode(errors="replace")
        super().__init__("%s failed with status %d: %s" % (where, status, msg))
        self.status = status


def _check(status: int, where: str):
    if status != PIC_OK:
        raise PicError(status, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# ------------------------------------------------------------- raw calls --


def pic_create_mesh(dim: int, n_cells, vertices, stream=None) -> int:
    """vertices: torch tensor [dim][nverts] float64 (device or host)."""
    nc = (C.c_int * dim)(*[int(v) for v in n_cells])
    out = C.c_void_p()
    on_dev = 1 if vertices.is_cuda else 0
    _check(_lib.pic_create_mesh(dim, nc, _ptr(vertices), on_dev, _stream(stream), C.byref(out)), "pic_create_mesh")
    return out.value


def pic_destroy_mesh(h: int):
    _check(_lib.pic_destroy_mesh(h), "pic_destroy_mesh")


def pic_set_velocity_dofs(h: int, U, stream=None, U_next=None):
    _check(_lib.pic_set_velocity_dofs(h, _ptr(U), _ptr(U_next), _stream(stream)), "pic_set_velocity_dofs")


def pic_seed_particles(mesh: int, per_cell=None, uniform_count: int = 0, seed: int = 0, first_id: int = 0,
                       n_props: int = 0, capacity: int = 0, stream=None) -> int:
    out = C.c_void_p()
    _check(_lib.pic_seed_particles(mesh, _ptr(per_cell), int(uniform_count), seed & (2**64 - 1), first_id, int(n_props),
                                   int(capacity), _stream(stream), C.byref(out)), "pic_seed_particles")
    return out.value


def pic_destroy_particles(h: int):
    _check(_lib.pic_destroy_particles(h), "pic_destroy_particles")


def pic_set_properties(h: int, prop: int, values, stream=None):
    _check(_lib.pic_set_properties(h, int(prop), _ptr(values), _stream(stream)), "pic_set_properties")


def pic_advect(parts: int, mesh: int, dt: float, integrator: int, precision: int, n_steps: int, stream=None):
    _check(_lib.pic_advect(parts, mesh, float(dt), int(integrator), int(precision), int(n_steps), _stream(stream)),
           "pic_advect")


def pic_stage_velocity_dofs(mesh: int, U, copy_stream=None):
    """U: pinned host tensor (asynchronous copy) or device tensor [dim][nnodes] float64."""
    _check(_lib.pic_stage_velocity_dofs(mesh, _ptr(U), _stream(copy_stream)), "pic_stage_velocity_dofs")


def pic_commit_velocity_dofs(mesh: int, stream=None):
    _check(_lib.pic_commit_velocity_dofs(mesh, _stream(stream)), "pic_commit_velocity_dofs")


def pic_cell_weights(mesh: int, rho, w, stream=None):
    _check(_lib.pic_cell_weights(mesh, _ptr(rho), _ptr(w), _stream(stream)), "pic_cell_weights")


def pic_draw_cell_counts(n_cells: int, w, n_particles: int, seed: int, counts, stream=None):
    _check(_lib.pic_draw_cell_counts(int(n_cells), _ptr(w), int(n_particles), int(seed) & (2**64 - 1), _ptr(counts),
                                     _stream(stream)), "pic_draw_cell_counts")


def pic_seed_particles_mh(mesh: int, per_cell, rho, thinning: int, seed: int, first_id: int = 0, n_props: int = 0,
                          capacity: int = 0, stream=None) -> int:
    out = C.c_void_p()
    _check(_lib.pic_seed_particles_mh(mesh, _ptr(per_cell), _ptr(rho), int(thinning), int(seed) & (2**64 - 1),
                                      int(first_id), int(n_props), int(capacity), _stream(stream), C.byref(out)),
           "pic_seed_particles_mh")
    return out.value


def pic_import_particles(mesh: int, n: int, x, first_id: int = 0, n_props: int = 0, capacity: int = 0,
                         stream=None) -> tuple[int, int]:
    out = C.c_void_p()
    outside = C.c_size_t(0)
    _check(_lib.pic_import_particles(mesh, int(n), _ptr(x), int(first_id), int(n_props), int(capacity),
                                     _stream(stream), C.byref(out), C.byref(outside)), "pic_import_particles")
    return out.value, int(outside.value)


class PropertyOdes(C.Structure):
    """pic_property_odes: damage slot (or -1), alpha, beta, first deformation slot (or -1)."""
    _fields_ = [("damage", C.c_int), ("alpha", C.c_double), ("beta", C.c_double), ("deformation", C.c_int)]


def pic_advect_properties(parts: int, mesh: int, dt: float, integrator: int, n_steps: int, damage: int = -1,
                          alpha: float = 0.0, beta: float = 0.0, deformation: int = -1, stream=None):
    odes = PropertyOdes(int(damage), float(alpha), float(beta), int(deformation))
    _check(_lib.pic_advect_properties(parts, mesh, float(dt), int(integrator), int(n_steps), C.byref(odes),
                                      _stream(stream)), "pic_advect_properties")


def pic_advect_record(parts: int, mesh: int, dt: float, integrator: int, n_steps: int, stream=None) -> int:
    out = C.c_void_p()
    _check(_lib.pic_advect_record(parts, mesh, float(dt), int(integrator), int(n_steps), _stream(stream), C.byref(out)),
           "pic_advect_record")
    return out.value


def pic_advect_record_tape(parts: int, mesh: int, dt: float, integrator: int, n_steps: int, kind: int,
                           stream=None) -> int:
    out = C.c_void_p()
    _check(_lib.pic_advect_record_tape(parts, mesh, float(dt), int(integrator), int(n_steps), int(kind),
                                       _stream(stream), C.byref(out)), "pic_advect_record_tape")
    return out.value


def pic_tape_adjoint(tape: int, dL_dxfinal, dL_dU, dL_dx0=None, stream=None):
    _check(_lib.pic_tape_adjoint(tape, _ptr(dL_dxfinal), _ptr(dL_dU), _ptr(dL_dx0), _stream(stream)),
           "pic_tape_adjoint")


def pic_destroy_tape(tape: int):
    _check(_lib.pic_destroy_tape(tape), "pic_destroy_tape")


def pic_locate(parts: int, mesh: int, stream=None):
    _check(_lib.pic_locate(parts, mesh, _stream(stream)), "pic_locate")


def pic_rebin(parts: int, stream=None):
    _check(_lib.pic_rebin(parts, _stream(stream)), "pic_rebin")


def pic_locate_points(mesh: int, x, hint=None, cell_out=None, xhat_out=None, stream=None):
    """x: device [dim][n] float64.  Returns (cell_out u32-as-int32 tensor,
    xhat_out [dim][n])."""
    import torch

    dim, n = x.shape
    if cell_out is None:
        cell_out = torch.empty(n, dtype=torch.int32, device=x.device)
    if xhat_out is None:
        xhat_out = torch.empty((dim, n), dtype=torch.float64, device=x.device)
    _check(_lib.pic_locate_points(mesh, n, _ptr(x), _ptr(hint), _ptr(cell_out), _ptr(xhat_out), _stream(stream)),
           "pic_locate_points")
    return cell_out, xhat_out


def pic_sort_by_cell(cell, id, n_cells: int, perm=None, cell_off=None, stream=None):
    """cell: device int32/uint32 [n]; id: device int64 [n].  Returns (perm,
    cell_off) device int32 tensors; perm[:cell_off[-1]] is the order."""
    import torch

    n = int(cell.shape[0])
    if perm is None:
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=cell.device)
    if cell_off is None:
        cell_off = torch.empty(n_cells + 1, dtype=torch.int32, device=cell.device)
    _check(_lib.pic_sort_by_cell(n, _ptr(cell), _ptr(id), int(n_cells), _ptr(perm), _ptr(cell_off), _stream(stream)),
           "pic_sort_by_cell")
    return perm, cell_off


def pic_sort_by_cell_noalloc(cell, id, n_cells: int, perm, cell_off, stream=None):
    """As pic_sort_by_cell, with caller-provided outputs and no device
    allocation inside the library (scratch in a fixed device array)."""
    n = int(cell.shape[0])
    _check(_lib.pic_sort_by_cell_noalloc(n, _ptr(cell), _ptr(id), int(n_cells), _ptr(perm), _ptr(cell_off),
                                         _stream(stream)), "pic_sort_by_cell_noalloc")
    return perm, cell_off


def pic_interpolate_to_cells(parts: int, mesh: int, prop: int, avg, count=None, empty_fill: float = 0.0,
                             kind: int = PIC_AVG_ARITHMETIC, stream=None):
    _check(_lib.pic_interpolate_to_cells(parts, mesh, int(prop), int(kind), _ptr(avg), _ptr(count), float(empty_fill),
                                         _stream(stream)), "pic_interpolate_to_cells")


def pic_interpolate_to_vertices(parts: int, mesh: int, prop: int, avg, weight=None, empty_fill: float = 0.0,
                                stream=None):
    _check(_lib.pic_interpolate_to_vertices(parts, mesh, int(prop), _ptr(avg), _ptr(weight), float(empty_fill),
                                            _stream(stream)), "pic_interpolate_to_vertices")


def pic_project_linear(parts: int, mesh: int, prop: int, coef, count=None, empty_fill: float = 0.0, stream=None):
    _check(_lib.pic_project_linear(parts, mesh, int(prop), _ptr(coef), _ptr(count), float(empty_fill),
                                   _stream(stream)), "pic_project_linear")


def pic_get_state(parts: int):
    na, nl, st = C.c_size_t(), C.c_size_t(), C.c_uint32()
    _check(_lib.pic_get_state(parts, C.byref(na), C.byref(nl), C.byref(st)), "pic_get_state")
    return int(na.value), int(nl.value), int(st.value)


def pic_get_stats(parts: int):
    v = [C.c_uint64() for _ in range(4)]
    _check(_lib.pic_get_stats(parts, *[C.byref(a) for a in v]), "pic_get_stats")
    return dict(zip(("particle_steps", "walks", "global_searches", "newton_iterations"), [int(a.value) for a in v]))


COUNTER_NAMES = ("particle_steps", "walks", "global_searches", "newton_iterations", "lost", "fallback64", "walk64",
                 "deferred")


def pic_get_counters(parts: int) -> dict:
    v = (C.c_uint64 * len(COUNTER_NAMES))()
    _check(_lib.pic_get_counters(parts, v, len(COUNTER_NAMES)), "pic_get_counters")
    return dict(zip(COUNTER_NAMES, [int(a) for a in v]))


def pic_export(parts: int, x=None, xhat=None, id=None, cell=None, props=None, stream=None):
    _check(_lib.pic_export(parts, _ptr(x), _ptr(xhat), _ptr(id), _ptr(cell), _ptr(props), _stream(stream)),
           "pic_export")


def pic_export_range(parts: int, first: int, count: int, x=None, xhat=None, id=None, cell=None, props=None,
                     cell_shift: int = 0, stream=None):
    _check(_lib.pic_export_range(parts, int(first), int(count), int(cell_shift), _ptr(x), _ptr(xhat), _ptr(id),
                                 _ptr(cell), _ptr(props), _stream(stream)), "pic_export_range")


def pic_merge_particles(parts: int, keep_lo: int, keep_hi: int, x_in, xhat_in, id_in, cell_in, cell_shift: int = 0,
                        props_in=None, stream=None):
    n = int(id_in.shape[0]) if id_in is not None else 0
    _check(_lib.pic_merge_particles(parts, int(keep_lo), int(keep_hi), n, _ptr(x_in) if n else None,
                                    _ptr(xhat_in) if n else None, _ptr(id_in) if n else None,
                                    _ptr(cell_in) if n else None, int(cell_shift),
                                    _ptr(props_in) if (n and props_in is not None) else None, _stream(stream)),
           "pic_merge_particles")


def pic_set_advect_staging(parts: int, on: bool):
    _check(_lib.pic_set_advect_staging(parts, 1 if on else 0), "pic_set_advect_staging")


def pic_cell_offsets(parts: int, off, stream=None):
    _check(_lib.pic_cell_offsets(parts, _ptr(off), _stream(stream)), "pic_cell_offsets")


def pic_timing_enable(parts: int, on: bool):
    _check(_lib.pic_timing_enable(parts, int(bool(on))), "pic_timing_enable")


def pic_timing_read(parts: int):
    a, r, n = C.c_double(), C.c_double(), C.c_uint64()
    _check(_lib.pic_timing_read(parts, C.byref(a), C.byref(r), C.byref(n)), "pic_timing_read")
    return float(a.value), float(r.value), int(n.value)


def pic_kernel_launches() -> int:
    return int(_lib.pic_kernel_launches())


def pic_version() -> str:
    return _lib.pic_version().decode()


# --------------------------------------------------------- conveniences --


class Mesh:
    """Owning wrapper of a pic_mesh handle."""

    def __init__(self, n_cells, vertices, U=None, device="cuda", stream=None):
        import torch

        self.dim = len(n_cells)
        self.n = tuple(int(v) for v in n_cells)
        self.ncells = int(np.prod(self.n))
        X = torch.as_tensor(np.ascontiguousarray(vertices, dtype=np.float64), device=device)
        self.h = pic_create_mesh(self.dim, self.n, X, stream)
        if U is not None:
            self.set_velocity(U, stream)

    def set_velocity(self, U, stream=None, U_next=None):
        import torch

        self.U = torch.as_tensor(np.ascontiguousarray(U, dtype=np.float64), device="cuda")
        self.U_next = None
        if U_next is not None:
            self.U_next = torch.as_tensor(np.ascontiguousarray(U_next, dtype=np.float64), device="cuda")
        pic_set_velocity_dofs(self.h, self.U, stream, self.U_next)

    def locate_points(self, x, hint=None, stream=None):
        return pic_locate_points(self.h, x, hint, stream=stream)

    def close(self):
        if getattr(self, "h", None):
            pic_destroy_mesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cell_weights(mesh: "Mesh", rho):
    """Sec. 2.2: w_K = int_K rho_h dx for vertex values rho -> device tensor [n_cells]."""
    import torch

    r = torch.as_tensor(np.ascontiguousarray(rho, dtype=np.float64), device="cuda") \
        if not isinstance(rho, torch.Tensor) else rho
    w = torch.empty(mesh.ncells, dtype=torch.float64, device="cuda")
    pic_cell_weights(mesh.h, r, w)
    return w


def draw_cell_counts(w, n_particles: int, seed: int):
    """Sec. 2.2: particles per cell for n_particles weighted draws -> device int32 tensor (u32 bits)."""
    import torch

    wt = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float64), device="cuda") \
        if not isinstance(w, torch.Tensor) else w
    counts = torch.empty(wt.shape[0], dtype=torch.int32, device="cuda")
    pic_draw_cell_counts(wt.shape[0], wt, n_particles, seed, counts)
    return counts


class Particles:
    """Owning wrapper of a pic_particles handle."""

    def __init__(self, mesh: Mesh, per_cell=None, uniform_count: int = 0, seed: int = 0, first_id: int = 0,
                 n_props: int = 0, capacity: int = 0, stream=None):
        import torch

        self.mesh = mesh
        self.dim = mesh.dim
        self.n_props = n_props
        pc = None
        if per_cell is not None:
            pc = torch.as_tensor(np.ascontiguousarray(per_cell, dtype=np.uint32).view(np.int32), device="cuda")
        self.h = pic_seed_particles(mesh.h, pc, uniform_count, seed, first_id, n_props, capacity, stream)

    @classmethod
    def _wrap(cls, mesh: Mesh, h: int, n_props: int) -> "Particles":
        obj = cls.__new__(cls)
        obj.mesh, obj.dim, obj.n_props, obj.h = mesh, mesh.dim, n_props, h
        return obj

    @classmethod
    def metropolis_hastings(cls, mesh: Mesh, per_cell, rho, thinning: int = 8, seed: int = 0, first_id: int = 0,
                            n_props: int = 0, capacity: int = 0, stream=None) -> "Particles":
        """Sec. 2.2 in-cell Metropolis-Hastings generation for a vertex density rho."""
        import torch

        pc = torch.as_tensor(np.ascontiguousarray(per_cell, dtype=np.uint32).view(np.int32), device="cuda") \
            if not isinstance(per_cell, torch.Tensor) else per_cell
        r = torch.as_tensor(np.ascontiguousarray(rho, dtype=np.float64), device="cuda") \
            if not isinstance(rho, torch.Tensor) else rho
        h = pic_seed_particles_mh(mesh.h, pc, r, thinning, seed, first_id, n_props, capacity, stream)
        return cls._wrap(mesh, h, n_props)

    @classmethod
    def import_points(cls, mesh: Mesh, x, first_id: int = 0, n_props: int = 0, capacity: int = 0,
                      stream=None) -> tuple["Particles", int]:
        """Sec. 2.2 prescribed locations: x [dim][n] -> (store, number of points outside)."""
        import torch

        xt = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda") \
            if not isinstance(x, torch.Tensor) else x.contiguous()
        n = int(xt.shape[1]) if xt.dim() == 2 else 0
        h, outside = pic_import_particles(mesh.h, n, xt, first_id, n_props, capacity, stream)
        return cls._wrap(mesh, h, n_props), outside

    def advect_properties(self, dt, integrator=PIC_RK4, n_steps=1, damage=-1, alpha=0.0, beta=0.0, deformation=-1,
                          stream=None):
        """advect() that also integrates the damage and deformation-gradient ODEs (Sec. 2.6)."""
        pic_advect_properties(self.h, self.mesh.h, dt, integrator, n_steps, damage, alpha, beta, deformation, stream)

    def advect(self, dt, integrator=PIC_RK4, n_steps=1, precision=PIC_FP64, stream=None):
        pic_advect(self.h, self.mesh.h, dt, integrator, precision, n_steps, stream)

    def locate(self, stream=None):
        pic_locate(self.h, self.mesh.h, stream)

    def rebin(self, stream=None):
        pic_rebin(self.h, stream)

    def set_property(self, prop, values, stream=None):
        pic_set_properties(self.h, prop, values, stream)

    def state(self):
        return pic_get_state(self.h)

    def stats(self):
        return pic_get_counters(self.h)

    def average(self, prop, empty_fill=0.0, kind=PIC_AVG_ARITHMETIC, stream=None):
        import torch

        avg = torch.empty(self.mesh.ncells, dtype=torch.float64, device="cuda")
        cnt = torch.empty(self.mesh.ncells, dtype=torch.int32, device="cuda")
        pic_interpolate_to_cells(self.h, self.mesh.h, prop, avg, cnt, empty_fill, kind=kind, stream=stream)
        return avg, cnt

    def vertex_average(self, prop, empty_fill=0.0, stream=None):
        """Sec. 2.7 (iv): shape-function-weighted averages at the vertices -> (avg, weight sums)."""
        import torch

        nv = int(np.prod([k + 1 for k in self.mesh.n]))
        avg = torch.empty(nv, dtype=torch.float64, device="cuda")
        w = torch.empty(nv, dtype=torch.float64, device="cuda")
        pic_interpolate_to_vertices(self.h, self.mesh.h, prop, avg, w, empty_fill, stream)
        return avg, w

    def project_linear(self, prop, empty_fill=0.0, stream=None):
        """Sec. 2.7 (v): per-cell linear least squares -> (coef [dim+1][C], counts)."""
        import torch

        coef = torch.empty((self.mesh.dim + 1, self.mesh.ncells), dtype=torch.float64, device="cuda")
        cnt = torch.empty(self.mesh.ncells, dtype=torch.int32, device="cuda")
        pic_project_linear(self.h, self.mesh.h, prop, coef, cnt, empty_fill, stream)
        return coef, cnt

    def export(self, stream=None):
        """Store contents as torch device tensors in (cell, id) order."""
        import torch

        n, _, _ = self.state()
        x = torch.empty((self.dim, n), dtype=torch.float64, device="cuda")
        xh = torch.empty((self.dim, n), dtype=torch.float64, device="cuda")
        ids = torch.empty(n, dtype=torch.int64, device="cuda")
        cell = torch.empty(n, dtype=torch.int32, device="cuda")
        props = torch.empty((max(self.n_props, 1), n), dtype=torch.float64, device="cuda")
        pic_export(self.h, x, xh, ids, cell, props if self.n_props else None, stream)
        return {"x": x, "xhat": xh, "id": ids, "cell": cell, "props": props[: self.n_props]}

    def export_range(self, first: int, count: int, cell_shift: int = 0, stream=None):
        """Particles [first, first + count) of the sorted store as torch device
        tensors, cells shifted by cell_shift."""
        import torch

        x = torch.empty((self.dim, count), dtype=torch.float64, device="cuda")
        xh = torch.empty((self.dim, count), dtype=torch.float64, device="cuda")
        ids = torch.empty(count, dtype=torch.int64, device="cuda")
        cell = torch.empty(count, dtype=torch.int32, device="cuda")
        props = torch.empty((max(self.n_props, 1), count), dtype=torch.float64, device="cuda")
        if count:
            pic_export_range(self.h, first, count, x, xh, ids, cell, props if self.n_props else None, cell_shift, stream)
        return {"x": x, "xhat": xh, "id": ids, "cell": cell, "props": props[: self.n_props]}

    def merge(self, keep_lo: int, keep_hi: int, incoming=None, cell_shift: int = 0, stream=None):
        """Keep the particles of cells [keep_lo, keep_hi), add `incoming` (as
        export_range returns it) at cell + cell_shift, re-sort."""
        if incoming is None or incoming["id"].shape[0] == 0:
            pic_merge_particles(self.h, keep_lo, keep_hi, None, None, None, None, 0, None, stream)
            return
        pic_merge_particles(self.h, keep_lo, keep_hi, incoming["x"].contiguous(), incoming["xhat"].contiguous(),
                            incoming["id"].contiguous(), incoming["cell"].contiguous(), cell_shift,
                            incoming["props"].contiguous() if self.n_props else None, stream)

    def cell_offsets(self, stream=None):
        import torch

        off = torch.empty(self.mesh.ncells + 1, dtype=torch.int32, device="cuda")
        pic_cell_offsets(self.h, off, stream)
        return off

    def close(self):
        if getattr(self, "h", None):
            pic_destroy_particles(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Tape:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            if self.h:
                pic_destroy_tape(self.h)
                self.h = None
        except Exception:
            pass


def _advect_function():
    import torch

    class AdvectFunction(torch.autograd.Function):
        """x_final, ids = AdvectFunction.apply(U, parts, dt, integrator, n_steps, tape_kind)

        Forward: sets the mesh velocity to U ([dim][nnodes] float64, CUDA) and
        advances `parts` n_steps with a recorded tape; returns the final
        positions [dim][N_final] and ids [N_final] in store order.
        Backward: the adjoint sweep (pic_tape_adjoint) turns dL/dx_final into
        dL/dU.  The particle store is advanced in place by the forward.
        tape_kind: PIC_TAPE_STAGES (faster sweep) or PIC_TAPE_CHECKPOINTS
        (about half the tape memory); the gradient is the same bit for bit."""

        @staticmethod
        def forward(ctx, U, parts, dt, integrator, n_steps, tape_kind):
            pic_set_velocity_dofs(parts.mesh.h, U.detach().contiguous())
            tape = _Tape(pic_advect_record_tape(parts.h, parts.mesh.h, dt, integrator, n_steps, tape_kind))
            st = parts.export()
            ctx.tape = tape
            ctx.U_shape = U.shape
            ctx.mark_non_differentiable(st["id"])
            return st["x"], st["id"]

        @staticmethod
        def backward(ctx, grad_x, grad_ids):
            dU = torch.empty(ctx.U_shape, dtype=torch.float64, device="cuda")
            pic_tape_adjoint(ctx.tape.h, grad_x.contiguous(), dU)
            return dU, None, None, None, None, None

    return AdvectFunction


def advect_differentiable(U, parts: "Particles", dt: float, integrator: int = PIC_RK4, n_steps: int = 1,
                          tape_kind: int = 0):
    """Differentiable advection: returns (x_final [dim][N], ids [N]); gradients
    flow from x_final back to the nodal velocities U.  tape_kind as in
    pic_advect_record_tape (PIC_TAPE_STAGES or PIC_TAPE_CHECKPOINTS)."""
    return _advect_function().apply(U, parts, dt, integrator, n_steps, int(tape_kind))


# ------------------------------------------------------------- ensemble --


def pic_barrier_selftest(timeout_s: float, stream=None) -> int:
    """Returns the status (PIC_ERR_TIMEOUT is the expected outcome)."""
    return int(_lib.pic_barrier_selftest(float(timeout_s), _stream(stream)))


class Ensemble:
    """Independent problems advanced together (pic_ensemble_*)."""

    def __init__(self, meshes, per_cell=None, uniform_counts=None, seeds=None, n_props=0, stream=None):
        import torch

        self.meshes = list(meshes)
        self.P = len(self.meshes)
        self.dim = self.meshes[0].dim
        hs = (C.c_void_p * self.P)(*[m.h for m in self.meshes])
        self._pc_tensors = []
        pc_arr = None
        if per_cell is not None:
            ptrs = []
            for a in per_cell:
                if a is None:
                    ptrs.append(None)
                else:
                    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32), device="cuda")
                    self._pc_tensors.append(t)
                    ptrs.append(t.data_ptr())
            pc_arr = (C.c_void_p * self.P)(*ptrs)
        uc = None
        if uniform_counts is not None:
            uc = (C.c_uint32 * self.P)(*[int(v) for v in uniform_counts])
        sd = (C.c_uint64 * self.P)(*[int(v) & (2**64 - 1) for v in (seeds or [0] * self.P)])
        out = C.c_void_p()
        _check(_lib.pic_ensemble_create(self.P, hs, pc_arr, uc, sd, int(n_props), _stream(stream), C.byref(out)),
               "pic_ensemble_create")
        self.h = out.value

    def set_dt(self, dts, stream=None):
        a = (C.c_double * self.P)(*[float(v) for v in dts])
        _check(_lib.pic_ensemble_set_dt(self.h, a, _stream(stream)), "pic_ensemble_set_dt")

    def run(self, integrator=PIC_RK4, n_steps=1, mode=1, use_graph=True, stream=None):
        _check(_lib.pic_ensemble_run(self.h, int(integrator), int(n_steps), int(mode), int(bool(use_graph)),
                                     _stream(stream)), "pic_ensemble_run")

    def tune(self, integrator=PIC_RK4, stream=None):
        b, t, ms = C.c_int(), C.c_int(), C.c_double()
        _check(_lib.pic_ensemble_tune(self.h, int(integrator), C.byref(b), C.byref(t), C.byref(ms), _stream(stream)),
               "pic_ensemble_tune")
        return int(b.value), int(t.value), float(ms.value)

    def state(self):
        na, nl, st = C.c_size_t(), C.c_size_t(), C.c_uint32()
        _check(_lib.pic_ensemble_state(self.h, C.byref(na), C.byref(nl), C.byref(st)), "pic_ensemble_state")
        return int(na.value), int(nl.value), int(st.value)

    def export(self, problem, stream=None):
        import torch

        n = C.c_size_t()
        _check(_lib.pic_ensemble_export(self.h, int(problem), None, None, None, None, C.byref(n), _stream(stream)),
               "pic_ensemble_export")
        n = int(n.value)
        x = torch.empty((self.dim, max(n, 1)), dtype=torch.float64, device="cuda")
        xh = torch.empty((self.dim, max(n, 1)), dtype=torch.float64, device="cuda")
        ids = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        cell = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        m = C.c_size_t()
        _check(_lib.pic_ensemble_export(self.h, int(problem), _ptr(x), _ptr(xh), _ptr(ids), _ptr(cell), C.byref(m),
                                        _stream(stream)), "pic_ensemble_export")
        torch.cuda.synchronize()
        return {"x": x[:, :n], "xhat": xh[:, :n], "id": ids[:n], "cell": cell[:n]}

    def close(self):
        if getattr(self, "h", None):
            pic_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_ensemble_destroy(h):
    _check(_lib.pic_ensemble_destroy(h), "pic_ensemble_destroy")
