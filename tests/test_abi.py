"""Host-side checks of the C ABI (no GPU needed, no kernel launched): the
library loads, exports every entry point include/frax.h declares, and
frax_model_create validates its arguments and derives the tree structure."""

import ctypes
import os
import re

import numpy as np
import pytest

import gen
import paper_2604_04310_gb300 as fx
from paper_2604_04310_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"FRAX_API\s+[\w\s\*]+?\b(frax_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared()
    assert {"frax_model_create", "frax_rnea", "frax_aba", "frax_crba", "frax_fk", "frax_jacobian",
            "frax_rnea_vjp", "frax_aba_vjp"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(_lib.SIGNATURES)


def test_model_dims_and_kinds():
    c = fx.Model.from_robot(gen.chain7(0))
    assert (c.nq, c.nv, c.n_bodies, c.kind) == (7, 7, 7, 0)
    h = fx.Model.from_robot(gen.humanoid(0))
    assert (h.nq, h.nv, h.n_bodies) == (36, 35, 30)
    t = fx.Model.from_robot(gen.random_tree(7, 64))
    assert (t.nq, t.nv, t.n_bodies, t.kind) == (64, 64, 64, 1)


def _valid(n=3):
    r = gen.random_tree(3, n)
    return dict(parent=r.parent.copy(), joint_type=r.joint_type.copy(), axis=r.axis.copy(),
                placement=r.placement.copy(), inertia=r.inertia.copy(), gravity=r.gravity.copy())


@pytest.mark.parametrize("mutate,msg", [
    (lambda a: a["parent"].__setitem__(1, 1), "parent"),
    (lambda a: a["parent"].__setitem__(0, 0), "parent"),
    (lambda a: a["joint_type"].__setitem__(1, 1), "free-flyer"),
    (lambda a: a["joint_type"].__setitem__(2, 5), "joint type"),
    (lambda a: a["axis"].__setitem__(1, [0.0, 0.0, 2.0]), "unit"),
    (lambda a: a["placement"].__setitem__((1, 0), 2.0), "rotation"),
    (lambda a: a["inertia"].__setitem__((2, 0), -1.0), "mass"),
    (lambda a: a["inertia"].__setitem__((2, 4), -1.0), "positive definite"),
    (lambda a: a["gravity"].__setitem__(0, np.nan), "gravity"),
])
def test_model_create_rejects(mutate, msg):
    a = _valid()
    mutate(a)
    with pytest.raises(fx.FraxError) as e:
        fx.Model(**a)
    assert msg in str(e.value) and e.value.status == 1


def test_model_create_limits():
    a = _valid()
    L = _lib.load()
    h = ctypes.c_void_p()
    i32 = lambda x: np.ascontiguousarray(x, np.int32).ctypes.data_as(_lib.c_i32)
    f64 = lambda x: np.ascontiguousarray(x, np.float64).ctypes.data_as(_lib.c_d)
    assert L.frax_model_create(0, i32(a["parent"]), i32(a["joint_type"]), f64(a["axis"]), f64(a["placement"]),
                               f64(a["inertia"]), f64(a["gravity"]), ctypes.byref(h)) == 1
    assert L.frax_model_create(65, i32(a["parent"]), i32(a["joint_type"]), f64(a["axis"]), f64(a["placement"]),
                               f64(a["inertia"]), f64(a["gravity"]), ctypes.byref(h)) == 1
    assert b"n_bodies" in L.frax_last_error()


def test_batch_argument_checks_before_any_launch():
    """Errors found on the host return before anything touches the GPU, and
    B == 0 is a no-op; both work without a device."""
    L = _lib.load()
    m = fx.Model.from_robot(gen.chain7(0))
    null = ctypes.c_void_p(0)
    assert L.frax_rnea(m.handle, 0, 0, null, null, null, null, null) == 0
    assert L.frax_rnea(m.handle, -1, 0, null, null, null, null, null) == 1
    assert L.frax_rnea(m.handle, 16, 8, null, null, null, null, null) == 1
    assert b"ld" in L.frax_last_error()
    assert L.frax_rnea(m.handle, 16, 1 << 30, null, null, null, null, null) == 1
    assert b"below 2^30" in L.frax_last_error()
    assert L.frax_rnea(m.handle, 16, 16, null, null, null, null, null) == 1
    assert b"q is NULL" in L.frax_last_error()
    assert L.frax_crba(m.handle, 16, 16, ctypes.c_void_p(16), null, null, null) == 1
    frames = np.array([7], np.int32)
    assert L.frax_jacobian(m.handle, 16, 16, ctypes.c_void_p(16), 1, frames.ctypes.data_as(_lib.c_i32), null,
                           ctypes.c_void_p(16), null) == 1
    assert L.frax_jacobian(m.handle, 16, 16, ctypes.c_void_p(16), 9, frames.ctypes.data_as(_lib.c_i32), null,
                           ctypes.c_void_p(16), null) == 1


def test_osc_argument_checks_before_any_launch():
    """frax_osc rejects a task body out of range, and one moved by fewer than
    six dofs (its 6-D task inertia is singular), before any launch."""
    L = _lib.load()
    null = ctypes.c_void_p(0)
    p = ctypes.c_void_p(16)
    ch = fx.Model.from_robot(gen.chain7(0))
    assert L.frax_osc(ch.handle, 7, 16, 16, p, p, p, p, null, null) == 1
    assert b"task_body" in L.frax_last_error()
    assert L.frax_osc(ch.handle, 4, 16, 16, p, p, p, p, null, null) == 1  # 5 dofs above body 4
    assert b"fewer than 6 dofs" in L.frax_last_error()
    assert L.frax_osc(ch.handle, 6, 0, 0, null, null, null, null, null, null) == 0
    assert L.frax_osc(ch.handle, 6, 16, 16, p, p, null, p, null, null) == 1
    assert b"xdd_des is NULL" in L.frax_last_error()
    hu = fx.Model.from_robot(gen.humanoid(0))
    assert L.frax_osc(hu.handle, 0, 0, 0, null, null, null, null, null, null) == 0  # free root: 6 dofs


def test_external_force_argument_checks():
    L = _lib.load()
    null = ctypes.c_void_p(0)
    p = ctypes.c_void_p(16)
    ch = fx.Model.from_robot(gen.chain7(0))
    assert L.frax_rnea_ext(ch.handle, 0, 0, null, null, null, null, null, null) == 0
    assert L.frax_rnea_ext(ch.handle, 16, 16, p, p, null, null, p, null) == 1
    assert b"fext is NULL" in L.frax_last_error()
    assert L.frax_aba_ext(ch.handle, 16, 16, p, p, p, p, null, null) == 1
    assert b"qdd is NULL" in L.frax_last_error()


def test_jvp_argument_checks():
    L = _lib.load()
    null = ctypes.c_void_p(0)
    p = ctypes.c_void_p(16)
    ch = fx.Model.from_robot(gen.chain7(0))
    frames = np.array([6], np.int32)
    assert L.frax_fk_jvp(ch.handle, 16, 16, p, null, 1, frames.ctypes.data_as(_lib.c_i32), p, null) == 1
    assert b"dq is NULL" in L.frax_last_error()
    assert L.frax_fk_jvp(ch.handle, 16, 16, p, p, 0, frames.ctypes.data_as(_lib.c_i32), p, null) == 1
    assert L.frax_rnea_jvp(ch.handle, 0, 0, null, null, null, null, null, null, null, null, null) == 0
    assert L.frax_rnea_jvp(ch.handle, 16, 16, p, p, null, p, p, null, null, null, null) == 1
    assert b"dtau is NULL" in L.frax_last_error()
    assert L.frax_aba_jvp(ch.handle, 16, 16, p, p, null, null, p, p, null, p, null) == 1
    assert b"qdd is NULL" in L.frax_last_error()


def test_fk_scan_requires_a_serial_chain():
    L = _lib.load()
    p = ctypes.c_void_p(16)
    tree = fx.Model.from_robot(gen.random_tree(101))
    assert L.frax_fk_scan(tree.handle, 4, 4, p, p, ctypes.c_void_p(0)) == 1
    assert b"serial chain" in L.frax_last_error()
    ch = fx.Model.from_robot(gen.serial_chain(1, 64, free_root=True))
    assert L.frax_fk_scan(ch.handle, 0, 0, ctypes.c_void_p(0), ctypes.c_void_p(0), ctypes.c_void_p(0)) == 0


def test_tree_path_setting_is_validated():
    import gen
    h = fx.Model.from_robot(gen.humanoid(0))
    L = fx.lib()
    assert L.frax_model_set_tree_path(h.handle, 2) == 0
    assert L.frax_model_set_tree_path(h.handle, 3) == 1 and "unknown path" in L.frax_last_error().decode()
    assert L.frax_model_set_tree_path(None, 0) == 1
    h.set_tree_path("auto")


def test_fp32_probe_argument_checks():
    """The probe rejects empty launches and a missing sink before any launch."""
    L = _lib.load()
    null = ctypes.c_void_p(0)
    flops = ctypes.c_double(-1.0)
    assert L.frax_fp32_probe(0, 0, 10, ctypes.c_void_p(16), ctypes.byref(flops), null) == 1
    assert b"blocks" in L.frax_last_error()
    assert L.frax_fp32_probe(1, 4, 0, ctypes.c_void_p(16), ctypes.byref(flops), null) == 1
    assert L.frax_fp32_probe(0, 4, 10, null, ctypes.byref(flops), null) == 1
    assert flops.value == -1.0
