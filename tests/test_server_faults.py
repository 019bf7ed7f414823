"""Host-side fault injection on the server's error paths (frax_debug_inject_fault).

Each injection makes one host allocation or CUDA call of the server behave as
failed; the public call must return the documented status (FRAX_ENOMEM or
FRAX_ECUDA), release what it had taken (no slab bytes, ring slots or device
memory left behind) and leave the server usable. Nothing is injected on the
GPU. Injection is armed only in a process started with FRAX_FAULT_INJECTION=1,
so each case runs in a child process of its own."""

import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(code, inject=True, timeout=300):
    env = dict(os.environ)
    env.pop("FRAX_FAULT_INJECTION", None)
    if inject:
        env["FRAX_FAULT_INJECTION"] = "1"
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_injection_is_refused_without_the_environment_switch():
    out = _child("""
        import paper_2604_04310_gb300 as fx
        st = fx.lib().frax_debug_inject_fault(1, 0)
        print(st, fx.lib().frax_last_error().decode())
    """, inject=False)
    assert out.startswith("1 ") and "FRAX_FAULT_INJECTION" in out


def test_server_create_host_allocation_failure():
    """The server's host struct is allocated before any CUDA call, so this
    case needs no GPU."""
    out = _child("""
        import ctypes
        import paper_2604_04310_gb300 as fx
        L = fx.lib()
        assert L.frax_debug_inject_fault(1, 0) == 0
        h = ctypes.c_void_p()
        st = L.frax_server_create(1 << 20, 10.0, ctypes.byref(h))
        print(st, h.value, L.frax_last_error().decode())
    """)
    st, handle = out.split()[:2]
    assert st == "3" and handle == "None"  # FRAX_ENOMEM, nothing returned


@pytest.mark.gpu
def test_server_error_paths_release_everything():
    _child("""
        import ctypes, time
        import numpy as np
        import torch
        import gen
        import paper_2604_04310_gb300 as fx
        from paper_2604_04310_gb300.serving import Server
        from oracle import rbd
        from tests.pins import normwise
        L = fx.lib()
        torch.cuda.init()
        robot = gen.chain7(0)
        model = fx.Model.from_robot(robot)
        B = 300
        s = gen.draw_states(robot, B, 41).as_f32()
        inp = [gen.to_soa(x) for x in (s.q, s.qd, s.qdd)]
        ref = rbd.rnea(robot, s.q, s.qd, s.qdd)

        # the pinned host mirror fails after the device slab was taken: the
        # slab must be given back
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert L.frax_debug_inject_fault(2, 0) == 0
        try:
            Server(budget_bytes=1 << 30)
            raise AssertionError("create succeeded")
        except fx.FraxError as e:
            assert e.status == 3, e
        free1 = torch.cuda.mem_get_info()[0]
        assert free0 - free1 < (64 << 20), (free0, free1)

        srv = Server(budget_bytes=256 << 20, idle_exit_ms=20.0)
        mid = srv.add_model(model)

        def run_one():
            req = srv.submit(mid, "rnea", inp, B)
            t_end = time.time() + 20
            while not srv.poll(req):
                assert time.time() < t_end
                time.sleep(1e-4)
            return req

        for point in (3, 4):  # the input copy, then the descriptor copy
            assert L.frax_debug_inject_fault(point, 0) == 0
            try:
                srv.submit(mid, "rnea", inp, B)
                raise AssertionError("submit succeeded")
            except fx.FraxError as e:
                assert e.status == 2, e  # FRAX_ECUDA
            info = srv.info()
            assert info["bytes_in_use"] == 0 and info["in_flight"] == 0, info
            outs, _ = srv.collect(run_one(), mid, "rnea", B)
            assert normwise(gen.from_soa(outs[0], B), ref) < 1e-4

        # the output copy fails: the request is still released
        req = run_one()
        assert L.frax_debug_inject_fault(5, 0) == 0
        try:
            srv.collect(req, mid, "rnea", B)
            raise AssertionError("collect succeeded")
        except fx.FraxError as e:
            assert e.status == 2, e
        info = srv.info()
        assert info["bytes_in_use"] == 0 and info["in_flight"] == 0, info
        outs, _ = srv.collect(run_one(), mid, "rnea", B)
        assert normwise(gen.from_soa(outs[0], B), ref) < 1e-4
        assert srv.info()["device_status"] == 0
        srv.close()
        print("ok")
    """)
