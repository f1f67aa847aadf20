"""ctypes binding of libdpsr (include/dpsr.h): the same entry points under the
same names, argument marshalling only. Every step of the computation runs in
the library's CUDA kernels; there is no CPU path.

The shared library is built in-tree by ``paper_2106_03452_gb300.build`` (or
``__graft_entry__.build()``); loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# DPSR_DEBUG_CHECKS=1 in the environment loads the bounds-checking build
# (build.build(debug=True)) instead of the release one
_DEBUG = os.environ.get("DPSR_DEBUG_CHECKS", "") == "1"
LIB_PATH = os.path.join(_HERE, "_build_debug" if _DEBUG else "_build", "libdpsr.so")
_lock = threading.Lock()
_lib = None

DPSR_OK = 0
DPSR_EINVAL = -1
DPSR_ENOMEM = -2
DPSR_ECUDA = -3
DPSR_EDEGENERATE = -4
DPSR_ESTATE = -5
DPSR_ETIMEOUT = -6
DPSR_EBUSY = -7
DPSR_ECANCELED = -8
DPSR_EBOUNDS = -9

_c_int, _c_i64, _c_sz, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
_PROTOS = {
    "dpsr_plan_create": (_c_int, [_c_int, ctypes.c_float, ctypes.POINTER(_vp)]),
    "dpsr_server_cancel": (_c_int, [_vp, _c_i64]),
    "dpsr_server_wait_any": (_c_int, [_vp, ctypes.POINTER(_c_i64), ctypes.POINTER(_c_int), _c_int,
                                      ctypes.c_double, ctypes.POINTER(_c_int)]),
    "dpsr_debug_checks": (_c_int, []),
    "dpsr_debug_read_spectrum": (_c_int, [_vp, _c_int, _vp]),
    "dpsr_debug_check_selftest": (_c_int, []),
    "dpsr_fp32_fma_peak": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_double)]),
    "dpsr_plan_create_box": (_c_int, [_c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_vp)]),
    "dpsr_plan_destroy": (_c_int, [_vp]),
    "dpsr_plan_set_stream": (_c_int, [_vp, _vp]),
    "dpsr_plan_reserve": (_c_int, [_vp, _c_i64]),
    "dpsr_plan_workspace_bytes": (_c_sz, [_c_int, _c_i64, _c_int]),
    "dpsr_forward": (_c_int, [_vp, _vp, _vp, _c_i64, _vp]),
    "dpsr_backward": (_c_int, [_vp, _vp, _vp, _vp]),
    "dpsr_forward_host": (_c_int, [_vp, _vp, _vp, _c_i64, _vp]),
    "dpsr_backward_host": (_c_int, [_vp, _vp, _vp, _vp]),
    "dpsr_solve_host": (_c_int, [_vp, _vp, _vp, _c_i64, _vp, _vp, _vp, _vp]),
    "dpsr_sync": (_c_int, [_vp]),
    "dpsr_get_scalars": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "dpsr_plan_last_launches": (_c_int, [_vp]),
    "dpsr_strerror": (ctypes.c_char_p, [_c_int]),
    "dpsr_check_bounded_wait": (_c_int, [ctypes.c_double]),
    "dpsr_plan_check_bounded_wait": (_c_int, [_vp, ctypes.c_double]),
    "dpsr_forward_static": (_c_int, [_c_int, ctypes.c_float, _vp, _vp, _c_i64, _vp, _vp]),
    "dpsr_grid_sample": (_c_int, [_vp, _c_int, _vp, _c_i64, _vp, _vp]),
    "dpsr_grid_splat": (_c_int, [_vp, _c_int, _vp, _vp, _c_i64, _c_int, _vp]),
    "dpsr_plan_profile": (_c_int, [_vp, _c_int]),
    "dpsr_plan_clusters": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "dpsr_batch_paths": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_int)]),
    "dpsr_mse_grad": (_c_int, [_vp, _vp, _vp]),
    "dpsr_get_loss": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "dpsr_batch_bind_target": (_c_int, [_vp, _c_int, _vp]),
    "dpsr_batch_train_step": (_c_int, [_vp]),
    "dpsr_batch_losses": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "dpsr_server_set_max_group": (_c_int, [_vp, _c_int]),
    "dpsr_server_group_stats": (_c_int, [_vp, ctypes.POINTER(_c_i64)]),
    "dpsr_mesh_extract": (_c_int, [_vp, _c_int, ctypes.c_float, _vp, _vp, _c_i64, _vp, _vp]),
    "dpsr_mesh_surrogate_splat": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _c_i64, _c_int, _vp]),
    "dpsr_chamfer": (_c_int, [_vp, _c_i64, _vp, _c_i64, _vp, _vp, _vp, _vp, _vp]),
    "dpsr_largest_region": (_c_int, [_vp, _c_int, ctypes.c_float, _vp, _vp, _vp, _vp, _vp]),
    "dpsr_mesh_extract_region": (_c_int, [_vp, _c_int, ctypes.c_float, _vp, _c_int, _vp, _vp, _c_i64, _vp, _vp]),
    "dpsr_mesh_sample": (_c_int, [_vp, _vp, _c_i64, _c_i64, ctypes.c_uint64, _vp, _vp, _vp, _vp]),
    "dpsr_batch_create": (_c_int, [_c_int, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(_c_i64), ctypes.POINTER(_vp)]),
    "dpsr_batch_create_box": (_c_int, [_c_int, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(_vp)]),
    "dpsr_batch_destroy": (_c_int, [_vp]),
    "dpsr_batch_set_stream": (_c_int, [_vp, _vp]),
    "dpsr_batch_bind": (_c_int, [_vp, _c_int, _vp, _vp, _c_i64, _vp, _vp, _vp, _vp]),
    "dpsr_batch_forward": (_c_int, [_vp]),
    "dpsr_batch_backward": (_c_int, [_vp]),
    "dpsr_batch_graph_launch": (_c_int, [_vp, _c_int]),
    "dpsr_batch_sync": (_c_int, [_vp]),
    "dpsr_batch_launches": (_c_int, [_vp, _c_int]),
    "dpsr_server_create": (_c_int, [_c_sz, _c_int, ctypes.c_float, ctypes.POINTER(_vp)]),
    "dpsr_server_destroy": (_c_int, [_vp]),
    "dpsr_server_submit": (_c_int, [_vp, _c_int, _vp, _vp, _c_i64, _vp, _vp, _vp, _vp,
                                    ctypes.POINTER(_c_i64)]),
    "dpsr_server_poll": (_c_int, [_vp, _c_i64, ctypes.POINTER(_c_int)]),
    "dpsr_server_wait": (_c_int, [_vp, _c_i64, ctypes.c_double]),
    "dpsr_server_stats": (_c_int, [_vp, ctypes.POINTER(_c_i64)]),
    "dpsr_plan_profile_read": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_int)]),
}

KERNEL_KINDS = ["bin", "plane_fwd", "xpass_fwd", "final_fwd", "plane_inv", "plane_bfwd", "final_bwd",
                "xpass_bwd", "plane_binv", "combine"]


class DPSRError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = load().dpsr_strerror(code).decode() if code is not None else "?"
        super().__init__(f"{what}: {msg} (status {code})")
        self.code = code


def load():
    """Load the in-tree libdpsr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libdpsr is not built ({LIB_PATH} missing): run "
                    f"`python -m paper_2106_03452_gb300.build{' --debug' if _DEBUG else ''}` (needs nvcc); "
                    "there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _PROTOS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(code: int, what: str) -> None:
    if code != DPSR_OK:
        raise DPSRError(code, what)


# Same-named thin wrappers.
def dpsr_plan_create(r: int, sigma: float) -> int:
    h = _vp()
    check(load().dpsr_plan_create(int(r), float(sigma), ctypes.byref(h)), "dpsr_plan_create")
    return h.value


def dpsr_plan_create_box(r: int, sigma: float, box) -> int:
    h = _vp()
    b = None if box is None else (ctypes.c_double * 3)(*[float(v) for v in box])
    check(load().dpsr_plan_create_box(int(r), float(sigma), b, ctypes.byref(h)), "dpsr_plan_create_box")
    return h.value


def dpsr_server_wait_any(server: int, max_n: int = 64, timeout_s: float = 0.0):
    """[(ticket, status), ...] of up to max_n completed requests, retired in
    completion order; [] when timeout_s passes first."""
    t = (_c_i64 * max_n)()
    st = (_c_int * max_n)()
    n = _c_int()
    rc = load().dpsr_server_wait_any(server, t, st, int(max_n), float(timeout_s), ctypes.byref(n))
    if rc == DPSR_ETIMEOUT:
        return []
    check(rc, "dpsr_server_wait_any")
    return [(int(t[i]), int(st[i])) for i in range(n.value)]


def dpsr_server_cancel(server: int, ticket: int) -> int:
    """DPSR_OK (cancelled before admission) or DPSR_EBUSY (admitted or done:
    it completes normally); raises for an unknown ticket."""
    rc = load().dpsr_server_cancel(server, int(ticket))
    if rc not in (DPSR_OK, DPSR_EBUSY):
        raise DPSRError(rc, "dpsr_server_cancel")
    return rc


def dpsr_debug_read_spectrum(plan: int, which: int, r: int):
    """One of the forward's intermediate spectra as a complex64 numpy array
    [x][ky][kz], kz = 0 .. r/2 (see include/dpsr.h)."""
    import numpy as np
    out = np.empty((r, r, r // 2 + 1), np.complex64)
    check(load().dpsr_debug_read_spectrum(plan, int(which), out.ctypes.data), "dpsr_debug_read_spectrum")
    return out


def dpsr_debug_checks() -> bool:
    return bool(load().dpsr_debug_checks())


def dpsr_debug_check_selftest() -> int:
    return int(load().dpsr_debug_check_selftest())


def dpsr_fp32_fma_peak(iters: int = 1 << 16) -> float:
    """FP32 FMA throughput of the current device, FLOP/s."""
    v = ctypes.c_double()
    check(load().dpsr_fp32_fma_peak(int(iters), ctypes.byref(v)), "dpsr_fp32_fma_peak")
    return v.value


def dpsr_plan_destroy(plan: int) -> None:
    check(load().dpsr_plan_destroy(plan), "dpsr_plan_destroy")


def dpsr_plan_set_stream(plan: int, stream: int) -> None:
    check(load().dpsr_plan_set_stream(plan, stream), "dpsr_plan_set_stream")


def dpsr_plan_reserve(plan: int, n_max: int) -> None:
    check(load().dpsr_plan_reserve(plan, int(n_max)), "dpsr_plan_reserve")


def dpsr_plan_workspace_bytes(r: int, n_max: int, with_bwd: bool = True) -> int:
    return int(load().dpsr_plan_workspace_bytes(int(r), int(n_max), 1 if with_bwd else 0))


def dpsr_forward(plan: int, points: int, normals: int, N: int, chi_out: int) -> None:
    check(load().dpsr_forward(plan, points, normals, int(N), chi_out), "dpsr_forward")


def dpsr_backward(plan: int, dchi: int, dpoints: int, dnormals: int) -> None:
    check(load().dpsr_backward(plan, dchi, dpoints, dnormals), "dpsr_backward")


def dpsr_forward_host(plan: int, points: int, normals: int, N: int, chi_out: int) -> None:
    check(load().dpsr_forward_host(plan, points, normals, int(N), chi_out), "dpsr_forward_host")


def dpsr_backward_host(plan: int, dchi: int, dpoints: int, dnormals: int) -> None:
    check(load().dpsr_backward_host(plan, dchi, dpoints, dnormals), "dpsr_backward_host")


def dpsr_solve_host(plan: int, points: int, normals: int, N: int, dchi: int, chi_out: int, dpoints: int,
                    dnormals: int) -> None:
    check(load().dpsr_solve_host(plan, points, normals, int(N), dchi, chi_out, dpoints, dnormals), "dpsr_solve_host")


def dpsr_sync(plan: int) -> int:
    """Returns the device status (DPSR_OK or an error code) without raising."""
    return int(load().dpsr_sync(plan))


def dpsr_get_scalars(plan: int):
    out = (ctypes.c_double * 3)()
    check(load().dpsr_get_scalars(plan, out), "dpsr_get_scalars")
    return float(out[0]), float(out[1]), float(out[2])


def dpsr_plan_last_launches(plan: int) -> int:
    return int(load().dpsr_plan_last_launches(plan))


def dpsr_strerror(code: int) -> str:
    return load().dpsr_strerror(int(code)).decode()


def dpsr_check_bounded_wait(limit_s: float) -> int:
    return int(load().dpsr_check_bounded_wait(float(limit_s)))


def dpsr_plan_check_bounded_wait(plan: int, limit_s: float) -> int:
    """Queues the never-completed bounded wait on the plan's stream; the next
    dpsr_sync(plan) reports DPSR_ETIMEOUT. Returns the call's status."""
    return int(load().dpsr_plan_check_bounded_wait(plan, float(limit_s)))


def dpsr_plan_profile(plan: int, enable: bool) -> None:
    check(load().dpsr_plan_profile(plan, 1 if enable else 0), "dpsr_plan_profile")


def dpsr_plan_profile_read(plan: int):
    """{kind: (total_ms, launches)} since profiling was enabled or last read."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    check(load().dpsr_plan_profile_read(plan, ms, cnt), "dpsr_plan_profile_read")
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}


def dpsr_forward_static(r: int, sigma: float, points: int, normals: int, N: int, chi_out: int,
                        stream: int = 0) -> int:
    """Forward pass with no device allocation (static scratch; r <= 64,
    N <= 65536). Returns the status code instead of raising."""
    return int(load().dpsr_forward_static(int(r), float(sigma), points, normals, int(N), chi_out,
                                          stream))


def dpsr_plan_clusters(plan: int):
    """Cluster sizes of the four plane kernels (forward, forward inverse,
    backward, backward inverse)."""
    out = (ctypes.c_int * 4)()
    check(load().dpsr_plan_clusters(plan, out), "dpsr_plan_clusters")
    return [int(x) for x in out]


def dpsr_batch_create(r, sigma, n_max) -> int:
    n = len(r)
    h = _vp()
    ra = (ctypes.c_int * n)(*[int(x) for x in r])
    sa = (ctypes.c_float * n)(*[float(x) for x in sigma])
    na = (ctypes.c_int64 * n)(*[int(x) for x in n_max])
    check(load().dpsr_batch_create(n, ra, sa, na, ctypes.byref(h)), "dpsr_batch_create")
    return h.value


def dpsr_batch_create_box(r, sigma, box, n_max) -> int:
    """box: count x 3 side lengths (one periodic box per instance)."""
    n = len(r)
    h = _vp()
    ra = (ctypes.c_int * n)(*[int(x) for x in r])
    sa = (ctypes.c_float * n)(*[float(x) for x in sigma])
    ba = (ctypes.c_double * (3 * n))(*[float(v) for b in box for v in b])
    na = (ctypes.c_int64 * n)(*[int(x) for x in n_max])
    check(load().dpsr_batch_create_box(n, ra, sa, ba, na, ctypes.byref(h)), "dpsr_batch_create_box")
    return h.value


def dpsr_batch_destroy(batch: int) -> None:
    check(load().dpsr_batch_destroy(batch), "dpsr_batch_destroy")


def dpsr_batch_set_stream(batch: int, stream: int) -> None:
    check(load().dpsr_batch_set_stream(batch, stream), "dpsr_batch_set_stream")


def dpsr_batch_bind(batch: int, i: int, points: int, normals: int, N: int, chi: int, dchi: int = 0,
                    dpoints: int = 0, dnormals: int = 0) -> None:
    check(load().dpsr_batch_bind(batch, int(i), points, normals, int(N), chi, dchi or None,
                                 dpoints or None, dnormals or None), "dpsr_batch_bind")


def dpsr_batch_forward(batch: int) -> None:
    check(load().dpsr_batch_forward(batch), "dpsr_batch_forward")


def dpsr_batch_backward(batch: int) -> None:
    check(load().dpsr_batch_backward(batch), "dpsr_batch_backward")


def dpsr_batch_graph_launch(batch: int, with_bwd: bool = True) -> None:
    check(load().dpsr_batch_graph_launch(batch, 1 if with_bwd else 0), "dpsr_batch_graph_launch")


def dpsr_batch_sync(batch: int) -> int:
    return int(load().dpsr_batch_sync(batch))


def dpsr_batch_launches(batch: int, with_bwd: bool = True) -> int:
    return int(load().dpsr_batch_launches(batch, 1 if with_bwd else 0))


def dpsr_mse_grad(plan: int, target: int, dchi: int) -> None:
    check(load().dpsr_mse_grad(plan, target, dchi), "dpsr_mse_grad")


def dpsr_get_loss(plan: int) -> float:
    out = ctypes.c_double()
    check(load().dpsr_get_loss(plan, ctypes.byref(out)), "dpsr_get_loss")
    return float(out.value)


def dpsr_batch_bind_target(batch: int, i: int, target: int) -> None:
    check(load().dpsr_batch_bind_target(batch, int(i), target), "dpsr_batch_bind_target")


def dpsr_batch_train_step(batch: int) -> None:
    check(load().dpsr_batch_train_step(batch), "dpsr_batch_train_step")


def dpsr_batch_losses(batch: int, count: int):
    out = (ctypes.c_double * count)()
    check(load().dpsr_batch_losses(batch, out), "dpsr_batch_losses")
    return [float(v) for v in out]


def dpsr_server_set_max_group(server: int, max_group: int) -> None:
    check(load().dpsr_server_set_max_group(server, int(max_group)), "dpsr_server_set_max_group")


def dpsr_mesh_extract(chi: int, r: int, level: float, tris: int, normals: int, max_tris: int, count: int,
                      stream: int = 0) -> None:
    check(load().dpsr_mesh_extract(chi, int(r), float(level), tris, normals, int(max_tris), count, stream),
          "dpsr_mesh_extract")


def dpsr_mesh_surrogate_splat(dchi: int, r: int, points: int, normals: int, dldp: int, M: int,
                              accumulate: bool = False, stream: int = 0) -> None:
    check(load().dpsr_mesh_surrogate_splat(dchi, int(r), points, normals, dldp, int(M), 1 if accumulate else 0,
                                           stream), "dpsr_mesh_surrogate_splat")


def dpsr_chamfer(a: int, na: int, b: int, nb: int, ws_idx: int, ws_d2: int, grad_a: int, loss: int,
                 stream: int = 0) -> None:
    check(load().dpsr_chamfer(a, int(na), b, int(nb), ws_idx, ws_d2, grad_a, loss, stream), "dpsr_chamfer")


def dpsr_largest_region(chi: int, r: int, level: float, labels: int, ws: int, best: int, err: int,
                        stream: int = 0) -> None:
    check(load().dpsr_largest_region(chi, int(r), float(level), labels, ws, best, err, stream),
          "dpsr_largest_region")


def dpsr_mesh_extract_region(chi: int, r: int, level: float, labels: int, keep: int, tris: int, normals: int,
                             max_tris: int, count: int, stream: int = 0) -> None:
    check(load().dpsr_mesh_extract_region(chi, int(r), float(level), labels, int(keep), tris, normals,
                                          int(max_tris), count, stream), "dpsr_mesh_extract_region")


def dpsr_mesh_sample(tris: int, normals: int, T: int, M: int, seed: int, ws: int, points: int, pnormals: int,
                     stream: int = 0) -> None:
    check(load().dpsr_mesh_sample(tris, normals, int(T), int(M), int(seed) & (2 ** 64 - 1), ws, points,
                                  pnormals, stream), "dpsr_mesh_sample")


def dpsr_batch_paths(batch: int, r: int):
    """The four plane paths of the batch's instances of grid size r."""
    out = (_c_int * 4)()
    check(load().dpsr_batch_paths(batch, int(r), out), "dpsr_batch_paths")
    return [int(v) for v in out]


def dpsr_server_create(hbm_budget_bytes: int, slots: int = 8, sigma: float = 2.0) -> int:
    h = _vp()
    check(load().dpsr_server_create(int(hbm_budget_bytes), int(slots), float(sigma), ctypes.byref(h)),
          "dpsr_server_create")
    return h.value


def dpsr_server_destroy(server: int) -> None:
    check(load().dpsr_server_destroy(server), "dpsr_server_destroy")


def dpsr_server_submit(server: int, r: int, points: int, normals: int, N: int, dchi: int, chi_out: int,
                       dpoints: int = 0, dnormals: int = 0) -> int:
    t = _c_i64()
    check(load().dpsr_server_submit(server, int(r), points, normals, int(N), dchi or None, chi_out,
                                    dpoints or None, dnormals or None, ctypes.byref(t)),
          "dpsr_server_submit")
    return t.value


def dpsr_server_poll(server: int, ticket: int):
    """(done, status)."""
    d = _c_int()
    st = int(load().dpsr_server_poll(server, int(ticket), ctypes.byref(d)))
    return bool(d.value), st


def dpsr_server_wait(server: int, ticket: int, timeout_s: float = 0.0) -> int:
    return int(load().dpsr_server_wait(server, int(ticket), float(timeout_s)))


def dpsr_server_group_stats(server: int):
    out = (_c_i64 * 2)()
    check(load().dpsr_server_group_stats(server, out), "dpsr_server_group_stats")
    return dict(groups=out[0], grouped_requests=out[1])


def dpsr_server_stats(server: int):
    out = (_c_i64 * 4)()
    check(load().dpsr_server_stats(server, out), "dpsr_server_stats")
    return dict(admitted=out[0], completed=out[1], max_in_flight=out[2], bytes_in_use=out[3])


def dpsr_grid_sample(grid: int, r: int, q: int, M: int, out: int, stream: int = 0) -> None:
    check(load().dpsr_grid_sample(grid, int(r), q, int(M), out, stream), "dpsr_grid_sample")


def dpsr_grid_splat(grid: int, r: int, q: int, vals: int, M: int, accumulate: bool = False,
                    stream: int = 0) -> None:
    check(load().dpsr_grid_splat(grid, int(r), q, vals, int(M), 1 if accumulate else 0, stream),
          "dpsr_grid_splat")
