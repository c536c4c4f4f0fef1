"""lbm_observables_noalloc: the allocation-free observables entry point.

It exists for callers that cannot allocate device memory: a host that hands
the library a fixed memory arena and forbids further allocation, or a
latency-critical loop where cudaMalloc would synchronise the device. Here it
is called through the C ABI on a state held by a lattice context, with
caller-owned device buffers for the probe tables and the output record, and
its result is compared with lbm_observables on two calls in a row. In-place
CS lattices alternate between two storage phases, so they are checked after
an odd and after an even number of steps, in both precisions. This file sorts
last so a run that stops at the first failure has already run every other
test; it also passes on its own.
"""
import ctypes
import math

import pytest

import lbm_workloads as wl
import paper_1904_02471_gb300 as pkg
from paper_1904_02471_gb300 import lbm

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _run_noalloc(L, comp, dpx, dpy, norm, out, stream_ptr):
    v = L.device_view()
    s = L.spec
    rc = lbm.lib().lbm_observables_noalloc(
        s.model, s.q_per_axis, s.precision, s.nx, s.ny, v.base, v.plane, v.pitch, v.cs_pull_phase, s.rho0, comp,
        dpx, dpy, norm, L.steps_done, s.dt, out, stream_ptr)
    assert rc == lbm.LBM_OK, lbm.last_error()


def _check(got, ref):
    assert got["step"] == ref["step"] and got["nonfinite"] == 0
    assert abs(got["time"] - ref["time"]) <= 1e-15 * max(1.0, abs(ref["time"]))
    m = ref["mass"]
    assert abs(got["mass"] - m) <= TOL * m
    assert abs(got["mom_x"] - ref["mom_x"]) <= TOL * m
    assert abs(got["mom_y"] - ref["mom_y"]) <= TOL * m
    assert abs(got["amp"] - ref["amp"]) <= TOL * abs(ref["amp"]) + 1e-18


@pytest.mark.parametrize("model,q,prec,nx,ny,storage,steps", [
    ("cs", 3, "fp32", 150, 90, "ab", (5, 12)),
    ("cs", 3, "fp64", 77, 31, "ab", (5, 12)),
    ("cs", 3, "fp32", 150, 90, "inplace", (5, 12)),   # phase 2 (odd), then 0 (even)
    ("cs", 3, "fp64", 77, 31, "inplace", (4, 7)),     # phase 0 (even), then 2 (odd)
    ("fd", 4, "fp64", 48, 40, "ab", (5, 12)),
    ("fd", 5, "fp32", 36, 20, "ab", (5, 12)),
])
def test_noalloc_matches_lbm_observables(model, q, prec, nx, ny, storage, steps):
    import torch
    assert torch.cuda.is_available()
    from paper_1904_02471_gb300 import build
    build.build()
    torch.cuda.init()
    # a shear wave along x gives a non-zero total momentum, so a flipped sign shows
    U = 0.02 * math.sqrt(3) if model == "cs" else 0.02
    kw = {} if model == "cs" else {"dt": 0.3 / (3.0 * nx)}
    if storage == "inplace":
        kw["storage"] = "inplace"
    tau = 0.5 if model == "cs" else 2.0 / (3.0 * nx)
    comp, px, py, norm = wl.probe_taylor_green(nx, ny)
    dpx = torch.tensor(px, dtype=torch.float64, device="cuda")
    dpy = torch.tensor(py, dtype=torch.float64, device="cuda")
    out = torch.zeros(ctypes.sizeof(lbm.lbm_obs), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rho, ux, uy = wl.taylor_green(nx, ny, U)
    ux = ux + 0.3 * U   # uniform drift: total momentum far from zero
    uy = uy - 0.2 * U
    with pkg.Lattice(model, q, nx, ny, tau, precision=prec, **kw) as L:
        L.init(rho, ux, uy)
        L.set_probe(comp, px, py, norm)
        phases = []
        done = 0
        for n in steps:  # two calls in a row on different states
            L.step(n - done)
            done = n
            L.sync()
            ref = L.observables()
            phases.append(L.device_view().cs_pull_phase)
            _run_noalloc(L, comp, dpx.data_ptr(), dpy.data_ptr(), norm, out.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            got = lbm.lbm_obs.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()
            assert abs(ref["mom_x"]) > 1e-3 * ref["mass"] * U
            _check(got, ref)
        if storage == "inplace":
            assert sorted(phases) == [0, 2]
        elif model == "cs":
            assert phases == [1, 1]
        else:
            assert phases == [0, 0]
        # without a probe the amplitude is reported as 0
        _run_noalloc(L, -1, None, None, 0.0, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = lbm.lbm_obs.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()
        assert got["amp"] == 0.0 and abs(got["mass"] - L.observables()["mass"]) <= TOL * got["mass"]


def test_noalloc_rejects_sizes_beyond_the_maximum():
    # rejected on the host before any launch: nothing is read through the pointer
    rc = lbm.lib().lbm_observables_noalloc(lbm.LBM_CS, 3, lbm.LBM_FP32_DEV, 65536, 32768, 0x1000, 1 << 40, 65536,
                                           1, 1.0, -1, None, None, 0.0, 0, 1.0, 0x2000, None)
    assert rc == lbm.LBM_EINVAL
    assert "maximum" in lbm.last_error()


@pytest.mark.parametrize("model,phase", [(0, -1), (0, 3), (1, 1), (1, 2)])
def test_noalloc_rejects_bad_phase(model, phase):
    # rejected on the host before any launch
    rc = lbm.lib().lbm_observables_noalloc(model, 3, lbm.LBM_FP64, 8, 8, 0x1000, 64, 8, phase, 1.0, -1, None,
                                           None, 0.0, 0, 1.0, 0x2000, None)
    assert rc == lbm.LBM_EINVAL
    assert "cs_phase" in lbm.last_error()
