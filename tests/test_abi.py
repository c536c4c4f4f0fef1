"""The C-ABI library on the CPU: it loads, exports every symbol include/lbm.h
declares, and its host-only logic (unit helpers, velocity sets, parameter
validation, decay fit) is right. No GPU compute is called here."""
import math
import os
import re

import numpy as np
import pytest

import oracle_pins as P
from paper_1904_02471_gb300 import lbm
import paper_1904_02471_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_02471_gb300 import build
    build.build()


def test_every_declared_symbol_is_exported():
    L = lbm.lib()
    declared = _declared()
    assert len(declared) > 30
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers every declared entry point
    assert declared <= set(lbm.exported_names()) | set(), sorted(declared - set(lbm.exported_names()))


def test_version_and_errors():
    assert "sm_103a" in lbm.lib().lbm_version().decode()
    for code in range(12):
        assert lbm.strerror(code) != "unknown error"


def test_velocity_sets_match_numpy_gauss_hermite():
    from numpy.polynomial.hermite_e import hermegauss
    for q in (3, 4, 5):
        vx, vy, w = pkg.lbm_velocity_set(q)
        x, wr = hermegauss(q)
        wr = wr / wr.sum()
        for k in range(q * q):
            assert abs(vx[k] - x[k % q]) < 1e-14 and abs(vy[k] - x[k // q]) < 1e-14
            assert abs(w[k] - wr[k % q] * wr[k // q]) < 1e-15


def test_unit_helpers_against_printed_values():
    g = P._golden("paper_values.json")
    t = g["tau_lu_tables"]
    for n, printed in t["rows"]:
        assert P._trunc(pkg.lbm_tau_lu_from_fd(n, t["tau_fd"]), t["digits"]) == printed
        assert abs(pkg.lbm_tau_fd_from_lu(n, pkg.lbm_tau_lu_from_fd(n, t["tau_fd"])) - t["tau_fd"]) < 1e-15
        # Eq. (nulu) with the CS dt: nu_LU = N nu_FD
        tl = pkg.lbm_tau_lu_from_fd(n, t["tau_fd"])
        assert abs(pkg.lbm_nu(lbm.LBM_CS, tl, 1 / math.sqrt(3)) - n * t["tau_fd"]) < 1e-14
    s = g["tau_lu_shock"]
    for tau_fd, printed, digits in s["rows"]:
        assert P._trunc(pkg.lbm_tau_lu_from_fd(s["n"], tau_fd), digits) == printed
    assert pkg.lbm_nu(lbm.LBM_FD, 5e-4, 1.0) == 5e-4
    assert abs(pkg.lbm_tau_star(0.8 / math.sqrt(3)) - 0.8) < 1e-15
    # CFL / stiffness bound (Sec. 4.1)
    assert abs(pkg.lbm_fd_max_dt(3, 1 / 2048, 1e-3) - 1 / (2048 * math.sqrt(3))) < 1e-18
    assert pkg.lbm_fd_max_dt(4, 1 / 256, 1e-5) == 1e-5


def test_fit_decay():
    t = np.linspace(0, 10, 50)
    a = 0.3 * np.exp(-0.25 * t)
    g, a0 = pkg.lbm_fit_decay(t, a, 1.0)
    assert abs(g - 0.25) < 1e-12 and abs(a0 - 0.3) < 1e-12
    with pytest.raises(lbm.LbmError):
        pkg.lbm_fit_decay(t[:1], a[:1])


@pytest.mark.parametrize("args,code", [
    (("cs", 3, 8, 8, 0.2), lbm.LBM_EINVAL),                       # tau_LU <= dt/2
    (("cs", 4, 8, 8, 0.5), lbm.LBM_EINVAL),                       # CS is D2Q9 only
    (("cs", 3, 8, 8, 0.5, 0.5, 1.0), lbm.LBM_EINVAL),             # dx/dt != sqrt(3)
    (("fd", 4, 32, 32, 1e-2, 1.5e-2), lbm.LBM_ECFL),              # 2.33 * 0.015 * 32 > 1
    (("fd", 4, 32, 32, 1e-4, 1e-3), lbm.LBM_ESTIFF),              # dt > tau
    (("fd", 6, 8, 8, 1.0, 1e-3), lbm.LBM_EINVAL),                 # no such set
    (("fd", 4, 0, 8, 1.0, 1e-3), lbm.LBM_EINVAL),                 # empty lattice
    (("fd", 4, 8, 8, -1.0, 1e-3), lbm.LBM_EINVAL),                # negative tau
    (("fd", 4, 8, 8, 1.0, 0.0), lbm.LBM_EINVAL),                  # dt = 0
])
def test_create_validation(args, code):
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Lattice(*args)
    assert ei.value.code == code


@pytest.mark.parametrize("model,q,storage", [("fd", 4, "inplace"), ("cs", 3, 2), ("cs", 3, -1)])
def test_storage_validation(model, q, storage):
    """In-place storage is a CS option; FD keeps its three stage buffers."""
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Lattice(model, q, 32, 32, 0.5 if model == "cs" else 1e-2, 0.0 if model == "cs" else 1e-3,
                    storage=storage)
    assert ei.value.code == lbm.LBM_EINVAL


def test_batch_validation_names_the_lattice():
    specs = [pkg.make_spec("cs", 3, 8, 8, 0.5), pkg.make_spec("fd", 4, 32, 32, 1e-4, 1e-3)]
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Batch(specs)
    assert ei.value.code == lbm.LBM_ESTIFF and "lattice 1" in str(ei.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        lbm.lib()


def test_kernel_digest_follows_code_not_comments():
    """The digest that ties a recorded DRAM-traffic figure to a kernel's
    sources ignores comments and layout, and changes with the code."""
    from paper_1904_02471_gb300 import build
    base = {"kernels_fd.cu": "int f(int a) { return a + 1; } // one\n", "fd_common.cuh": "int g();\n",
            "common.cuh": "/* c */ #define X 1\n",
            "ptx.cuh": 'const char* s = "a // not a comment";\n', "kernels.h": ""}
    d0 = build.kernel_digest("fd_stage", base.__getitem__)
    relaid = dict(base, **{"kernels_fd.cu": "// header\nint f(int a)\n{\n    return a + 1;  /* two */\n}\n"})
    assert build.kernel_digest("fd_stage", relaid.__getitem__) == d0
    changed = dict(base, **{"kernels_fd.cu": "int f(int a) { return a + 2; }\n"})
    assert build.kernel_digest("fd_stage", changed.__getitem__) != d0
    in_string = dict(base, **{"ptx.cuh": 'const char* s = "a // now different";\n'})
    assert build.kernel_digest("fd_stage", in_string.__getitem__) != d0


def test_recorded_dram_traffic_matches_the_kernel_sources():
    """Every DRAM-traffic entry under profiles/ was taken on the kernel code
    in the tree (its digest matches), and its bytes are within 10% of the
    algorithmic bytes, as the profile summaries state."""
    import json
    import os
    from paper_1904_02471_gb300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    assert set(rec["kernels"]) == set(build.KERNEL_SOURCES)
    for name, e in rec["kernels"].items():
        assert e["source_digest"] == build.kernel_digest(name), name
        assert 0.9 < e["bytes_per_launch"] / e["algorithmic_bytes_per_launch"] <= 1.1, name


def test_server_round_plan():
    """The server's round allotment (host logic, no GPU): equal device time per
    run by the step-cost estimate, at least one step, never more than left."""
    import math
    import paper_1904_02471_gb300 as pkg
    from paper_1904_02471_gb300 import lbm
    sq3 = math.sqrt(3.0)

    def fd(n):
        tau = pkg.lbm_tau_fd_from_lu(n, 0.9 / sq3)
        return pkg.make_spec("fd", 4, n, n, tau, min(tau, 0.4 * pkg.lbm_fd_max_dt(4, 1.0 / n, 1e300)), 0.0, "fp32")

    def cs(n, prec="fp32"):
        return pkg.make_spec("cs", 3, n, n, 0.6, 0.0, 0.0, prec)

    # FD 1024^2 step ~ 20 us + 1 M nodes x 0.227 ns, CS 64^2 ~ 20 us: ratio ~12.9 -> 32 / 12.9 = 2
    assert lbm.plan_round([fd(1024), cs(64)], [300, 1000], 32) == [2, 32]
    assert lbm.plan_round([fd(4096), cs(64)], [300, 1000], 32) == [1, 32]       # at least one
    assert lbm.plan_round([fd(1024), cs(64)], [1, 5], 32) == [1, 5]             # never more than left
    assert lbm.plan_round([cs(64), cs(64)], [0, 100], 32) == [0, 32]            # finished runs get none
    assert lbm.plan_round([fd(4096)], [10 ** 6], 64) == [64]                    # a run alone: the chunk
    assert lbm.plan_round([cs(256), cs(256)], [500, 500], 16) == [16, 16]       # equal costs, equal steps
    a, b = lbm.plan_round([cs(2048), cs(2048, "fp64")], [10 ** 6, 10 ** 6], 64)
    assert a == 64 and 1 <= b < a                                               # FP64 costs more
    fused = fd(512)
    fused.scheme = lbm.LBM_TS_RK3_FUSED
    a, b = lbm.plan_round([fd(512), fused], [10 ** 6, 10 ** 6], 64)
    assert a == 64 and 1 <= b < a                                               # the blocked step costs more
    assert lbm.plan_round([], [], 8) == []
    for args in (([cs(64)], [1], 0), ([cs(64)], [-1], 8)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.plan_round(*args)
        assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:                                      # a bad spec as in lbm_create
        lbm.plan_round([pkg.make_spec("cs", 4, 64, 64, 0.6, 0.0, 0.0, "fp32")], [10], 8)
    assert e.value.code == lbm.LBM_EINVAL


def test_spec_from_nu_against_printed_tau_lu():
    """lbm_spec_from_nu (Sec. 3): a CS lattice from the FD viscosity
    nu_FD = 5e-4 (or from nu_LU = 5e-4 N in its own units) gets the tau_LU
    column of Tables 1-2; an FD lattice from either gets tau_FD = 5e-4."""
    g = P._golden("paper_values.json")
    t = g["tau_lu_tables"]
    nu_fd = t["tau_fd"]
    for n, printed in t["rows"]:
        for nu, units in ((nu_fd, "fd"), (nu_fd * n, "cs")):
            s = pkg.spec_from_nu("cs", 3, n, 1, nu, units)
            assert P._trunc(s.tau, t["digits"]) == printed
            assert abs(s.tau - pkg.lbm_tau_lu_from_fd(n, nu_fd)) < 1e-15
            assert abs(s.dt - 1 / math.sqrt(3)) < 1e-16 and s.dx == 1.0
            f = pkg.spec_from_nu("fd", 4, n, n, nu, units, dt=nu_fd)
            assert abs(f.tau - nu_fd) < 1e-18 and abs(f.dx - 1.0 / n) < 1e-18
    # the shock-tube pair of Sec. 4.1 (N = 2048), with the reference length
    # given apart from the lattice width
    s = g["tau_lu_shock"]
    for tau_fd, printed, digits in s["rows"]:
        c = pkg.spec_from_nu("cs", 3, 2048, 4, tau_fd, "fd", n_ref=s["n"])
        assert P._trunc(c.tau, digits) == printed
    # a CS dt other than the default enters through Eq. (nulu)
    c = pkg.spec_from_nu("cs", 3, 16, 16, 0.1, "cs", dt=0.5, dx=0.5 * math.sqrt(3))
    assert abs(c.tau - 0.35) < 1e-15


@pytest.mark.parametrize("args,code", [
    (dict(model="cs", q=3, nx=8, ny=8, nu=0.0), lbm.LBM_EINVAL),           # nu must be positive
    (dict(model="cs", q=3, nx=8, ny=8, nu=float("nan")), lbm.LBM_EINVAL),
    (dict(model="cs", q=3, nx=8, ny=8, nu=0.1, nu_model=7), lbm.LBM_EINVAL),
    (dict(model="cs", q=3, nx=8, ny=8, nu=0.1, n_ref=-1), lbm.LBM_EINVAL),
    (dict(model="fd", q=4, nx=32, ny=32, nu=1e-4, dt=1e-3), lbm.LBM_ESTIFF),  # dt > tau_FD = nu
    (dict(model="fd", q=4, nx=32, ny=32, nu=1e-2, dt=1.5e-2), lbm.LBM_ECFL),
])
def test_spec_from_nu_validation(args, code):
    a = dict(args)
    with pytest.raises(lbm.LbmError) as ei:
        pkg.spec_from_nu(a.pop("model"), a.pop("q"), a.pop("nx"), a.pop("ny"), a.pop("nu"), **a)
    assert ei.value.code == code
    # lbm_create_nu refuses the same before any device work
    a = dict(args)
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Lattice(a.pop("model"), a.pop("q"), a.pop("nx"), a.pop("ny"), None, **a)
    assert ei.value.code == code


@pytest.mark.parametrize("kw,code", [
    (dict(model="fd", q=4, tau=1e-4, dt=1e-3, scheme="rk3"), lbm.LBM_ESTIFF),   # RK3 needs dt <= tau
    (dict(model="cs", q=3, tau=0.5, dt=0.0, scheme="imex"), lbm.LBM_EINVAL),    # the scheme is an FD choice
    (dict(model="fd", q=4, tau=1e-4, dt=1e-3, scheme=7), lbm.LBM_EINVAL),
    (dict(model="fd", q=4, tau=1e-4, dt=2e-2, scheme="imex"), lbm.LBM_ECFL),    # IMEX keeps the CFL bound
    (dict(model="fd", q=4, tau=1e-4, dt=1e-3, scheme="rk3_fused"), lbm.LBM_ESTIFF),  # the fused RK3 step too
    (dict(model="cs", q=3, tau=0.5, dt=0.0, scheme="rk3_fused"), lbm.LBM_EINVAL),
    (dict(model="fd", q=4, tau=1e-2, dt=2e-2, scheme="rk3_fused"), lbm.LBM_ECFL),
])
def test_scheme_validation(kw, code):
    """IMEX lifts dt <= tau (Sec. 4.1) and nothing else; the RK3 default
    keeps it (checked on the host before any device work)."""
    s = pkg.make_spec(kw["model"], kw["q"], 32, 32, kw["tau"], kw["dt"], 0.0, "fp64", scheme=kw["scheme"])
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Batch([s])
    assert ei.value.code == code
    s = pkg.make_spec("fd", 4, 32, 32, 1e-4, 1e-3, 0.0, "fp64", scheme="imex")
    s.reserved = 1
    with pytest.raises(lbm.LbmError) as ei:
        pkg.Batch([s])
    assert ei.value.code == lbm.LBM_EINVAL
    # an IMEX lattice with dt = 10 tau passes validation (spec_from_nu only resolves)
    ok = pkg.spec_from_nu("fd", 4, 32, 32, 1e-4, "fd", dt=1e-3, precision="fp32", scheme="imex")
    assert ok.scheme == lbm.LBM_TS_IMEX and ok.tau == 1e-4
    with pytest.raises(lbm.LbmError) as ei:
        pkg.spec_from_nu("fd", 4, 32, 32, 1e-4, "fd", dt=1e-3, precision="fp32")
    assert ei.value.code == lbm.LBM_ESTIFF


def test_footprint_follows_the_state_buffers():
    """Device bytes per lattice (host only): in-place CS holds one copy of the
    9 planes against two, the temporally blocked FD step two copies of the
    Q^2 planes against three, FP64 twice the FP32 bytes; rows are padded to
    a pitch of 32 (plus 8 nodes of slack) and each lattice has 32 KiB of
    observables scratch."""
    from paper_1904_02471_gb300 import lbm
    scratch = 8 * 4 * 1024

    def fp(*a, **kw):
        return lbm.footprint(pkg.make_spec(*a, **kw)) - scratch

    n = 1000
    plane = ((n + 8 + 31) // 32 * 32) * n           # pitch 1024
    tail = 1024                                      # spare elements per buffer
    assert fp("cs", 3, n, n, 0.6, 0.0, 0.0, "fp32") == 2 * (9 * plane + tail) * 4
    assert fp("cs", 3, n, n, 0.6, 0.0, 0.0, "fp32", storage="inplace") == (9 * plane + tail) * 4
    assert fp("cs", 3, n, n, 0.6, 0.0, 0.0, "fp64") == 2 * (9 * plane + tail) * 8
    tau = dt = 1e-4
    assert fp("fd", 4, n, n, tau, dt, 0.0, "fp32") == 3 * (16 * plane + tail) * 4
    assert fp("fd", 4, n, n, tau, dt, 0.0, "fp32", scheme="imex") == 3 * (16 * plane + tail) * 4
    assert fp("fd", 4, n, n, tau, dt, 0.0, "fp32", scheme="rk3_fused") == 2 * (16 * plane + tail) * 4
    assert fp("fd", 5, n, n, tau, dt, 0.0, "fp64", scheme="rk3_fused") == 2 * (25 * plane + tail) * 8
    with pytest.raises(lbm.LbmError) as e:
        lbm.footprint(pkg.make_spec("fd", 4, n, n, 1e-4, 2e-4, 0.0, "fp32"))   # dt > tau
    assert e.value.code == lbm.LBM_ESTIFF
