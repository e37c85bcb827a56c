"""The C-ABI library: it builds, loads, exports every entry point of include/qg.h,
and its host-side validation rejects bad inputs before touching a device."""
import dataclasses
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qg():
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


def _header_functions():
    src = open(os.path.join(ROOT, "include", "qg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_header_symbol(qg):
    import ctypes
    lib = ctypes.CDLL(qg.LIB)
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(qg.EXPORTED)
    assert qg.qg_version() >= 100


def test_default_options(qg):
    o = qg.qg_default_options()
    assert (o.c_p, o.c_q, o.c_s, o.c_rz, o.rho, o.eps, o.beta, o.adam_eps) == (1e4, 1e4, 1e3, 1e3, 1e3, 1e-3, 1.0, 1e-8)
    assert o.precision == qg.QG_FP64 and o.lodf_dtype == qg.QG_LODF_F32


def _expect(qg, case, code, **opt):
    with pytest.raises(qg.QGError) as ei:
        qg.qg_create(case, qg.case_options(case, **opt))
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device path")
def test_valid_case_reaches_device_check(qg):
    msg = _expect(qg, synth.tiny(), qg.QG_ERR_NO_DEVICE)
    assert "device" in msg


def test_invalid_inputs_are_rejected(qg):
    c = synth.tiny()
    bad_from = c.br_from.copy(); bad_from[3] = c.n_bus
    _expect(qg, dataclasses.replace(c, br_from=bad_from), qg.QG_ERR_INVALID_ARG)
    loop = c.br_to.copy(); loop[0] = c.br_from[0]
    _expect(qg, dataclasses.replace(c, br_to=loop), qg.QG_ERR_INVALID_ARG)
    bx = c.br_x.copy(); bx[1] = 0.0
    _expect(qg, dataclasses.replace(c, br_x=bx), qg.QG_ERR_INVALID_ARG)
    dup = c.ctg.copy(); dup[1] = dup[0]
    _expect(qg, dataclasses.replace(c, ctg=dup), qg.QG_ERR_INVALID_ARG)
    lp = c.load_p.copy(); lp[0, 0] = np.nan
    _expect(qg, dataclasses.replace(c, load_p=lp), qg.QG_ERR_INVALID_ARG)
    gz = c.gen_zone.copy(); gz[0] = 5
    _expect(qg, dataclasses.replace(c, gen_zone=gz), qg.QG_ERR_INVALID_ARG)
    _expect(qg, c, qg.QG_ERR_INVALID_ARG, eps=-1.0)
    _expect(qg, c, qg.QG_ERR_INVALID_ARG, precision=7)


def _radial(n=5):
    """A path graph: every branch is a bridge, so every outage islands the grid."""
    c = synth.tiny()
    M = n - 1
    frm = np.arange(M, dtype=np.int32)
    to = np.arange(1, n, dtype=np.int32)
    return dataclasses.replace(
        c, n_bus=n, n_branch=M, br_from=frm, br_to=to, br_r=np.full(M, 0.01), br_x=np.full(M, 0.1),
        br_b=np.zeros(M), s_max=np.ones(M), s_max_ctg=np.ones(M), n_gen=1, gen_bus=np.array([0], np.int32),
        gen_zone=np.array([0], np.int32), cost_a=np.ones(1), cost_b=np.ones(1), cost_r=np.ones(1), pmin=np.zeros(1),
        pmax=np.ones(1), qmin=-np.ones(1), qmax=np.ones(1), ramp=np.ones(1), vmin=np.full(n, 0.9),
        vmax=np.full(n, 1.1), load_p=np.full((c.T, n), 0.1), load_q=np.zeros((c.T, n)),
        bus_zone=np.zeros(n, np.int32), ctg=np.array([1, 2], np.int32))


def test_islanding_outage_is_rejected(qg):
    msg = _expect(qg, _radial(), qg.QG_ERR_ISLANDING)
    assert "islands" in msg


def test_disconnected_grid_is_rejected(qg):
    c = _radial()
    c = dataclasses.replace(c, br_from=np.array([0, 1, 3, 0], np.int32), br_to=np.array([1, 2, 4, 2], np.int32),
                            ctg=np.zeros(0, np.int32))
    _expect(qg, c, qg.QG_ERR_ISLANDING)


def test_sparse_dc_solver_options_are_validated(qg):
    c = synth.tiny()
    _expect(qg, c, qg.QG_ERR_INVALID_ARG, dc_solver=3)
    with pytest.raises(qg.QGError) as ei:
        qg.qg_create_batch([c, c], qg.case_options(c, dc_solver=qg.QG_DC_SPARSE))
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED and "one instance" in str(ei.value)


def test_sparse_dc_set_up_rejects_islanding_and_disconnected_grids(qg):
    msg = _expect(qg, _radial(), qg.QG_ERR_ISLANDING, dc_solver=qg.QG_DC_SPARSE)
    assert "islands" in msg
    c = _radial()
    c = dataclasses.replace(c, br_from=np.array([0, 1, 3, 0], np.int32), br_to=np.array([1, 2, 4, 2], np.int32),
                            ctg=np.zeros(0, np.int32))
    _expect(qg, c, qg.QG_ERR_ISLANDING, dc_solver=qg.QG_DC_SPARSE)


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device path")
@pytest.mark.parametrize("name", ["tiny", "rt617"])
def test_sparse_dc_set_up_runs_on_the_host(qg, name):
    """The whole FP64 set-up of the sparse solver (factor, dense tail inverse, gather lists,
    line-outage block) runs before the device is needed."""
    c = {"tiny": synth.tiny, "rt617": synth.rt617}[name]()
    _expect(qg, c, qg.QG_ERR_NO_DEVICE, dc_solver=qg.QG_DC_SPARSE)


def test_transformer_inputs_are_validated(qg):
    c = synth.with_transformers(synth.tiny(), 0.3, 4)
    dup = c.xf_branch.copy(); dup[1] = dup[0]
    _expect(qg, dataclasses.replace(c, xf_branch=dup), qg.QG_ERR_INVALID_ARG)
    far = c.xf_branch.copy(); far[0] = c.n_branch
    _expect(qg, dataclasses.replace(c, xf_branch=far), qg.QG_ERR_INVALID_ARG)
    tl = c.tau_min.copy(); tl[0] = 0.0
    _expect(qg, dataclasses.replace(c, tau_min=tl), qg.QG_ERR_INVALID_ARG)
    ph = c.phi_min.copy(); ph[0] = 1.0
    _expect(qg, dataclasses.replace(c, phi_min=ph), qg.QG_ERR_INVALID_ARG)


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device path")
def test_transformer_case_reaches_device_check(qg):
    c = synth.with_transformers(synth.mid(), 0.15, 5)
    for dc in (qg.QG_DC_DENSE, qg.QG_DC_SPARSE):
        _expect(qg, c, qg.QG_ERR_NO_DEVICE, dc_solver=dc)


def _devices_case():
    return synth.with_commitment(synth.with_block_bids(synth.tiny(), 3, 0.3, 1), seed=1)


def test_device_model_inputs_are_validated(qg):
    c = _devices_case()
    w = c.blk_width.copy(); w[2, 1] = -0.1
    _expect(qg, dataclasses.replace(c, blk_width=w), qg.QG_ERR_INVALID_ARG)
    pr = c.blk_price.copy(); pr[0, 0] = np.nan
    _expect(qg, dataclasses.replace(c, blk_price=pr), qg.QG_ERR_INVALID_ARG)
    big = np.ones((c.n_gen, 65))
    _expect(qg, dataclasses.replace(c, blk_price=big, blk_width=big), qg.QG_ERR_INVALID_ARG)
    su = c.c_su.copy(); su[0] = -1.0
    _expect(qg, dataclasses.replace(c, c_su=su), qg.QG_ERR_INVALID_ARG)
    ui = c.u_init.copy(); ui[0] = 1.5
    _expect(qg, dataclasses.replace(c, u_init=ui), qg.QG_ERR_INVALID_ARG)


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device path")
def test_device_model_case_reaches_device_check(qg):
    c = _devices_case()
    for dc in (qg.QG_DC_DENSE, qg.QG_DC_SPARSE):
        _expect(qg, c, qg.QG_ERR_NO_DEVICE, dc_solver=dc)


def _star(leaves):
    """A hub bus joined to `leaves` buses, the generator on the first leaf: the hub's balance and
    adjoint rows hold one entry per incident branch end."""
    c = synth.tiny()
    n = leaves + 1
    M = leaves
    return dataclasses.replace(
        c, name="star", n_bus=n, n_branch=M, br_from=np.zeros(M, np.int32), br_to=np.arange(1, n, dtype=np.int32),
        br_r=np.full(M, 0.01), br_x=np.full(M, 0.1), br_b=np.zeros(M), s_max=np.ones(M), s_max_ctg=np.ones(M),
        n_gen=1, gen_bus=np.array([1], np.int32), gen_zone=np.array([0], np.int32), cost_a=np.ones(1),
        cost_b=np.ones(1), cost_r=np.ones(1), pmin=np.zeros(1), pmax=np.full(1, 9.0), qmin=-np.ones(1),
        qmax=np.ones(1), ramp=np.ones(1), vmin=np.full(n, 0.9), vmax=np.full(n, 1.1),
        load_p=np.full((c.T, n), 0.01), load_q=np.zeros((c.T, n)), bus_zone=np.zeros(n, np.int32),
        ctg=np.zeros(0, np.int32))


def test_sizes_beyond_32_bit_indices_are_rejected(qg):
    """Per-instance counts are indexed in 32 bits: a horizon that would take an instance's variable
    count past 2^31 is refused from the sizes alone, before any array is read (the arrays here keep
    their small shapes, so reading them would run past their ends)."""
    c = synth.tiny()
    msg = _expect(qg, dataclasses.replace(c, T=2 ** 26), qg.QG_ERR_INVALID_ARG)
    assert "sizes too large" in msg


def test_instance_count_limit(qg):
    c = synth.tiny()
    with pytest.raises(qg.QGError) as ei:
        qg.qg_create_batch([c] * 33, qg.case_options(c))
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED and "at most 32" in str(ei.value)
    import ctypes
    h = ctypes.c_void_p()
    opt = qg.case_options(c)
    assert qg._lib.qg_create_batch(ctypes.byref(h), 0, None, None, None, ctypes.byref(opt)) == qg.QG_ERR_INVALID_ARG
    assert h.value is None


def test_bus_incidence_limit(qg):
    """A bus's balance and adjoint rows are reduced by one warp: more than 32 incident entries is a
    size this build rejects (before any device work)."""
    msg = _expect(qg, _star(33), qg.QG_ERR_UNSUPPORTED)
    assert "more than 32" in msg


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device path")
def test_limit_and_degenerate_inputs_reach_device_check(qg):
    """32 entries at a bus, 64 bid blocks per device, no outages (K = 0), a single period and the
    two-bus grid pass validation and the whole host set-up."""
    c = synth.tiny()
    cases = [_star(32), synth.with_block_bids(c, 64, 0.3, 5), dataclasses.replace(c, ctg=np.zeros(0, np.int32)),
             dataclasses.replace(c, T=1, dt=c.dt[:1], load_p=c.load_p[:1], load_q=c.load_q[:1],
                                 reserve_req=c.reserve_req[:1]),
             dataclasses.replace(_star(1), gen_bus=np.array([0], np.int32))]
    for case in cases:
        for dc in (qg.QG_DC_DENSE, qg.QG_DC_SPARSE):
            _expect(qg, case, qg.QG_ERR_NO_DEVICE, dc_solver=dc)


@pytest.mark.parametrize("iters", [1, 2, 7, 500])
def test_library_schedule_matches_the_closed_forms(qg, iters):
    """qg_schedule (host code of the library) against Eqs. norm_t, mag_scale and step_size as the
    oracle writes them (pinned in test_oracle_pins), plus the eps lag and the linear beta."""
    got = qg.qg_schedule(iters, 5e-3, 1e-5, 1e-1, 1e-5, 0.1, 1.0, 0.25)
    ref = oracle.schedule_table(iters, 5e-3, 1e-5, 1e-1, 1e-5, 0.1, 1.0, 0.25)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    assert got[0, 2] == pytest.approx(0.1) and got[-1, 2] == pytest.approx(1.0 if iters > 1 else 0.1)
    assert np.all(np.diff(got[:, 0]) <= 0) and np.all(np.diff(got[:, 1]) <= 0)
    with pytest.raises(qg.QGError):
        qg.qg_schedule(0, 5e-3, 1e-5, 1e-1, 1e-5)


def test_normal_build_has_no_index_checks(qg):
    """qg_bounds_report answers only in the index-checked build."""
    with pytest.raises(qg.QGError) as ei:
        qg.qg_bounds_report()
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED


def test_checked_source_transform():
    """The checked build's rewrite of qg_kernels.cu: every d.<array>[i] (nested ones too) becomes a
    checked access; other subscripts are untouched and no line is added."""
    from paper_2310_06650_gb300.build import CSRC, checked_source
    t = "a = d.x[d.y[i] + 1] * ad.z[3] + d.w + d.q[t[2]];\nb = tab.I[0]; d.g[k] = v;"
    out = checked_source(t)
    assert out == ("a = qg_at(d.x, (long long)(qg_at(d.y, (long long)(i), __LINE__) + 1), __LINE__) * ad.z[3] + d.w + "
                   "qg_at(d.q, (long long)(t[2]), __LINE__);\nb = tab.I[0]; qg_at(d.g, (long long)(k), __LINE__) = v;")
    src = open(os.path.join(CSRC, "qg_kernels.cu")).read()
    chk = checked_source(src)
    assert chk.count("\n") == src.count("\n")
    assert chk.count("qg_at(d.") > 200
