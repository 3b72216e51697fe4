"""Batched solves and the continuous-batching server (GPU): every result
matches the CPU oracle's solution of its system (oracle GMRES to 1e-12,
relative error <= 1e-6) and is the same alone and in the mix, admission never
exceeds the device budget, oversized requests are rejected, and a poisoned
request fails alone."""
import ctypes
import threading
import time

import numpy as np
import pytest

from gpu_common import cuda_or_fail, relerr
from oracle import solve as osolve
from paper_1903_07884_gb300 import inputs, vie
from paper_1903_07884_gb300.solver import Plan, make_opts, to_device

pytestmark = pytest.mark.gpu


def _problems():
    return [inputs.straight_guide(96, 8, 4, 0.05, 1.55, absorber=8, name="a"),
            inputs.bragg_grating(128, 12, 4, 0.025, 1.50, wide=8, narrow=6, period=16, name="b"),
            inputs.directional_coupler(80, 0.025, 1.58, ny=24, nz=4, core_w=8, gap=4, margin=2, name="c"),
            inputs.straight_guide(131, 8, 4, 0.025, 1.52, core_ny=6, core_nz=4, name="d")]


_ORACLE = {}


def _oracle_solution(p):
    """The oracle's solution of a request's system, cached per problem name."""
    if p.name not in _ORACLE:
        s = osolve.iterative_solve(p, tol=1e-12, tau=1e-3, max_iter=20000)
        assert s.relres <= 1e-12, (p.name, s.relres)
        _ORACLE[p.name] = s.w
    return _ORACLE[p.name]


def _opts(p, precision=vie.VIE_MIXED):
    return make_opts(precision=precision, boxes=p.boxes or None, homog=p.homog)


def test_batch_equals_individual_solves():
    torch = cuda_or_fail()
    probs = _problems()
    alone = []
    for p in probs:
        plan = Plan.for_problem(p)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        alone.append(w.cpu().numpy())
        plan.close()
    plans, es, ws, streams = [], [], [], []
    for p in probs:
        s = torch.cuda.Stream()
        pl = Plan(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, _opts(p), stream=s)
        with torch.cuda.stream(s):
            pl.set_permittivity(p.eps)
            e = to_device(p.e_inc)
            es.append(e)
            ws.append(torch.empty_like(e))
        torch.cuda.synchronize()
        plans.append(pl)
        streams.append(s)
    infos = vie.vie_solve_batch([pl.handle for pl in plans], [e.data_ptr() for e in es], [w.data_ptr() for w in ws])
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        assert infos[i].relres <= 1e-9
        np.testing.assert_array_equal(ws[i].cpu().numpy(), alone[i])
        assert relerr(alone[i], _oracle_solution(p)) <= 1e-6, p.name
    for pl in plans:
        pl.close()


def test_batch_mixes_precisions_and_uneven_lengths():
    """One lockstep batch of plans of different lengths (nx 96, 131, 200),
    cross-sections and precisions (two complex-FP32 GMRES-IR solves and one
    FP64 solve): the Arnoldi kernels of each step run as one launch over the
    work-list of all plans of a precision, and every result is bitwise the
    result of the same plan solved alone."""
    torch = cuda_or_fail()
    probs = [inputs.straight_guide(96, 8, 4, 0.05, 1.55, absorber=8, name="u0"),
             inputs.straight_guide(131, 8, 4, 0.025, 1.52, core_ny=6, core_nz=4, name="u1"),
             inputs.bragg_grating(200, 12, 4, 0.025, 1.50, wide=8, narrow=6, period=16, name="u2")]
    precs = [vie.VIE_MIXED, vie.VIE_FP64, vie.VIE_MIXED]
    alone = []
    for p, pr in zip(probs, precs):
        plan = Plan.for_problem(p, precision=pr)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        alone.append(w.cpu().numpy())
        plan.close()
    plans, es, ws = [], [], []
    for p, pr in zip(probs, precs):
        pl = Plan.for_problem(p, precision=pr)
        pl.set_permittivity(p.eps)
        e = to_device(p.e_inc)
        es.append(e)
        ws.append(torch.empty_like(e))
        plans.append(pl)
    torch.cuda.synchronize()
    launches0 = vie.vie_kernel_launches()
    infos = vie.vie_solve_batch([pl.handle for pl in plans], [e.data_ptr() for e in es], [w.data_ptr() for w in ws])
    torch.cuda.synchronize()
    assert vie.vie_kernel_launches() > launches0
    for i, p in enumerate(probs):
        assert infos[i].relres <= 1e-9
        np.testing.assert_array_equal(ws[i].cpu().numpy(), alone[i])
        assert relerr(alone[i], _oracle_solution(p)) <= 1e-6, p.name
    for pl in plans:
        pl.close()


def _submit(srv, p, w_out, opts=None):
    eps = np.ascontiguousarray(p.eps)
    e = np.ascontiguousarray(p.e_inc)
    st, t = vie.vie_server_submit(srv, p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, opts or _opts(p),
                                  eps.ctypes.data, e.ctypes.data, w_out.ctypes.data)
    return st, t


def _wait(srv, tickets, timeout=120.0):
    t0 = time.time()
    out = {}
    while len(out) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t in out:
                continue
            st, info = vie.vie_server_poll(srv, t)
            if st != vie.VIE_PENDING:
                out[t] = (st, info)
        time.sleep(0.002)
    return out


def test_server_results_alone_equal_results_in_the_mix():
    cuda_or_fail()
    probs = _problems()
    srv = vie.vie_server_create(40 << 30, 4)
    try:
        alone = []
        for p in probs:
            w = np.empty(p.e_inc.shape, dtype=np.complex128)
            st, t = _submit(srv, p, w)
            assert st == vie.VIE_OK
            res = _wait(srv, [t])
            assert res[t][0] == vie.VIE_OK, vie.last_error()
            assert relerr(w, _oracle_solution(p)) <= 1e-6, p.name
            alone.append(w)
        # all at once, twice over, arriving while others run
        outs, tickets = [], []
        for rep in range(2):
            for p in probs:
                w = np.empty(p.e_inc.shape, dtype=np.complex128)
                st, t = _submit(srv, p, w)
                assert st == vie.VIE_OK
                outs.append(w)
                tickets.append(t)
        res = _wait(srv, tickets)
        assert all(res[t][0] == vie.VIE_OK for t in tickets)
        for i, w in enumerate(outs):
            ref = alone[i % len(probs)]
            # the same kernels with the same launch shapes run on the same data
            assert relerr(w, ref) <= 1e-12
            assert res[tickets[i]][1].relres <= 1e-9
    finally:
        vie.vie_server_destroy(srv)


def test_server_admission_respects_budget_and_rejects_oversized():
    cuda_or_fail()
    probs = _problems()
    need = max(vie.vie_estimate_bytes(p.nx, p.ny, p.nz, _opts(p)) for p in probs)
    budget = int(need * 1.5)             # at most one request fits at a time
    srv = vie.vie_server_create(budget, 4)
    try:
        outs, tickets = [], []
        for p in probs:
            w = np.empty(p.e_inc.shape, dtype=np.complex128)
            st, t = _submit(srv, p, w)
            assert st == vie.VIE_OK
            outs.append(w)
            tickets.append(t)
        peak = 0
        t0 = time.time()
        done = {}
        while len(done) < len(tickets) and time.time() - t0 < 120:
            peak = max(peak, vie.vie_server_reserved_bytes(srv))
            for t in tickets:
                if t not in done:
                    st, _ = vie.vie_server_poll(srv, t)
                    if st != vie.VIE_PENDING:
                        done[t] = st
        assert all(st == vie.VIE_OK for st in done.values()) and len(done) == len(tickets)
        assert 0 < peak <= budget
        big = inputs.straight_guide(4096, 24, 8, 0.025, 1.55)
        w = np.empty(big.e_inc.shape, dtype=np.complex128)
        st, t = _submit(srv, big, w, make_opts())
        assert st == vie.VIE_EREJECTED
    finally:
        vie.vie_server_destroy(srv)


def test_server_poisoned_request_fails_alone():
    cuda_or_fail()
    probs = _problems()[:2]
    bad = inputs.straight_guide(64, 8, 4, 0.05, 1.55, absorber=4, name="bad")
    bad.eps[1, 2, 3] = np.nan
    srv = vie.vie_server_create(40 << 30, 3)
    try:
        ws = [np.empty(p.e_inc.shape, dtype=np.complex128) for p in probs + [bad]]
        tickets = []
        for p, w in zip(probs + [bad], ws):
            st, t = _submit(srv, p, w)
            assert st == vie.VIE_OK
            tickets.append(t)
        res = _wait(srv, tickets)
        assert res[tickets[0]][0] == vie.VIE_OK and res[tickets[1]][0] == vie.VIE_OK
        assert res[tickets[2]][0] == vie.VIE_EINVAL
    finally:
        vie.vie_server_destroy(srv)


def test_server_concurrent_medium_requests_bitwise():
    """Eight medium requests (1500..3250 x 16 x 8 wires and Bragg gratings, so
    that every SM carries blocks of several plans at once) through the server
    with all eight in flight: each result is bitwise the result of the same
    request solved alone.  Plans share no device state, so concurrency may
    change timing but never a single bit."""
    cuda_or_fail()
    probs = []
    for i in range(8):
        nx = 1500 + 250 * i
        if i % 2 == 0:
            probs.append(inputs.straight_guide(nx, 16, 8, 0.025, 1.50 + 0.01 * i, name=f"m{i}"))
        else:
            probs.append(inputs.bragg_grating(nx, 16, 8, 0.025, 1.50 + 0.01 * i, name=f"m{i}"))
    alone = []
    for p in probs:
        plan = Plan.for_problem(p)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        assert info["relres"] <= 1e-9
        alone.append(w.cpu().numpy())
        plan.close()
    srv = vie.vie_server_create(64 << 30, 8)
    bufs, tickets = [], {}
    for i, p in enumerate(probs):
        eps, e = np.ascontiguousarray(p.eps), np.ascontiguousarray(p.e_inc)
        w = np.empty(p.e_inc.shape, dtype=np.complex128)
        bufs.append((eps, e, w))
        st, t = vie.vie_server_submit(srv, p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, _opts(p), eps.ctypes.data,
                                      e.ctypes.data, w.ctypes.data)
        assert st == vie.VIE_OK
        tickets[t] = i
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < 300:
        for t, i in tickets.items():
            if i not in done:
                st, info = vie.vie_server_poll(srv, t)
                if st != vie.VIE_PENDING:
                    done[i] = (st, info.relres)
        time.sleep(0.01)
    vie.vie_server_destroy(srv)
    assert len(done) == len(probs)
    for i in range(len(probs)):
        assert done[i][0] == vie.VIE_OK, (i, done[i], vie.last_error())
        np.testing.assert_array_equal(bufs[i][2], alone[i])


def test_server_twelve_requests_join_and_leave_the_lockstep_set():
    """Twelve small requests of uneven lengths, both precisions, submitted in
    two waves: the driver's lockstep set grows beyond eight runs and changes
    as requests join and finish; every result is bitwise the solo result."""
    cuda_or_fail()
    probs, precs = [], []
    for i in range(12):
        nx = 40 + 13 * i
        if i % 3 == 2:
            probs.append(inputs.bragg_grating(nx, 12, 4, 0.025, 1.50 + 0.005 * i, wide=8, narrow=6, period=16,
                                              name=f"t{i}"))
        else:
            probs.append(inputs.straight_guide(nx, 8, 4, 0.05, 1.50 + 0.005 * i, absorber=4, name=f"t{i}"))
        precs.append(vie.VIE_FP64 if i % 4 == 3 else vie.VIE_MIXED)
    alone = []
    for p, pr in zip(probs, precs):
        plan = Plan.for_problem(p, precision=pr)
        plan.set_permittivity(p.eps)
        w, info = plan.solve(p.e_inc)
        alone.append(w.cpu().numpy())
        plan.close()
    srv = vie.vie_server_create(64 << 30, 12)
    outs, tickets = [], []
    try:
        for wave in (range(0, 7), range(7, 12)):
            for i in wave:
                p = probs[i]
                w = np.empty(p.e_inc.shape, dtype=np.complex128)
                st, t = _submit(srv, p, w, _opts(p, precs[i]))
                assert st == vie.VIE_OK
                outs.append(w)
                tickets.append(t)
            time.sleep(0.05)
        res = _wait(srv, tickets, timeout=300)
    finally:
        vie.vie_server_destroy(srv)
    assert len(res) == len(tickets)
    for i, t in enumerate(tickets):
        assert res[t][0] == vie.VIE_OK, (i, res[t])
        np.testing.assert_array_equal(outs[i], alone[i])
