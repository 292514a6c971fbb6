"""Heterogeneous CPU + GPU co-execution (Sec. 4 workflow; Sec. 6 Eq. hete):
one block split into k-slabs between the GPU and the host worker, the cut's
ghost layers exchanged every Runge-Kutta stage.

  * stage-by-stage GPU stepping (sensei_rk_stage) is bitwise the one-call
    step (sensei_rk_step) with the same dt;
  * the face exchange moves exactly the two layers next to a face;
  * the co-executed state equals the GPU-only state of the same block to
    1e-9 after 40 steps (periodic k: two cuts; k-faces with extrapolation
    and inflow rules: one cut), and the oracle's to 1e-9 after 10 steps."""
import numpy as np
import pytest

import oracle
from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import build as libbuild
from paper_2305_18057_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sensei():
    libbuild.build()
    from paper_2305_18057_gb300 import sensei as s
    s.load()
    return s


def test_stage_by_stage_equals_one_step(sensei):
    w = wl.ramp_3d(ni=40, nj=20, nk=12, perturb=0.05, seed=41)
    a, b = gpu_grid(w), gpu_grid(w)
    Ua, Ub = gpu_states(a, w), gpu_states(b, w)
    s = torch.cuda.current_stream().cuda_stream
    dt = sensei.sensei_dt_min(a.handle, [U.data_ptr() for U in Ua], 0.5, s)
    for rk in (sensei.RK3_SSP, sensei.RK2_SSP, sensei.RK4_SSP2):
        a.rk_step(Ua, rk, cfl=0.0, dt=dt)
        for st in range(sensei.RK_STAGES[rk]):
            sensei.sensei_rk_stage(b.handle, [U.data_ptr() for U in Ub], rk, st, dt, s)
    torch.cuda.synchronize()
    assert torch.equal(a.interior_view(Ua[0], 0), b.interior_view(Ub[0], 0))


def test_face_exchange_moves_two_layers(sensei):
    w = wl.periodic_3d(n=20, nj=12, nk=10, seed=42)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    g.fill_ghosts(Us)
    ni, nj, nk = w.dims[0]
    s = torch.cuda.current_stream().cuda_stream
    L = sensei.sensei_state_layout(g.handle, 0)
    full = Us[0].as_strided((5, nk + 4, nj + 4, ni + 4), (L.stride_var, L.stride_k, L.stride_j, 1),
                            L.offset - 2 * L.stride_k - 2 * L.stride_j - 2)
    for face in range(6):
        n1 = nj if face < 2 else ni
        n2 = nk if face < 4 else nj
        buf = torch.empty(5 * 2 * n1 * n2, dtype=torch.float64, device="cuda")
        sensei.sensei_face_exchange(g.handle, [Us[0].data_ptr()], 0, 0, face, buf.data_ptr(), 0, s)
        b = buf.view(5, 2, n2, n1)
        inner = [full[:, 2:-2, 2:-2, 2 + l] if face == 0 else full[:, 2:-2, 2:-2, -3 - l] if face == 1 else
                 full[:, 2:-2, 2 + l, 2:-2] if face == 2 else full[:, 2:-2, -3 - l, 2:-2] if face == 3 else
                 full[:, 2 + l, 2:-2, 2:-2] if face == 4 else full[:, -3 - l, 2:-2, 2:-2] for l in range(2)]
        for l in range(2):
            assert torch.equal(b[:, l], inner[l]), (face, l)
        # unpack a marker into the ghosts and read it back
        buf.copy_(torch.arange(buf.numel(), dtype=torch.float64, device="cuda"))
        sensei.sensei_face_exchange(g.handle, [Us[0].data_ptr()], 0, 0, face, buf.data_ptr(), 1, s)
        ghost = [full[:, 2:-2, 2:-2, 1 - l] if face == 0 else full[:, 2:-2, 2:-2, -2 + l] if face == 1 else
                 full[:, 2:-2, 1 - l, 2:-2] if face == 2 else full[:, 2:-2, -2 + l, 2:-2] if face == 3 else
                 full[:, 1 - l, 2:-2, 2:-2] if face == 4 else full[:, -2 + l, 2:-2, 2:-2] for l in range(2)]
        for l in range(2):
            assert torch.equal(ghost[l], b[:, l]), ("unpack", face, l)


def _bcs(w):
    return [(bc.type, bc.prim) for bc in w.bcs[0]]


def _kfaces_physical(w):
    """The same workload with its k-faces under the extrapolation (kmin) and
    freestream-inflow (kmax) rules instead of periodic ones."""
    import dataclasses
    prim = np.array([w.U0[0][0].mean(), *(w.U0[0][a].mean() / w.U0[0][0].mean() for a in (1, 2, 3)), 1.0 / w.gamma])
    faces = list(w.bcs[0])
    faces[4] = wl.BC(wl.EXTRAPOLATE, None, -1, -1)
    faces[5] = wl.BC(wl.INFLOW, prim, -1, -1)
    return dataclasses.replace(w, bcs=[faces])


@pytest.mark.parametrize("case", ["periodic", "ramp", "kfaces_physical"])
def test_coexecution_equals_gpu_only(sensei, case):
    if case == "periodic":
        w, nk_host = wl.periodic_3d(n=32, nj=24, nk=40, seed=43), 12
    elif case == "ramp":
        w, nk_host = wl.ramp_3d(ni=40, nj=24, nk=24, perturb=0.05, seed=44), 8
    else:
        w, nk_host = _kfaces_physical(wl.periodic_3d(n=24, nj=20, nk=30, seed=46)), 9
    h = sensei.Hetero(w.dims[0], w.nodes[0], _bcs(w), nk_host, threads=4, limiter=wl.LIMITERS[w.limiter],
                      entropy_fix=w.fix)
    h.upload(w.U0[0])
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    dt_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(40):
        dt, _t = h.step(sensei.RK3_SSP, cfl=0.5)
        g.rk_step(Us, sensei.RK3_SSP, cfl=0.5, dt_used=dt_t)
        torch.cuda.synchronize()
        assert abs(dt - dt_t.item()) <= 1e-12 * dt
    got = h.download()
    want = g.download(Us[0], 0)
    err = per_var_rel(got, want)
    print(f"{case}: co-executed vs GPU-only after 40 steps: {err:.3g}")
    assert err < 1e-9
    h.close()


def test_coexecution_against_oracle(sensei):
    w = wl.ramp_3d(ni=24, nj=16, nk=20, perturb=0.05, seed=45)
    h = sensei.Hetero(w.dims[0], w.nodes[0], _bcs(w), 6, threads=2, limiter=wl.LIMITERS[w.limiter], entropy_fix=w.fix)
    h.upload(w.U0[0])
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    for _ in range(10):
        dt, _t = h.step(sensei.RK3_SSP, cfl=0.5)
        og.rk_step(Uo, oracle.RK3_SSP, dt=dt)
    err = per_var_rel(h.download(), og.interior(Uo[0], 0))
    assert err < 1e-9
    h.close()


def test_coexecution_rejects_bad_splits(sensei):
    w = wl.periodic_3d(n=16, nj=12, nk=10, seed=47)
    for nk_host in (1, 9):
        with pytest.raises(sensei.SenseiError):
            sensei.Hetero(w.dims[0], w.nodes[0], _bcs(w), nk_host, threads=1)
