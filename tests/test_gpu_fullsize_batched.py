"""Parity at the full batched size: 256 independent fields, N log-uniform in [50, 5000],
unit masses, kappa_* ~ U[0.1, 0.8], gamma ~ U[0, 0.8], kappa_s ~ U[0, 0.3], m = 5000 phi
steps each (about 2.75*10^9 root points), in one persistent launch replayed from a CUDA
graph with the autotuner's tile shape, as the benchmark's batched section runs it.

What the oracle can compute in test time:
- the fields of smallest N: whole rows solved cold, compared root for root;
- sampled fields across the N range (the largest included): at sampled roots of sampled
  rows, the FP64 Newton step |F/F'| and the lens map w, and the rows' root separation.
Vieta's sums of each field's rationalised polynomial are checked on every row of every
field (on the device, in FP64)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import autotune, cc, synth
from tests.gpu_util import match_row

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def run():
    wl = synth.workload_batched()
    fields = [cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma) for f in wl.fields]
    ms = [wl.msteps] * len(fields)
    t, items, _ = autotune.tune(fields, ms, probe_steps=32, repeats=1)
    b = cc.cc_batch_create(fields, ms, t, items)
    z = [torch.empty((m + 1, fl.n_roots), dtype=torch.complex128, device="cuda") for fl, m in zip(fields, ms)]
    w = [torch.empty_like(a) for a in z]
    ws = cc.workspace(cc.cc_batch_workspace_bytes(b))
    cc.cc_batch_bind(b, z, w, ws)
    stream = torch.cuda.Stream()
    cc.cc_batch_launch(b, True, stream)
    stream.synchronize()
    st, per, tot = cc.cc_batch_report(b)
    yield dict(wl=wl, z=z, w=w, st=st, per=per, tot=tot)
    del z, w, ws, b, fields
    torch.cuda.empty_cache()


def test_report_clean(run):
    tot = run["tot"]
    assert run["st"] == cc.CC_OK, tot
    assert tot["unconverged"] == 0 and tot["uncertified"] == 0 and tot["seam_ambiguous"] == 0
    assert tot["max_err_est"] < 1e-10
    assert len(run["z"]) == 256
    assert sum(a.numel() for a in run["z"]) > 2.5e9


def test_every_row_of_every_field_vieta(run):
    wl, z = run["wl"], run["z"]
    m = wl.msteps
    phis = np.array([oracle.phi(j, m) for j in range(m + 1)])
    for f, zz in zip(wl.fields, z):
        nr = zz.shape[1]
        zs = f.x + 1j * f.y
        c = f.gamma - (1 - f.kappa_s) * np.exp(-1j * phis)
        s1 = zz.sum(dim=1).cpu().numpy()
        s2 = (zz * zz).sum(dim=1).cpu().numpy()
        a1 = zz.abs().sum(dim=1).cpu().numpy()
        zmax = float(zz.abs().max())
        tol1 = 2e-10 * nr + 1e-13 * a1
        tol2 = 4e-10 * nr * zmax + 1e-13 * a1 * zmax
        assert np.all(np.abs(s1 - 2 * zs.sum()) < tol1), len(f.x)
        assert np.all(np.abs(s2 - (2 * (zs * zs).sum() - 2 * f.m.sum() / c)) < tol2), len(f.x)


def test_smallest_fields_match_cold_oracle_rows(run):
    wl, z, w = run["wl"], run["z"], run["w"]
    m = wl.msteps
    order = np.argsort([len(f.x) for f in wl.fields])
    for i in order[:4]:
        f = wl.fields[i]
        for j in (0, 1, m // 3, m // 2, m):
            zo, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m))
            assert left == 0
            zg = z[i][j].cpu().numpy()
            idx, dist, sep = match_row(zg, zo)
            assert len(set(idx.tolist())) == len(idx), (int(i), j)
            assert dist < TOL and dist < 1e-3 * sep, (int(i), j, dist)
            wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo[idx])
            assert np.abs(w[i][j].cpu().numpy() - wo).max() < TOL, (int(i), j)


def test_sampled_fields_roots_are_fp64_zeros(run):
    wl, z, w = run["wl"], run["z"], run["w"]
    m = wl.msteps
    n_of = [len(f.x) for f in wl.fields]
    u = synth.uniform(5150, 10)
    pick = sorted({int(np.argmax(n_of))} | {int(v * len(wl.fields)) for v in u})
    for i in pick:
        f = wl.fields[i]
        nr = z[i].shape[1]
        for j in (0, m // 2 + 1, int(u[i % 10] * m)):
            zr = z[i][j].cpu().numpy()
            wr = w[i][j].cpu().numpy()
            ks = np.unique((synth.uniform(7000 + 31 * i + j, 120) * nr).astype(np.int64))
            ph = oracle.phi(j, m)
            for k in ks:
                step = oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, zr[k]) / oracle.dF(f.x, f.y, f.m, zr[k])
                assert abs(step) < TOL, (i, j, int(k), abs(step))
            wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zr[ks])
            assert np.abs(wr[ks] - wo).max() < TOL, (i, j)
            assert oracle.min_separation(zr) > 1e-7, (i, j)
