"""The C-ABI IRLS drivers tf_gkb / tf_rsvd against the FP64 oracle (same inputs, same
readings of the paper), with the tolerances of the Python-level driver's tests: one step
(alpha^(1) from Eq. (11)) to 1e-11 in FP64 and 2e-5 in FP32, three steps with the oracle's
alphas fixed to 1e-9, and the quality of a full 20-iteration GKB run on c1."""
import numpy as np
import pytest

import synth
from oracle import irls as oirls
from oracle import operator as oop

pytestmark = pytest.mark.gpu


def _c1_problem(seed=0):
    g = synth.config_grid("c1")
    T = oop.layer_tables(g, "gravity")
    m_true = synth.config_model("c1", seed)
    d = oop.fft_matvec(g, T, m_true)
    sigma = 0.01 * np.abs(d) + 0.001 * np.abs(d).max()
    d_obs = d + sigma * synth.unit_noise(g.m, seed)
    return g, T, m_true, d_obs, sigma


def _oracle(c, solver, tp, kmax, alphas=None):
    g = c["g"]
    wz = oirls.depth_weights(g.z_edges, g.station_z, g.ny, g.nx, 0.8)
    p = oirls.IRLSParams(solver=solver, t=c["t"], tp=tp, kmax=kmax, chi2_stop=False, alphas=alphas)
    return oirls.irls(lambda x: oop.fft_matvec(g, c["T"], x), lambda y: oop.fft_rmatvec(g, c["T"], y),
                      c["d_obs"], c["sigma"], g.n, wz, p, c["omega"] if solver == "rsvd" else None)


def _native(c, dtype, solver, tp, kmax, reorth="cgs2", alphas=None):
    import torch
    from paper_2004_13904_gb300 import Operator
    from paper_2004_13904_gb300.irls import IRLSOptions, invert_native
    op = Operator(c["g"], "gravity", dtype=dtype)
    opts = IRLSOptions(solver=solver, t=c["t"], tp=tp, kmax=kmax, chi2_stop=False, reorth=reorth,
                       alphas=alphas)
    om = torch.tensor(c["omega"], dtype=dtype, device="cuda") if solver == "rsvd" else None
    r = invert_native(op, torch.tensor(c["d_obs"], dtype=dtype, device="cuda"),
                      torch.tensor(c["sigma"], dtype=dtype, device="cuda"), opts, om)
    return r.model.double().cpu().numpy(), r


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def c1():
    g, T, m_true, d_obs, sigma = _c1_problem()
    t = g.m // 8
    return dict(g=g, T=T, m_true=m_true, d_obs=d_obs, sigma=sigma, t=t, tp_gkb=int(1.05 * t),
                tp_rsvd=t + 10, omega=synth.gaussian_columns(g.m, t + 10, seed=17))


@pytest.mark.parametrize("reorth", ["mgs", "cgs2"])
def test_native_gkb_first_step_fp64(c1, reorth):
    import torch
    m_ref, rep = _oracle(c1, "gkb", c1["tp_gkb"], 1)
    m, r = _native(c1, torch.float64, "gkb", c1["tp_gkb"], 1, reorth)
    print(f"tf_gkb {reorth} step 1: {rel(m, m_ref):.3e}, alpha {r.alphas[0]:.6e} vs {rep.alphas[0]:.6e}")
    assert r.alphas and abs(r.alphas[0] - rep.alphas[0]) <= 1e-12 * rep.alphas[0]
    assert rel(m, m_ref) <= 1e-11
    assert abs(r.chi2[0] - rep.chi2[0]) <= 1e-9 * rep.chi2[0]


def test_native_rsvd_first_step_fp64(c1):
    import torch
    m_ref, rep = _oracle(c1, "rsvd", c1["tp_rsvd"], 1)
    m, r = _native(c1, torch.float64, "rsvd", c1["tp_rsvd"], 1)
    print(f"tf_rsvd step 1: {rel(m, m_ref):.3e}")
    assert abs(r.alphas[0] - rep.alphas[0]) <= 1e-12 * rep.alphas[0]
    assert rel(m, m_ref) <= 1e-11


@pytest.mark.parametrize("solver", ["gkb", "rsvd"])
def test_native_fixed_alpha_three_steps_fp64(c1, solver):
    import torch
    tp = c1["tp_gkb"] if solver == "gkb" else c1["tp_rsvd"]
    _, rep = _oracle(c1, solver, tp, 3)
    m_ref, _ = _oracle(c1, solver, tp, 3, alphas=rep.alphas)
    m, r = _native(c1, torch.float64, solver, tp, 3, alphas=rep.alphas)
    print(f"native {solver} 3 steps, fixed alpha: {rel(m, m_ref):.3e}")
    assert r.alphas == list(rep.alphas)
    assert rel(m, m_ref) <= 1e-9


@pytest.mark.parametrize("solver", ["gkb", "rsvd"])
def test_native_first_step_fp32(c1, solver):
    import torch
    tp = c1["tp_gkb"] if solver == "gkb" else c1["tp_rsvd"]
    m_ref, _ = _oracle(c1, solver, tp, 1)
    m, _ = _native(c1, torch.float32, solver, tp, 1)
    print(f"native {solver} FP32 step 1 vs FP64 oracle: {rel(m, m_ref):.3e}")
    assert rel(m, m_ref) <= 2e-5


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_native_full_gkb_irls_c1(c1, dtn):
    """c1 as specified: GKB-IRLS, t = m/8 = 128, t_p = 134, 20 iterations, 0-1 g/cc."""
    import torch
    dt = torch.float64 if dtn == "f64" else torch.float32
    m_ref, rep = _oracle(c1, "gkb", c1["tp_gkb"], 20)
    m, r = _native(c1, dt, "gkb", c1["tp_gkb"], 20)
    re, re_ref = rel(m, c1["m_true"]), rel(m_ref, c1["m_true"])
    print(f"tf_gkb {dtn}: RE {re:.4f} (oracle {re_ref:.4f}), alphas {r.alphas[:3]}")
    a_tol = 1e-6 if dtn == "f64" else 1e-2
    assert len(r.alphas) == 20
    assert np.allclose(r.alphas[:5], rep.alphas[:5], rtol=a_tol)
    assert abs(re - re_ref) < (0.01 if dtn == "f64" else 0.05)
    assert m.min() >= 0.0 and m.max() <= 1.0


def test_native_chi2_stop_and_errors(c1):
    import torch
    from paper_2004_13904_gb300 import Operator, _lib
    from paper_2004_13904_gb300.irls import IRLSOptions, invert_native
    op = Operator(c1["g"], "gravity", dtype=torch.float32)
    d = torch.tensor(c1["d_obs"], dtype=torch.float32, device="cuda")
    s = torch.tensor(c1["sigma"], dtype=torch.float32, device="cuda")
    r = invert_native(op, d, s, IRLSOptions(t=c1["t"], tp=c1["tp_gkb"], kmax=25, chi2_stop=True))
    m = c1["g"].m
    assert r.chi2[-1] <= m + np.sqrt(2 * m) or len(r.chi2) == 25
    assert all(c > m + np.sqrt(2 * m) for c in r.chi2[:-1])
    with pytest.raises(_lib.TFError) as e:
        invert_native(op, d, s, IRLSOptions(t=20, tp=10, kmax=1))
    assert e.value.status == _lib.TF_EINVAL
    with pytest.raises(ValueError):
        invert_native(op, d, s, IRLSOptions(solver="rsvd", t=10, tp=12, kmax=1))
