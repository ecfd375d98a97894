"""The C-ABI IRLS drivers at their named configurations against the FP64 oracle.

* tf_rsvd on c2 (100 x 100 stations, 110 x 110 x 10 cells, t = 1250, t_p = 1260, one power
  iteration, Alg. 2): the first IRLS step (alpha^(1) from Eq. (11)), FP64 and FP32, the
  model against the oracle's (the oracle's step takes about 2.5 minutes: 5040 FFT-route
  products and two tall QRs; later steps differ only by the elementwise W_L^(k), which the
  three-step fixed-alpha tests at c1 cover);
* tf_gkb on the c3 magnetic geometry (150 x 150 stations, 150 x 150 x 20 cells) with a
  reduced t_p = 150 (the oracle keeps dense FP64 bases and runs modified Gram-Schmidt in
  Python loops, so the configuration's t_p = 2952 is beyond it), FP32 with double-float
  re-orthogonalisation and FP64, first step against the oracle (Alg. 1);
* at full size, where the oracle's step would take hours, the FP32 driver against the FP64
  driver: tf_rsvd on c4 (t_p = 2510, tall-skinny QR of the 10^6-row bases) and tf_gkb on
  c3 (t_p = 2952).

Tolerances: FP64 <= 1e-11 (rounding differences of two FP64 implementations of the same
steps, through t_p-term projections), FP32 <= 2e-5 per step against the FP64 oracle.
"""
import numpy as np
import pytest

import synth
from oracle import irls as oirls
from oracle import operator as oop

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _problem(cfg, kind, inc, dec, beta, seed=0):
    g = synth.config_grid(cfg)
    T = oop.layer_tables(g, kind, inc, dec)
    m_true = synth.config_model(cfg, seed)
    d = oop.fft_matvec(g, T, m_true)
    sigma = 0.01 * np.abs(d) + 0.001 * np.abs(d).max()
    d_obs = d + sigma * synth.unit_noise(g.m, seed)
    wz = oirls.depth_weights(g.z_edges, g.station_z, g.ny, g.nx, beta)
    return dict(g=g, T=T, d_obs=d_obs, sigma=sigma, wz=wz, kind=kind, inc=inc, dec=dec,
                beta=beta, upper=0.1 if kind == "magnetic" else 1.0)


def _oracle(c, solver, t, tp, kmax, omega=None, alphas=None):
    g = c["g"]
    p = oirls.IRLSParams(solver=solver, t=t, tp=tp, beta=c["beta"], upper=c["upper"], kmax=kmax,
                         chi2_stop=False, alphas=alphas)
    return oirls.irls(lambda x: oop.fft_matvec(g, c["T"], x),
                      lambda y: oop.fft_rmatvec(g, c["T"], y),
                      c["d_obs"], c["sigma"], g.n, c["wz"], p, omega)


def _native(c, dtn, solver, t, tp, kmax, omega=None, alphas=None):
    import torch
    from paper_2004_13904_gb300 import Operator
    from paper_2004_13904_gb300.irls import IRLSOptions, invert_native
    dt = torch.float32 if dtn == "f32" else torch.float64
    op = Operator(c["g"], c["kind"], c["inc"], c["dec"], dtype=dt)
    opts = IRLSOptions(solver=solver, t=t, tp=tp, beta=c["beta"], upper=c["upper"], kmax=kmax,
                       chi2_stop=False, alphas=alphas)
    om = torch.tensor(omega, dtype=dt, device="cuda") if omega is not None else None
    r = invert_native(op, torch.tensor(c["d_obs"], dtype=dt, device="cuda"),
                      torch.tensor(c["sigma"], dtype=dt, device="cuda"), opts, om)
    out = r.model.double().cpu().numpy()
    op.close()
    return out, r


TOL = {"f64": 1e-11, "f32": 2e-5}


@pytest.fixture(scope="module")
def c2_rsvd():
    c = _problem("c2", "gravity", 90.0, 0.0, 0.8)
    t = c["g"].m // 8                      # 1250
    tp = t + 10                            # 1260: the configuration's block
    omega = synth.gaussian_columns(c["g"].m, tp, seed=17)
    m1, rep1 = _oracle(c, "rsvd", t, tp, 1, omega)
    return dict(c=c, t=t, tp=tp, omega=omega, m1=m1, rep1=rep1)


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_rsvd_c2_first_step(c2_rsvd, dtn):
    f = c2_rsvd
    m, r = _native(f["c"], dtn, "rsvd", f["t"], f["tp"], 1, f["omega"])
    err = rel(m, f["m1"])
    print(f"tf_rsvd c2 {dtn} step 1: {err:.3e}, alpha {r.alphas[0]:.6e} vs {f['rep1'].alphas[0]:.6e}")
    assert abs(r.alphas[0] - f["rep1"].alphas[0]) <= (1e-10 if dtn == "f64" else 1e-4) * f["rep1"].alphas[0]
    assert err <= TOL[dtn]


def test_rsvd_c2_tall_skinny_qr(c2_rsvd, monkeypatch):
    """The RSVD driver's tall-skinny QR (row blocks factored separately, their stacked R
    factored again), which it takes when a basis block exceeds the 32-bit solver interface
    (c4: 10^6 x 2510); forced here on c2 by a lower block bound (3 row blocks of the
    121000 x 1260 basis), FP64 against the oracle's Householder QR step."""
    f = c2_rsvd
    monkeypatch.setenv("TF_QR_BLOCK_ELEMS", str(60_000_000))
    m, r = _native(f["c"], "f64", "rsvd", f["t"], f["tp"], 1, f["omega"])
    err = rel(m, f["m1"])
    print(f"tf_rsvd c2 with tall-skinny QR: {err:.3e}")
    assert abs(r.alphas[0] - f["rep1"].alphas[0]) <= 1e-10 * f["rep1"].alphas[0]
    assert err <= TOL["f64"]


@pytest.fixture(scope="module")
def c3_gkb():
    c = _problem("c3", "magnetic", 50.0, 10.0, 1.4)
    tp = 150
    t = int(tp / 1.05)
    m1, rep1 = _oracle(c, "gkb", t, tp, 1)
    return dict(c=c, t=t, tp=tp, m1=m1, rep1=rep1)


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_gkb_c3_first_step(c3_gkb, dtn):
    f = c3_gkb
    m, r = _native(f["c"], dtn, "gkb", f["t"], f["tp"], 1)
    err = rel(m, f["m1"])
    print(f"tf_gkb c3 {dtn} step 1 (t_p = {f['tp']}): {err:.3e}, alpha {r.alphas[0]:.6e} vs "
          f"{f['rep1'].alphas[0]:.6e}")
    assert abs(r.alphas[0] - f["rep1"].alphas[0]) <= (1e-10 if dtn == "f64" else 1e-4) * f["rep1"].alphas[0]
    assert err <= TOL[dtn]


def test_rsvd_c4_fp32_matches_fp64():
    """c4 at paper scale (250 x 200 stations, 250 x 200 x 20 cells), RSVD-IRLS with
    k = m/20 = 2500 and oversampling 10 (t_p = 2510), one step: the FP32 driver's recovered
    model against the FP64 driver's (itself pinned to the oracle at c1 and c2; the
    oracle's own RSVD step at this size would take about an hour on the host)."""
    c = _problem("c4", "gravity", 90.0, 0.0, 0.8)
    t = c["g"].m // 20
    tp = t + 10
    omega = synth.gaussian_columns(c["g"].m, tp, seed=17)
    m64, r64 = _native(c, "f64", "rsvd", t, tp, 1, omega)
    m32, r32 = _native(c, "f32", "rsvd", t, tp, 1, omega)
    err = rel(m32, m64)
    print(f"tf_rsvd c4 step 1, FP32 vs FP64: {err:.3e}; alpha {r32.alphas[0]:.6e} vs {r64.alphas[0]:.6e}; "
          f"seconds FP32 {r32.seconds[0]:.2f}, FP64 {r64.seconds[0]:.2f}")
    assert abs(r32.alphas[0] - r64.alphas[0]) <= 1e-4 * r64.alphas[0]
    assert err <= TOL["f32"]


def test_gkb_c3_full_fp32_matches_fp64():
    """c3 at its full size (magnetic 150 x 150 stations, 150 x 150 x 20 cells), GKB-IRLS
    with t = m/8 = 2812 and t_p = 1.05 t = 2952 Lanczos steps, one step: the FP32 driver
    (double-float re-orthogonalisation) against the FP64 driver (pinned to the oracle at
    t_p = 150 above and at c1; the oracle's dense Python Gram-Schmidt would take hours at
    t_p = 2952)."""
    c = _problem("c3", "magnetic", 50.0, 10.0, 1.4)
    t = c["g"].m // 8
    tp = int(1.05 * t)
    m64, r64 = _native(c, "f64", "gkb", t, tp, 1)
    m32, r32 = _native(c, "f32", "gkb", t, tp, 1)
    err = rel(m32, m64)
    print(f"tf_gkb c3 step 1 (t_p = {tp}), FP32 vs FP64: {err:.3e}; alpha {r32.alphas[0]:.6e} vs "
          f"{r64.alphas[0]:.6e}; seconds FP32 {r32.seconds[0]:.2f}, FP64 {r64.seconds[0]:.2f}")
    assert abs(r32.alphas[0] - r64.alphas[0]) <= 1e-4 * r64.alphas[0]
    assert err <= TOL["f32"]
