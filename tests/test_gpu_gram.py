"""Gram-Schmidt kernels (tf_rows_dot / tf_rows_axpy) against FP64 references: FP64 data
to rounding, FP32 data (double-float accumulation) to ~1e-12 of the exact sums."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtn,tol", [("f64", 1e-14), ("f32", 1e-11)])
@pytest.mark.parametrize("k,length", [(1, 1000), (37, 100003), (2500, 4097)])
def test_rows_dot_and_axpy(dtn, tol, k, length):
    import torch
    from paper_2004_13904_gb300.irls import rows_axpy as _rows_axpy, rows_dot as _rows_dot
    dt = torch.float64 if dtn == "f64" else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(k)
    A = torch.randn(k, length + 3, generator=gen, device="cuda", dtype=dt)[:, :length]
    x = torch.randn(length, generator=gen, device="cuda", dtype=dt)
    y = _rows_dot(A, k, x)
    ref = A.double() @ x.double()
    scale = A.double().abs() @ x.double().abs()
    assert torch.all((y - ref).abs() <= tol * scale + 1e-300)
    c = torch.randn(k, generator=gen, device="cuda", dtype=torch.float64)
    x0 = x.clone()
    _rows_axpy(A, k, c, x)
    refx = x0.double() - c @ A.double()
    # result rounded once to the data type
    ulp = 2.0 ** -52 if dtn == "f64" else 2.0 ** -23
    bound = ulp * refx.abs() + tol * ((c.abs() @ A.double().abs()) + x0.double().abs())
    assert torch.all((x.double() - refx).abs() <= bound)
