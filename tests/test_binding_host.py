"""The Python binding without a GPU: every entry point checks its tensors
before anything reaches the library, so host memory is never handed to a
kernel as if it were device memory (and there is no CPU fallback)."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    from paper_2604_27210_gb300 import build
    build.build()
    from paper_2604_27210_gb300 import fv as mod
    return mod


def _quotes(n=8):
    f = lambda v: torch.full((n,), v, dtype=torch.float64)
    return dict(price=f(5.0), S_or_F=f(100.0), K=f(100.0), T=f(1.0), r=f(0.01), q=f(0.0),
                flag=torch.ones(n, dtype=torch.int8))


def test_host_tensors_are_rejected_before_the_library(fv):
    w = _quotes()
    args = [w[k] for k in ("price", "S_or_F", "K", "T", "r", "q", "flag")]
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_implied_vol(fv.FV_BSM, fv.FV_LBR, *args)
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_implied_vol_ex(fv.FV_BSM, fv.FV_LBR, fv.FV_MIXED, *args)
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_price(fv.FV_BSM, w["flag"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["price"])
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_greeks(fv.FV_BSM, w["flag"], w["S_or_F"], w["K"], w["T"], w["r"], w["q"], w["price"])
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_math(fv.FV_MATH_ERFCX_SQRT2, w["price"])
    with pytest.raises(TypeError, match="CUDA tensor"):
        fv.fv_normalised_black(w["price"], w["T"], w["flag"])


def test_pointer_checks(fv):
    t = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="required"):
        fv._ptr(None, 4, fv._F64, "price")
    assert fv._ptr(None, 4, fv._F64, "q", allow_none=True) is None
    # host-array entry points take CPU tensors of the stated dtype and length
    assert fv._host_ptr(t, 4, fv._F64, "price").value == t.data_ptr()
    with pytest.raises(ValueError):
        fv._host_ptr(t, 5, fv._F64, "price")
    with pytest.raises(ValueError):
        fv._host_ptr(t.to(torch.float32), 4, fv._F64, "price")
    with pytest.raises(ValueError):
        fv._host_ptr(torch.zeros(8, dtype=torch.float64)[::2], 4, fv._F64, "price")
    with pytest.raises(ValueError, match="required"):
        fv._host_ptr(None, 4, fv._F64, "price")
