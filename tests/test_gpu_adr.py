"""The ADR analysis through the C ABI (paper_1808_00037_gb300.adr): the
GPU right-hand sides of the 128 modes, projected with torch.fft, give the same
modified wavenumbers as the oracle's right-hand sides projected with numpy
(FP64 to 1e-12, both schemes, cutoff on and off); FP32 follows FP64 to 1e-4
below the wavenumber where the selection starts to act."""
import numpy as np
import pytest

import oracle
from paper_1808_00037_gb300 import adr as ADR
from paper_1808_00037_gb300 import binding as B
from test_oracle_adr import N, oracle_adr

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")


@pytest.mark.parametrize("CT", [1e-5, 1e-300])
@pytest.mark.parametrize("scheme,osch", [(B.T7_TENO7EXT, oracle.SCHEME_TENO7EXT), (B.T7_TENO5, oracle.SCHEME_TENO5)],
                         ids=["teno7ext", "teno5"])
def test_adr_gpu_equals_oracle(scheme, osch, CT):
    phi, got = ADR.adr(N, scheme=scheme, CT=CT)
    phio, want = oracle_adr(osch, CT)
    assert np.allclose(phi, phio, rtol=0, atol=1e-15)
    assert np.max(np.abs(got - want)) < 1e-12


def test_adr_f32_follows_f64():
    phi, a64 = ADR.adr(N, prec=B.T7_F64)
    _, a32 = ADR.adr(N, prec=B.T7_F32)
    k = np.argmax(phi > 0.5 * np.pi)
    assert np.max(np.abs(a32[:k] - a64[:k])) < 1e-4
    assert ADR.resolving_wavenumber(phi, a64, 1e-2) > 1.0
